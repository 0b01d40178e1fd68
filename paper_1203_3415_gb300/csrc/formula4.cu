// k = 4 by the paper's edge formulas (Thm lema4d, Cor coro:a, Alg mine,
// Fact correction): no 4-set is visited one by one.
//
// For an edge e = {u, v} of G* the other vertices adjacent to u or v fall
// into the paper's 15 sets of e (Fig. edgesets: A1, B1, C1 touch u only,
// A2, B2, C2 touch v only, AA .. CC touch both), here the 4-bit bin
// state(u, x) | state(v, x) << 2.  Every pair {x, y} of them forms a
// 4-set {u, v, x, y} whose class is fixed by the state of e, the two bins
// and the state of {x, y}.  So, as in Thm lema4d, the pairs are counted per
// pair of bins from the bin sizes (C(n, 2) or n_i n_j) as if x and y were not
// linked, and each linked pair (the paper's m and m' variables) moves one
// 4-set from the unlinked class to its own.  Cor coro:a (e one-way) needs
// nothing extra: the state of e is part of the class lookup.
//
// A 4-set is reached from every G* edge of it whose other two vertices each
// touch an end of the edge: 1 (path), 3 (star, tailed triangle), 4 (cycle),
// 5 (diamond), 6 (complete) edges (Fact correction).  The sums are divided
// by that multiplicity at the end, which leaves the exact counts.
//
// Warp per edge, taken from its smaller end; the linked pairs come from
// scanning the lists of the union's members (each pair once, from its smaller
// vertex), the entries spread over the lanes.
#include "formula.cuh"

namespace acc {

namespace {

constexpr int kF4Classes = 199;
constexpr int kF4Warps = 8;

// True when the launch just enqueued was accepted; a refused launch's error
// is cleared, and the caller launches nothing that would read its output.
bool launch_ok() {
    if (cudaPeekAtLastError() == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

__device__ __forceinline__ uint32_t probe4(const uint32_t *__restrict__ st, long long pitch, uint32_t a, uint32_t b) {
    return (__ldg(st + (long long)a * pitch + (b >> 4)) >> ((b & 15u) << 1)) & 3u;
}

// Canonical-layout code of the tuple (u, v, x, y): bin_x = state(u, x) |
// state(v, x) << 2, the same for y; s_uv and s_xy are the states of those
// pairs.  Arc w_i -> w_j is bit i * 3 + j - [j > i].
__device__ __forceinline__ uint32_t code4(uint32_t s_uv, uint32_t bx, uint32_t by, uint32_t s_xy) {
    const uint32_t s[4][4] = {{0u, s_uv, bx & 3u, by & 3u}, {0u, 0u, bx >> 2, by >> 2}, {0u, 0u, 0u, s_xy}, {0u, 0u, 0u, 0u}};
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = i + 1; j < 4; j++) {
            c |= (s[i][j] & 1u) << (i * 3 + j - 1);  // w_i -> w_j
            c |= (s[i][j] >> 1) << (j * 3 + i);      // w_j -> w_i
        }
    return c;
}

__global__ void __launch_bounds__(kF4Warps * 32) k_formula4(GSet gs, const uint32_t *__restrict__ state,
                                                            const long long *__restrict__ nptr,
                                                            const int *__restrict__ deg, const int *__restrict__ lo,
                                                            const uint32_t *__restrict__ nbr,
                                                            const int16_t *__restrict__ lut, const GraphInfo *info,
                                                            unsigned long long *counts, int *status) {
    __shared__ unsigned long long hist[kF4Classes];
    __shared__ int bins[kF4Warps][16];
    const bool several = gs.B > 1;  // several graphs: straight to each graph's counts
    for (int i = threadIdx.x; i < kF4Classes; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nnz = info->nnz;
    auto add = [&](unsigned long long *cnt, uint32_t code, long long delta) {
        const int cls = lut[code];
        if (cls < 0 || cls >= kF4Classes) {
            set_status(status, ACC_ERR_INTERNAL);
            return;
        }
        atomicAdd(several ? &cnt[cls] : &hist[cls], (unsigned long long)delta);
    };
    for (long long p = warp; p < nnz; p += nwarps) {
        // the vertex whose list holds entry p
        long long a = 0, b = gs.NV - 1;
        while (a < b) {
            const long long mid = (a + b + 1) >> 1;
            if (nptr[mid] <= p) a = mid;
            else b = mid - 1;
        }
        const long long ug = a;
        if (p - nptr[ug] < lo[ug]) continue;  // each edge once, from its smaller end
        const int g = gs.graph_of((int)ug);
        const GMeta mt = gs.meta(g);
        unsigned long long *cnt = counts + (size_t)g * kF4Classes;
        const uint32_t *st = state + mt.soff;
        const uint32_t e_uv = __ldg(nbr + p);
        const uint32_t u = (uint32_t)(ug - mt.voff), v = e_uv >> 2, s_uv = e_uv & 3u;
        const long long vg = mt.voff + v;
        const long long bu = nptr[ug], bv = nptr[vg];
        const int du = deg[ug], dv = deg[vg];

        // bin sizes: N(u) \ {v}, then the members of N(v) \ {u} outside N(u)
        if (lane < 16) bins[wib][lane] = 0;
        __syncwarp();
        for (int q = lane; q < du; q += kWarp) {
            const uint32_t ex = __ldg(nbr + bu + q), x = ex >> 2;
            if (x != v) atomicAdd(&bins[wib][(ex & 3u) | (probe4(st, mt.pitch, v, x) << 2)], 1);
        }
        for (int q = lane; q < dv; q += kWarp) {
            const uint32_t ex = __ldg(nbr + bv + q), x = ex >> 2;
            if (x != u && probe4(st, mt.pitch, u, x) == 0u) atomicAdd(&bins[wib][(ex & 3u) << 2], 1);
        }
        __syncwarp();
        // every pair of bins as if unlinked (120 pairs i <= j of bins 1..15)
        for (int t = lane; t < 120; t += kWarp) {
            int i = 1, r = t;
            while (r >= 16 - i) {
                r -= 16 - i;
                i++;
            }
            const int j = i + r;
            const long long ni = bins[wib][i], nj = bins[wib][j];
            const long long pairs = i == j ? ni * (ni - 1) / 2 : ni * nj;
            if (pairs) add(cnt, code4(s_uv, (uint32_t)i, (uint32_t)j, 0u), pairs);
        }
        // linked pairs {x, y} of the union, x < y: members in chunks of 32
        // (pass 0: N(u) \ {v}; pass 1: N(v) \ {u} outside N(u)), their lists'
        // entries spread over the lanes (every shuffle on all lanes)
        for (int pass = 0; pass < 2; pass++) {
            const long long bl = pass ? bv : bu;
            const int dl = pass ? dv : du;
            for (int c0 = 0; c0 < dl; c0 += kWarp) {
                const int q = c0 + lane;
                uint32_t x = 0, bx = 0;
                int dx = 0;
                long long bxl = 0;
                if (q < dl) {
                    const uint32_t ex = __ldg(nbr + bl + q);
                    x = ex >> 2;
                    bool member;
                    if (pass == 0) {
                        member = x != v;
                        bx = (ex & 3u) | (probe4(st, mt.pitch, v, x) << 2);
                    } else {
                        member = x != u && probe4(st, mt.pitch, u, x) == 0u;
                        bx = (ex & 3u) << 2;
                    }
                    if (member) {
                        dx = deg[mt.voff + x];
                        bxl = nptr[mt.voff + x];
                    }
                }
                int pre = dx;  // inclusive prefix of the members' degrees
#pragma unroll
                for (int o = 1; o < kWarp; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, pre, o);
                    if (lane >= o) pre += y;
                }
                const int total = __shfl_sync(kFull, pre, kWarp - 1);
                pre -= dx;  // exclusive
                for (int i0 = 0; i0 < total; i0 += kWarp) {
                    const int idx = i0 + lane;
                    int owner = 0;
#pragma unroll
                    for (int step = 16; step; step >>= 1) {
                        const int cand = owner + step;
                        const int pc = __shfl_sync(kFull, pre, cand & 31);
                        if (cand < kWarp && pc <= idx) owner = cand;
                    }
                    const uint32_t xo = __shfl_sync(kFull, x, owner);
                    const uint32_t bxo = __shfl_sync(kFull, bx, owner);
                    const long long blo = __shfl_sync(kFull, bxl, owner);
                    const int preo = __shfl_sync(kFull, pre, owner);
                    if (idx < total) {
                        const uint32_t ey = __ldg(nbr + blo + (idx - preo)), y = ey >> 2;
                        if (y > xo && y != u && y != v) {
                            const uint32_t by = probe4(st, mt.pitch, u, y) | (probe4(st, mt.pitch, v, y) << 2);
                            if (by) {
                                add(cnt, code4(s_uv, bxo, by, 0u), -1);
                                add(cnt, code4(s_uv, bxo, by, ey & 3u), 1);
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    if (!several)
        for (int i = threadIdx.x; i < kF4Classes; i += blockDim.x)
            if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

// counts[g][c] /= the number of G* edges of class c's pattern whose other two
// vertices each touch an end of the edge (Fact correction).
__global__ void k_formula4_divide(unsigned long long *counts, long long n, const uint32_t *__restrict__ class_code,
                                  int *status) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t code = class_code[i % kF4Classes];
        bool adj[4][4];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++)
                adj[a][b] = a != b && (((code >> code_bit(4, a, b)) & 1u) || ((code >> code_bit(4, b, a)) & 1u));
        int mult = 0;
        for (int a = 0; a < 4; a++)
            for (int b = a + 1; b < 4; b++) {
                if (!adj[a][b]) continue;
                bool dom = true;
                for (int w = 0; w < 4; w++)
                    if (w != a && w != b && !adj[w][a] && !adj[w][b]) dom = false;
                mult += dom;
            }
        const unsigned long long c = counts[i];
        if (mult == 0 || c % (unsigned long long)mult) {
            set_status(status, ACC_ERR_INTERNAL);
            continue;
        }
        counts[i] = c / (unsigned long long)mult;
    }
}

}  // namespace

int launch_formula4(const GSet &gs, const uint32_t *state, const long long *nptr, const int *deg, const int *lo,
                    const uint32_t *nbr, const int16_t *lut, const uint32_t *class_code, const GraphInfo *info,
                    unsigned long long *counts, int *status, int num_sms, cudaStream_t s) {
    if (gs.NV == 0) return 0;
    // at most 2 entries per arc
    long long blocks = (2 * gs.M * kWarp + kF4Warps * 32 - 1) / (kF4Warps * 32);
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    int launches = 0;
    if (blocks > 0) {
        k_formula4<<<(int)blocks, kF4Warps * 32, 0, s>>>(gs, state, nptr, deg, lo, nbr, lut, info, counts, status);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches++;
    }
    const long long n = (long long)gs.B * kF4Classes;
    long long db = (n + 255) / 256;
    if (db > (long long)num_sms * 4) db = (long long)num_sms * 4;
    k_formula4_divide<<<(int)db, 256, 0, s>>>(counts, n, class_code, status);
    launches++;
    return cudaGetLastError() == cudaSuccess ? launches : ACC_ERR_CUDA;
}

}  // namespace acc
