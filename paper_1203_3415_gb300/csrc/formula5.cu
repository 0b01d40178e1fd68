// k = 5 by the paper's Δ-pattern formulas (Lemma lema5d, Algorithm fived,
// Algorithm partfive, Fact basefive): no 5-set is visited one by one.
//
// For a connected 3-set {p1, p2, p3} of G* (the paper's induced Δ), the other
// vertices adjacent to some p_i fall into the paper's 63 sets (Algorithm
// partfive), here the 6-bit bin state(p1, x) | state(p2, x) << 2 |
// state(p3, x) << 4.  Every pair {x, y} of them forms a 5-set whose class is
// fixed by the three states inside Δ, the two bins and the state of {x, y}:
// pairs are counted per pair of bins from the bin sizes as if unlinked, and
// every linked pair moves one 5-set from the unlinked class to its own
// (Lemma lema5d).  A 5-set is reached from each connected 3-subset of it
// whose other two vertices each touch it, so each class is divided by that
// number for its pattern at the end (Algorithm fived's constants, derived
// here from the class's code).
//
// Each connected 3-set is taken once: an open one (p2, p3 not adjacent) at
// its middle vertex p1, a triangle at its smallest vertex.  A work item is a
// pair of entries of one list, the items of all lists numbered through a
// prefix sum of C(deg, 2), a warp per item.
#include "formula.cuh"

namespace acc {

namespace {

constexpr int kF5Classes = 9364;
constexpr int kF5Warps = 8;
constexpr int kF5Bins = 64;

// True when the launch just enqueued was accepted; a refused launch's error
// is cleared, and the caller launches nothing that would read its output.
bool launch_ok() {
    if (cudaPeekAtLastError() == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

__device__ __forceinline__ uint32_t probe5(const uint32_t *__restrict__ st, long long pitch, uint32_t a, uint32_t b) {
    return (__ldg(st + (long long)a * pitch + (b >> 4)) >> ((b & 15u) << 1)) & 3u;
}

// Canonical-layout code of (p1, p2, p3, x, y): d = state(p1, p2) |
// state(p1, p3) << 2 | state(p2, p3) << 4, bx / by the bins of x / y, s_xy the
// state of {x, y}.  Arc w_i -> w_j is bit i * 4 + j - [j > i].
__device__ __forceinline__ uint32_t code5(uint32_t d, uint32_t bx, uint32_t by, uint32_t s_xy) {
    uint32_t s[5][5] = {};
    s[0][1] = d & 3u;
    s[0][2] = (d >> 2) & 3u;
    s[1][2] = (d >> 4) & 3u;
    s[0][3] = bx & 3u;
    s[1][3] = (bx >> 2) & 3u;
    s[2][3] = (bx >> 4) & 3u;
    s[0][4] = by & 3u;
    s[1][4] = (by >> 2) & 3u;
    s[2][4] = (by >> 4) & 3u;
    s[3][4] = s_xy;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = i + 1; j < 5; j++) {
            c |= (s[i][j] & 1u) << (i * 4 + j - 1);  // w_i -> w_j
            c |= (s[i][j] >> 1) << (j * 4 + i);      // w_j -> w_i
        }
    return c;
}

// items[v] = C(deg v, 2); exclusive prefix into pre[0..NV] (one block walks
// the vertices in tiles of 1024 with a running carry).
__global__ void __launch_bounds__(1024) k_f5_prefix(const int *__restrict__ deg, long long NV, long long *pre) {
    __shared__ long long ws[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (long long base = 0; base < NV; base += 1024) {
        const long long i = base + t;
        const long long d = i < NV ? deg[i] : 0;
        const long long v = d * (d - 1) / 2;
        long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const long long w0 = ws[lane];
            long long wi = w0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += y;
            }
            ws[lane] = wi - w0;
        }
        __syncthreads();
        const long long c0 = carry;
        if (i < NV) pre[i] = c0 + ws[wid] + incl - v;
        __syncthreads();
        if (t == 1023) carry = c0 + ws[wid] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) pre[NV] = carry;
}

__global__ void __launch_bounds__(kF5Warps * 32) k_formula5(GSet gs, const uint32_t *__restrict__ state,
                                                            const long long *__restrict__ nptr,
                                                            const int *__restrict__ deg,
                                                            const uint32_t *__restrict__ nbr,
                                                            const int16_t *__restrict__ lut,
                                                            const long long *__restrict__ pre,
                                                            unsigned long long *counts, int *status) {
    __shared__ int bins[kF5Warps][kF5Bins];
    __shared__ unsigned char nonempty[kF5Warps][kF5Bins];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long items = pre[gs.NV];
    auto add = [&](unsigned long long *cnt, uint32_t code, long long delta) {
        const int cls = lut[code];
        if (cls < 0 || cls >= kF5Classes) {
            set_status(status, ACC_ERR_INTERNAL);
            return;
        }
        atomicAdd(&cnt[cls], (unsigned long long)delta);
    };
    for (long long q = warp; q < items; q += nwarps) {
        // the vertex p1 and the pair (i, j), i < j, of its list
        long long a0 = 0, b0 = gs.NV - 1;
        while (a0 < b0) {
            const long long mid = (a0 + b0 + 1) >> 1;
            if (pre[mid] <= q) a0 = mid;
            else b0 = mid - 1;
        }
        const long long xg = a0;
        const long long r = q - pre[xg];
        const long long dd = deg[xg];
        // row i holds pairs (i, i+1 .. dd-1): start(i) = i (2 dd - i - 1) / 2
        long long i = (long long)((2.0 * dd - 1.0 - sqrt((2.0 * dd - 1.0) * (2.0 * dd - 1.0) - 8.0 * (double)r)) / 2.0);
        if (i < 0) i = 0;
        while (i > 0 && i * (2 * dd - i - 1) / 2 > r) i--;
        while ((i + 1) * (2 * dd - i - 2) / 2 <= r) i++;
        const long long j = i + 1 + (r - i * (2 * dd - i - 1) / 2);
        const int g = gs.graph_of((int)xg);
        const GMeta mt = gs.meta(g);
        const uint32_t *st = state + mt.soff;
        unsigned long long *cnt = counts + (size_t)g * kF5Classes;
        const long long bx1 = nptr[xg];
        const uint32_t ea = __ldg(nbr + bx1 + i), eb = __ldg(nbr + bx1 + j);
        const uint32_t p1 = (uint32_t)(xg - mt.voff), p2 = ea >> 2, p3 = eb >> 2;
        const uint32_t s23 = probe5(st, mt.pitch, p2, p3);
        if (s23 && (p2 < p1 || p3 < p1)) continue;  // a triangle, taken at its smallest vertex
        const uint32_t dcode = (ea & 3u) | ((eb & 3u) << 2) | (s23 << 4);
        const uint32_t pv[3] = {p1, p2, p3};
        long long lb[3];
        int ld[3];
#pragma unroll
        for (int t = 0; t < 3; t++) {
            lb[t] = nptr[mt.voff + pv[t]];
            ld[t] = deg[mt.voff + pv[t]];
        }
        // bin of y in the union from list t (0 if y is in an earlier list or is a p)
        auto bin_of = [&](int t, uint32_t ey) -> uint32_t {
            const uint32_t y = ey >> 2;
            if (y == p1 || y == p2 || y == p3) return 0u;
            uint32_t b = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k == t) b |= (ey & 3u) << (2 * k);
                else {
                    const uint32_t sk = probe5(st, mt.pitch, pv[k], y);
                    if (k < t && sk) return 0u;  // counted from list k
                    b |= sk << (2 * k);
                }
            }
            return b;
        };
        for (int k = lane; k < kF5Bins; k += kWarp) bins[wib][k] = 0;
        __syncwarp();
        for (int t = 0; t < 3; t++)
            for (int e = lane; e < ld[t]; e += kWarp) {
                const uint32_t b = bin_of(t, __ldg(nbr + lb[t] + e));
                if (b) atomicAdd(&bins[wib][b], 1);
            }
        __syncwarp();
        // non-empty bins, in order
        int ne = 0;
        for (int k0 = 0; k0 < kF5Bins; k0 += kWarp) {
            const int k = k0 + lane;
            const bool has = bins[wib][k] > 0;
            const unsigned m = __ballot_sync(kFull, has);
            if (has) nonempty[wib][ne + __popc(m & ((1u << lane) - 1u))] = (unsigned char)k;
            ne += __popc(m);
        }
        __syncwarp();
        // every pair of non-empty bins as if unlinked
        const int npairs = ne * (ne + 1) / 2;
        for (int t = lane; t < npairs; t += kWarp) {
            int a = 0, rr = t;
            while (rr >= ne - a) {
                rr -= ne - a;
                a++;
            }
            const int b = a + rr;
            const int ba = nonempty[wib][a], bb = nonempty[wib][b];
            const long long na = bins[wib][ba], nb = bins[wib][bb];
            const long long pairs = a == b ? na * (na - 1) / 2 : na * nb;
            if (pairs) add(cnt, code5(dcode, (uint32_t)ba, (uint32_t)bb, 0u), pairs);
        }
        // linked pairs {y, z} of the union, y < z: members in chunks of 32,
        // their lists' entries spread over the lanes (every shuffle on all lanes)
        for (int t = 0; t < 3; t++)
            for (int c0 = 0; c0 < ld[t]; c0 += kWarp) {
                const int e = c0 + lane;
                uint32_t y = 0, by = 0;
                int dy = 0;
                long long bly = 0;
                if (e < ld[t]) {
                    const uint32_t ey = __ldg(nbr + lb[t] + e);
                    by = bin_of(t, ey);
                    y = ey >> 2;
                    if (by) {
                        dy = deg[mt.voff + y];
                        bly = nptr[mt.voff + y];
                    }
                }
                int pfx = dy;
#pragma unroll
                for (int o = 1; o < kWarp; o <<= 1) {
                    const int v = __shfl_up_sync(kFull, pfx, o);
                    if (lane >= o) pfx += v;
                }
                const int total = __shfl_sync(kFull, pfx, kWarp - 1);
                pfx -= dy;
                for (int i0 = 0; i0 < total; i0 += kWarp) {
                    const int idx = i0 + lane;
                    int owner = 0;
#pragma unroll
                    for (int step = 16; step; step >>= 1) {
                        const int cand = owner + step;
                        const int pc = __shfl_sync(kFull, pfx, cand & 31);
                        if (cand < kWarp && pc <= idx) owner = cand;
                    }
                    const uint32_t yo = __shfl_sync(kFull, y, owner);
                    const uint32_t byo = __shfl_sync(kFull, by, owner);
                    const long long blo = __shfl_sync(kFull, bly, owner);
                    const int po = __shfl_sync(kFull, pfx, owner);
                    if (idx < total) {
                        const uint32_t ez = __ldg(nbr + blo + (idx - po)), z = ez >> 2;
                        if (z > yo && z != p1 && z != p2 && z != p3) {
                            const uint32_t bz = probe5(st, mt.pitch, p1, z) | (probe5(st, mt.pitch, p2, z) << 2) |
                                                (probe5(st, mt.pitch, p3, z) << 4);
                            if (bz) {
                                add(cnt, code5(dcode, byo, bz, 0u), -1);
                                add(cnt, code5(dcode, byo, bz, ez & 3u), 1);
                            }
                        }
                    }
                }
            }
        __syncwarp();
    }
}

// counts[g][c] /= the number of connected 3-subsets of class c's pattern
// whose other two vertices each touch one of them.
__global__ void k_formula5_divide(unsigned long long *counts, long long n, const uint32_t *__restrict__ class_code,
                                  int *status) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t code = class_code[i % kF5Classes];
        bool adj[5][5];
        for (int a = 0; a < 5; a++)
            for (int b = 0; b < 5; b++)
                adj[a][b] = a != b && (((code >> code_bit(5, a, b)) & 1u) || ((code >> code_bit(5, b, a)) & 1u));
        int mult = 0;
        for (int a = 0; a < 5; a++)
            for (int b = a + 1; b < 5; b++)
                for (int c = b + 1; c < 5; c++) {
                    const int links = adj[a][b] + adj[a][c] + adj[b][c];
                    if (links < 2) continue;  // not connected
                    bool dom = true;
                    for (int w = 0; w < 5; w++)
                        if (w != a && w != b && w != c && !adj[w][a] && !adj[w][b] && !adj[w][c]) dom = false;
                    mult += dom;
                }
        const unsigned long long v = counts[i];
        if (mult == 0 || v % (unsigned long long)mult) {
            set_status(status, ACC_ERR_INTERNAL);
            continue;
        }
        counts[i] = v / (unsigned long long)mult;
    }
}

}  // namespace

int launch_formula5(const GSet &gs, const uint32_t *state, const long long *nptr, const int *deg, const uint32_t *nbr,
                    const int16_t *lut, const uint32_t *class_code, long long *pre, unsigned long long *counts,
                    int *status, int num_sms, cudaStream_t s) {
    if (gs.NV == 0) return 0;
    k_f5_prefix<<<1, 1024, 0, s>>>(deg, gs.NV, pre);
    if (!launch_ok()) return ACC_ERR_CUDA;
    k_formula5<<<num_sms * 8, kF5Warps * 32, 0, s>>>(gs, state, nptr, deg, nbr, lut, pre, counts, status);
    if (!launch_ok()) return ACC_ERR_CUDA;
    const long long n = (long long)gs.B * kF5Classes;
    long long db = (n + 255) / 256;
    if (db > (long long)num_sms * 4) db = (long long)num_sms * 4;
    k_formula5_divide<<<(int)db, 256, 0, s>>>(counts, n, class_code, status);
    return cudaGetLastError() == cudaSuccess ? 3 : ACC_ERR_CUDA;
}

}  // namespace acc
