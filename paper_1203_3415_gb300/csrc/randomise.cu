// Randomised copies on the device: the random ensemble of the significance
// step (Implementation section, steps i and iii: the real graph and a set of
// random graphs are counted; the paper fixes no generator).
//
// Double-edge swaps on the out-CSR: arc e runs from the row holding position
// e to col[e].  A copy starts as col and keeps rowptr; an attempt draws two
// positions e1, e2 uniformly and, for arcs a -> b and c -> d, retargets them
// to a -> d and c -> b unless that makes a self-loop or a repeated arc, so
// every out- and in-degree is kept.  The mutual mode also keeps mutual arcs
// mutual (two single arcs swap as above; two mutual pairs a <-> b and c <-> d
// become a <-> d and c <-> b; mixed draws are rejected), so every vertex keeps
// its single in-, single out- and mutual degree.
//
// Random numbers: SplitMix64 (Steele, Lea and Flood, 2014), one stream per
// copy started at its seed, two draws per attempt, a draw mapped below m by
// the high half of its 64 x 64-bit product with m (Lemire, 2019).
//
// Layout: a warp per copy; positions are grouped by row, so the rows of e1
// and e2 (the rows of a and c) come from a per-position table shared by every
// copy ({begin, end, source}).  Two forms:
//  - speculative (when the copies' adjacency bitmaps fit the context's
//    limit): the stream is counter-based (draw k is the mix of seed + (k + 1)
//    * increment), so the warp draws 16 attempts at once, two lanes each, and
//    decides all of them against the copy as it stands: one round trip for
//    both targets and rows, one for the bitmap bits.  In the plain mode an
//    attempt reads and writes only its own two rows (targets, bits); in the
//    mutual mode it also reads the rows of b and d (and each copy keeps the
//    position of every arc's reverse), and an accepted swap of mutual pairs
//    writes them.  The decisions are exact up to the first attempt that
//    reads a row an earlier accepted one writes; that prefix is applied and
//    the next batch starts there.  The copies equal the one-by-one
//    procedure's.
//  - one by one (bitmaps over the limit): "is a -> d an arc?" is a scan of
//    row a of the copy itself, each half-warp holding one of the two rows;
//    the next attempt's draws and rows are read ahead.  An attempt costs one
//    round trip in the plain mode, two more in the mutual mode (the rows of b
//    and d).
#include "randomise.cuh"

namespace acc {

namespace {

constexpr int kRandThreads = 128;
constexpr int kRandU = 4;  // row entries per lane read with the attempt's first loads
constexpr int kHalf = 16;

// True when the launch just enqueued was accepted; a refused launch's error
// is cleared, and the caller launches nothing that would read its output.
bool launch_ok() {
    if (cudaPeekAtLastError() == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

__device__ __forceinline__ uint64_t splitmix_next(uint64_t &s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int splitmix_below(uint64_t &s, int bound) {
    return (int)__umul64hi(splitmix_next(s), (uint64_t)bound);
}

__device__ __forceinline__ int find_graph(const RGraph *gr, int G, long long q, bool by_vertex) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_vertex ? (long long)gr[mid].voff : gr[mid].moff) <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-position row table and input validation (thread per arc, then thread
// per vertex).  Malformed rows (rowptr[0] != 0, decreasing, outside [0, m],
// rowptr[n] != m), targets outside [0, n) and self-loops set *status; every
// table entry stays inside the graph's positions.
__global__ void k_rand_rows(const RGraph *__restrict__ gr, int G, long long M, long long NV, int4 *rows,
                            int *rpart, int *status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long q = t0; q < M; q += stride) {
        const RGraph rg = gr[find_graph(gr, G, q, false)];
        const int p = (int)(q - rg.moff);
        int lo = 0, hi = rg.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rg.rowptr[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        const long long beg = rg.n > 0 ? rg.rowptr[lo] : 1, end = rg.n > 0 ? rg.rowptr[lo + 1] : 0;
        const int u = rg.col[p];
        int4 e = make_int4(p, p + 1, lo, 0);
        const bool bad = beg < 0 || beg > p || end <= p || end > rg.m || u < 0 || u >= rg.n || u == lo;
        if (bad)
            set_status(status, ACC_ERR_INPUT);
        else
            e = make_int4((int)beg, (int)end, lo, 0);
        rows[q] = e;
        if (rpart) {
            // position of the reverse arc u -> lo in row u, or -1
            int rp = -1;
            if (!bad) {
                const long long rb = min(max(rg.rowptr[u], 0ll), rg.m), re = min(max(rg.rowptr[u + 1], rb), rg.m);
                for (long long k = rb; k < re; k++)
                    if (rg.col[k] == lo) {
                        rp = (int)k;
                        break;
                    }
            }
            rpart[q] = rp;
        }
    }
    for (long long x = t0; x < NV; x += stride) {
        const RGraph rg = gr[find_graph(gr, G, x, true)];
        const int v = (int)(x - rg.voff);
        const long long b = rg.rowptr[v], e = rg.rowptr[v + 1];
        if (b < 0 || e < b || e > rg.m || (v == 0 && b != 0) || (v == rg.n - 1 && e != rg.m))
            set_status(status, ACC_ERR_INPUT);
    }
}

// In this half-warp's row cp[beg, end): the position of w1 (or -1) and
// whether w2 occurs.  The first kRandU * 16 entries were read into v.
__device__ __forceinline__ void half_search(const int *cp, int beg, int end, int hl, const int (&v)[kRandU], int w1,
                                            int w2, int &pos1, bool &has2) {
    pos1 = -1;
    has2 = false;
#pragma unroll
    for (int j = 0; j < kRandU; j++) {
        const int q = beg + hl + kHalf * j;
        if (q < end) {
            if (v[j] == w1) pos1 = q;
            has2 |= v[j] == w2;
        }
    }
    for (int q = beg + kHalf * kRandU + hl; q < end; q += kHalf) {
        const int x = cp[q];
        if (x == w1) pos1 = q;
        has2 |= x == w2;
    }
}

__device__ __forceinline__ void half_load(const int *cp, int beg, int end, int hl, int (&v)[kRandU]) {
#pragma unroll
    for (int j = 0; j < kRandU; j++) {
        const int q = beg + hl + kHalf * j;
        v[j] = q < end ? cp[q] : -1;
    }
}

// One attempt on copy cp (e1 != e2; r1, r2 the rows of e1 and e2).  Returns
// whether it was accepted; the copy is updated and the update is visible to
// the whole warp on return.
template <bool MUTUAL>
__device__ __forceinline__ bool attempt(int *cp, const long long *__restrict__ rowptr, int m, int e1, int e2,
                                        int4 r1, int4 r2, int lane) {
    const int half = lane >> 4, hl = lane & 15;
    const int4 rr = half ? r2 : r1;  // half 0: row a (arc e1), half 1: row c (arc e2)
    const int x = cp[half ? e2 : e1];
    int v[kRandU];
    half_load(cp, rr.x, rr.y, hl, v);
    const int b = __shfl_sync(kFull, x, 0), d = __shfl_sync(kFull, x, kHalf);
    const int a = r1.z, c = r2.z;
    if (a == d || c == b) return false;
    int p;
    bool unused;
    half_search(cp, rr.x, rr.y, hl, v, half ? b : d, -2, p, unused);  // a -> d (half 0), c -> b (half 1)
    if (__any_sync(kFull, p >= 0)) return false;
    int p1 = -1, p2 = -1;
    if (MUTUAL) {
        // rows of b (half 0) and d (half 1): the reverse arcs b -> a and d -> c
        // (mutual arcs) and the arcs b -> c and d -> a (adjacency)
        const int y = half ? d : b;
        const int beg = (int)min(max(rowptr[y], 0ll), (long long)m);
        const int end = (int)min(max(rowptr[y + 1], (long long)beg), (long long)m);
        int u[kRandU];
        half_load(cp, beg, end, hl, u);
        int pm;
        bool rev;
        half_search(cp, beg, end, hl, u, half ? c : a, half ? a : c, pm, rev);
        if (__any_sync(kFull, rev)) return false;
        p1 = __reduce_max_sync(kFull, half ? -1 : pm);
        p2 = __reduce_max_sync(kFull, half ? pm : -1);
        if ((p1 >= 0) != (p2 >= 0)) return false;
    }
    if (lane == 0) {
        cp[e1] = d;
        cp[e2] = b;
        if (MUTUAL && p1 >= 0) {
            cp[p1] = c;
            cp[p2] = a;
        }
    }
    __syncwarp();
    return true;
}

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// Draw k (0-based) of the stream seeded `seed`, mapped below `bound`.
__device__ __forceinline__ int splitmix_draw_below(uint64_t seed, unsigned long long k, int bound) {
    uint64_t s = seed + (uint64_t)k * kGamma;  // the state before draw k
    return splitmix_below(s, bound);
}

// Plain mode, speculative batches of 16 attempts (lanes 2p and 2p + 1 hold
// the arcs e1 and e2 of attempt t + p).  bits: the copies' adjacency bitmaps,
// row a of a copy at a * bw words.
__global__ void __launch_bounds__(kRandThreads) k_rand_swap_spec(const RGraph *__restrict__ gr, int G, int R,
                                                                 const int4 *__restrict__ rows, int *out,
                                                                 uint32_t *bits, long long *accepted,
                                                                 int *status) {
    if (*(volatile const int *)status) return;
    const int lane = threadIdx.x & 31;
    const unsigned earlier = (1u << (lane & ~1)) - 1u;  // lanes of the batch's earlier attempts
    const long long items = (long long)G * R;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < items; w += nw) {
        const int g = (int)(w / R), r = (int)(w - (long long)g * R);
        const RGraph rg = gr[g];
        const int m = (int)rg.m, bw = rg.bw;
        const int4 *rw = rows + rg.moff;
        int *cp = out + rg.ooff + (long long)r * rg.m;
        uint32_t *bm = bits + rg.boff + (long long)r * rg.n * bw;
        uint4 *bm4 = reinterpret_cast<uint4 *>(bm);
        const long long words4 = (long long)rg.n * bw / 4;
        for (long long i = lane; i < words4; i += kWarp) bm4[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        for (int e = lane; e < m; e += kWarp) {
            const int u = __ldg(rg.col + e);
            cp[e] = u;
            atomicOr(&bm[(long long)__ldg(&rw[e].z) * bw + (u >> 5)], 1u << (u & 31));
        }
        __syncwarp();
        long long acc = 0;
        const uint64_t seed = rg.seed + (uint64_t)r;
        long long t = 0, batches = 0;
        while (m >= 2 && t < rg.attempts) {
            if (++batches > rg.attempts) {  // every batch applies at least one attempt
                set_status(status, ACC_ERR_INTERNAL);
                break;
            }
            const long long left = rg.attempts - t;
            const int P = left < 16 ? (int)left : 16;
            const bool live = (lane >> 1) < P;
            const int e = splitmix_draw_below(seed, (unsigned long long)(2 * t + lane), m);
            const int src = __ldg(&rw[e].z);
            const int x = cp[e];                              // this arc's target
            const int y = __shfl_xor_sync(kFull, x, 1);       // the other arc's target
            const int ep = __shfl_xor_sync(kFull, e, 1);
            // even lane: a -> b with b = x, looks up a -> d (d = y); odd lane:
            // c -> d with d = x, looks up c -> b (b = y)
            // (every lane takes part in each shuffle: none sits behind && or ?:)
            const bool ok = live && e != ep && src != y;
            const bool ok_other = __shfl_xor_sync(kFull, ok, 1);
            const bool pair_ok = ok && ok_other;
            bool hit = false;
            if (pair_ok) hit = (bm[(long long)src * bw + (y >> 5)] >> (y & 31)) & 1u;
            const bool hit_other = __shfl_xor_sync(kFull, hit, 1);
            const bool take = pair_ok && !hit && !hit_other;
            const unsigned A = __ballot_sync(kFull, take);
            const unsigned same_row = __match_any_sync(kFull, src);
            const unsigned C = __ballot_sync(kFull, live && (same_row & A & earlier) != 0u);
            const unsigned Cp = (C | (C >> 1)) & 0x55555555u;  // bit 2p: attempt p shares a row
            const int adv = Cp ? min(P, (__ffs(Cp) - 1) >> 1) : P;
            const bool commit = take && (lane >> 1) < adv;
            if (commit) {
                uint32_t *row = bm + (long long)src * bw;
                cp[e] = y;
                atomicAnd(&row[x >> 5], ~(1u << (x & 31)));
                atomicOr(&row[y >> 5], 1u << (y & 31));
            }
            acc += __popc(__ballot_sync(kFull, commit)) >> 1;
            __syncwarp();
            t += adv;
        }
        if (lane == 0 && accepted) accepted[w] = acc;
        __syncwarp();
    }
}

// Mutual mode, speculative batches of 16 attempts.  pt: each copy's reverse
// position of every arc (-1 for a single arc), started from the graph's
// (rpart).  An attempt reads rows a, b, c, d; an accepted swap of two single
// arcs writes rows a and c, of two mutual pairs all four; the batch applies
// the attempts before the first one that reads a row an earlier accepted
// one writes.
__global__ void __launch_bounds__(kRandThreads) k_rand_swap_spec_mutual(const RGraph *__restrict__ gr, int G, int R,
                                                                        const int4 *__restrict__ rows,
                                                                        const int *__restrict__ rpart, int *out,
                                                                        int *pts, uint32_t *bits,
                                                                        long long *accepted, int *status) {
    if (*(volatile const int *)status) return;
    const int lane = threadIdx.x & 31;
    const long long items = (long long)G * R;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < items; w += nw) {
        const int g = (int)(w / R), r = (int)(w - (long long)g * R);
        const RGraph rg = gr[g];
        const int m = (int)rg.m, bw = rg.bw;
        const int4 *rw = rows + rg.moff;
        int *cp = out + rg.ooff + (long long)r * rg.m;
        int *pt = pts + rg.ooff + (long long)r * rg.m;
        uint32_t *bm = bits + rg.boff + (long long)r * rg.n * bw;
        uint4 *bm4 = reinterpret_cast<uint4 *>(bm);
        const long long words4 = (long long)rg.n * bw / 4;
        for (long long i = lane; i < words4; i += kWarp) bm4[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        for (int e = lane; e < m; e += kWarp) {
            const int u = __ldg(rg.col + e);
            cp[e] = u;
            pt[e] = __ldg(rpart + rg.moff + e);
            atomicOr(&bm[(long long)__ldg(&rw[e].z) * bw + (u >> 5)], 1u << (u & 31));
        }
        __syncwarp();
        long long acc = 0;
        const uint64_t seed = rg.seed + (uint64_t)r;
        long long t = 0, batches = 0;
        while (m >= 2 && t < rg.attempts) {
            if (++batches > rg.attempts) {  // every batch applies at least one attempt
                set_status(status, ACC_ERR_INTERNAL);
                break;
            }
            const long long left = rg.attempts - t;
            const int P = left < 16 ? (int)left : 16;
            const bool live = (lane >> 1) < P;
            // even lane: arc e1 = a -> b; odd lane: arc e2 = c -> d.  src is
            // a (c), x is b (d), y the other arc's target, so the arcs to be
            // made are src -> y on both lanes
            const int e = splitmix_draw_below(seed, (unsigned long long)(2 * t + lane), m);
            const int src = __ldg(&rw[e].z);
            const int x = cp[e];
            const int pe = pt[e];
            const int y = __shfl_xor_sync(kFull, x, 1);
            const int ep = __shfl_xor_sync(kFull, e, 1);
            const int pe_o = __shfl_xor_sync(kFull, pe, 1);
            const int src_o = __shfl_xor_sync(kFull, src, 1);
            const bool ok = live && e != ep && src != y && (pe >= 0) == (pe_o >= 0);
            const bool ok_other = __shfl_xor_sync(kFull, ok, 1);
            const bool pair_ok = ok && ok_other;
            bool hit = false;
            if (pair_ok) {
                const uint32_t f = (bm[(long long)src * bw + (y >> 5)] >> (y & 31)) & 1u;   // a -> d / c -> b
                const uint32_t b2 = (bm[(long long)y * bw + (src >> 5)] >> (src & 31)) & 1u; // d -> a / b -> c
                hit = (f | b2) != 0u;
            }
            const bool hit_other = __shfl_xor_sync(kFull, hit, 1);
            const bool take = pair_ok && !hit && !hit_other;
            const bool mut = pe >= 0;
            // rows this lane's attempt reads: src and x (with the other lane's, a b c d)
            bool clash = false;
#pragma unroll 1
            for (int jp = 0; jp < 16; jp++) {
                const bool tj = __shfl_sync(kFull, take, 2 * jp);
                const bool mj = __shfl_sync(kFull, mut, 2 * jp);
                const int a_j = __shfl_sync(kFull, src, 2 * jp), c_j = __shfl_sync(kFull, src, 2 * jp + 1);
                const int b_j = __shfl_sync(kFull, x, 2 * jp), d_j = __shfl_sync(kFull, x, 2 * jp + 1);
                if (tj && jp < (lane >> 1)) {
                    clash |= src == a_j || src == c_j || x == a_j || x == c_j;
                    if (mj) clash |= src == b_j || src == d_j || x == b_j || x == d_j;
                }
            }
            const unsigned C = __ballot_sync(kFull, live && clash);
            const unsigned Cp = (C | (C >> 1)) & 0x55555555u;
            const int adv = Cp ? min(P, (__ffs(Cp) - 1) >> 1) : P;
            const bool commit = take && (lane >> 1) < adv;
            if (commit) {
                uint32_t *row = bm + (long long)src * bw;
                cp[e] = y;
                atomicAnd(&row[x >> 5], ~(1u << (x & 31)));
                atomicOr(&row[y >> 5], 1u << (y & 31));
                if (mut) {
                    // the reverse arc x -> src becomes x -> (the other arc's source);
                    // new pairs: src <-> y (this arc, the other's reverse) and
                    // x <-> other source (this reverse, the other arc)
                    uint32_t *rrow = bm + (long long)x * bw;
                    cp[pe] = src_o;
                    atomicAnd(&rrow[src >> 5], ~(1u << (src & 31)));
                    atomicOr(&rrow[src_o >> 5], 1u << (src_o & 31));
                    pt[e] = pe_o;
                    pt[pe] = ep;
                }
            }
            acc += __popc(__ballot_sync(kFull, commit)) >> 1;
            __syncwarp();
            t += adv;
        }
        if (lane == 0 && accepted) accepted[w] = acc;
        __syncwarp();
    }
}

template <bool MUTUAL>
__global__ void __launch_bounds__(kRandThreads) k_rand_swap(const RGraph *__restrict__ gr, int G, int R,
                                                            const int4 *__restrict__ rows, int *out,
                                                            long long *accepted, const int *status) {
    if (*(volatile const int *)status) return;
    const int lane = threadIdx.x & 31;
    const long long items = (long long)G * R;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < items; w += nw) {
        const int g = (int)(w / R), r = (int)(w - (long long)g * R);
        const RGraph rg = gr[g];
        const int m = (int)rg.m;
        int *cp = out + rg.ooff + (long long)r * rg.m;
        for (int e = lane; e < m; e += kWarp) cp[e] = __ldg(rg.col + e);
        __syncwarp();
        long long acc = 0;
        if (m >= 2 && rg.attempts > 0) {
            const int4 *rw = rows + rg.moff;
            uint64_t s = rg.seed + (uint64_t)r;
            int e1 = splitmix_below(s, m);
            int e2 = splitmix_below(s, m);
            int4 r1 = __ldg(rw + e1), r2 = __ldg(rw + e2);
            for (long long t = 0; t < rg.attempts; t++) {
                // the next attempt's draws and rows do not depend on this one
                int f1 = 0, f2 = 0;
                int4 q1 = r1, q2 = r2;
                if (t + 1 < rg.attempts) {
                    f1 = splitmix_below(s, m);
                    f2 = splitmix_below(s, m);
                    q1 = __ldg(rw + f1);
                    q2 = __ldg(rw + f2);
                }
                if (e1 != e2 && attempt<MUTUAL>(cp, rg.rowptr, m, e1, e2, r1, r2, lane)) acc++;
                e1 = f1;
                e2 = f2;
                r1 = q1;
                r2 = q2;
            }
        }
        if (lane == 0 && accepted) accepted[w] = acc;
        __syncwarp();
    }
}

}  // namespace

int launch_randomise(const RGraph *meta, int G, int R, long long M, long long NV, int mode, int4 *rows, int *out,
                     uint32_t *bits, int *rpart, int *pts, long long *accepted, int *status, int num_sms,
                     cudaStream_t s) {
    const bool mutual_spec = mode == ACC_RAND_MUTUAL && bits && rpart && pts;
    int launches = 0;
    const long long work = M > NV ? M : NV;
    if (work > 0) {
        long long blocks = (work + 255) / 256;
        if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
        k_rand_rows<<<(int)blocks, 256, 0, s>>>(meta, G, M, NV, rows, mutual_spec ? rpart : nullptr, status);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches++;
    }
    const long long items = (long long)G * R;
    if (items > 0) {
        long long blocks = (items * kWarp + kRandThreads - 1) / kRandThreads;
        if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
        if (mutual_spec)
            k_rand_swap_spec_mutual<<<(int)blocks, kRandThreads, 0, s>>>(meta, G, R, rows, rpart, out, pts, bits,
                                                                          accepted, status);
        else if (mode == ACC_RAND_MUTUAL)
            k_rand_swap<true><<<(int)blocks, kRandThreads, 0, s>>>(meta, G, R, rows, out, accepted, status);
        else if (bits)
            k_rand_swap_spec<<<(int)blocks, kRandThreads, 0, s>>>(meta, G, R, rows, out, bits, accepted, status);
        else
            k_rand_swap<false><<<(int)blocks, kRandThreads, 0, s>>>(meta, G, R, rows, out, accepted, status);
        launches++;
    }
    return cudaGetLastError() == cudaSuccess ? launches : ACC_ERR_CUDA;
}

}  // namespace acc
