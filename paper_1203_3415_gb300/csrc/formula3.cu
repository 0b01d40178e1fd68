// k = 3 by the paper's per-vertex formulas (Thm teo3, Algorithm s3, Table
// starb): no subset is visited.
//
// At a vertex c the neighbours fall into three sets by their pair state to c
// (out-only, in-only, bidirected: the paper's B, C, A).  Every pair {a, b} of
// neighbours of c is a connected triple with c in the middle; its class is
// fixed by the two states and by the arcs between a and b.  So the paper
// counts the pairs per pair of sets from the set sizes (|S|(|S|-1)/2 or
// |S||T|) as if a and b were not adjacent, and corrects with the pairs that
// are adjacent; those are the triangles through c, which it counts once per
// vertex and divides by 3.  Here each triangle v < x < u is found once, at its
// middle vertex x (a lower neighbour v of x adjacent to an upper neighbour u
// of x, one pair-state probe), adds 1 to its own class and moves the three
// pairs it was counted as (one per centre) out of their open-triple classes.
// Warp per vertex; classes come from the canonical-layout code table.
#include "formula.cuh"

namespace acc {

namespace {

constexpr int kF3Classes = 13;

// State of a pair seen from the other end (arc directions swapped).
__device__ __forceinline__ uint32_t swap_state(uint32_t s) { return ((s & 1u) << 1) | (s >> 1); }

// Canonical-layout adjacency code of the tuple (c, a, b) (bit i*2 + j - [j>i]
// is the arc w_i -> w_j) from state(c, a), state(c, b), state(a, b).
__device__ __forceinline__ uint32_t code3(uint32_t s_ca, uint32_t s_cb, uint32_t s_ab) {
    return (s_ca & 1u) | ((s_ca >> 1) << 2) | ((s_cb & 1u) << 1) | ((s_cb >> 1) << 4) | ((s_ab & 1u) << 3) |
           ((s_ab >> 1) << 5);
}

__device__ __forceinline__ uint32_t probe3(const uint32_t *__restrict__ st, long long pitch, uint32_t a, uint32_t b) {
    return (__ldg(st + (long long)a * pitch + (b >> 4)) >> ((b & 15u) << 1)) & 3u;
}

__global__ void k_formula3(GSet gs, const uint32_t *__restrict__ state, const long long *__restrict__ nptr,
                           const int *__restrict__ deg, const int *__restrict__ lo, const uint32_t *__restrict__ nbr,
                           const int16_t *__restrict__ lut, unsigned long long *counts, int *status) {
    grid_dep_wait();
    __shared__ unsigned long long hist[kF3Classes];
    const bool several = gs.B > 1;  // several graphs: straight to each graph's counts
    for (int i = threadIdx.x; i < kF3Classes; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    auto add = [&](unsigned long long *cnt, uint32_t code, long long delta) {
        const int cls = lut[code];
        if (cls < 0 || cls >= kF3Classes) {
            set_status(status, ACC_ERR_INTERNAL);
            return;
        }
        atomicAdd(several ? &cnt[cls] : &hist[cls], (unsigned long long)delta);
    };
    for (long long x = warp; x < gs.NV; x += nwarps) {
        const GMeta mt = gs.meta(gs.graph_of((int)x));
        unsigned long long *cnt = counts + (size_t)gs.graph_of((int)x) * kF3Classes;
        const uint32_t *st = state + mt.soff;
        const long long base = nptr[x];
        const int d = deg[x], l = lo[x];
        // neighbours of x per pair state: open triples with x in the middle
        long long n1 = 0, n2 = 0, n3 = 0;
        for (int q = lane; q < d; q += kWarp) {
            const uint32_t s = __ldg(nbr + base + q) & 3u;
            n1 += s == 1u;
            n2 += s == 2u;
            n3 += s == 3u;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            n1 += __shfl_xor_sync(kFull, n1, o);
            n2 += __shfl_xor_sync(kFull, n2, o);
            n3 += __shfl_xor_sync(kFull, n3, o);
        }
        if (lane < 6) {
            // (1,1) (2,2) (3,3) (1,2) (1,3) (2,3)
            const uint32_t sa = lane < 3 ? (uint32_t)lane + 1u : (lane == 5 ? 2u : 1u);
            const uint32_t sb = lane < 3 ? sa : (lane == 3 ? 2u : 3u);
            const long long na = sa == 1u ? n1 : (sa == 2u ? n2 : n3);
            const long long nb = sb == 1u ? n1 : (sb == 2u ? n2 : n3);
            const long long pairs = sa == sb ? na * (na - 1) / 2 : na * nb;
            if (pairs) add(cnt, code3(sa, sb, 0u), pairs);
        }
        // triangles v < x < u: v among the first l entries, u among the rest
        const long long npairs = (long long)l * (d - l);
        const int hi = d - l;
        for (long long p = lane; p < npairs; p += kWarp) {
            const int i = (int)(p / hi), j = (int)(p % hi);
            const uint32_t ev = __ldg(nbr + base + i), eu = __ldg(nbr + base + l + j);
            const uint32_t v = ev >> 2, u = eu >> 2;
            const uint32_t s_vu = probe3(st, mt.pitch, v, u);
            if (!s_vu) continue;
            const uint32_t s_vx = swap_state(ev & 3u), s_xu = eu & 3u;
            add(cnt, code3(s_vx, s_vu, s_xu), 1);                        // the triangle (v, x, u)
            add(cnt, code3(s_vx, s_vu, 0u), -1);                         // counted open at v
            add(cnt, code3(ev & 3u, s_xu, 0u), -1);                      // at x
            add(cnt, code3(swap_state(s_vu), swap_state(s_xu), 0u), -1); // at u
        }
    }
    __syncthreads();
    if (!several)
        for (int i = threadIdx.x; i < kF3Classes; i += blockDim.x)
            if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

}  // namespace

int launch_formula3(const GSet &gs, const uint32_t *state, const long long *nptr, const int *deg, const int *lo,
                    const uint32_t *nbr, const int16_t *lut, unsigned long long *counts, int *status, int num_sms,
                    cudaStream_t s) {
    if (gs.NV == 0) return 0;
    long long blocks = (gs.NV * kWarp + 255) / 256;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    launch_pdl(k_formula3, (int)blocks, 256, 0, s, gs, state, nptr, deg, lo, nbr, lut, counts, status);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

}  // namespace acc
