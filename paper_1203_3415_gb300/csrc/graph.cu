// Graph ingest: out-CSR -> dense pair-state matrix -> sorted G* neighbour
// lists with the 2-bit pair state attached to every entry.
//
// The pair state is the paper's three-way neighbour partition (Notation
// section; Algorithm table1a builds the same sets A, B, C by bucketing arcs):
// a neighbour u of v is bidirected (state 3), out-only (state 1) or in-only
// (state 2).  Here the partition is a 2-bit field of an n x n matrix, which
// also answers every "are a and b adjacent, and how" question of the
// enumeration in one 4-byte load.
#include "common.cuh"

namespace acc {

namespace {

__device__ __forceinline__ int warp_excl_scan(int x, int lane, int *total) {
    int incl = x;
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
        int y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    *total = __shfl_sync(kFull, incl, kWarp - 1);
    return incl - x;
}

__global__ void k_zero(uint4 *p, size_t n16, unsigned char *tail, size_t ntail, int *status,
                       unsigned long long *counts, int ncounts, int *ints, int nints) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j = i; j < n16; j += stride) p[j] = make_uint4(0, 0, 0, 0);
    if (i < ntail) tail[i] = 0;
    for (size_t j = i; j < (size_t)ncounts; j += stride) counts[j] = 0;
    for (size_t j = i; j < (size_t)nints; j += stride) ints[j] = 0;
    if (i == 0 && status) *status = 0;
}

// Warp per source row: set the pair-state bits of every arc, validating the
// CSR on the way.  Invalid rows and arcs are skipped (never read out of
// range) and reported through *status.  With `label` non-null, vertex x is
// written as label[x] (the relabelled matrix).
__global__ void k_ingest(const long long *__restrict__ rowptr, const int *__restrict__ col, int n,
                         long long m, uint32_t *state, long long pitch, const int *__restrict__ label,
                         int *status) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    if (warp == 0 && lane == 0) {
        if (rowptr[0] != 0 || rowptr[n] != m) set_status(status, ACC_ERR_INPUT);
    }
    for (long long v = warp; v < n; v += nwarps) {
        const long long b = rowptr[v], e = rowptr[v + 1];
        if (b < 0 || e < b || e > m) {
            if (lane == 0) set_status(status, ACC_ERR_INPUT);
            continue;
        }
        const long long a = label ? label[v] : v;
        for (long long p = b + lane; p < e; p += kWarp) {
            const int u0 = col[p];
            if (u0 < 0 || u0 >= n || u0 == (int)v) {
                set_status(status, ACC_ERR_INPUT);
                continue;
            }
            const int u = label ? label[u0] : u0;
            atomicOr(&state[a * pitch + (u >> 4)], 1u << ((u & 15) * 2));
            atomicOr(&state[(long long)u * pitch + (a >> 4)], 2u << ((a & 15) * 2));
        }
    }
}

// Degree-descending relabelling: start[d] = vertices of degree above d.
// One block; dhist[d] = vertices of degree d, d < n.
__global__ void k_desc_starts(const int *__restrict__ dhist, int n, int *start) {
    __shared__ int warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    // position i of the scan is degree n - 1 - i
    const int b = min(n, t * chunk), e = min(n, b + chunk);
    int s = 0;
    for (int i = b; i < e; i++) s += dhist[n - 1 - i];
    int incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        const int ws = lane < nw ? warp_sum[lane] : 0;
        int wi = ws;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < nw) warp_sum[lane] = wi - ws;
    }
    __syncthreads();
    int run = warp_sum[wid] + (incl - s);
    for (int i = b; i < e; i++) {
        start[n - 1 - i] = run;
        run += dhist[n - 1 - i];
    }
}

// label[v] = the next free position of v's degree class (ties in any order).
__global__ void k_desc_scatter(const int *__restrict__ deg, int n, int *start, int *label) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        label[v] = atomicAdd(&start[deg[v]], 1);
}

// Warp per row: degree of v in G* and the number of its neighbours below v.
__global__ void k_degrees(const uint32_t *__restrict__ state, long long pitch, int n, int *deg, int *lo,
                          int *dhist) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int words = (n + 15) >> 4;
    for (long long v = warp; v < n; v += nwarps) {
        const uint4 *row4 = reinterpret_cast<const uint4 *>(state + v * pitch);
        const int vw = (int)(v >> 4);
        const uint32_t below_mask = (1u << ((v & 15) * 2)) - 1u;
        int cnt = 0, below = 0;
        for (int w4 = lane; w4 * 4 < words; w4 += kWarp) {
            uint4 q = row4[w4];
            uint32_t ws[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int w = w4 * 4 + t;
                const uint32_t nz = (ws[t] | (ws[t] >> 1)) & 0x55555555u;
                const int c = __popc(nz);
                cnt += c;
                if (w < vw) below += c;
                else if (w == vw) below += __popc(nz & below_mask);
            }
        }
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            cnt += __shfl_xor_sync(kFull, cnt, d);
            below += __shfl_xor_sync(kFull, below, d);
        }
        if (lane == 0) {
            deg[v] = cnt;
            if (lo) lo[v] = below;
            if (dhist) atomicAdd(&dhist[cnt], 1);
        }
    }
}

// One block: exclusive scan of the degrees into nptr, the largest degree,
// and the reset of the per-graph work counters.
__global__ void k_scan_degrees(const int *__restrict__ deg, int n, long long *nptr, GraphInfo *info) {
    __shared__ long long warp_sum[32];
    __shared__ int warp_max[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int nthreads = blockDim.x;
    const int chunk = (n + nthreads - 1) / nthreads;
    const int b = min(n, t * chunk), e = min(n, b + chunk);
    long long s = 0;
    int mx = 0;
    for (int i = b; i < e; i++) {
        s += deg[i];
        mx = max(mx, deg[i]);
    }
    long long incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, d));
    if (lane == 31) warp_sum[wid] = incl;
    if (lane == 0) warp_max[wid] = mx;
    __syncthreads();
    if (wid == 0) {
        const int nw = nthreads >> 5;
        long long ws = lane < nw ? warp_sum[lane] : 0;
        int wm = lane < nw ? warp_max[lane] : 0;
        long long wi = ws;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
#pragma unroll
        for (int d = 16; d; d >>= 1) wm = max(wm, __shfl_xor_sync(kFull, wm, d));
        if (lane < nw) warp_sum[lane] = wi - ws;  // exclusive warp offsets
        if (lane == 0) warp_max[0] = wm;
        if (lane == nw - 1) {
            info->nnz = wi;
            nptr[n] = wi;
        }
    }
    __syncthreads();
    long long run = warp_sum[wid] + (incl - s);
    for (int i = b; i < e; i++) {
        nptr[i] = run;
        run += deg[i];
    }
    if (t == 0) {
        info->maxdeg = warp_max[0];
        info->queue_tail = 0;
        info->queue_head = 0;
        info->unit_ctr = 0;
        info->chunks_pushed = 0;
    }
}

// Warp per row: write the sorted neighbour entries (u << 2) | state(v, u).
__global__ void k_fill(const uint32_t *__restrict__ state, long long pitch, int n,
                       const long long *__restrict__ nptr, uint32_t *nbr) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int words = (n + 15) >> 4;
    for (long long v = warp; v < n; v += nwarps) {
        const uint32_t *row = state + v * pitch;
        long long base = nptr[v];
        for (int w0 = 0; w0 < words; w0 += kWarp) {
            const int w = w0 + lane;
            const uint32_t x = w < words ? row[w] : 0u;
            uint32_t nz = (x | (x >> 1)) & 0x55555555u;
            int total;
            const int off = warp_excl_scan(__popc(nz), lane, &total);
            long long pos = base + off;
            while (nz) {
                const int bit = __ffs(nz) - 1;
                const uint32_t u = (uint32_t)(w * 16 + (bit >> 1));
                nbr[pos++] = (u << 2) | ((x >> bit) & 3u);
                nz &= nz - 1;
            }
            base += total;
        }
    }
}

int grid_for(long long work_items, int per_block, int num_sms) {
    long long b = (work_items + per_block - 1) / per_block;
    long long cap = (long long)num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int launch_zero(void *p, size_t bytes, int num_sms, cudaStream_t s, int *status,
                unsigned long long *counts, int ncounts, int *ints, int nints) {
    const size_t n16 = bytes / 16, ntail = bytes % 16;
    const int grid = grid_for((long long)(n16 > 0 ? n16 : 1), 256 * 4, num_sms);
    k_zero<<<grid, 256, 0, s>>>(reinterpret_cast<uint4 *>(p), n16,
                                reinterpret_cast<unsigned char *>(p) + n16 * 16, ntail, status, counts, ncounts,
                                ints, nints);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

int launch_build_graph(const long long *rowptr, const int *col, int n, long long m,
                       uint32_t *state, long long pitch, int *deg, int *lo, long long *nptr,
                       uint32_t *nbr, int *label, GraphInfo *info, int *status, unsigned long long *counts,
                       int ncounts, bool relabel, int num_sms, cudaStream_t s) {
    int launches = 0;
    const size_t state_bytes = (size_t)n * (size_t)pitch * 4;
    const int rows_grid = grid_for((long long)n * kWarp, 256, num_sms);
    // zero the pair-state matrix, the counts, the status word and (for the
    // relabelling) the degree histogram kept in lo[]
    int r = launch_zero(state, state_bytes, num_sms, s, status, counts, ncounts, relabel ? lo : nullptr,
                        relabel ? n + 1 : 0);
    if (r < 0) return r;
    launches += r;
    k_ingest<<<rows_grid, 256, 0, s>>>(rowptr, col, n, m, state, pitch, nullptr, status);
    launches++;
    if (relabel) {
        // G* degrees under the input labels, then vertices renumbered by
        // descending degree and the matrix rebuilt under the new numbers
        int *dhist = lo;
        int *start = reinterpret_cast<int *>(nptr);
        k_degrees<<<rows_grid, 256, 0, s>>>(state, pitch, n, deg, nullptr, dhist);
        k_desc_starts<<<1, 1024, 0, s>>>(dhist, n, start);
        k_desc_scatter<<<grid_for(n, 256, num_sms), 256, 0, s>>>(deg, n, start, label);
        launches += 3;
        r = launch_zero(state, state_bytes, num_sms, s);
        if (r < 0) return r;
        launches += r;
        k_ingest<<<rows_grid, 256, 0, s>>>(rowptr, col, n, m, state, pitch, label, nullptr);
        launches++;
    }
    k_degrees<<<rows_grid, 256, 0, s>>>(state, pitch, n, deg, lo, nullptr);
    k_scan_degrees<<<1, 1024, 0, s>>>(deg, n, nptr, info);
    k_fill<<<rows_grid, 256, 0, s>>>(state, pitch, n, nptr, nbr);
    launches += 3;
    return cudaGetLastError() == cudaSuccess ? launches : ACC_ERR_CUDA;
}

}  // namespace acc
