// Graph ingest for a set of graphs (one graph is a set of one): out-CSR ->
// dense pair-state block per graph -> sorted G* neighbour lists with the
// 2-bit pair state attached to every entry.
//
// The pair state is the paper's three-way neighbour partition (Notation
// section; Algorithm table1a builds the same sets A, B, C by bucketing arcs):
// a neighbour u of v is bidirected (state 3), out-only (state 1) or in-only
// (state 2).  Here the partition is a 2-bit field of an n x n block per graph,
// which also answers every "are a and b adjacent, and how" question of the
// enumeration in one 4-byte load.
//
// Vertices of graph g occupy the global range [voff_g, voff_g + n_g); its
// pair-state block starts at word soff_g.  deg, lo, label, nptr are indexed
// by global vertex; neighbour entries and block rows/columns use local ids.
//
// The pair-state buffer is all zero between calls: a build sets only the
// words its arcs touch and the call ends by clearing exactly those words
// (k_clear_arcs), so no pass ever sweeps the whole n x n block.  G* degrees
// come out of the ingest itself: of the atomics that touch the field of pair
// {a, u} in row a (arc a -> u sets bit 0, arc u -> a sets bit 1 as its
// mirror), exactly one finds the field still zero, and that one counts u as
// a neighbour of a.  Repeated arcs therefore count once.
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

struct IntRanges {
    int *p[3];
    long long n[3];
};

__global__ void k_zero(uint4 *p, size_t n16, unsigned char *tail, size_t ntail, int *status,
                       unsigned long long *counts, long long ncounts, IntRanges ints) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j = i; j < n16; j += stride) p[j] = make_uint4(0, 0, 0, 0);
    if (i < ntail) tail[i] = 0;
    for (size_t j = i; j < (size_t)ncounts; j += stride) counts[j] = 0;
#pragma unroll
    for (int r = 0; r < 3; r++)
        for (size_t j = i; j < (size_t)ints.n[r]; j += stride) ints.p[r][j] = 0;
    if (i == 0 && status) *status = 0;
}

// Warp per global row: set the pair-state bits of every arc, validating the
// CSR on the way.  Invalid rows and arcs are skipped (never read out of
// range) and reported through *status.  With `label` non-null, vertex x is
// written as label[x] (the renumbered block).  deg[voff + a] counts the G*
// neighbours of block vertex a; lo (if non-null) those below a.
__global__ void k_ingest(GSet gs, uint32_t *state, const int *__restrict__ label, int *status, int *deg, int *lo) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < gs.NV; v += nwarps) {
        const GMeta mt = gs.meta(gs.graph_of((int)v));
        const int lv = (int)v - mt.voff;
        if (lv == 0 && lane == 0 && (mt.rowptr[0] != 0 || mt.rowptr[mt.n] != mt.m))
            set_status(status, ACC_ERR_INPUT);
        const long long b = mt.rowptr[lv], e = mt.rowptr[lv + 1];
        if (b < 0 || e < b || e > mt.m) {
            if (lane == 0) set_status(status, ACC_ERR_INPUT);
            continue;
        }
        const long long a = label ? label[v] - mt.voff : lv;
        uint32_t *blk = state + mt.soff;
        for (long long p = b + lane; p < e; p += kWarp) {
            const int u0 = mt.col[p];
            if (u0 < 0 || u0 >= mt.n || u0 == lv) {
                set_status(status, ACC_ERR_INPUT);
                continue;
            }
            const int u = label ? label[mt.voff + u0] - mt.voff : u0;
            const int su = (u & 15) * 2, sa = (int)(a & 15) * 2;
            const uint32_t oa = atomicOr(&blk[a * mt.pitch + (u >> 4)], 1u << su);
            const uint32_t ou = atomicOr(&blk[(long long)u * mt.pitch + (a >> 4)], 2u << sa);
            if (((oa >> su) & 3u) == 0u) {
                atomicAdd(&deg[mt.voff + a], 1);
                if (lo && u < a) atomicAdd(&lo[mt.voff + a], 1);
            }
            if (((ou >> sa) & 3u) == 0u) {
                atomicAdd(&deg[mt.voff + u], 1);
                if (lo && a < u) atomicAdd(&lo[mt.voff + u], 1);
            }
        }
    }
}

// Warp per global row: zero the pair-state words the arcs of the row set
// (the same rows and arcs k_ingest accepted, under the same labels), and
// with zero_deg the degree counters of the row's vertex.
__global__ void k_clear_arcs(GSet gs, uint32_t *state, const int *__restrict__ label, int *deg, int *lo) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < gs.NV; v += nwarps) {
        if (lane == 0 && deg) {
            deg[v] = 0;
            lo[v] = 0;
        }
        const GMeta mt = gs.meta(gs.graph_of((int)v));
        const int lv = (int)v - mt.voff;
        const long long b = mt.rowptr[lv], e = mt.rowptr[lv + 1];
        if (b < 0 || e < b || e > mt.m) continue;
        const long long a = label ? label[v] - mt.voff : lv;
        uint32_t *blk = state + mt.soff;
        for (long long p = b + lane; p < e; p += kWarp) {
            const int u0 = mt.col[p];
            if (u0 < 0 || u0 >= mt.n || u0 == lv) continue;
            const int u = label ? label[mt.voff + u0] - mt.voff : u0;
            blk[a * mt.pitch + (u >> 4)] = 0u;
            blk[(long long)u * mt.pitch + (a >> 4)] = 0u;
        }
    }
}

// Per-graph degree histogram dhist[voff + degree] (for the renumbering).
__global__ void k_dhist(GSet gs, const int *__restrict__ deg, int *dhist) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < gs.NV;
         v += (long long)gridDim.x * blockDim.x)
        atomicAdd(&dhist[gs.meta(gs.graph_of((int)v)).voff + deg[v]], 1);
}

// Block per graph: start[voff + d] = vertices of the graph with degree above d.
__global__ void k_desc_starts(GSet gs, const int *__restrict__ dhist, int *start) {
    __shared__ int warp_sum[32];
    const GMeta mt = gs.meta(blockIdx.x);
    const int n = mt.n;
    const int *h = dhist + mt.voff;
    int *st = start + mt.voff;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    // position i of the scan is degree n - 1 - i
    const int b = min(n, t * chunk), e = min(n, b + chunk);
    int s = 0;
    for (int i = b; i < e; i++) s += h[n - 1 - i];
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
        st[n - 1 - i] = run;
        run += h[n - 1 - i];
    }
}

// label[v] = voff + the next free position of v's degree class in its graph
// (ties in any order).
__global__ void k_desc_scatter(GSet gs, const int *__restrict__ deg, int *start, int *label) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < gs.NV;
         v += (long long)gridDim.x * blockDim.x) {
        const int voff = gs.meta(gs.graph_of((int)v)).voff;
        label[v] = voff + atomicAdd(&start[voff + deg[v]], 1);
    }
}

// Exclusive scan of the degrees into nptr, with the largest degree and the
// reset of the work counters.  Small sets: one block.
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
        info->scanned = 0;
    }
}

// Large sets, three passes over tiles of kScanTile degrees: tile sums (and
// the largest degree), a one-block scan of the tile sums, then each tile's
// own scan plus its offset.  The caller zeroes info->maxdeg first.
constexpr int kScanTile = 4096;

__global__ void k_scan_tiles(const int *__restrict__ deg, int n, long long *tile_sum, GraphInfo *info) {
    __shared__ long long ws[32];
    __shared__ int wm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kScanTile;
    long long s = 0;
    int mx = 0;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        const long long j = base + i;
        if (j < n) {
            s += deg[j];
            mx = max(mx, deg[j]);
        }
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        s += __shfl_xor_sync(kFull, s, d);
        mx = max(mx, __shfl_xor_sync(kFull, mx, d));
    }
    if (lane == 0) {
        ws[wid] = s;
        wm[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        int m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            t += ws[w];
            m = max(m, wm[w]);
        }
        tile_sum[blockIdx.x] = t;
        atomicMax(&info->maxdeg, m);
    }
}

__global__ void k_scan_top(long long *tile_sum, int ntiles, long long *nptr, int n, GraphInfo *info) {
    __shared__ long long warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int chunk = (ntiles + blockDim.x - 1) / blockDim.x;
    const int b = min(ntiles, t * chunk), e = min(ntiles, b + chunk);
    long long s = 0;
    for (int i = b; i < e; i++) s += tile_sum[i];
    long long incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        long long w0 = lane < nw ? warp_sum[lane] : 0;
        long long wi = w0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < nw) warp_sum[lane] = wi - w0;
        if (lane == nw - 1) {
            info->nnz = wi;
            nptr[n] = wi;
        }
    }
    __syncthreads();
    long long run = warp_sum[wid] + (incl - s);
    for (int i = b; i < e; i++) {
        const long long v = tile_sum[i];
        tile_sum[i] = run;
        run += v;
    }
    if (t == 0) {
        info->queue_tail = 0;
        info->queue_head = 0;
        info->unit_ctr = 0;
        info->chunks_pushed = 0;
        info->scanned = 0;
    }
}

__global__ void k_scan_apply(const int *__restrict__ deg, int n, const long long *__restrict__ tile_off,
                             long long *nptr) {
    __shared__ long long warp_sum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int per = kScanTile / 1024;  // elements per thread (blockDim 1024)
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * per;
    int vals[per];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < per; i++) {
        vals[i] = base + i < n ? deg[base + i] : 0;
        s += vals[i];
    }
    long long incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w0 = warp_sum[lane];
        long long wi = w0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
        warp_sum[lane] = wi - w0;
    }
    __syncthreads();
    long long run = tile_off[blockIdx.x] + warp_sum[wid] + (incl - s);
#pragma unroll
    for (int i = 0; i < per; i++) {
        if (base + i < n) nptr[base + i] = run;
        run += vals[i];
    }
}

// Warp per global row: write the sorted neighbour entries (u << 2) | state(v, u)
// with local u.  Each lane reads 16 bytes (64 columns) per step; steps where
// the whole warp's 2048 columns are empty are skipped after one ballot.
__global__ void k_fill(GSet gs, const uint32_t *__restrict__ state, const long long *__restrict__ nptr,
                       uint32_t *nbr) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < gs.NV; v += nwarps) {
        const GMeta mt = gs.meta(gs.graph_of((int)v));
        const int lv = (int)v - mt.voff;
        const int quads = (((mt.n + 15) >> 4) + 3) >> 2;  // within the pitch (a multiple of 4 words)
        const uint4 *row4 = reinterpret_cast<const uint4 *>(state + mt.soff + (long long)lv * mt.pitch);
        long long base = nptr[v];
        for (int q0 = 0; q0 < quads; q0 += kWarp) {
            const int q = q0 + lane;
            const uint4 x4 = q < quads ? row4[q] : make_uint4(0, 0, 0, 0);
            const uint32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
            uint32_t nz[4];
            int c = 0;
#pragma unroll
            for (int t = 0; t < 4; t++) {
                nz[t] = (xs[t] | (xs[t] >> 1)) & 0x55555555u;
                c += __popc(nz[t]);
            }
            if (!__ballot_sync(kFull, c != 0)) continue;
            int total;
            const int off = warp_excl_scan(c, lane, &total);
            long long pos = base + off;
#pragma unroll
            for (int t = 0; t < 4; t++) {
                uint32_t m = nz[t];
                while (m) {
                    const int bit = __ffs(m) - 1;
                    const uint32_t u = (uint32_t)((q * 4 + t) * 16 + (bit >> 1));
                    nbr[pos++] = (u << 2) | ((xs[t] >> bit) & 3u);
                    m &= m - 1;
                }
            }
            base += total;
        }
    }
}

// gid[v] = graph of global vertex v (block per graph).
__global__ void k_graph_ids(GSet gs, int *gid) {
    const GMeta mt = gs.meta(blockIdx.x);
    for (int i = threadIdx.x; i < mt.n; i += blockDim.x) gid[mt.voff + i] = blockIdx.x;
}

__global__ void k_reset_maxdeg(GraphInfo *info) { info->maxdeg = 0; }

int grid_for(long long work_items, int per_block, int num_sms) {
    long long b = (work_items + per_block - 1) / per_block;
    long long cap = (long long)num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int launch_zero(void *p, size_t bytes, int num_sms, cudaStream_t s, int *status, unsigned long long *counts,
                long long ncounts, int *ints, long long nints) {
    IntRanges r = {{ints, nullptr, nullptr}, {ints ? nints : 0, 0, 0}};
    const size_t n16 = bytes / 16, ntail = bytes % 16;
    const int grid = grid_for((long long)(n16 > 0 ? n16 : 1), 256 * 4, num_sms);
    k_zero<<<grid, 256, 0, s>>>(reinterpret_cast<uint4 *>(p), n16,
                                reinterpret_cast<unsigned char *>(p) + n16 * 16, ntail, status, counts, ncounts, r);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

int launch_graph_ids(const GSet &gs, int *gid, cudaStream_t s) {
    if (gs.B <= 1) return 0;
    k_graph_ids<<<gs.B, 256, 0, s>>>(gs, gid);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

long long scan_tiles_needed(long long NV) { return NV <= kScanSingleMax ? 0 : (NV + kScanTile - 1) / kScanTile; }

int launch_build_graph(const GSet &gs, long long state_words, uint32_t *state, bool state_clean, int *deg, int *lo,
                       int *deg_in, long long *nptr, long long *tile_scratch, uint32_t *nbr, int *label,
                       GraphInfo *info, int *status, unsigned long long *counts, long long ncounts, bool relabel,
                       int num_sms, cudaStream_t s) {
    int launches = 0;
    const long long NV = gs.NV;
    const int rows_grid = grid_for(NV * kWarp, 256, num_sms);
    // zero the counts, the status word, the degree counters and, unless the
    // previous call left it clean, the pair-state buffer
    {
        const size_t bytes = state_clean ? 0 : (size_t)state_words * 4;
        IntRanges r = {{deg, lo, deg_in}, {NV, NV, relabel ? NV : 0}};
        const size_t n16 = bytes / 16, ntail = bytes % 16;
        const long long items = (long long)max((size_t)1, max(n16, (size_t)max(NV, ncounts)));
        k_zero<<<grid_for(items, 256 * 4, num_sms), 256, 0, s>>>(reinterpret_cast<uint4 *>(state), n16,
                                                                 reinterpret_cast<unsigned char *>(state) + n16 * 16,
                                                                 ntail, status, counts, ncounts, r);
        launches++;
    }
    if (relabel) {
        // G* degrees under the input labels; each graph's vertices renumbered
        // by descending degree; the arcs' words cleared and the block rebuilt
        int *dhist = lo;  // zeroed above, cleared again by k_clear_arcs
        int *start = reinterpret_cast<int *>(nptr);
        k_ingest<<<rows_grid, 256, 0, s>>>(gs, state, nullptr, status, deg_in, nullptr);
        k_dhist<<<grid_for(NV, 256, num_sms), 256, 0, s>>>(gs, deg_in, dhist);
        k_desc_starts<<<gs.B, 1024, 0, s>>>(gs, dhist, start);
        k_desc_scatter<<<grid_for(NV, 256, num_sms), 256, 0, s>>>(gs, deg_in, start, label);
        k_clear_arcs<<<rows_grid, 256, 0, s>>>(gs, state, nullptr, deg, lo);
        k_ingest<<<rows_grid, 256, 0, s>>>(gs, state, label, nullptr, deg, lo);
        launches += 6;
    } else {
        k_ingest<<<rows_grid, 256, 0, s>>>(gs, state, nullptr, status, deg, lo);
        launches++;
    }
    if (NV <= kScanSingleMax) {
        k_scan_degrees<<<1, 1024, 0, s>>>(deg, (int)NV, nptr, info);
        launches++;
    } else {
        const int ntiles = (int)scan_tiles_needed(NV);
        k_reset_maxdeg<<<1, 1, 0, s>>>(info);
        k_scan_tiles<<<ntiles, 1024, 0, s>>>(deg, (int)NV, tile_scratch, info);
        k_scan_top<<<1, 1024, 0, s>>>(tile_scratch, ntiles, nptr, (int)NV, info);
        k_scan_apply<<<ntiles, 1024, 0, s>>>(deg, (int)NV, tile_scratch, nptr);
        launches += 4;
    }
    k_fill<<<rows_grid, 256, 0, s>>>(gs, state, nptr, nbr);
    launches++;
    return cudaGetLastError() == cudaSuccess ? launches : ACC_ERR_CUDA;
}

int launch_clear_graph(const GSet &gs, uint32_t *state, const int *label, bool relabel, int num_sms, cudaStream_t s) {
    if (gs.NV == 0) return 0;
    k_clear_arcs<<<grid_for(gs.NV * kWarp, 256, num_sms), 256, 0, s>>>(gs, state, relabel ? label : nullptr, nullptr,
                                                                       nullptr);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

}  // namespace acc
