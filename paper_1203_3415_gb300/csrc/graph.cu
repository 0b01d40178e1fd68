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
// words its arcs touch, marking their 128-byte chunks in a per-row
// occupancy bitmap, and the call ends by zeroing the marked chunks
// (k_clear_chunks; it reads neither the input nor the labels), so no pass
// ever sweeps the whole n x n block.  G* degrees
// come out of the ingest itself: of the atomics that touch the field of pair
// {a, u} in row a (arc a -> u sets bit 0, arc u -> a sets bit 1 as its
// mirror), exactly one finds the field still zero, and that one counts u as
// a neighbour of a.  Repeated arcs therefore count once.
//
// The degree-descending renumbering only needs high-degree vertices first
// (the counts do not depend on the numbering), so it orders by out- plus
// in-degree taken straight from the CSR, before any pair state exists.
//
// Arc kernels run a thread per arc of the whole set: the arc's graph and row
// are found by binary search (arc offsets of the graphs, then the graph's
// rowptr), so a hub row costs no more than any other and ingest and clear
// attribute every arc identically, malformed rows included (those are
// reported by the ingest's row check).
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
    int *p[4];
    long long n[4];
};

__global__ void k_zero(uint4 *p, size_t n16, unsigned char *tail, size_t ntail, int *status,
                       unsigned long long *counts, long long ncounts, IntRanges ints) {
    grid_dep_wait();
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j = i; j < n16; j += stride) p[j] = make_uint4(0, 0, 0, 0);
    if (i < ntail) tail[i] = 0;
    for (size_t j = i; j < (size_t)ncounts; j += stride) counts[j] = 0;
#pragma unroll
    for (int r = 0; r < 4; r++)
        for (size_t j = i; j < (size_t)ints.n[r]; j += stride) ints.p[r][j] = 0;
    if (i == 0 && status) *status = 0;
}

// Graph of arc p of the set: the last graph whose first arc is at most p.
__device__ __forceinline__ int graph_of_arc(const GSet &gs, long long p) {
    if (gs.B == 1) return 0;
    int lo = 0, hi = gs.B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gs.many[mid].moff <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Row of local arc position p: the last row whose rowptr is at most p, or
// -1 when there is none (rowptr[0] > p, or no rows: a malformed graph).
__device__ __forceinline__ int row_of_arc(const GMeta &mt, long long p) {
    if (mt.n <= 0 || mt.rowptr[0] > p) return -1;
    int lo = 0, hi = mt.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mt.rowptr[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// f(v, mt, lv, p) for every arc p of the set, thread per arc (grid-stride).
template <typename F>
__device__ __forceinline__ void for_each_arc(const GSet &gs, F f) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < gs.M; q += stride) {
        const GMeta mt = gs.meta(graph_of_arc(gs, q));
        const long long p = q - mt.moff;
        const int lv = row_of_arc(mt, p);
        if (lv >= 0) f(mt.voff + lv, mt, lv, p);
    }
}

// Out- plus in-degree of every vertex from the CSR alone (repeated arcs and
// both arcs of a mutual pair counted), the key of the renumbering.  Arcs
// with a bad target are skipped here (k_ingest reports them).
__global__ void k_arc_degrees(GSet gs, int *deg_io) {
    grid_dep_wait();
    for_each_arc(gs, [&](int v, const GMeta &mt, int lv, long long p) {
        const int u0 = mt.col[p];
        if (u0 < 0 || u0 >= mt.n || u0 == lv) return;
        atomicAdd(&deg_io[v], 1);
        atomicAdd(&deg_io[mt.voff + u0], 1);
    });
}

// Set the pair-state bits of every arc, validating the CSR on the way:
// malformed rows (rowptr decreasing or outside [0, m], rowptr[0] != 0,
// rowptr[n] != m), targets out of range and self-loops are reported through
// *status; nothing is read out of range.  With `label` non-null, vertex x is
// written as label[x] (the renumbered block).  deg[voff + a] counts the G*
// neighbours of block vertex a; lo (if non-null) those below a.  The atomic
// that finds a state word empty marks the word's 32-word chunk in its row's
// occupancy bitmap.
// Row checks of the input CSRs (grid-stride): rowptr non-decreasing within
// [0, m], rowptr[0] = 0, rowptr[n] = m; no arcs in a graph without vertices.
__device__ __forceinline__ void validate_rows(const GSet &gs, int *status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < gs.NV; v += stride) {
        const GMeta mt = gs.meta(gs.graph_of((int)v));
        const int lv = (int)v - mt.voff;
        const long long b = mt.rowptr[lv], e = mt.rowptr[lv + 1];
        if (b < 0 || e < b || e > mt.m || (lv == 0 && b != 0) || (lv == mt.n - 1 && e != mt.m))
            set_status(status, ACC_ERR_INPUT);
    }
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < gs.B; g += stride) {
        const GMeta mt = gs.meta((int)g);  // arcs of a graph without vertices
        if (mt.n == 0 && mt.m != 0) set_status(status, ACC_ERR_INPUT);
    }
}

__global__ void k_ingest(GSet gs, uint32_t *state, const int *__restrict__ label, int *status, int *deg, int *lo,
                         uint32_t *occ, int occ_w) {
    grid_dep_wait();
    validate_rows(gs, status);
    for_each_arc(gs, [&](int v, const GMeta &mt, int lv, long long p) {
        const int u0 = mt.col[p];
        if (u0 < 0 || u0 >= mt.n || u0 == lv) {
            set_status(status, ACC_ERR_INPUT);
            return;
        }
        const long long a = label ? label[v] - mt.voff : lv;
        const int u = label ? label[mt.voff + u0] - mt.voff : u0;
        uint32_t *blk = state + mt.soff;
        const int su = (u & 15) * 2, sa = (int)(a & 15) * 2;
        const uint32_t oa = atomicOr(&blk[a * mt.pitch + (u >> 4)], 1u << su);
        const uint32_t ou = atomicOr(&blk[(long long)u * mt.pitch + (a >> 4)], 2u << sa);
        if (oa == 0u) atomicOr(&occ[(mt.voff + a) * occ_w + (u >> 14)], 1u << ((u >> 9) & 31));
        if (ou == 0u) atomicOr(&occ[((long long)mt.voff + u) * occ_w + (a >> 14)], 1u << ((a >> 9) & 31));
        if (((oa >> su) & 3u) == 0u) {
            atomicAdd(&deg[mt.voff + a], 1);
            if (lo && u < a) atomicAdd(&lo[mt.voff + a], 1);
        }
        if (((ou >> sa) & 3u) == 0u) {
            atomicAdd(&deg[mt.voff + u], 1);
            if (lo && a < u) atomicAdd(&lo[mt.voff + u], 1);
        }
    });
}

// Warp per global row: zero the 32-word chunks of the row that the occupancy
// bitmap marks (every word the ingest set lies in one), lane j taking the
// j-th marked chunk of a bitmap word.  The buffer is all zero afterwards.
__global__ void k_clear_chunks(GSet gs, uint32_t *state, const uint32_t *__restrict__ occ, int occ_w) {
    grid_dep_wait();
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < gs.NV; v += nwarps) {
        const GMeta mt = gs.meta(gs.graph_of((int)v));
        const int quads = (((mt.n + 15) >> 4) + 3) >> 2;
        uint4 *row4 = reinterpret_cast<uint4 *>(state + mt.soff + (long long)(v - mt.voff) * mt.pitch);
        for (int mw = 0; mw < occ_w; mw++) {
            const uint32_t mask = occ[v * occ_w + mw];
            if (lane < __popc(mask)) {
                const int q0 = (mw * 32 + (int)__fns(mask, 0, lane + 1)) * 8;
#pragma unroll
                for (int g = 0; g < 8; g++)
                    if (q0 + g < quads) row4[q0 + g] = make_uint4(0, 0, 0, 0);
            }
        }
    }
}

// Per-graph histogram dhist[voff + key] of the renumbering keys (clamped to
// n - 1: the out- plus in-degree can exceed it).
__global__ void k_dhist(GSet gs, const int *__restrict__ key, int *dhist) {
    grid_dep_wait();
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < gs.NV;
         v += (long long)gridDim.x * blockDim.x) {
        const GMeta mt = gs.meta(gs.graph_of((int)v));
        atomicAdd(&dhist[mt.voff + min(key[v], mt.n - 1)], 1);
    }
}

// Block per graph: start[voff + d] = vertices of the graph with degree above d.
__global__ void __launch_bounds__(1024) k_desc_starts(GSet gs, const int *__restrict__ dhist, int *start) {
    grid_dep_wait();
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

// label[v] = voff + the next free position of v's key class in its graph
// (ties in any order); also zeroes dhist (dead once the starts exist).
__global__ void k_desc_scatter(GSet gs, const int *__restrict__ key, int *start, int *label, int *dhist) {
    grid_dep_wait();
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < gs.NV;
         v += (long long)gridDim.x * blockDim.x) {
        const GMeta mt = gs.meta(gs.graph_of((int)v));
        label[v] = mt.voff + atomicAdd(&start[mt.voff + min(key[v], mt.n - 1)], 1);
        dhist[v] = 0;
    }
}

// Exclusive scan of the degrees into nptr, with the largest degree and the
// reset of the work counters.  Small sets: one block, the degrees staged in
// shared memory by coalesced loads (n ints of dynamic shared memory).
__global__ void __launch_bounds__(1024) k_scan_degrees(const int *__restrict__ deg_g, int n, long long *nptr, GraphInfo *info,
                                                       int k, int max_n, int *status) {
    grid_dep_wait();
    extern __shared__ int deg[];
    __shared__ long long warp_sum[32];
    __shared__ int warp_max[32];
    __shared__ float warp_bound[32][3];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    {
        constexpr int kPer = (int)(kScanSingleMax / 1024);  // n <= kPer * blockDim.x
        int dv[kPer];
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const int i = t + j * (int)blockDim.x;
            dv[j] = i < n ? deg_g[i] : 0;
        }
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const int i = t + j * (int)blockDim.x;
            if (i < n) deg[i] = dv[j];
        }
    }
    __syncthreads();
    const int nthreads = blockDim.x;
    const int chunk = (n + nthreads - 1) / nthreads;
    const int b = min(n, t * chunk), e = min(n, b + chunk);
    long long s = 0;
    int mx = 0;
    float bs[3] = {0.0f, 0.0f, 0.0f};
    for (int i = b; i < e; i++) {
        s += deg[i];
        mx = max(mx, deg[i]);
        if (k) count_bound_terms(k, deg[i], bs);
    }
    long long incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, d));
    if (k) {
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int d = 16; d; d >>= 1) bs[j] += __shfl_xor_sync(kFull, bs[j], d);
        if (lane == 0)
            for (int j = 0; j < 3; j++) warp_bound[wid][j] = bs[j];
    }
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
    // offsets back into shared memory (below 2^32: they count 2 |E*| < 2^32
    // entries), then written out coalesced
    unsigned run = (unsigned)(warp_sum[wid] + (incl - s));
    for (int i = b; i < e; i++) {
        const int d = deg[i];
        deg[i] = (int)run;
        run += (unsigned)d;
    }
    __syncthreads();
    for (int i = t; i < n; i += blockDim.x) nptr[i] = (long long)(unsigned)deg[i];
    if (t == 0) {
        if (k) {
            float tb[3] = {0.0f, 0.0f, 0.0f};
            for (int w = 0; w < (int)(blockDim.x >> 5); w++)
                for (int j = 0; j < 3; j++) tb[j] += warp_bound[w][j];
            if (count_bound(k, max_n, warp_max[0], tb) > kCountLimit) set_status(status, ACC_ERR_OVERFLOW);
        }
        info->maxdeg = warp_max[0];
        info->big_rows = 0;
        info->big_head = 0;
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

__global__ void __launch_bounds__(1024) k_scan_tiles(const int *__restrict__ deg, int n, long long *tile_sum, GraphInfo *info,
                                                     int k) {
    grid_dep_wait();
    __shared__ long long ws[32];
    __shared__ int wm[32];
    __shared__ float wb[32][3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kScanTile;
    long long s = 0;
    int mx = 0;
    float bs[3] = {0.0f, 0.0f, 0.0f};
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        const long long j = base + i;
        if (j < n) {
            s += deg[j];
            mx = max(mx, deg[j]);
            if (k) count_bound_terms(k, deg[j], bs);
        }
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        s += __shfl_xor_sync(kFull, s, d);
        mx = max(mx, __shfl_xor_sync(kFull, mx, d));
#pragma unroll
        for (int j = 0; j < 3; j++) bs[j] += __shfl_xor_sync(kFull, bs[j], d);
    }
    if (lane == 0) {
        ws[wid] = s;
        wm[wid] = mx;
        for (int j = 0; j < 3; j++) wb[wid][j] = bs[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        int m = 0;
        float tb[3] = {0.0f, 0.0f, 0.0f};
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            t += ws[w];
            m = max(m, wm[w]);
            for (int j = 0; j < 3; j++) tb[j] += wb[w][j];
        }
        tile_sum[blockIdx.x] = t;
        atomicMax(&info->maxdeg, m);
        if (k)
            for (int j = 0; j < 3; j++) atomicAdd(&info->bound[j], tb[j]);
    }
}

__global__ void __launch_bounds__(1024) k_scan_top(long long *tile_sum, int ntiles, long long *nptr, int n, GraphInfo *info,
                                                   int k, int max_n, int *status) {
    grid_dep_wait();
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
        if (k && count_bound(k, max_n, info->maxdeg, info->bound) > kCountLimit) set_status(status, ACC_ERR_OVERFLOW);
        info->big_rows = 0;
        info->big_head = 0;
        info->queue_tail = 0;
        info->queue_head = 0;
        info->unit_ctr = 0;
        info->chunks_pushed = 0;
        info->scanned = 0;
    }
}

__global__ void __launch_bounds__(1024) k_scan_apply(const int *__restrict__ deg, int n, const long long *__restrict__ tile_off,
                             long long *nptr) {
    grid_dep_wait();
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

// Warp per rw consecutive global rows (a power of two up to 32): write the
// sorted neighbour entries (u << 2) | state(v, u) with local u, reading only
// the 32-word chunks the occupancy bitmap marks.  The rows' marked chunks are
// numbered row by row
// and spread over the lanes (a lane per chunk, 128 bytes each); a chunk's
// entries go to its row's offset plus the entries of the row's earlier
// chunks (a scan over the lanes, segmented by row and carried from one round
// to the next), so rows with few neighbours share a warp.
//
// With src non-NULL, each entry's position also records its row: src[pos] =
// global row vertex, bit 31 set when the neighbour is below the row's vertex
// (the enumeration's phase 1 reads a work unit's vertex from it).
__global__ void k_fill(GSet gs, const uint32_t *__restrict__ state, const uint32_t *__restrict__ occ, int occ_w,
                       const long long *__restrict__ nptr, uint32_t *nbr, uint32_t *src, int rw) {
    grid_dep_wait();
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r0 = warp * rw; r0 < gs.NV; r0 += nwarps * rw) {
        const long long v = r0 + lane;
        int nch = 0, quads = 0, vloc = 0;
        long long row_word = 0, rbase = 0;
        if (lane < rw && v < gs.NV) {
            for (int w = 0; w < occ_w; w++) nch += __popc(occ[v * occ_w + w]);
            const GMeta mt = gs.meta(gs.graph_of((int)v));
            vloc = (int)v - mt.voff;
            row_word = mt.soff + (long long)vloc * mt.pitch;
            quads = (((mt.n + 15) >> 4) + 3) >> 2;  // 16-byte groups within the pitch
            rbase = nptr[v];
        }
        int total;
        const int pre = warp_excl_scan(nch, lane, &total);
        int carry_row = -1, carry = 0;  // the row the last round ended in, and its entries so far
        for (int i0 = 0; i0 < total; i0 += kWarp) {
            const int idx = i0 + lane;
            const bool act = idx < total;
            // owner: the last lane whose chunks start at or before idx
            int owner = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const int cand = owner + step;
                const int pc = __shfl_sync(kFull, pre, cand & 31);
                if (cand < kWarp && pc <= idx) owner = cand;
            }
            const int o_pre = __shfl_sync(kFull, pre, owner);
            const long long o_word = __shfl_sync(kFull, row_word, owner);
            const long long o_base = __shfl_sync(kFull, rbase, owner);
            const int o_quads = __shfl_sync(kFull, quads, owner);
            const int o_vloc = __shfl_sync(kFull, vloc, owner);
            uint32_t xs[32];
            int cnt = 0, q0 = 0;
            if (act) {
                // the (idx - o_pre)-th marked chunk of the owner's row
                const long long vo = r0 + owner;
                int j = idx - o_pre;
                for (int w = 0; w < occ_w; w++) {
                    const uint32_t mk = occ[vo * occ_w + w];
                    const int pc = __popc(mk);
                    if (j < pc) {
                        q0 = (w * 32 + (int)__fns(mk, 0, j + 1)) * 8;  // first 16-byte group of the chunk
                        break;
                    }
                    j -= pc;
                }
                const uint4 *row4 = reinterpret_cast<const uint4 *>(state + o_word);
#pragma unroll
                for (int g = 0; g < 8; g++) {
                    const uint4 x4 = q0 + g < o_quads ? row4[q0 + g] : make_uint4(0, 0, 0, 0);
                    xs[4 * g] = x4.x;
                    xs[4 * g + 1] = x4.y;
                    xs[4 * g + 2] = x4.z;
                    xs[4 * g + 3] = x4.w;
                }
#pragma unroll
                for (int t = 0; t < 32; t++) cnt += __popc((xs[t] | (xs[t] >> 1)) & 0x55555555u);
            }
            int round_total;
            const int ex = warp_excl_scan(cnt, lane, &round_total);
            // chunks of a row sit on consecutive lanes: the row's first lane here
            const unsigned same = __match_any_sync(kFull, act ? owner : -1 - lane);
            const int first = __ffs(same) - 1;
            const int ex_first = __shfl_sync(kFull, ex, first);
            if (act) {
                long long pos = o_base + (ex - ex_first) + (owner == carry_row ? carry : 0);
#pragma unroll
                for (int t = 0; t < 32; t++) {
                    uint32_t nz = (xs[t] | (xs[t] >> 1)) & 0x55555555u;
                    while (nz) {
                        const int bit = __ffs(nz) - 1;
                        const int col = (q0 * 4 + t) * 16 + (bit >> 1);
                        nbr[pos] = ((uint32_t)col << 2) | ((xs[t] >> bit) & 3u);
                        if (src) src[pos] = (uint32_t)(r0 + owner) | (col < o_vloc ? 0x80000000u : 0u);
                        pos++;
                        nz &= nz - 1;
                    }
                }
            }
            // the round's last row may go on in the next round
            const int last = min(total - i0, kWarp) - 1;
            const int last_owner = __shfl_sync(kFull, owner, last);
            const int last_first = __shfl_sync(kFull, first, last);
            const int in_round = __shfl_sync(kFull, ex + cnt, last) - __shfl_sync(kFull, ex, last_first);
            carry = (last_owner == carry_row ? carry : 0) + in_round;
            carry_row = last_owner;
        }
    }
}

// ---------------------------------------------------------------------------
// Sparse build: the same G* neighbour lists without the dense pair-state
// block (for graphs above its size limit, or on request).  Each arc puts one
// raw entry (u << 2) | state bit into each endpoint's row (bit 0 at the
// tail's row: arc a -> u; bit 1 at the head's row); each row is then sorted
// and the entries of one neighbour merged (their state bits OR'd, so repeated
// arcs count once and a mutual pair becomes state 3), and the merged rows are
// compacted into the lists.
// ---------------------------------------------------------------------------

constexpr int kSortSmall = 2048;  // raw entries of a row one warp sorts in shared memory
constexpr int kSortWarps = 4;     // warps per block of the small-row sort

// Raw entries per row (cnt[v], both directions of each arc), after the row
// checks of the input; arcs with a bad target or self-loops are reported
// and not counted.
__global__ void k_sp_count(GSet gs, const int *__restrict__ label, int *status, int *cnt) {
    grid_dep_wait();
    validate_rows(gs, status);
    for_each_arc(gs, [&](int v, const GMeta &mt, int lv, long long p) {
        const int u0 = mt.col[p];
        if (u0 < 0 || u0 >= mt.n || u0 == lv) {
            set_status(status, ACC_ERR_INPUT);
            return;
        }
        const int a = label ? label[v] - mt.voff : lv;
        const int u = label ? label[mt.voff + u0] - mt.voff : u0;
        atomicAdd(&cnt[mt.voff + a], 1);
        atomicAdd(&cnt[mt.voff + u], 1);
    });
}

// The raw entries into their rows (row v from roff[v]; cur[v] counts the
// entries placed, in any order).
__global__ void k_sp_scatter(GSet gs, const int *__restrict__ label, const long long *__restrict__ roff, int *cur,
                             uint32_t *raw) {
    grid_dep_wait();
    for_each_arc(gs, [&](int v, const GMeta &mt, int lv, long long p) {
        const int u0 = mt.col[p];
        if (u0 < 0 || u0 >= mt.n || u0 == lv) return;
        const int a = label ? label[v] - mt.voff : lv;
        const int u = label ? label[mt.voff + u0] - mt.voff : u0;
        raw[roff[mt.voff + a] + atomicAdd(&cur[mt.voff + a], 1)] = ((uint32_t)u << 2) | 1u;
        raw[roff[mt.voff + u] + atomicAdd(&cur[mt.voff + u], 1)] = ((uint32_t)a << 2) | 2u;
    });
}

// Ascending sort of x[0..n) by compare-exchanges that always put the smaller
// value at the lower index (the bitonic network in its flipped form: each
// merge of size k first compares i with its mirror i ^ (k - 1), then i with
// i ^ j); the comparators reaching past n meet virtual maxima that never
// move, so any n works without padding.  Thread t of nt runs indexes t, t +
// nt, ...; sync() separates the stages.
template <typename Sync>
__device__ __forceinline__ void flip_sort(uint32_t *x, int n, int t, int nt, Sync sync) {
    for (int k = 2; (k >> 1) < n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = t; i < n; i += nt) {
                const int l = j == (k >> 1) ? (i ^ (k - 1)) : (i ^ j);
                if (l > i && l < n) {
                    const uint32_t a = x[i], b = x[l];
                    if (a > b) {
                        x[i] = b;
                        x[l] = a;
                    }
                }
            }
            sync();
        }
    }
}

// Warp per row of at most kSortSmall raw entries (longer rows are listed in
// big[] for k_sp_sort_big): sort in the warp's shared buffer, then OR every
// entry into merged[roff[v] + (its neighbour's rank in the row)] (merged is
// zero beforehand); deg[v], lo[v] = neighbours of v, those below v.
__global__ void __launch_bounds__(kSortWarps * kWarp) k_sp_sort_small(GSet gs, const long long *__restrict__ roff,
                                                                   const uint32_t *__restrict__ raw,
                                                                   uint32_t *merged, int *deg, int *lo, int *big,
                                                                   GraphInfo *info) {
    grid_dep_wait();
    __shared__ uint32_t buf[kSortWarps][kSortSmall];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *x = buf[wib];
    const long long nw = (long long)gridDim.x * kSortWarps;
    for (long long v = blockIdx.x * (long long)kSortWarps + wib; v < gs.NV; v += nw) {
        const long long r0 = roff[v];
        const int R = (int)(roff[v + 1] - r0);
        if (R > kSortSmall) {
            if (lane == 0) big[atomicAdd(&info->big_rows, 1u)] = (int)v;
            continue;
        }
        for (int i = lane; i < R; i += kWarp) x[i] = raw[r0 + i];
        __syncwarp();
        flip_sort(x, R, lane, kWarp, [] { __syncwarp(); });
        const uint32_t vloc = (uint32_t)((int)v - gs.meta(gs.graph_of((int)v)).voff);
        int runs = 0, below = 0;
        for (int c0 = 0; c0 < R; c0 += kWarp) {
            const int i = c0 + lane;
            const uint32_t e = i < R ? x[i] : 0u;
            const bool start = i < R && (i == 0 || (x[i - 1] >> 2) != (e >> 2));
            const unsigned ball = __ballot_sync(kFull, start);
            if (i < R) atomicOr(&merged[r0 + runs + __popc(ball & (0xFFFFFFFFu >> (31 - lane))) - 1], e);
            below += __popc(__ballot_sync(kFull, start && (e >> 2) < vloc));
            runs += __popc(ball);
        }
        if (lane == 0) {
            deg[v] = runs;
            lo[v] = below;
        }
        __syncwarp();
    }
}

// Block per listed long row (taken one at a time through info->big_head):
// the same sort in place in raw (global memory), then the same merge.
__global__ void k_sp_sort_big(GSet gs, const long long *__restrict__ roff, uint32_t *raw, uint32_t *merged, int *deg,
                              int *lo, const int *__restrict__ big, GraphInfo *info) {
    grid_dep_wait();
    __shared__ int row, warp_cnt[32], warp_below[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nwarps = blockDim.x >> 5;
    for (;;) {
        if (t == 0) {
            const unsigned i = atomicAdd(&info->big_head, 1u);
            row = i < info->big_rows ? big[i] : -1;
        }
        __syncthreads();
        const int v = row;
        if (v < 0) return;
        const long long r0 = roff[v];
        const int R = (int)(roff[v + 1] - r0);
        uint32_t *x = raw + r0;
        flip_sort(x, R, t, (int)blockDim.x, [] {
            __threadfence_block();
            __syncthreads();
        });
        const uint32_t vloc = (uint32_t)(v - gs.meta(gs.graph_of(v)).voff);
        int runs = 0, below = 0;
        for (int c0 = 0; c0 < R; c0 += (int)blockDim.x) {
            const int i = c0 + t;
            const uint32_t e = i < R ? x[i] : 0u;
            const bool start = i < R && (i == 0 || (x[i - 1] >> 2) != (e >> 2));
            const unsigned ball = __ballot_sync(kFull, start);
            const unsigned bbelow = __ballot_sync(kFull, start && (e >> 2) < vloc);
            if (lane == 0) {
                warp_cnt[wid] = __popc(ball);
                warp_below[wid] = __popc(bbelow);
            }
            __syncthreads();
            int before = 0, total = 0, tb = 0;
            for (int w = 0; w < nwarps; w++) {
                if (w < wid) before += warp_cnt[w];
                total += warp_cnt[w];
                tb += warp_below[w];
            }
            if (i < R) atomicOr(&merged[r0 + runs + before + __popc(ball & (0xFFFFFFFFu >> (31 - lane))) - 1], e);
            runs += total;
            below += tb;
            __syncthreads();
        }
        if (t == 0) {
            deg[v] = runs;
            lo[v] = below;
        }
        __syncthreads();
    }
}

// Warp per row: the merged row into the neighbour lists at nptr (the scan of
// the final degrees), and each entry's row into src (bit 31: a neighbour
// below the row's vertex).
__global__ void k_sp_compact(GSet gs, const long long *__restrict__ roff, const uint32_t *__restrict__ merged,
                             const int *__restrict__ deg, const long long *__restrict__ nptr, uint32_t *nbr,
                             uint32_t *src) {
    grid_dep_wait();
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; v < gs.NV; v += nw) {
        const long long r0 = roff[v], b = nptr[v];
        const int d = deg[v];
        const uint32_t vloc = (uint32_t)((int)v - gs.meta(gs.graph_of((int)v)).voff);
        for (int i = lane; i < d; i += kWarp) {
            const uint32_t e = merged[r0 + i];
            nbr[b + i] = e;
            src[b + i] = (uint32_t)v | ((e >> 2) < vloc ? 0x80000000u : 0u);
        }
    }
}

// Block per graph (every graph of the set has at most kRelabelSmemMax
// vertices): renumber the graph's vertices by descending key, ties in any
// order, with the key histogram and its starts in shared memory.
__global__ void __launch_bounds__(1024) k_relabel_graph(GSet gs, const int *__restrict__ key, int *label) {
    grid_dep_wait();
    extern __shared__ int h[];
    __shared__ int warp_sum[32];
    const GMeta mt = gs.meta(blockIdx.x);
    const int n = mt.n;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // this thread's keys, loaded in one batch (n <= 32 * blockDim.x)
    constexpr int kPer = kRelabelSmemMax / 1024;
    int kv[kPer];
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        const int v = t + j * (int)blockDim.x;
        kv[j] = v < n ? min(key[mt.voff + v], n - 1) : 0;
    }
    for (int i = t; i < n; i += blockDim.x) h[i] = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; j++)
        if (t + j * (int)blockDim.x < n) atomicAdd(&h[kv[j]], 1);
    __syncthreads();
    // h[d] <- vertices with key above d (position i of the scan is key n-1-i)
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    const int b = min(n, t * chunk), e = min(n, b + chunk);
    int sum = 0;
    for (int i = b; i < e; i++) sum += h[n - 1 - i];
    int incl = sum;
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
    int run = warp_sum[wid] + (incl - sum);
    for (int i = b; i < e; i++) {
        const int c = h[n - 1 - i];
        h[n - 1 - i] = run;
        run += c;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        const int v = t + j * (int)blockDim.x;
        if (v < n) label[mt.voff + v] = mt.voff + atomicAdd(&h[kv[j]], 1);
    }
}

// Thread per neighbour entry p (row vertex a = src[p], neighbour x): the
// index i of a in N*(x), found by binary search of x's sorted list (a is
// there: the lists are symmetric), stored as the part of N*(x) above a:
// its first position nptr[x] + i + 1 and its length deg(x) - i - 1.
__global__ void k_rev(GSet gs, const long long *__restrict__ nptr, const int *__restrict__ deg,
                      const uint32_t *__restrict__ nbr, const uint32_t *__restrict__ src,
                      const GraphInfo *__restrict__ info, uint2 *rev) {
    grid_dep_wait();
    const long long nnz = info->nnz;
    for (long long pos = blockIdx.x * (long long)blockDim.x + threadIdx.x; pos < nnz;
         pos += (long long)gridDim.x * blockDim.x) {
        const uint32_t a = src[pos] & 0x7FFFFFFFu;  // global
        const int voff = gs.meta(gs.graph_of((int)a)).voff;
        const uint32_t x = (uint32_t)voff + (nbr[pos] >> 2);
        const uint32_t key = (a - (uint32_t)voff) << 2;
        const long long base = nptr[x];
        const int d = deg[x];
        int lo = 0, hi = d;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (nbr[base + mid] < key) lo = mid + 1;
            else hi = mid;
        }
        rev[pos] = make_uint2((uint32_t)(base + lo + 1), (uint32_t)(d - lo - 1));
    }
}

// gid[v] = graph of global vertex v (block per graph).
__global__ void k_graph_ids(GSet gs, int *gid) {
    grid_dep_wait();
    const GMeta mt = gs.meta(blockIdx.x);
    for (int i = threadIdx.x; i < mt.n; i += blockDim.x) gid[mt.voff + i] = blockIdx.x;
}

__global__ void k_reset_maxdeg(GraphInfo *info) {
    grid_dep_wait();
    info->maxdeg = 0;
    info->bound[0] = info->bound[1] = info->bound[2] = 0.0f;
}

// True when the launch just enqueued was accepted; a refused launch's error
// is cleared, and the caller launches nothing that would read its output.
bool launch_ok() {
    if (cudaPeekAtLastError() == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}


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
    IntRanges r = {{ints, nullptr, nullptr, nullptr}, {ints ? nints : 0, 0, 0, 0}};
    const size_t n16 = bytes / 16, ntail = bytes % 16;
    const int grid = grid_for((long long)(n16 > 0 ? n16 : 1), 256 * 4, num_sms);
    launch_pdl(k_zero, grid, 256, 0, s, reinterpret_cast<uint4 *>(p), n16,
                                reinterpret_cast<unsigned char *>(p) + n16 * 16, ntail, status, counts, ncounts, r);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

int launch_graph_ids(const GSet &gs, int *gid, cudaStream_t s) {
    if (gs.B <= 1) return 0;
    launch_pdl(k_graph_ids, gs.B, 256, 0, s, gs, gid);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

long long scan_tiles_needed(long long NV) { return NV <= kScanSingleMax ? 0 : (NV + kScanTile - 1) / kScanTile; }

int launch_build_graph(const GSet &gs, const BuildBufs &bb, int max_n, int *status, unsigned long long *counts,
                       long long ncounts, bool relabel, int num_sms, cudaStream_t s) {
    static bool smem_opt_in = false;
    if (!smem_opt_in) {
        if (cudaFuncSetAttribute(k_scan_degrees, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kScanSingleMax * 4)) != cudaSuccess ||
            cudaFuncSetAttribute(k_relabel_graph, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kRelabelSmemMax * 4) != cudaSuccess)
            return ACC_ERR_CUDA;
        smem_opt_in = true;
    }
    int launches = 0;
    const long long NV = gs.NV;
    const int arcs_grid = grid_for(max(gs.M, NV), 256, num_sms);
    // zero the counts, the status word, the degree counters, the occupancy
    // bitmap and, unless the previous call left it clean, the pair-state buffer
    {
        const size_t bytes = bb.state_clean ? 0 : (size_t)bb.state_words * 4;
        const long long nocc = NV * bb.occ_w;
        IntRanges r = {{bb.deg, bb.lo, bb.deg_in, reinterpret_cast<int *>(bb.occ)},
                       {NV, NV, relabel ? NV : 0, nocc}};
        const size_t n16 = bytes / 16, ntail = bytes % 16;
        const long long items = (long long)max((size_t)1, max(n16, (size_t)max(max(NV, ncounts), nocc)));
        launch_pdl(k_zero, grid_for(items, 256 * 4, num_sms), 256, 0, s, reinterpret_cast<uint4 *>(bb.state), n16,
                                                                 reinterpret_cast<unsigned char *>(bb.state) + n16 * 16,
                                                                 ntail, status, counts, ncounts, r);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches++;
    }
    if (relabel) {
        // each graph's vertices renumbered by descending out- plus in-degree,
        // then the block built under the new ids
        launch_pdl(k_arc_degrees, arcs_grid, 256, 0, s, gs, bb.deg_in);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches++;
        if (max_n <= kRelabelSmemMax) {
            launch_pdl(k_relabel_graph, gs.B, 1024, (size_t)max_n * 4, s, gs, bb.deg_in, bb.label);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launches++;
        } else {
            int *dhist = bb.deg;  // zeroed above, zeroed again by k_desc_scatter
            int *start = reinterpret_cast<int *>(bb.nptr);
            launch_pdl(k_dhist, grid_for(NV, 256, num_sms), 256, 0, s, gs, bb.deg_in, dhist);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launch_pdl(k_desc_starts, gs.B, 1024, 0, s, gs, dhist, start);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launch_pdl(k_desc_scatter, grid_for(NV, 256, num_sms), 256, 0, s, gs, bb.deg_in, start, bb.label, dhist);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launches += 3;
        }
    }
    launch_pdl(k_ingest, arcs_grid, 256, 0, s, gs, bb.state, relabel ? bb.label : nullptr, status, bb.deg, bb.lo, bb.occ,
                                       bb.occ_w);
    if (!launch_ok()) return ACC_ERR_CUDA;
    launches++;
    if (NV <= kScanSingleMax) {
        launch_pdl(k_scan_degrees, 1, 1024, (size_t)(NV > 0 ? NV : 1) * 4, s, bb.deg, (int)NV, bb.nptr, bb.info, bb.k, max_n,
                                                                      status);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches++;
    } else {
        const int ntiles = (int)scan_tiles_needed(NV);
        launch_pdl(k_reset_maxdeg, 1, 1, 0, s, bb.info);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launch_pdl(k_scan_tiles, ntiles, 1024, 0, s, bb.deg, (int)NV, bb.tiles, bb.info, bb.k);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launch_pdl(k_scan_top, 1, 1024, 0, s, bb.tiles, ntiles, bb.nptr, (int)NV, bb.info, bb.k, max_n, status);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launch_pdl(k_scan_apply, ntiles, 1024, 0, s, bb.deg, (int)NV, bb.tiles, bb.nptr);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches += 4;
    }
    // rows per warp: enough warps to fill the GPU (64 per SM) first
    int rw = 1;
    while (rw < kWarp && (long long)rw * 2 * num_sms * 64 <= NV) rw *= 2;
    launch_pdl(k_fill, grid_for((NV + rw - 1) / rw * kWarp, 256, num_sms), 256, 0, s, gs, bb.state, bb.occ, bb.occ_w,
                                                                              bb.nptr, bb.nbr, bb.src, rw);
    launches++;
    return cudaGetLastError() == cudaSuccess ? launches : ACC_ERR_CUDA;
}

int sparse_big_rows_cap(long long arcs) { return (int)(2 * arcs / kSortSmall + 2); }

int launch_build_graph_sparse(const GSet &gs, const BuildBufs &bb, const SparseBufs &sb, int max_n, int *status,
                              unsigned long long *counts, long long ncounts, bool relabel, int num_sms,
                              cudaStream_t s) {
    static bool smem_opt_in = false;
    if (!smem_opt_in) {
        if (cudaFuncSetAttribute(k_scan_degrees, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kScanSingleMax * 4)) != cudaSuccess ||
            cudaFuncSetAttribute(k_relabel_graph, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kRelabelSmemMax * 4) != cudaSuccess)
            return ACC_ERR_CUDA;
        smem_opt_in = true;
    }
    int launches = 0;
    const long long NV = gs.NV;
    const int arcs_grid = grid_for(max(gs.M, NV), 256, num_sms);
    int *cnt = bb.lo, *cur = bb.deg;  // raw entries per row, then the final neighbours below each vertex
    {
        IntRanges r = {{bb.deg, bb.lo, bb.deg_in, nullptr}, {NV, NV, relabel ? NV : 0, 0}};
        const long long items = max(NV, ncounts) > 0 ? max(NV, ncounts) : 1;
        launch_pdl(k_zero, grid_for(items, 256 * 4, num_sms), 256, 0, s, nullptr, 0, nullptr, 0, status, counts, ncounts, r);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches++;
    }
    if (relabel) {
        launch_pdl(k_arc_degrees, arcs_grid, 256, 0, s, gs, bb.deg_in);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launches++;
        if (max_n <= kRelabelSmemMax) {
            launch_pdl(k_relabel_graph, gs.B, 1024, (size_t)max_n * 4, s, gs, bb.deg_in, bb.label);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launches++;
        } else {
            int *dhist = bb.deg;  // zeroed above, zeroed again by k_desc_scatter
            int *start = reinterpret_cast<int *>(bb.nptr);
            launch_pdl(k_dhist, grid_for(NV, 256, num_sms), 256, 0, s, gs, bb.deg_in, dhist);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launch_pdl(k_desc_starts, gs.B, 1024, 0, s, gs, dhist, start);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launch_pdl(k_desc_scatter, grid_for(NV, 256, num_sms), 256, 0, s, gs, bb.deg_in, start, bb.label, dhist);
            if (!launch_ok()) return ACC_ERR_CUDA;
            launches += 3;
        }
    }
    launch_pdl(k_sp_count, arcs_grid, 256, 0, s, gs, relabel ? bb.label : nullptr, status, cnt);
    if (!launch_ok()) return ACC_ERR_CUDA;
    launches++;
    // degree scans: the raw counts into the row offsets (no count bound), and
    // after the sort the final degrees into nptr (with it)
    auto scan = [&](const int *d, long long *out, int k) -> int {
        if (NV <= kScanSingleMax) {
            launch_pdl(k_scan_degrees, 1, 1024, (size_t)(NV > 0 ? NV : 1) * 4, s, d, (int)NV, out, bb.info, k, max_n, status);
            return launch_ok() ? 1 : ACC_ERR_CUDA;
        }
        const int ntiles = (int)scan_tiles_needed(NV);
        launch_pdl(k_reset_maxdeg, 1, 1, 0, s, bb.info);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launch_pdl(k_scan_tiles, ntiles, 1024, 0, s, d, (int)NV, bb.tiles, bb.info, k);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launch_pdl(k_scan_top, 1, 1024, 0, s, bb.tiles, ntiles, out, (int)NV, bb.info, k, max_n, status);
        if (!launch_ok()) return ACC_ERR_CUDA;
        launch_pdl(k_scan_apply, ntiles, 1024, 0, s, d, (int)NV, bb.tiles, out);
        return launch_ok() ? 4 : ACC_ERR_CUDA;
    };
    int rc = scan(cnt, sb.roff, 0);
    if (rc < 0) return rc;
    launches += rc;
    launch_pdl(k_sp_scatter, arcs_grid, 256, 0, s, gs, relabel ? bb.label : nullptr, sb.roff, cur, sb.raw);
    if (!launch_ok()) return ACC_ERR_CUDA;
    launches++;
    if (gs.M > 0 && cudaMemsetAsync(sb.merged, 0, (size_t)(2 * gs.M) * sizeof(uint32_t), s) != cudaSuccess)
        return ACC_ERR_CUDA;
    launch_pdl(k_sp_sort_small, grid_for((NV + kSortWarps - 1) / kSortWarps, 1, num_sms), kSortWarps * kWarp, 0, s, 
        gs, sb.roff, sb.raw, sb.merged, bb.deg, bb.lo, sb.big, bb.info);
    if (!launch_ok()) return ACC_ERR_CUDA;
    launch_pdl(k_sp_sort_big, num_sms, 256, 0, s, gs, sb.roff, sb.raw, sb.merged, bb.deg, bb.lo, sb.big, bb.info);
    if (!launch_ok()) return ACC_ERR_CUDA;
    launches += 2;
    if ((rc = scan(bb.deg, bb.nptr, bb.k)) < 0) return rc;
    launches += rc;
    launch_pdl(k_sp_compact, grid_for(NV * kWarp, 256, num_sms), 256, 0, s, gs, sb.roff, sb.merged, bb.deg, bb.nptr, bb.nbr,
                                                                   bb.src);
    if (!launch_ok()) return ACC_ERR_CUDA;
    launches++;
    return launches;
}

int launch_rev_build(const GSet &gs, const long long *nptr, const int *deg, const uint32_t *nbr, const uint32_t *src,
                     const GraphInfo *info, long long max_entries, uint2 *rev, int num_sms, cudaStream_t s) {
    if (max_entries <= 0) return 0;
    launch_pdl(k_rev, grid_for(max_entries, 256, num_sms), 256, 0, s, gs, nptr, deg, nbr, src, info, rev);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

int launch_clear_graph(const GSet &gs, uint32_t *state, const uint32_t *occ, int occ_w, int num_sms, cudaStream_t s) {
    if (gs.NV == 0) return 0;
    launch_pdl(k_clear_chunks, grid_for(gs.NV * kWarp, 256, num_sms), 256, 0, s, gs, state, occ, occ_w);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

}  // namespace acc
