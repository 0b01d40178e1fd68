// Internal declarations shared by the library's CUDA translation units.
//
// Data layout on the device for one graph (all owned by the context's
// workspace):
//   state   uint32[n * pitch]   dense pair-state matrix, 2 bits per ordered
//                               pair: bits of (a, b) = [arc a->b] | [arc b->a] << 1,
//                               16 pairs per word, rows padded to 16 bytes.
//                               The paper's neighbour partition (Notation
//                               section): state 3 = bidirected (delta*),
//                               1 = out only (delta+), 2 = in only (delta-).
//   deg     int32[n]            degree of v in G*
//   lo      int32[n]            neighbours of v below v (N*(v) is sorted, so
//                               the neighbours above v start at lo[v])
//   nptr    int64[n+1]          CSR offsets of the G* neighbour lists
//   nbr     uint32[2|E*|]       neighbour entries (u << 2) | state(v, u),
//                               sorted by u
//   src     uint32[2|E*|]       global row vertex of each entry, bit 31 set
//                               when the neighbour is below the row's vertex
//   label   int32[n]            new number of each input vertex (vertices
//                               are renumbered by descending G* degree, so
//                               hubs become the roots of their subsets)
// All of the above except label are in the renumbered ids.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/acc_motif.h"

namespace acc {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Block shape of the enumeration kernels.
constexpr int kWarpsPerBlock = 8;
#ifndef ACC_PARTB_ROWS
#define ACC_PARTB_ROWS 1024
#endif
// k = 5 count mode: part-B rows of a tile's level-3 lists a warp collects (two
// words each, at the end of its scratch) before scanning them in one pass
constexpr int kPartBRows = ACC_PARTB_ROWS;
constexpr int kThreads = kWarpsPerBlock * kWarp;

// Per-call scalars the builder leaves on the device.
struct GraphInfo {
    long long nnz;     // entries of nbr = sum over graphs of 2 |E*|
    int maxdeg;        // largest degree in G*
    int pad;
    unsigned long long queue_tail;  // heavy-unit chunks pushed by phase 1
    unsigned long long queue_head;  // chunks taken by phase 2
    unsigned long long unit_ctr;    // base units taken by phase 1
    unsigned long long chunks_pushed;
    unsigned long long scanned;     // count mode: neighbour entries the last two levels scanned
    unsigned big_rows;              // sparse build: rows listed for the block sort
    unsigned big_head;              // sparse build: listed rows taken
    float bound[3];                 // degree sums of the count bound (count_bound_terms)
};

// Largest count the library reports: a set whose upper bound on N_k (below)
// exceeds it is refused with ACC_ERR_OVERFLOW (int64 holds 2^63 - 1).
constexpr double kCountLimit = 4611686018427387904.0;  // 2^62

// Upper bound on the connected induced k-subsets of a graph from its G*
// degrees.  Every connected k-set has a spanning tree, so it is reached by
// choosing one embedded tree shape: k = 3 the path a-c-b from its centre c,
// C(d_c, 2); k = 4 the star at its centre, C(d_c, 3), or the path a-b-c-d
// from its middle edge, (d_b - 1)(d_c - 1); k = 5 the star, C(d_c, 4), the
// fork (centre c of degree 3, one leg b extended), C(d_c - 1, 2) sum_b (d_b
// - 1), or the path from its centre, at most (sum_b (d_b - 1))^2 / 2.  With
// every neighbour's degree taken as the largest degree D, the bound is
//   s0 + (D - 1) s1 + (D - 1)^2 s2,  per-vertex sums of count_bound_terms,
// and never above C(n, k).  The terms are single precision (FP64 is slow on
// this GPU and the scan runs on one SM for small sets); count_bound raises
// the sums by 1% to cover their rounding (at most a few 1e-4 relative for
// any set size the library takes).
__host__ __device__ inline void count_bound_terms(int k, int d, float *s) {
    const float x = (float)d;
    if (k == 3) {
        s[0] += x * (x - 1.0f) * 0.5f;
    } else if (k == 4) {
        s[0] += x * (x - 1.0f) * (x - 2.0f) * (1.0f / 6.0f);
        s[1] += x * (x - 1.0f) * 0.5f;
    } else if (k == 5) {
        s[0] += x * (x - 1.0f) * (x - 2.0f) * (x - 3.0f) * (1.0f / 24.0f);
        s[1] += x * (x - 1.0f) * (x - 2.0f) * 0.5f;
        s[2] += x * x * 0.5f;
    }
}
__host__ __device__ inline double count_bound(int k, int max_n, int maxdeg, const float *s) {
    const double dm = maxdeg > 0 ? maxdeg - 1.0 : 0.0;
    double b = 1.01 * ((double)s[0] + dm * (double)s[1] + dm * dm * (double)s[2]);
    double c = max_n >= k ? 1.0 : 0.0;
    for (int i = 0; i < k; i++) c = c * (double)(max_n - i) / (double)(i + 1);
    return c < b ? c : b;
}

// One graph of a set.  Its vertices are the global ids [voff, voff + n); its
// pair-state block is n rows of `pitch` words starting at word soff.
struct GMeta {
    const long long *rowptr;  // input out-CSR (device)
    const int *col;
    long long m;
    long long soff;
    long long pitch;
    long long moff;           // first arc of the graph in the set's arc numbering
    int n;
    int voff;
};

// A set of graphs counted together (B == 1: a single graph, held by value).
struct GSet {
    GMeta one;            // the graph when B == 1
    const GMeta *many;    // device array of B entries when B > 1
    const int *gid;       // graph of each global vertex when B > 1
    int B;
    long long NV;         // total vertices
    long long M;          // total arcs
    __device__ __forceinline__ GMeta meta(int g) const { return B == 1 ? one : many[g]; }
    __device__ __forceinline__ int graph_of(int v) const { return B == 1 ? 0 : gid[v]; }
};

// Sets with at most this many vertices scan their degrees in one block,
// through shared memory; larger sets scan in tiles.
constexpr long long kScanSingleMax = 1 << 15;
// Graph sets whose graphs all have at most this many vertices renumber each
// graph in one block with a shared-memory degree histogram.
constexpr int kRelabelSmemMax = 1 << 15;

// Occupancy bitmap of the pair-state rows: one bit per 32-word (128-byte)
// chunk of a row, set by the ingest when it first writes a word of the chunk,
// so the neighbour-list fill reads only chunks that hold neighbours.
// Words of bitmap per row for graphs of up to max_n vertices.
inline int occ_words(int max_n) {
    const long long pitch = ((long long)max_n + 15) / 16;
    const long long chunks = (pitch + 31) / 32;
    return (int)((chunks + 31) / 32 > 0 ? (chunks + 31) / 32 : 1);
}

// Bit of the adjacency code for the arc from tuple slot i to slot j.
__host__ __device__ constexpr int code_bit(int k, int i, int j) {
    return i * (k - 1) + (j - (j > i ? 1 : 0));
}

__host__ __device__ constexpr int num_classes(int k) {
    return k == 3 ? 13 : (k == 4 ? 199 : (k == 5 ? 9364 : 0));
}

__host__ __device__ constexpr int code_bits(int k) { return k * (k - 1); }

// Pitch (32-bit words per row) of the pair-state matrix for n vertices.
inline long long state_pitch(int n) {
    long long w = (n + 15) / 16;
    return (w + 3) & ~3LL;
}

// Hashed adjacency (for graphs whose dense pair-state block would not stay
// in L2): vertex p's neighbour entries (u << 2) | state(p, u) sit in an
// open-addressing table of 2^lg buckets of four 32-bit slots, lg = ceil(log2
// deg(p)) (at most one entry per bucket on average), at word kNhWords *
// nptr[p] of the table array (the region of kNhWords * deg(p) words holds
// it).  0 marks an empty slot (no entry is 0: its state is nonzero).  An
// entry goes to the bucket of its neighbour's hash, or the next bucket with a
// free slot, cyclically.
constexpr int kNhWords = 8;
__host__ __device__ inline uint32_t nh_lg(int d) {
    uint32_t lg = 0;
    while ((1 << lg) < d) lg++;
    return lg;
}
__host__ __device__ inline uint32_t nh_bucket(uint32_t u, uint32_t lg) {
    return lg ? (u * 0x9E3779B1u) >> (32u - lg) : 0u;  // multiplicative hash, top lg bits
}

// Programmatic dependent launch: a kernel launched with launch_pdl may have
// its blocks scheduled while the previous kernel of the stream finishes; it
// waits in grid_dep_wait(), its first statement, until that kernel has
// completed and its writes are visible (a no-op after a plain launch).
__device__ __forceinline__ void grid_dep_wait() {
#ifdef __CUDA_ARCH__
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
#ifdef __CUDACC__
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
#endif

// First-error-wins status update.
__device__ inline void set_status(int *status, int err) {
    if (status) atomicCAS(status, 0, err);
}

// --------------------------------------------------------------------------
// Launchers (each enqueues on `s` and returns the number of kernels it
// launched, or a negative ACC_ERR_* code).
// --------------------------------------------------------------------------

// graph.cu.  Builds the pair-state blocks and the G* neighbour lists of a
// graph set; with `relabel` each graph's vertices are first renumbered by
// descending G* degree (label[v] = new global id of input vertex v), which
// leaves the counts unchanged.  tile_scratch holds scan_tiles_needed(NV)
// values.
// Device buffers of the graph builder (sizes for NV vertices, at most max_n
// per graph).
struct BuildBufs {
    uint32_t *state;         // pair-state buffer of state_words words
    long long state_words;   // swept whole unless state_clean
    bool state_clean;        // known to be all zero
    int *deg, *lo, *label;   // NV each
    int *deg_in;             // NV: renumbering keys
    long long *nptr;         // NV + 1
    long long *tiles;        // scan_tiles_needed(NV) + 1
    uint32_t *nbr;           // 2 |E*|
    uint32_t *src = nullptr; // 2 |E*| or NULL: row of each entry (k_fill)
    uint32_t *occ;           // NV * occ_words(max_n)
    int occ_w;               // occ_words(max_n)
    GraphInfo *info;
    int k = 0;               // 3..5: refuse (ACC_ERR_OVERFLOW) a set whose count bound
                             // exceeds kCountLimit; 0: no check
};
int launch_build_graph(const GSet &gs, const BuildBufs &b, int max_n, int *status, unsigned long long *counts,
                       long long ncounts, bool relabel, int num_sms, cudaStream_t s);
// The sparse build: the same lists, degrees, renumbering, status and count
// bound from sorted rows of raw entries, without the dense block (b.state,
// b.occ unused).  Buffers: raw and merged 2 M words each, roff NV + 1, big
// sparse_big_rows_cap(M) ints.
struct SparseBufs {
    uint32_t *raw;
    uint32_t *merged;
    long long *roff;
    int *big;
};
int sparse_big_rows_cap(long long arcs);
int launch_build_graph_sparse(const GSet &gs, const BuildBufs &b, const SparseBufs &sb, int max_n, int *status,
                              unsigned long long *counts, long long ncounts, bool relabel, int num_sms,
                              cudaStream_t s);
// Hashed adjacency of a built set: nh (kNhWords * max_entries words) is
// cleared and every neighbour entry inserted; max_entries bounds the set's
// 2 |E*| (the exact count is read on the device).
int launch_nh_build(const long long *nptr, const int *deg, const uint32_t *nbr, const uint32_t *src,
                    const GraphInfo *info, long long max_entries, uint32_t *nh, int num_sms, cudaStream_t s);
// Reverse positions of a built set: for the entry p of row a holding x,
// the part of N*(x) above a (each list holds the other end of every edge,
// sorted by local id), as rev[p] = (first position, length).  The count mode
// stages a list row x that is a neighbour of the root v from rev(v -> x)
// instead of searching N*(x).  max_entries bounds 2 |E*|.
int launch_rev_build(const GSet &gs, const long long *nptr, const int *deg, const uint32_t *nbr, const uint32_t *src,
                     const GraphInfo *info, long long max_entries, uint2 *rev, int num_sms, cudaStream_t s);
// Zero the pair-state chunks a build set (by its occupancy bitmap), leaving
// the buffer all zero.
int launch_clear_graph(const GSet &gs, uint32_t *state, const uint32_t *occ, int occ_w, int num_sms, cudaStream_t s);
long long scan_tiles_needed(long long NV);
// gid[v] for a set of several graphs (no launch for one graph).
int launch_graph_ids(const GSet &gs, int *gid, cudaStream_t s);
// Zero `bytes` at p, plus counts[0..ncounts), ints[0..nints) and *status
// when not NULL.
int launch_zero(void *p, size_t bytes, int num_sms, cudaStream_t s, int *status = nullptr,
                unsigned long long *counts = nullptr, long long ncounts = 0, int *ints = nullptr,
                long long nints = 0);

// lut.cu: lut = code -> class in the canonical code layout (public API),
// lut_sv = the same classes indexed in the state-vector layout (kernels).
// scratch_canon holds 2^(k(k-1)) words, scratch_rank rank_ints(k) ints.
int rank_ints(int k);
int launch_build_lut(int k, uint32_t *scratch_canon, int *scratch_rank, int16_t *lut,
                     uint32_t *class_code, int16_t *lut_sv, cudaStream_t s);

// enum.cu
struct EnumArgs {
    const uint32_t *state;      // pair-state blocks of all graphs
    const int *deg;             // by global vertex
    const int *lo;
    const long long *nptr;
    const uint32_t *nbr;        // entries hold local ids
    const uint32_t *src;        // global row vertex of each entry, bit 31: neighbour below it
    const uint4 *nh;            // hashed adjacency (count mode), or NULL: probes read the dense block
    const uint2 *rev;           // count mode: reverse positions (launch_rev_build), or NULL
    const int16_t *lut;         // class table in the state-vector layout
    GSet gs;
    int max_n;                  // largest graph of the set
    GraphInfo *info;
    uint4 *queue;               // heavy-unit chunks (unit, lo, hi, global root)
    unsigned long long queue_cap;
    uint32_t *scratch;          // per-warp overflow buffers for the extension sets
    long long scratch_per_warp; // entries per warp
    int mode;                   // 0: count the last two levels by groups, 1: enumerate every leaf
    long long light;            // schedule: phase 1 runs units of at most this much work whole
    long long target;           // schedule: work of one queued chunk of a heavy unit
    unsigned long long *counts; // int64[B * num_classes]
    int *status;
};
// batch.cu: Z-scores of each group's real graph against its randomisations.
int launch_zscores(const long long *counts, int groups, int group_size, int K, double *z, cudaStream_t s);

// phase 1: light units run, heavy units queued; phase 2: the queue drained.
// The grid is the full persistent grid times grid_num / grid_den (at least
// one block per SM).
int launch_enumerate(int k, const EnumArgs &a, int num_sms, int phase, cudaStream_t s, int grid_num = 1,
                     int grid_den = 1);
// Default schedule of the enumeration kernels (see EnumArgs::light, target).
long long enum_default_light(int k, bool count_mode);
long long enum_default_target(int k, bool count_mode);
int enum_grid_warps(int k, int num_sms);

}  // namespace acc
