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
};

// One graph of a set.  Its vertices are the global ids [voff, voff + n); its
// pair-state block is n rows of `pitch` words starting at word soff.
struct GMeta {
    const long long *rowptr;  // input out-CSR (device)
    const int *col;
    long long m;
    long long soff;
    long long pitch;
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
    __device__ __forceinline__ GMeta meta(int g) const { return B == 1 ? one : many[g]; }
    __device__ __forceinline__ int graph_of(int v) const { return B == 1 ? 0 : gid[v]; }
};

// Sets with at most this many vertices scan their degrees in one block.
constexpr long long kScanSingleMax = 1 << 17;

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
// state_words: the whole pair-state buffer, swept unless state_clean says it
// is known to be all zero; deg_in: NV ints of scratch for the renumbering.
int launch_build_graph(const GSet &gs, long long state_words, uint32_t *state, bool state_clean, int *deg, int *lo,
                       int *deg_in, long long *nptr, long long *tile_scratch, uint32_t *nbr, int *label,
                       GraphInfo *info, int *status, unsigned long long *counts, long long ncounts, bool relabel,
                       int num_sms, cudaStream_t s);
// Zero the pair-state words a build set, leaving the buffer all zero.
int launch_clear_graph(const GSet &gs, uint32_t *state, const int *label, bool relabel, int num_sms, cudaStream_t s);
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
int launch_build_lut(int k, uint32_t *scratch_canon, int *scratch_rank, int16_t *lut,
                     uint32_t *class_code, int16_t *lut_sv, cudaStream_t s);

// enum.cu
struct EnumArgs {
    const uint32_t *state;      // pair-state blocks of all graphs
    const int *deg;             // by global vertex
    const int *lo;
    const long long *nptr;
    const uint32_t *nbr;        // entries hold local ids
    const int16_t *lut;         // class table in the state-vector layout
    GSet gs;
    int max_n;                  // largest graph of the set
    GraphInfo *info;
    uint4 *queue;               // heavy-unit chunks (unit, lo, hi, global root)
    unsigned long long queue_cap;
    uint32_t *scratch;          // per-warp overflow buffers for the extension sets
    long long scratch_per_warp; // entries per warp
    int mode;                   // 0: count the last two levels by groups, 1: enumerate every leaf
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
int enum_grid_warps(int k, int num_sms);

}  // namespace acc
