// The library context (private to the library's translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"
#include "randomise.cuh"

using acc::GMeta;
using acc::GSet;
using acc::GraphInfo;

struct acc_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t own = nullptr;  // stream of the host-buffer entry points

    // code -> class tables per k
    int16_t *lut[6] = {};
    int16_t *lut_sv[6] = {};
    uint32_t *class_code_dev[6] = {};
    int16_t *lut_host[6] = {};
    uint32_t *class_code_host[6] = {};

    // workspace (grow-only)
    uint32_t *state = nullptr;
    size_t state_cap = 0;
    bool state_clean = false;  // every pair-state word is zero (each call clears what it set)
    int *deg = nullptr, *lo = nullptr, *label = nullptr, *deg_in = nullptr;
    long long *nptr = nullptr;
    size_t n_cap = 0;
    long long *tiles = nullptr;
    size_t tiles_cap = 0;
    long long *f5_pre = nullptr;  // k = 5 formula path: prefix of C(deg, 2)
    size_t f5_pre_cap = 0;
    uint32_t *nbr = nullptr;
    uint32_t *src = nullptr;  // row of each neighbour entry
    size_t src_cap = 0;
    uint2 *rev = nullptr;     // count mode: reverse position of each neighbour entry
    size_t rev_cap = 0;
    uint32_t *nh = nullptr;   // hashed adjacency tables
    size_t nh_cap = 0;
    int adjacency = ACC_ADJ_AUTO;
    // sparse build: raw and merged rows, row offsets, rows for the block sort
    uint32_t *sp_raw = nullptr, *sp_merged = nullptr;
    size_t sp_raw_cap = 0, sp_merged_cap = 0;
    long long *sp_roff = nullptr;
    size_t sp_roff_cap = 0;
    int *sp_big = nullptr;
    size_t sp_big_cap = 0;
    int *maxdeg_host = nullptr;  // pinned
    uint32_t *occ = nullptr;  // pair-state row occupancy bitmaps
    size_t occ_cap = 0;
    size_t nbr_cap = 0;
    GraphInfo *info = nullptr;
    uint4 *queue = nullptr;
    unsigned long long queue_cap = 0;
    uint32_t *scratch = nullptr;
    size_t scratch_cap = 0;
    int mode = 0;             // ACC_MODE_COUNT, _ENUMERATE, _FORMULA or _AUTO
    long long sched_light = 0;   // enumeration schedule (0: the kernels' default)
    long long sched_target = 0;
    int *status_dev = nullptr;
    int *status_host = nullptr;  // pinned

    // prepared batch
    GMeta *meta_dev = nullptr;
    size_t meta_cap = 0;
    int *gid = nullptr;
    size_t gid_cap = 0;
    bool batch_ready = false;
    int batch_k = 0;
    GSet batch_set = {};
    long long batch_words = 0, batch_arcs = 0;
    int batch_max_n = 0;

    // randomised copies: graph descriptors and the per-position row table
    acc::RGraph *rand_meta = nullptr;
    size_t rand_meta_cap = 0;
    int4 *rand_rows = nullptr;
    size_t rand_rows_cap = 0;
    std::vector<acc::RGraph> rand_host;  // the descriptors on the device
    uint32_t *rand_bits = nullptr;       // the copies' adjacency bitmaps
    size_t rand_bits_cap = 0;
    long long rand_bits_limit = 16ll << 30;  // bytes the bitmaps (and reverse positions) may take
    int *rand_rpart = nullptr;           // mutual mode: reverse position of each arc of the graphs
    size_t rand_rpart_cap = 0;
    int *rand_pts = nullptr;             // mutual mode: the copies' reverse positions
    size_t rand_pts_cap = 0;

    // host-buffer entry point
    long long *h2d_rowptr = nullptr;
    size_t h2d_rowptr_cap = 0;
    int *h2d_col = nullptr;
    size_t h2d_col_cap = 0;
    unsigned long long *h2d_counts = nullptr;

    // launch graph of the last single count, replayed while a count repeats
    // it (same buffers, sizes, k, mode, schedule and workspace)
    bool graphs = true;
    cudaGraphExec_t cg_exec = nullptr;
    struct CountKey {
        const void *rowptr, *col, *counts, *status;
        long long m, light, target;
        int n, k, mode, grid_num, grid_den, adjacency;
        const void *ws[21];
    } cg_key = {}, cg_seen = {};  // the captured graph's key; the last key counted one by one
    int cg_launches = 0;
    long long cg_units = 0;
    int cg_blocks = 0;

    // stage timing
    bool timing = false;
    bool timed_call = false;
    cudaEvent_t ev[4] = {};

    // statistics of the last count
    int last_launches = 0;
    int last_k = 0;
    long long last_units = 0;
    int last_blocks = 0;

    // enumeration grid cap as a fraction of the full persistent grid
    // (1 = whole GPU); the request server lowers it so requests overlap
    int grid_num = 1, grid_den = 1;
};


namespace acc {
// Device bytes a context's workspace needs for one graph of n vertices and m
// arcs at k (with the growth margin), and pre-sizing it (plus the tables of
// every k) so later counts of graphs up to that size allocate nothing.
long long ctx_footprint(const acc_ctx *c, long long n, long long m, int k);
int ctx_reserve(acc_ctx *c, long long n, long long m, int k);
}  // namespace acc
