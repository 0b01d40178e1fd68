// C ABI: context, workspace and the counting entry points.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "context.cuh"
#include "formula.cuh"
#include "randomise.cuh"

using namespace acc;

namespace {

constexpr unsigned long long kQueueCap = 1ull << 22;
// ACC_ADJ_AUTO: count-mode probes read hashed tables for sets whose largest
// graph has at least this many vertices (k = 5; k = 3, 4), where the dense
// block's probes (n^2/4 bytes, out of L2) get slower than the hashed ones
// (measured on GB300: k = 5 dense/hashed 82/87 scanned entries per ns at
// n = 40000, 53/87 at 80000; k = 4 149/107 at 40000, 122/108 at 80000).
constexpr int kHashMinN5 = 49152;
constexpr int kHashMinN34 = 131072;
bool hash_auto(int k, int max_n) { return max_n >= (k == 5 ? kHashMinN5 : kHashMinN34); }
// Below this many vertices the renumbering pass costs more than it saves.
constexpr int kRelabelMinN = 1024;
// ACC_MODE_AUTO: largest graph (vertices) for which k = 3 takes the formula path.
constexpr int kAutoFormulaMaxN = 16384;

bool ok(cudaError_t e) { return e == cudaSuccess; }

template <typename T>
int grow(T **p, size_t *cap, size_t need) {
    if (need <= *cap && *p) return ACC_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    const size_t alloc = need + need / 4 + 64;
    if (!ok(cudaMalloc((void **)p, alloc * sizeof(T)))) {
        cudaGetLastError();
        *p = nullptr;
        return ACC_ERR_NOMEM;
    }
    *cap = alloc;
    return ACC_OK;
}

bool valid_k(int k) { return k >= 3 && k <= 5; }

// Class tables are built once per device and k and shared by every context
// on that device (the request server runs one context per slot); each
// context holds a reference, and the last one released frees the table.
struct SharedTable {
    int refs = 0;
    int16_t *lut = nullptr, *lut_sv = nullptr;
    uint32_t *class_code = nullptr;
    int16_t *lut_host = nullptr;
    uint32_t *class_code_host = nullptr;
};
constexpr int kTableDevices = 64;
SharedTable g_tables[kTableDevices][6];
std::mutex g_tables_mu;

// Build the table for k on stream s (waits for it) into t; on failure t is
// left empty.
int build_table(int k, cudaStream_t s, SharedTable &t) {
    const size_t ncodes = size_t(1) << code_bits(k);
    const int ncls = num_classes(k);
    uint32_t *canon = nullptr;
    int *rank = nullptr;
    int16_t *lut = nullptr, *lut_sv = nullptr;
    uint32_t *cc = nullptr;
    int16_t *lut_host = new (std::nothrow) int16_t[ncodes];
    uint32_t *cc_host = new (std::nothrow) uint32_t[ncls];
    int rc = ACC_ERR_NOMEM;
    if (!lut_host || !cc_host) goto fail;
    if (!ok(cudaMalloc(&canon, ncodes * 4)) || !ok(cudaMalloc(&rank, (size_t)rank_ints(k) * 4)) ||
        !ok(cudaMalloc(&lut, ncodes * 2)) || !ok(cudaMalloc(&lut_sv, ncodes * 2)) ||
        !ok(cudaMalloc(&cc, ncls * 4)))
        goto fail;
    rc = launch_build_lut(k, canon, rank, lut, cc, lut_sv, s);
    if (rc < 0) goto fail;
    rc = ACC_ERR_CUDA;
    if (!ok(cudaMemcpyAsync(lut_host, lut, ncodes * 2, cudaMemcpyDeviceToHost, s))) goto fail;
    if (!ok(cudaMemcpyAsync(cc_host, cc, ncls * 4, cudaMemcpyDeviceToHost, s))) goto fail;
    if (!ok(cudaStreamSynchronize(s))) goto fail;
    {
        // the table must use every class index exactly up to ncls - 1
        int mx = -1;
        for (size_t i = 0; i < ncodes; i++) {
            if (lut_host[i] < -1) mx = 1 << 20;
            if (lut_host[i] > mx) mx = lut_host[i];
        }
        if (mx != ncls - 1) {
            rc = ACC_ERR_INTERNAL;
            goto fail;
        }
    }
    cudaFree(canon);
    cudaFree(rank);
    t.lut = lut;
    t.lut_sv = lut_sv;
    t.class_code = cc;
    t.lut_host = lut_host;
    t.class_code_host = cc_host;
    return ACC_OK;
fail:
    cudaGetLastError();
    cudaFree(canon);
    cudaFree(rank);
    cudaFree(lut);
    cudaFree(lut_sv);
    cudaFree(cc);
    delete[] lut_host;
    delete[] cc_host;
    return rc;
}

int ensure_lut(acc_ctx *c, int k, cudaStream_t s) {
    if (c->lut[k]) return ACC_OK;
    if (c->device < 0 || c->device >= kTableDevices) return ACC_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tables_mu);
    SharedTable &t = g_tables[c->device][k];
    if (t.refs == 0) {
        const int rc = build_table(k, s, t);
        if (rc) return rc;
    }
    t.refs++;
    c->lut[k] = t.lut;
    c->lut_sv[k] = t.lut_sv;
    c->class_code_dev[k] = t.class_code;
    c->lut_host[k] = t.lut_host;
    c->class_code_host[k] = t.class_code_host;
    return ACC_OK;
}

// Drop the context's references to the shared tables (the device is current).
void release_luts(acc_ctx *c) {
    std::lock_guard<std::mutex> lock(g_tables_mu);
    for (int k = 3; k <= 5; k++) {
        if (!c->lut[k]) continue;
        SharedTable &t = g_tables[c->device][k];
        if (--t.refs == 0) {
            cudaFree(t.lut);
            cudaFree(t.lut_sv);
            cudaFree(t.class_code);
            delete[] t.lut_host;
            delete[] t.class_code_host;
            t = SharedTable();
        }
        c->lut[k] = c->lut_sv[k] = nullptr;
        c->class_code_dev[k] = nullptr;
        c->lut_host[k] = nullptr;
        c->class_code_host[k] = nullptr;
    }
}

// per warp: two overflow lists of up to max_n entries, then the k = 5 count
// mode's collected part-B rows
long long scratch_per_warp(int max_n) { return 2 * (((long long)max_n + 32 + 31) & ~31LL) + 2 * kPartBRows; }

// The count mode, and the automatic mode that runs it for k = 4, 5 and for
// any graph above the dense block's limit.
bool count_family(const acc_ctx *c) { return c->mode == ACC_MODE_COUNT || c->mode == ACC_MODE_AUTO; }

// The count mode builds the lists without the dense block (and probes
// hashed tables) above the dense block's limit, or when asked to.
bool sparse_build(const acc_ctx *c, int max_n) {
    return count_family(c) && (c->adjacency == ACC_ADJ_SPARSE || max_n > ACC_MAX_N);
}

bool uses_hash(const acc_ctx *c, int k, int max_n) {
    return count_family(c) &&
           (c->adjacency == ACC_ADJ_HASH || c->adjacency == ACC_ADJ_SPARSE || max_n > ACC_MAX_N ||
            (c->adjacency == ACC_ADJ_AUTO && hash_auto(k, max_n)));
}

// The count mode's scans stage the list rows that are neighbours of the
// root from the reverse positions of the root's entries (ACC_REV=0 at build
// time: by binary search, as for every other row).  Sets of fewer than
// ACC_REV_MIN_ARCS arcs skip them: building them costs about 4 us, more than
// the searches they save on small graphs (k = 3 count on 1000 vertices and
// 5000 arcs: 0.035 ms per count without, 0.039 with; k = 4 on 20000 vertices
// and 100000 arcs: 0.604 without, 0.572 with).
#ifndef ACC_REV
#define ACC_REV 1
#endif
#ifndef ACC_REV_MIN_ARCS
#define ACC_REV_MIN_ARCS 8192
#endif
bool uses_rev(const acc_ctx *c, long long arcs) { return ACC_REV && count_family(c) && arcs >= ACC_REV_MIN_ARCS; }

// Size limit of one graph: the dense block's, or the sparse build's for the
// count mode (local ids fill 26 bits of the extension-list entries).
int size_check(const acc_ctx *c, long long n) {
    if (n > ACC_MAX_N_SPARSE) return ACC_ERR_TOO_LARGE;
    if (n > ACC_MAX_N && !count_family(c)) return ACC_ERR_TOO_LARGE;
    return ACC_OK;
}

// Entries of one per-warp overflow list for the sparse build: an extension
// list holds at most 3 maxdeg vertices (k = 5: the level-2 list after w2
// and the neighbours of w2; k = 4: two neighbour lists; k = 3: one).
long long sparse_list_entries(int maxdeg) { return (3LL * maxdeg + 64 + 31) & ~31LL; }

// Workspace for a set of NV vertices in blocks of state_words words, with at
// most `arcs` arcs and graphs of at most max_n vertices.
int ensure_workspace(acc_ctx *c, long long NV, long long state_words, long long arcs, int max_n, int k) {
    int rc;
    const bool sparse = sparse_build(c, max_n);
    if (uses_hash(c, k, max_n) && (rc = grow(&c->nh, &c->nh_cap, (size_t)kNhWords * (size_t)(2 * arcs) + 4)))
        return rc;
    if (sparse) {
        if ((rc = grow(&c->sp_raw, &c->sp_raw_cap, (size_t)(2 * arcs) + 1))) return rc;
        if ((rc = grow(&c->sp_merged, &c->sp_merged_cap, (size_t)(2 * arcs) + 1))) return rc;
        if ((rc = grow(&c->sp_roff, &c->sp_roff_cap, (size_t)NV + 1))) return rc;
        if ((rc = grow(&c->sp_big, &c->sp_big_cap, (size_t)sparse_big_rows_cap(arcs)))) return rc;
    }
    if (!sparse) {
        // a reallocation (the capacity changes; the address may not) brings
        // memory that is not zero: the next build sweeps it
        const size_t cap_before = c->state_cap;
        if ((rc = grow(&c->state, &c->state_cap, (size_t)state_words + 4))) {
            c->state_clean = false;
            return rc;
        }
        if (c->state_cap != cap_before) c->state_clean = false;
    }
    if ((size_t)NV + 1 > c->n_cap || !c->deg) {
        size_t a = 0, b = 0, d = 0, e = 0;
        cudaFree(c->deg);
        cudaFree(c->lo);
        cudaFree(c->nptr);
        cudaFree(c->label);
        cudaFree(c->deg_in);
        c->deg = c->lo = c->label = c->deg_in = nullptr;
        c->nptr = nullptr;
        c->n_cap = 0;
        if ((rc = grow(&c->deg, &a, (size_t)NV + 1))) return rc;
        if ((rc = grow(&c->lo, &b, (size_t)NV + 1))) return rc;
        if ((rc = grow(&c->nptr, &d, (size_t)NV + 1))) return rc;
        if ((rc = grow(&c->label, &e, (size_t)NV + 1))) return rc;
        e = 0;
        if ((rc = grow(&c->deg_in, &e, (size_t)NV + 1))) return rc;
        c->n_cap = a;
    }
    if ((rc = grow(&c->tiles, &c->tiles_cap, (size_t)scan_tiles_needed(NV) + 1))) return rc;
    if ((rc = grow(&c->f5_pre, &c->f5_pre_cap, (size_t)NV + 1))) return rc;
    if ((rc = grow(&c->nbr, &c->nbr_cap, (size_t)(2 * arcs) + 1))) return rc;
    if ((rc = grow(&c->src, &c->src_cap, (size_t)(2 * arcs) + 1))) return rc;
    if (uses_rev(c, arcs) && (rc = grow(&c->rev, &c->rev_cap, (size_t)(2 * arcs) + 1))) return rc;
    if (!sparse && (rc = grow(&c->occ, &c->occ_cap, (size_t)NV * (size_t)occ_words(max_n) + 1))) return rc;
    if (!c->info) {
        if (!ok(cudaMalloc(&c->info, sizeof(GraphInfo)))) return ACC_ERR_NOMEM;
        if (!ok(cudaMemset(c->info, 0, sizeof(GraphInfo)))) return ACC_ERR_CUDA;
    }
    if (!c->queue) {
        if (!ok(cudaMalloc(&c->queue, kQueueCap * sizeof(uint4)))) return ACC_ERR_NOMEM;
        c->queue_cap = kQueueCap;
    }
    if (!c->status_dev) {
        if (!ok(cudaMalloc(&c->status_dev, sizeof(int)))) return ACC_ERR_NOMEM;
    }
    const int warps = enum_grid_warps(k, c->num_sms);
    if (warps < 0) return warps;
    // the sparse build sizes the overflow lists by the largest degree, once
    // it is known (run_set)
    if (!sparse && (rc = grow(&c->scratch, &c->scratch_cap, (size_t)scratch_per_warp(max_n) * (size_t)warps)))
        return rc;
    if (!c->maxdeg_host && !ok(cudaMallocHost(&c->maxdeg_host, sizeof(int)))) return ACC_ERR_NOMEM;
    return ACC_OK;
}

// Build + enumerate one graph set into counts[B * num_classes(k)].
int run_set(acc_ctx *c, const GSet &gs, int max_n, int k, bool relabel, cudaStream_t s,
            int64_t *counts, int *status) {
    int launches = 0;
    c->timed_call = c->timing;
    if (c->timing && !ok(cudaEventRecord(c->ev[0], s))) return ACC_ERR_CUDA;
    const bool clean = c->state_clean;
    const bool sparse = sparse_build(c, max_n);
    if (!sparse) c->state_clean = false;  // until the closing clear below is enqueued
    // a buffer not known to be clean is swept whole (capacity, not just this
    // set's blocks): a later, larger set may use any part of it
    BuildBufs bb;
    bb.state = c->state;
    bb.state_words = (long long)c->state_cap;
    bb.state_clean = clean;
    bb.deg = c->deg;
    bb.lo = c->lo;
    bb.label = c->label;
    bb.deg_in = c->deg_in;
    bb.nptr = c->nptr;
    bb.tiles = c->tiles;
    bb.nbr = c->nbr;
    bb.src = c->src;
    bb.occ = c->occ;
    bb.occ_w = occ_words(max_n);
    bb.info = c->info;
    bb.k = k;
    int rc;
    if (sparse) {
        const SparseBufs sb = {c->sp_raw, c->sp_merged, c->sp_roff, c->sp_big};
        rc = launch_build_graph_sparse(gs, bb, sb, max_n, status, reinterpret_cast<unsigned long long *>(counts),
                                       (long long)gs.B * num_classes(k), relabel, c->num_sms, s);
    } else {
        rc = launch_build_graph(gs, bb, max_n, status, reinterpret_cast<unsigned long long *>(counts),
                                (long long)gs.B * num_classes(k), relabel, c->num_sms, s);
    }
    if (rc < 0) return rc;
    launches += rc;
    long long spw = scratch_per_warp(max_n);
    if (sparse) {
        // overflow lists sized by the largest degree: wait for the build
        if (!ok(cudaMemcpyAsync(c->maxdeg_host, &c->info->maxdeg, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
            !ok(cudaStreamSynchronize(s)))
            return ACC_ERR_CUDA;
        spw = 2 * sparse_list_entries(*c->maxdeg_host) + 2 * kPartBRows;
        const int warps = enum_grid_warps(k, c->num_sms);
        if (warps < 0) return warps;
        if ((rc = grow(&c->scratch, &c->scratch_cap, (size_t)spw * (size_t)warps))) return rc;
    }
    // count mode on a large set: probes read hashed tables, built from the
    // sorted neighbour lists
    const bool hash = gs.NV > 0 && uses_hash(c, k, max_n);
    // the automatic mode takes the k = 3 formula path on graphs of up to
    // kAutoFormulaMaxN vertices (measured faster there: 0.028 against 0.034 ms
    // at 1000 vertices, 0.065 against 0.100 at 5000; slower at 20000 with
    // hubs of degree 470, 0.208 against 0.181)
    if (hash) {
        rc = launch_nh_build(c->nptr, c->deg, c->nbr, c->src, c->info, 2 * gs.M, c->nh, c->num_sms, s);
        if (rc < 0) return rc;
        launches += rc;
    }
    const bool formula = c->mode == ACC_MODE_FORMULA ||
                         (c->mode == ACC_MODE_AUTO && k == 3 && max_n <= kAutoFormulaMaxN && !sparse &&
                          !uses_hash(c, k, max_n));
    const bool rev = gs.NV > 0 && !formula && uses_rev(c, gs.M);
    if (rev) {
        rc = launch_rev_build(gs, c->nptr, c->deg, c->nbr, c->src, c->info, 2 * gs.M, c->rev, c->num_sms, s);
        if (rc < 0) return rc;
        launches += rc;
    }
    if (c->timing && !ok(cudaEventRecord(c->ev[1], s))) return ACC_ERR_CUDA;
    EnumArgs a;
    a.state = c->state;
    a.deg = c->deg;
    a.lo = c->lo;
    a.nptr = c->nptr;
    a.nbr = c->nbr;
    a.src = c->src;
    a.nh = hash ? reinterpret_cast<const uint4 *>(c->nh) : nullptr;
    a.rev = rev ? c->rev : nullptr;
    a.lut = c->lut_sv[k];
    a.gs = gs;
    a.max_n = max_n;
    a.info = c->info;
    a.queue = c->queue;
    a.queue_cap = c->queue_cap;
    a.scratch = c->scratch;
    a.scratch_per_warp = spw;
    a.mode = c->mode == ACC_MODE_ENUMERATE ? 1 : 0;
    a.light = c->sched_light > 0 ? c->sched_light : enum_default_light(k, a.mode == 0);
    a.target = c->sched_target > 0 ? c->sched_target : enum_default_target(k, a.mode == 0);
    a.counts = reinterpret_cast<unsigned long long *>(counts);
    a.status = status;
    const bool any = gs.NV > 0;
    if (any && formula) {
        if (k == 3)
            rc = launch_formula3(gs, c->state, c->nptr, c->deg, c->lo, c->nbr, c->lut[3],
                                 reinterpret_cast<unsigned long long *>(counts), status, c->num_sms, s);
        else if (k == 4)
            rc = launch_formula4(gs, c->state, c->nptr, c->deg, c->lo, c->nbr, c->lut[4], c->class_code_dev[4],
                                 c->info, reinterpret_cast<unsigned long long *>(counts), status, c->num_sms, s);
        else
            rc = launch_formula5(gs, c->state, c->nptr, c->deg, c->nbr, c->lut[5], c->class_code_dev[5], c->f5_pre,
                                 reinterpret_cast<unsigned long long *>(counts), status, c->num_sms, s);
        if (rc < 0) return rc;
        launches += rc;
    } else if (any) {
        rc = launch_enumerate(k, a, c->num_sms, 1, s, c->grid_num, c->grid_den);
        if (rc < 0) return rc;
        launches += rc;
    }
    if (c->timing && !ok(cudaEventRecord(c->ev[3], s))) return ACC_ERR_CUDA;
    if (any && !formula) {
        rc = launch_enumerate(k, a, c->num_sms, 2, s, c->grid_num, c->grid_den);
        if (rc < 0) return rc;
        launches += rc;
    }
    if (c->timing && !ok(cudaEventRecord(c->ev[2], s))) return ACC_ERR_CUDA;
    if (!sparse) {
        rc = launch_clear_graph(gs, c->state, c->occ, occ_words(max_n), c->num_sms, s);
        if (rc < 0) return rc;
        launches += rc;
        c->state_clean = true;
    }
    c->last_launches = launches;
    c->last_k = k;
    c->last_units = gs.NV;
    c->last_blocks = enum_grid_warps(k, c->num_sms) / kWarpsPerBlock * c->grid_num / c->grid_den;
    return ACC_OK;
}

// Wait for the call's device status when the caller gave no status word.
int finish(acc_ctx *c, cudaStream_t s, int32_t *status_user) {
    if (status_user) return ACC_OK;
    if (!ok(cudaMemcpyAsync(c->status_host, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s)))
        return ACC_ERR_CUDA;
    if (!ok(cudaStreamSynchronize(s))) return ACC_ERR_CUDA;
    return *c->status_host;
}

int count_impl(acc_ctx *c, const int64_t *rowptr, const int32_t *col, int32_t n, int64_t m, int k,
               cudaStream_t s, int64_t *counts, int32_t *status_user) {
    if (!c || !rowptr || !counts || (m > 0 && !col)) return ACC_ERR_ARG;
    if (!valid_k(k)) return ACC_ERR_K;
    if (n < 0 || m < 0 || m >= (1ll << 31)) return ACC_ERR_INPUT;
    if (size_check(c, n)) return ACC_ERR_TOO_LARGE;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    int rc = ensure_lut(c, k, s);
    if (rc) return rc;
    const long long pitch = state_pitch(n);
    if ((rc = ensure_workspace(c, n, sparse_build(c, n) ? 0 : (long long)n * pitch, m, n, k))) return rc;
    GSet gs = {};
    gs.one.rowptr = reinterpret_cast<const long long *>(rowptr);
    gs.one.col = col;
    gs.one.m = m;
    gs.one.soff = 0;
    gs.one.moff = 0;
    gs.one.pitch = pitch;
    gs.one.n = n;
    gs.one.voff = 0;
    gs.B = 1;
    gs.NV = n;
    gs.M = m;
    int *status = status_user ? status_user : c->status_dev;
    const bool relabel = n >= kRelabelMinN;
    if (c->graphs && !c->timing && c->state_clean && n > 0 && !sparse_build(c, n)) {
        // repeat counts replay one CUDA graph of the whole launch sequence;
        // it is captured (on the context's stream, not run) at the second
        // count with the same key, and only while the pair-state buffer is
        // known clean, so it holds no full sweep
        acc_ctx::CountKey key;
        memset(&key, 0, sizeof(key));
        key.rowptr = rowptr;
        key.col = col;
        key.counts = counts;
        key.status = status;
        key.m = m;
        key.light = c->sched_light;
        key.target = c->sched_target;
        key.n = n;
        key.k = k;
        key.mode = c->mode;
        key.grid_num = c->grid_num;
        key.grid_den = c->grid_den;
        key.adjacency = c->adjacency;
        const void *ws[21] = {c->state, c->deg, c->lo, c->label, c->deg_in, c->nptr, c->tiles, c->nbr, c->occ,
                              c->info, c->queue, c->scratch, c->lut[k], c->lut_sv[k], c->class_code_dev[k],
                              c->f5_pre, c->status_dev, c->src, c->nh, c->rev, nullptr};
        memcpy(key.ws, ws, sizeof(ws));
        bool have = c->cg_exec && memcmp(&key, &c->cg_key, sizeof(key)) == 0;
        // capture only when a count repeats: a one-off count runs one by one
        const bool repeat = memcmp(&key, &c->cg_seen, sizeof(key)) == 0;
        if (!have && !repeat) c->cg_seen = key;
        if (!have && repeat) {
            if (c->cg_exec) cudaGraphExecDestroy(c->cg_exec);
            c->cg_exec = nullptr;
            cudaGraph_t g = nullptr;
            if (ok(cudaStreamBeginCapture(c->own, cudaStreamCaptureModeRelaxed))) {
                rc = run_set(c, gs, n, k, relabel, c->own, counts, status);
                const cudaError_t ce = cudaStreamEndCapture(c->own, &g);
                c->state_clean = true;  // nothing ran
                if (rc) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                if (ce == cudaSuccess && g && ok(cudaGraphInstantiate(&c->cg_exec, g, 0))) {
                    c->cg_key = key;
                    c->cg_launches = c->last_launches;
                    c->cg_units = c->last_units;
                    c->cg_blocks = c->last_blocks;
                    have = true;
                } else {
                    c->cg_exec = nullptr;
                }
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();  // a refused capture leaves the eager path below
        }
        if (have) {
            if (!ok(cudaGraphLaunch(c->cg_exec, s))) return ACC_ERR_CUDA;
            c->state_clean = true;  // the sequence ends with the clear
            c->last_launches = c->cg_launches;
            c->last_k = k;
            c->last_units = c->cg_units;
            c->last_blocks = c->cg_blocks;
            return finish(c, s, status_user);
        }
    }
    rc = run_set(c, gs, n, k, relabel, s, counts, status);
    if (rc) return rc;
    return finish(c, s, status_user);
}

// The workspace a run of the prepared batch needs under the context's
// current mode and adjacency choice, which may differ from those at the
// prepare (the count mode's reverse positions, hashed tables or sparse
// build): grows nothing when they are the same.
int batch_workspace(acc_ctx *c) {
    if (size_check(c, c->batch_max_n)) return ACC_ERR_TOO_LARGE;
    return ensure_workspace(c, c->batch_set.NV, sparse_build(c, c->batch_max_n) ? 0 : c->batch_words, c->batch_arcs,
                            c->batch_max_n, c->batch_k);
}

}  // namespace

namespace acc {

long long ctx_footprint(const acc_ctx *c, long long n, long long m, int k) {
    const long long pitch = state_pitch((int)n);
    const long long warps = enum_grid_warps(k, c->num_sms);
    const long long hash_bytes = uses_hash(c, k, (int)n) ? 4LL * kNhWords * (2 * m + 1) : 0;
    const bool sparse = sparse_build(c, (int)n);
    // the sparse build keeps raw and merged rows (2 m words each) and row
    // offsets instead of the dense block and its bitmap; its overflow lists
    // are bounded by the largest degree, itself at most 2m and n
    const long long list_n = sparse ? (2 * m < n ? 2 * m : n) : n;
    const long long bytes = (sparse ? 16 * (m + 1) + 8 * (n + 1) : n * pitch * 4 + 4 * n * occ_words((int)n)) +
                            5 * 4 * (n + 1) + 8 * (n + 1) + (uses_rev(c, m) ? 16 : 8) * (2 * m + 1) + hash_bytes +
                            (long long)kQueueCap * 16 +
                            (sparse ? 2 * sparse_list_entries((int)list_n) + 2 * kPartBRows : scratch_per_warp((int)n)) *
                                (warps > 0 ? warps : 0) * 4;
    return bytes + bytes / 4;
}

int ctx_reserve(acc_ctx *c, long long n, long long m, int k) {
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    for (int kk = 3; kk <= 5; kk++) {
        const int rc = ensure_lut(c, kk, c->own);
        if (rc) return rc;
    }
    return ensure_workspace(c, n, n * state_pitch((int)n), m, (int)n, k);
}

}  // namespace acc

extern "C" {

const char *acc_strerror(int code) {
    switch (code) {
    case ACC_OK: return "ok";
    case ACC_ERR_K: return "k must be 3, 4 or 5";
    case ACC_ERR_INPUT: return "malformed graph (rowptr, column range, self-loop or size)";
    case ACC_ERR_NOMEM: return "device or pinned-host allocation failed";
    case ACC_ERR_TIMEOUT: return "a bounded device wait gave up";
    case ACC_ERR_OVERFLOW: return "a count or an index would not fit its type";
    case ACC_ERR_CUDA: return "a CUDA runtime call failed";
    case ACC_ERR_ARG: return "null pointer, bad handle or bad option";
    case ACC_ERR_TOO_LARGE: return "n above ACC_MAX_N (ACC_MAX_N_SPARSE in the count mode)";
    case ACC_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown error";
    }
}

int acc_motif_num_classes(int k) { return valid_k(k) ? num_classes(k) : ACC_ERR_K; }

int acc_ctx_create(acc_ctx **out, int device) {
    if (!out) return ACC_ERR_ARG;
    *out = nullptr;
    acc_ctx *c = new (std::nothrow) acc_ctx();
    if (!c) return ACC_ERR_NOMEM;
    c->device = device;
    if (!ok(cudaSetDevice(device)) ||
        !ok(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device)) ||
        !ok(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking)) ||
        !ok(cudaMallocHost(&c->status_host, sizeof(int)))) {
        cudaGetLastError();
        acc_ctx_destroy(c);
        return ACC_ERR_CUDA;
    }
    *out = c;
    return ACC_OK;
}

void acc_ctx_destroy(acc_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    release_luts(c);
    cudaFree(c->state);
    cudaFree(c->deg);
    cudaFree(c->lo);
    cudaFree(c->nptr);
    cudaFree(c->label);
    cudaFree(c->deg_in);
    cudaFree(c->tiles);
    cudaFree(c->f5_pre);
    cudaFree(c->occ);
    cudaFree(c->nbr);
    cudaFree(c->src);
    cudaFree(c->rev);
    cudaFree(c->nh);
    cudaFree(c->sp_raw);
    cudaFree(c->sp_merged);
    cudaFree(c->sp_roff);
    cudaFree(c->sp_big);
    if (c->maxdeg_host) cudaFreeHost(c->maxdeg_host);
    cudaFree(c->info);
    cudaFree(c->queue);
    cudaFree(c->scratch);
    cudaFree(c->status_dev);
    cudaFree(c->meta_dev);
    cudaFree(c->gid);
    if (c->cg_exec) cudaGraphExecDestroy(c->cg_exec);
    cudaFree(c->rand_meta);
    cudaFree(c->rand_rows);
    cudaFree(c->rand_bits);
    cudaFree(c->rand_rpart);
    cudaFree(c->rand_pts);
    cudaFree(c->h2d_rowptr);
    cudaFree(c->h2d_col);
    cudaFree(c->h2d_counts);
    for (int i = 0; i < 4; i++)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->status_host) cudaFreeHost(c->status_host);
    if (c->own) cudaStreamDestroy(c->own);
    cudaGetLastError();
    delete c;
}

int acc_motif_prepare(acc_ctx *c, int k, void *stream) {
    if (!c) return ACC_ERR_ARG;
    if (!valid_k(k)) return ACC_ERR_K;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_lut(c, k, s);
    if (rc) return rc;
    return ok(cudaStreamSynchronize(s)) ? ACC_OK : ACC_ERR_CUDA;
}

int acc_motif_count(acc_ctx *c, const int64_t *d_rowptr, const int32_t *d_col, int32_t n, int64_t m, int k,
                    void *stream, int64_t *d_counts, int32_t *d_status) {
    return count_impl(c, d_rowptr, d_col, n, m, k, (cudaStream_t)stream, d_counts, d_status);
}

int acc_motif_count_host(acc_ctx *c, const int64_t *h_rowptr, const int32_t *h_col, int32_t n, int64_t m, int k,
                         int64_t *h_counts) {
    if (!c || !h_rowptr || !h_counts || (m > 0 && !h_col)) return ACC_ERR_ARG;
    if (!valid_k(k)) return ACC_ERR_K;
    if (n < 0 || m < 0 || m >= (1ll << 31)) return ACC_ERR_INPUT;
    if (size_check(c, n)) return ACC_ERR_TOO_LARGE;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    int rc;
    size_t cnt_cap = c->h2d_counts ? 9364 : 0;
    if ((rc = grow(&c->h2d_rowptr, &c->h2d_rowptr_cap, (size_t)n + 1))) return rc;
    if ((rc = grow(&c->h2d_col, &c->h2d_col_cap, (size_t)m + 1))) return rc;
    if ((rc = grow(&c->h2d_counts, &cnt_cap, 9364))) return rc;
    cudaStream_t s = c->own;
    if (!ok(cudaMemcpyAsync(c->h2d_rowptr, h_rowptr, ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, s)))
        return ACC_ERR_CUDA;
    if (m > 0 && !ok(cudaMemcpyAsync(c->h2d_col, h_col, (size_t)m * 4, cudaMemcpyHostToDevice, s)))
        return ACC_ERR_CUDA;
    rc = count_impl(c, reinterpret_cast<const int64_t *>(c->h2d_rowptr), c->h2d_col, n, m, k, s,
                    reinterpret_cast<int64_t *>(c->h2d_counts), c->status_dev);
    if (rc) return rc;
    if (!ok(cudaMemcpyAsync(h_counts, c->h2d_counts, (size_t)num_classes(k) * 8, cudaMemcpyDeviceToHost, s)))
        return ACC_ERR_CUDA;
    if (!ok(cudaMemcpyAsync(c->status_host, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s)))
        return ACC_ERR_CUDA;
    if (!ok(cudaStreamSynchronize(s))) return ACC_ERR_CUDA;
    return *c->status_host;
}

int acc_motif_batch_prepare(acc_ctx *c, const acc_graph_desc *graphs, int32_t B, int k, void *stream) {
    if (!c || (B > 0 && !graphs) || B < 0) return ACC_ERR_ARG;
    if (!valid_k(k)) return ACC_ERR_K;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    c->batch_ready = false;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<GMeta> metas((size_t)B);
    long long NV = 0, words = 0, arcs = 0;
    int max_n = 0;
    for (int g = 0; g < B; g++) {
        const acc_graph_desc &d = graphs[g];
        if (!d.rowptr || (d.m > 0 && !d.col)) return ACC_ERR_ARG;
        if (d.n < 0 || d.m < 0 || d.m >= (1ll << 31)) return ACC_ERR_INPUT;
        if (size_check(c, d.n)) return ACC_ERR_TOO_LARGE;
        GMeta &mt = metas[(size_t)g];
        mt.rowptr = reinterpret_cast<const long long *>(d.rowptr);
        mt.col = d.col;
        mt.m = d.m;
        mt.n = d.n;
        mt.pitch = state_pitch(d.n);
        mt.soff = words;
        mt.moff = arcs;
        mt.voff = (int)NV;
        words += (long long)d.n * mt.pitch;
        NV += d.n;
        arcs += d.m;
        if (d.n > max_n) max_n = d.n;
        if (NV >= (1ll << 31) || arcs >= (1ll << 31)) return ACC_ERR_OVERFLOW;
    }
    // an earlier run on this stream (enqueued only, when it had a status
    // word) may still read the descriptors and graph ids rewritten below;
    // the pageable copy would not wait for it
    if (!ok(cudaStreamSynchronize(s))) return ACC_ERR_CUDA;
    int rc = ensure_lut(c, k, s);
    if (rc) return rc;
    if ((rc = ensure_workspace(c, NV, sparse_build(c, max_n) ? 0 : words, arcs, max_n, k))) return rc;
    if ((rc = grow(&c->meta_dev, &c->meta_cap, (size_t)B + 1))) return rc;
    if ((rc = grow(&c->gid, &c->gid_cap, (size_t)NV + 1))) return rc;
    if (B > 0 && !ok(cudaMemcpy(c->meta_dev, metas.data(), sizeof(GMeta) * (size_t)B, cudaMemcpyHostToDevice)))
        return ACC_ERR_CUDA;
    GSet gs = {};
    if (B == 1) gs.one = metas[0];
    gs.many = c->meta_dev;
    gs.gid = c->gid;
    gs.B = B;
    gs.NV = NV;
    gs.M = arcs;
    if ((rc = launch_graph_ids(gs, c->gid, s)) < 0) return rc;
    if (!ok(cudaStreamSynchronize(s))) return ACC_ERR_CUDA;
    c->batch_set = gs;
    c->batch_k = k;
    c->batch_words = words;
    c->batch_arcs = arcs;
    c->batch_max_n = max_n;
    c->batch_ready = true;
    return ACC_OK;
}

int acc_motif_batch_run(acc_ctx *c, void *stream, int64_t *d_counts, int32_t *d_status) {
    if (!c || !d_counts || !c->batch_ready) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->batch_set.B == 0) return ACC_OK;
    int rc = batch_workspace(c);
    if (rc) return rc;
    int *status = d_status ? d_status : c->status_dev;
    rc = run_set(c, c->batch_set, c->batch_max_n, c->batch_k, true, s, d_counts, status);
    if (rc) return rc;
    return finish(c, s, d_status);
}

int acc_motif_count_batch(acc_ctx *c, const acc_graph_desc *graphs, int32_t B, int k, void *stream,
                          int64_t *d_counts, int32_t *d_status) {
    const int rc = acc_motif_batch_prepare(c, graphs, B, k, stream);
    if (rc) return rc;
    return acc_motif_batch_run(c, stream, d_counts, d_status);
}

int acc_motif_zscores(const int64_t *d_counts, int32_t groups, int32_t group_size, int k, void *stream,
                      double *d_z) {
    if (!valid_k(k)) return ACC_ERR_K;
    if (groups < 0 || group_size < 2) return ACC_ERR_ARG;
    if (groups > 0 && (!d_counts || !d_z)) return ACC_ERR_ARG;
    const int rc = launch_zscores(reinterpret_cast<const long long *>(d_counts), groups, group_size, num_classes(k),
                                  d_z, (cudaStream_t)stream);
    return rc < 0 ? rc : ACC_OK;
}

int acc_swap_randomise(acc_ctx *c, const acc_graph_desc *graphs, int32_t G, int32_t R, int64_t attempts_per_arc,
                       const uint64_t *seeds, int mode, void *stream, int32_t *d_out, int64_t *d_accepted,
                       int32_t *d_status) {
    if (!c || G < 0 || R < 0 || attempts_per_arc < 0) return ACC_ERR_ARG;
    if (mode != ACC_RAND_SWAP && mode != ACC_RAND_MUTUAL) return ACC_ERR_ARG;
    if (G > 0 && (!graphs || !seeds)) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<RGraph> metas((size_t)G);
    long long M = 0, NV = 0, bwords = 0;
    for (int g = 0; g < G; g++) {
        const acc_graph_desc &d = graphs[g];
        if (!d.rowptr || (d.m > 0 && !d.col)) return ACC_ERR_ARG;
        if (d.n < 0 || d.m < 0 || d.m >= (1ll << 31) || (d.n == 0 && d.m > 0)) return ACC_ERR_INPUT;
        if (d.m > 0 && attempts_per_arc > (1ll << 62) / d.m) return ACC_ERR_OVERFLOW;
        RGraph &rg = metas[(size_t)g];
        rg.rowptr = reinterpret_cast<const long long *>(d.rowptr);
        rg.col = d.col;
        rg.m = d.m;
        rg.n = d.n;
        rg.moff = M;
        rg.ooff = M * (long long)R;
        rg.attempts = attempts_per_arc * d.m;
        rg.seed = seeds[g];
        rg.voff = (int)NV;
        rg.bw = (int)((((long long)d.n + 31) / 32 + 3) & ~3ll);
        rg.boff = bwords;
        M += d.m;
        NV += d.n;
        if (M >= (1ll << 40) || NV >= (1ll << 31)) return ACC_ERR_OVERFLOW;
        const long long per_copy = (long long)d.n * rg.bw;
        bwords = (R > 0 && per_copy > ((1ll << 60) - bwords) / R) ? (1ll << 60) : bwords + per_copy * R;
    }
    if (R > 0 && M > (1ll << 62) / R) return ACC_ERR_OVERFLOW;
    if (M * (long long)R > 0 && !d_out) return ACC_ERR_ARG;
    int rc;
    const bool same = c->rand_meta && c->rand_rows && c->rand_host.size() == metas.size() &&
                      (G == 0 || memcmp(c->rand_host.data(), metas.data(), sizeof(RGraph) * (size_t)G) == 0);
    if (!same) {
        // the previous call on this stream may still read the descriptors
        if (!ok(cudaStreamSynchronize(s))) return ACC_ERR_CUDA;
        c->rand_host.clear();
        if ((rc = grow(&c->rand_meta, &c->rand_meta_cap, (size_t)G + 1))) return rc;
        if ((rc = grow(&c->rand_rows, &c->rand_rows_cap, (size_t)M + 1))) return rc;
        if (G > 0 &&
            !ok(cudaMemcpy(c->rand_meta, metas.data(), sizeof(RGraph) * (size_t)G, cudaMemcpyHostToDevice)))
            return ACC_ERR_CUDA;
        c->rand_host = metas;
    }
    // both modes run speculatively when the copies' adjacency bitmaps (and,
    // for the mutual mode, the reverse positions of the graphs' and the
    // copies' arcs) fit the limit, and half of the free device memory when
    // they must grow
    uint32_t *bits = nullptr;
    int *rpart = nullptr, *pts = nullptr;
    const bool mutual = mode == ACC_RAND_MUTUAL;
    const long long extra = mutual ? M + M * (long long)R : 0;  // ints
    if (bwords > 0 && bwords < (1ll << 60) && (bwords + extra) * 4 <= c->rand_bits_limit) {
        bool fits = (size_t)bwords <= c->rand_bits_cap &&
                    (!mutual || ((size_t)M <= c->rand_rpart_cap && (size_t)(M * (long long)R) <= c->rand_pts_cap));
        if (!fits) {
            size_t free_b = 0, total_b = 0;
            fits = ok(cudaMemGetInfo(&free_b, &total_b)) && (size_t)(bwords + extra) * 4 * 2 <= free_b;
            cudaGetLastError();
            if (fits && grow(&c->rand_bits, &c->rand_bits_cap, (size_t)bwords) != ACC_OK) fits = false;
            if (fits && mutual &&
                (grow(&c->rand_rpart, &c->rand_rpart_cap, (size_t)M) != ACC_OK ||
                 grow(&c->rand_pts, &c->rand_pts_cap, (size_t)(M * (long long)R)) != ACC_OK))
                fits = false;
        }
        if (fits) {
            bits = c->rand_bits;
            if (mutual) {
                rpart = c->rand_rpart;
                pts = c->rand_pts;
            }
        }
    }
    if (!c->status_dev && !ok(cudaMalloc(&c->status_dev, sizeof(int)))) return ACC_ERR_NOMEM;
    int *status = d_status ? d_status : c->status_dev;
    if (!ok(cudaMemsetAsync(status, 0, sizeof(int), s))) return ACC_ERR_CUDA;
    rc = launch_randomise(c->rand_meta, G, R, M, NV, mode, c->rand_rows, d_out, bits, rpart, pts,
                          reinterpret_cast<long long *>(d_accepted), status, c->num_sms, s);
    if (rc < 0) return rc;
    return finish(c, s, d_status);
}

int acc_ctx_set_launch_graphs(acc_ctx *c, int on) {
    if (!c || (on != 0 && on != 1)) return ACC_ERR_ARG;
    c->graphs = on != 0;
    return ACC_OK;
}

int acc_ctx_set_randomise_memory(acc_ctx *c, int64_t bytes) {
    if (!c || bytes < 0) return ACC_ERR_ARG;
    c->rand_bits_limit = bytes;
    return ACC_OK;
}

int acc_motif_class_code(acc_ctx *c, int k, int32_t cls, uint32_t *code) {
    if (!c || !code) return ACC_ERR_ARG;
    if (!valid_k(k)) return ACC_ERR_K;
    if (cls < 0 || cls >= num_classes(k)) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    int rc = ensure_lut(c, k, c->own);
    if (rc) return rc;
    *code = c->class_code_host[k][cls];
    return ACC_OK;
}

int acc_motif_classify_code(acc_ctx *c, int k, uint32_t code, int32_t *cls) {
    if (!c || !cls) return ACC_ERR_ARG;
    if (!valid_k(k)) return ACC_ERR_K;
    if (code >= (1u << code_bits(k))) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    int rc = ensure_lut(c, k, c->own);
    if (rc) return rc;
    *cls = c->lut_host[k][code];
    return ACC_OK;
}

int acc_motif_copy_table(acc_ctx *c, int k, int16_t *h_table) {
    if (!c || !h_table) return ACC_ERR_ARG;
    if (!valid_k(k)) return ACC_ERR_K;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    int rc = ensure_lut(c, k, c->own);
    if (rc) return rc;
    memcpy(h_table, c->lut_host[k], (size_t(1) << code_bits(k)) * 2);
    return ACC_OK;
}

int acc_motif_last_stats(acc_ctx *c, int64_t *h_stats) {
    if (!c || !h_stats) return ACC_ERR_ARG;
    if (!c->info) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device)) || !ok(cudaDeviceSynchronize())) return ACC_ERR_CUDA;
    GraphInfo gi;
    if (!ok(cudaMemcpy(&gi, c->info, sizeof(gi), cudaMemcpyDeviceToHost))) return ACC_ERR_CUDA;
    h_stats[0] = c->last_launches;
    h_stats[1] = c->last_k == 3 ? (int64_t)c->last_units : (int64_t)gi.nnz;
    h_stats[2] = (int64_t)gi.queue_tail;
    h_stats[3] = (int64_t)(gi.nnz / 2);
    h_stats[4] = gi.maxdeg;
    h_stats[5] = c->last_blocks;
    h_stats[6] = (int64_t)gi.scanned;
    return ACC_OK;
}

int acc_ctx_set_adjacency(acc_ctx *c, int adjacency) {
    if (!c || (adjacency != ACC_ADJ_AUTO && adjacency != ACC_ADJ_DENSE && adjacency != ACC_ADJ_HASH &&
               adjacency != ACC_ADJ_SPARSE))
        return ACC_ERR_ARG;
    c->adjacency = adjacency;
    return ACC_OK;
}

int acc_ctx_set_mode(acc_ctx *c, int mode) {
    if (!c || (mode != ACC_MODE_COUNT && mode != ACC_MODE_ENUMERATE && mode != ACC_MODE_FORMULA &&
               mode != ACC_MODE_AUTO))
        return ACC_ERR_ARG;
    c->mode = mode;
    return ACC_OK;
}

int acc_ctx_set_schedule(acc_ctx *c, int64_t light, int64_t target) {
    constexpr int64_t kMax = 1ll << 40;
    if (!c || light < 0 || target < 0 || light > kMax || target > kMax) return ACC_ERR_ARG;
    c->sched_light = light;
    c->sched_target = target;
    return ACC_OK;
}

int acc_ctx_get_schedule(acc_ctx *c, int64_t *light, int64_t *target) {
    if (!c || !light || !target) return ACC_ERR_ARG;
    *light = c->sched_light > 0 ? c->sched_light : enum_default_light(3, true);
    *target = c->sched_target > 0 ? c->sched_target : enum_default_target(3, true);
    return ACC_OK;
}

int acc_motif_batch_autotune(acc_ctx *c, void *stream, int64_t *h_light, int64_t *h_target, float *h_ms) {
    if (!c || !c->batch_ready) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const long long B = c->batch_set.B;
    const long long light0 = c->sched_light, target0 = c->sched_target;
    // candidate schedules: light units from a warp each up to large units,
    // heavy units cut into small or large row tiles
    const long long lights[] = {512, 2048, 8192, 32768, 131072, 1ll << 20};
    const long long targets[] = {1024, 4096, 16384};
    int64_t *counts = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = ACC_OK;
    long long best_l = 0, best_t = 0;
    float best = -1.0f;
    if (B == 0) {
        best_l = enum_default_light(c->batch_k, c->mode != ACC_MODE_ENUMERATE);
        best_t = enum_default_target(c->batch_k, c->mode != ACC_MODE_ENUMERATE);
        best = 0.0f;
        goto done;
    }
    if ((rc = batch_workspace(c))) return rc;
    if (!ok(cudaMalloc(&counts, (size_t)B * num_classes(c->batch_k) * sizeof(int64_t)))) return ACC_ERR_NOMEM;
    if (!ok(cudaEventCreate(&e0)) || !ok(cudaEventCreate(&e1))) {
        rc = ACC_ERR_CUDA;
        goto done;
    }
    for (long long l : lights) {
        for (long long t : targets) {
            c->sched_light = l;
            c->sched_target = t;
            if (!ok(cudaEventRecord(e0, s))) {
                rc = ACC_ERR_CUDA;
                goto done;
            }
            rc = run_set(c, c->batch_set, c->batch_max_n, c->batch_k, true, s, counts, c->status_dev);
            if (rc) goto done;
            float ms = 0.0f;
            if (!ok(cudaEventRecord(e1, s)) || !ok(cudaEventSynchronize(e1)) ||
                !ok(cudaEventElapsedTime(&ms, e0, e1))) {
                rc = ACC_ERR_CUDA;
                goto done;
            }
            if ((rc = finish(c, s, nullptr))) goto done;  // a failing batch fails the tuning
            if (best < 0.0f || ms < best) {
                best = ms;
                best_l = l;
                best_t = t;
            }
        }
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(counts);
    if (rc) {
        c->sched_light = light0;
        c->sched_target = target0;
        return rc;
    }
    c->sched_light = best_l;
    c->sched_target = best_t;
    if (h_light) *h_light = best_l;
    if (h_target) *h_target = best_t;
    if (h_ms) *h_ms = best;
    return ACC_OK;
}

int acc_ctx_set_timing(acc_ctx *c, int on) {
    if (!c) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device))) return ACC_ERR_CUDA;
    if (on && !c->ev[0]) {
        for (int i = 0; i < 4; i++)
            if (!ok(cudaEventCreate(&c->ev[i]))) {
                cudaGetLastError();
                return ACC_ERR_CUDA;
            }
    }
    c->timing = on != 0;
    return ACC_OK;
}

int acc_motif_last_timing(acc_ctx *c, float *h_ms) {
    if (!c || !h_ms || !c->timed_call) return ACC_ERR_ARG;
    if (!ok(cudaSetDevice(c->device)) || !ok(cudaEventSynchronize(c->ev[2]))) return ACC_ERR_CUDA;
    if (!ok(cudaEventElapsedTime(&h_ms[0], c->ev[0], c->ev[1])) ||
        !ok(cudaEventElapsedTime(&h_ms[1], c->ev[1], c->ev[2])) ||
        !ok(cudaEventElapsedTime(&h_ms[2], c->ev[1], c->ev[3])) ||
        !ok(cudaEventElapsedTime(&h_ms[3], c->ev[3], c->ev[2])))
        return ACC_ERR_CUDA;
    return ACC_OK;
}

}  // extern "C"
