// Request server: continuous batching of counting requests on one GPU.
//
// Serving form of the counter: requests (resident graph, k) arrive at any
// time; each is admitted as soon as a slot is free and its device-memory
// footprint fits the budget, so requests that arrive while others run on the
// GPU start without waiting for a batch boundary and overlap on the device.
// Each slot owns a context (workspace) and a CUDA stream; completion is
// detected with CUDA events, results are copied to pinned host memory in
// stream order.  A small graph (at most 4096 vertices) takes 1/8 of the GPU's
// persistent enumeration grid, which its few units cannot fill anyway, so
// that it runs beside a large request instead of behind it; a large graph
// takes the whole grid (capping it at 5/8 to make room for small requests
// measured slower in throughput and in tail latency at saturation).
// Admission takes the queued request with the smallest aged work estimate (or
// FIFO order).
// Host work happens only inside the caller's calls (no threads).
#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cmath>
#include <new>
#include <vector>

#include "context.cuh"

namespace {

constexpr int kSmallGraph = 4096;  // vertices; smaller graphs get the small grid share
constexpr int kSmallShare = 1, kBigShare = 8;  // eighths of the persistent grid a request takes

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Slot {
    acc_ctx *ctx = nullptr;
    cudaStream_t s = nullptr;
    int64_t *d_counts = nullptr;
    int32_t *d_status = nullptr;
    int64_t *h_counts = nullptr;  // pinned
    int32_t *h_status = nullptr;  // pinned
    cudaEvent_t ev = nullptr;
    long long req = -1;
    long long footprint = 0;  // device bytes this slot's workspace may hold
};

struct Graph {
    const int64_t *rowptr;
    const int32_t *col;
    int32_t n;
    int64_t m;
    double est[3];  // work estimate for k = 3, 4, 5: sum over v of d(v)^(k-1)
};

constexpr int64_t kEstimateCopyMax = 1ll << 26;  // arcs; larger graphs are estimated from n and m

// Work estimate of a registered graph: sum over vertices of d^(k-1), with d
// the out- plus in-degree (ESU's work grows with the (k-1)-th power of the
// degrees; the ordering of requests is all it is used for).
int estimate_work(Graph &g) {
    for (int k = 3; k <= 5; k++) {
        const double d = g.n > 0 ? 2.0 * (double)g.m / g.n : 0.0;
        g.est[k - 3] = (double)g.n * std::pow(d, k - 1);
    }
    if (g.n == 0 || g.m == 0 || g.m > kEstimateCopyMax) return ACC_OK;
    std::vector<int64_t> rp((size_t)g.n + 1);
    std::vector<int32_t> col((size_t)g.m);
    if (cudaMemcpy(rp.data(), g.rowptr, rp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(col.data(), g.col, col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return ACC_ERR_CUDA;
    }
    std::vector<double> deg((size_t)g.n, 0.0);
    for (int32_t v = 0; v < g.n; v++) {
        const int64_t b = rp[(size_t)v], e = rp[(size_t)v + 1];
        if (b < 0 || e < b || e > g.m) continue;  // malformed: the count reports it
        deg[(size_t)v] += (double)(e - b);
        for (int64_t p = b; p < e; p++)
            if (col[(size_t)p] >= 0 && col[(size_t)p] < g.n) deg[(size_t)col[(size_t)p]] += 1.0;
    }
    for (int k = 3; k <= 5; k++) {
        double s = 0.0;
        for (double d : deg) s += std::pow(d, k - 1);
        g.est[k - 3] = s;
    }
    return ACC_OK;
}

struct Req {
    int32_t graph;
    int k;
    int32_t state;
    double t_submit = 0, t_start = 0, t_done = 0;
    std::vector<int64_t> counts;
};

}  // namespace

struct acc_server {
    int device = 0;
    long long budget = 0;
    int policy = ACC_SERVE_SHORTEST;
    double aging_s = 1.0;
    std::vector<Slot> slots;
    std::vector<Graph> graphs;
    std::vector<Req> reqs;
    std::vector<long long> queue;  // request ids in submission order
};

namespace {

bool ok(cudaError_t e) { return e == cudaSuccess; }

long long used_except(const acc_server *sv, size_t skip) {
    long long t = 0;
    for (size_t i = 0; i < sv->slots.size(); i++)
        if (i != skip) t += sv->slots[i].footprint;
    return t;
}

// Completed requests leave their slots; queued requests enter free slots.
int progress(acc_server *sv) {
    for (Slot &sl : sv->slots) {
        if (sl.req < 0) continue;
        const cudaError_t q = cudaEventQuery(sl.ev);
        if (q == cudaErrorNotReady) continue;
        Req &r = sv->reqs[(size_t)sl.req];
        r.t_done = now_s();
        if (q != cudaSuccess) {
            cudaGetLastError();
            r.state = ACC_ERR_CUDA;
        } else if (*sl.h_status != 0) {
            r.state = *sl.h_status;
        } else {
            r.counts.assign(sl.h_counts, sl.h_counts + acc_motif_num_classes(r.k));
            r.state = ACC_REQ_DONE;
        }
        sl.req = -1;
    }
    while (!sv->queue.empty()) {
        bool any_free = false;
        for (const Slot &sl : sv->slots) any_free = any_free || sl.req < 0;
        if (!any_free) break;
        // the request to admit next
        size_t pick = 0;
        if (sv->policy == ACC_SERVE_SHORTEST) {
            const double t = now_s();
            double best_key = 0.0;
            for (size_t q = 0; q < sv->queue.size(); q++) {
                const Req &c = sv->reqs[(size_t)sv->queue[q]];
                const double key = sv->graphs[(size_t)c.graph].est[c.k - 3] * std::exp(-(t - c.t_submit) / sv->aging_s);
                if (q == 0 || key < best_key) {
                    best_key = key;
                    pick = q;
                }
            }
        }
        const long long id = sv->queue[pick];
        Req &r = sv->reqs[(size_t)id];
        const Graph &g = sv->graphs[(size_t)r.graph];
        // the free slot that needs the least growth and stays within budget
        int best = -1;
        long long best_fp = 0;
        for (size_t i = 0; i < sv->slots.size(); i++) {
            Slot &sl = sv->slots[i];
            if (sl.req >= 0) continue;
            const long long need = acc::ctx_footprint(sl.ctx, g.n, g.m, r.k);
            const long long fp = need > sl.footprint ? need : sl.footprint;
            if (used_except(sv, i) + fp > sv->budget) continue;
            if (best < 0 || fp < best_fp) {
                best = (int)i;
                best_fp = fp;
            }
        }
        if (best < 0) {
            bool idle = true;
            for (const Slot &sl : sv->slots) idle = idle && sl.req < 0;
            if (!idle) break;  // wait for a running request to free its slot
            // nothing runs and it still does not fit: it never will
            r.state = ACC_ERR_NOMEM;
            r.t_done = now_s();
            sv->queue.erase(sv->queue.begin() + (long)pick);
            continue;
        }
        Slot &sl = sv->slots[(size_t)best];
        sl.footprint = best_fp;
        sl.ctx->grid_num = g.n <= kSmallGraph ? kSmallShare : kBigShare;
        sl.ctx->grid_den = 8;
        r.t_start = now_s();
        const int rc = acc_motif_count(sl.ctx, g.rowptr, g.col, g.n, g.m, r.k, sl.s, sl.d_counts, sl.d_status);
        sv->queue.erase(sv->queue.begin() + (long)pick);
        if (rc != ACC_OK) {
            r.state = rc;
            r.t_done = now_s();
            continue;
        }
        if (!ok(cudaMemcpyAsync(sl.h_counts, sl.d_counts, sizeof(int64_t) * (size_t)acc_motif_num_classes(r.k),
                                cudaMemcpyDeviceToHost, sl.s)) ||
            !ok(cudaMemcpyAsync(sl.h_status, sl.d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, sl.s)) ||
            !ok(cudaEventRecord(sl.ev, sl.s))) {
            cudaGetLastError();
            r.state = ACC_ERR_CUDA;
            r.t_done = now_s();
            continue;
        }
        r.state = ACC_REQ_RUNNING;
        sl.req = id;
    }
    return ACC_OK;
}

}  // namespace

extern "C" {

int acc_server_create(acc_server **out, int device, int32_t slots, int64_t mem_budget_bytes) {
    if (!out || slots < 1 || slots > 64 || mem_budget_bytes <= 0) return ACC_ERR_ARG;
    *out = nullptr;
    acc_server *sv = new (std::nothrow) acc_server();
    if (!sv) return ACC_ERR_NOMEM;
    sv->device = device;
    sv->budget = mem_budget_bytes;
    sv->slots.resize((size_t)slots);
    for (Slot &sl : sv->slots) {
        int rc = acc_ctx_create(&sl.ctx, device);
        if (rc) {
            acc_server_destroy(sv);
            return rc;
        }
        // a slot's consecutive requests are rarely the same graph and k:
        // launch one by one rather than capture a graph per request
        acc_ctx_set_launch_graphs(sl.ctx, 0);
        if (!ok(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking)) ||
            !ok(cudaMalloc(&sl.d_counts, sizeof(int64_t) * 9364)) || !ok(cudaMalloc(&sl.d_status, sizeof(int32_t))) ||
            !ok(cudaMallocHost(&sl.h_counts, sizeof(int64_t) * 9364)) ||
            !ok(cudaMallocHost(&sl.h_status, sizeof(int32_t))) ||
            !ok(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming))) {
            cudaGetLastError();
            acc_server_destroy(sv);
            return ACC_ERR_NOMEM;
        }
    }
    *out = sv;
    return ACC_OK;
}

void acc_server_destroy(acc_server *sv) {
    if (!sv) return;
    cudaSetDevice(sv->device);
    for (Slot &sl : sv->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        acc_ctx_destroy(sl.ctx);
        cudaFree(sl.d_counts);
        cudaFree(sl.d_status);
        if (sl.h_counts) cudaFreeHost(sl.h_counts);
        if (sl.h_status) cudaFreeHost(sl.h_status);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    cudaGetLastError();
    delete sv;
}

int acc_server_add_graph(acc_server *sv, const int64_t *d_rowptr, const int32_t *d_col, int32_t n, int64_t m,
                         int32_t *graph_id) {
    if (!sv || !d_rowptr || !graph_id || (m > 0 && !d_col)) return ACC_ERR_ARG;
    if (n < 0 || m < 0 || m >= (1ll << 31)) return ACC_ERR_INPUT;
    if (n > ACC_MAX_N_SPARSE) return ACC_ERR_TOO_LARGE;  // requests are counted in the count mode
    Graph g{d_rowptr, d_col, n, m, {0.0, 0.0, 0.0}};
    if (!ok(cudaSetDevice(sv->device))) return ACC_ERR_CUDA;
    const int rc = estimate_work(g);
    if (rc) return rc;
    sv->graphs.push_back(g);
    *graph_id = (int32_t)sv->graphs.size() - 1;
    return ACC_OK;
}

int acc_server_set_policy(acc_server *sv, int policy, double aging_s) {
    if (!sv || (policy != ACC_SERVE_FIFO && policy != ACC_SERVE_SHORTEST) || !(aging_s > 0.0)) return ACC_ERR_ARG;
    sv->policy = policy;
    sv->aging_s = aging_s;
    return ACC_OK;
}

int acc_server_reserve(acc_server *sv) {
    if (!sv) return ACC_ERR_ARG;
    long long n = 0, m = 0;
    for (const Graph &g : sv->graphs) {
        if (g.n > n) n = g.n;
        if (g.m > m) m = g.m;
    }
    for (size_t i = 0; i < sv->slots.size(); i++) {
        Slot &sl = sv->slots[i];
        long long fp = 0;
        for (int k = 3; k <= 5; k++) {
            const long long f = acc::ctx_footprint(sl.ctx, n, m, k);
            if (f > fp) fp = f;
        }
        if (used_except(sv, i) + fp > sv->budget) continue;  // this slot grows on demand
        for (int k = 3; k <= 5; k++) {
            const int rc = acc::ctx_reserve(sl.ctx, n, m, k);
            if (rc) return rc;
        }
        if (fp > sl.footprint) sl.footprint = fp;
    }
    return ok(cudaDeviceSynchronize()) ? ACC_OK : ACC_ERR_CUDA;
}

int acc_server_submit(acc_server *sv, int32_t graph_id, int k, int64_t *request_id) {
    if (!sv || !request_id) return ACC_ERR_ARG;
    if (graph_id < 0 || (size_t)graph_id >= sv->graphs.size()) return ACC_ERR_ARG;
    if (k < 3 || k > 5) return ACC_ERR_K;
    Req r;
    r.graph = graph_id;
    r.k = k;
    r.state = ACC_REQ_QUEUED;
    r.t_submit = now_s();
    sv->reqs.push_back(r);
    *request_id = (int64_t)sv->reqs.size() - 1;
    sv->queue.push_back(*request_id);
    return progress(sv);
}

int acc_server_progress(acc_server *sv, int32_t *running, int32_t *queued) {
    if (!sv) return ACC_ERR_ARG;
    const int rc = progress(sv);
    int run = 0;
    for (const Slot &sl : sv->slots) run += sl.req >= 0;
    if (running) *running = run;
    if (queued) *queued = (int32_t)sv->queue.size();
    return rc;
}

int acc_server_poll(acc_server *sv, int64_t request_id, int32_t *state, int64_t *h_counts, double *latency_s) {
    if (!sv || !state || request_id < 0 || (size_t)request_id >= sv->reqs.size()) return ACC_ERR_ARG;
    const int rc = progress(sv);
    const Req &r = sv->reqs[(size_t)request_id];
    *state = r.state;
    if (r.state == ACC_REQ_DONE && h_counts)
        for (size_t i = 0; i < r.counts.size(); i++) h_counts[i] = r.counts[i];
    if (latency_s) *latency_s = (r.state == ACC_REQ_DONE || r.state < 0) ? r.t_done - r.t_submit : -1.0;
    return rc;
}

int acc_server_drain(acc_server *sv) {
    if (!sv) return ACC_ERR_ARG;
    for (;;) {
        const int rc = progress(sv);
        if (rc) return rc;
        bool busy = !sv->queue.empty();
        for (const Slot &sl : sv->slots) busy = busy || sl.req >= 0;
        if (!busy) return ACC_OK;
        for (const Slot &sl : sv->slots)
            if (sl.req >= 0) {
                cudaEventSynchronize(sl.ev);
                break;
            }
    }
}

}  // extern "C"
