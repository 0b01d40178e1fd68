// Enumeration kernels: every connected induced k-subset exactly once,
// classified by the code -> class table and counted in shared-memory
// histograms.
//
// Which subsets: the problem of the paper (Problems Motifs-3/4/5), i.e. the
// k-sets S whose undirected version G*[S] is connected (Notation section).
// The paper counts them through per-vertex / per-edge / per-triple
// combinatorial formulas; here they are enumerated, which makes the cost
// proportional to the count but lets one kernel serve every class.
//
// Exactly-once rule (ESU, Wernicke 2006, the FANMOD algorithm the paper
// cites): a set is grown from its smallest vertex v (the root).  The current
// set Vsub carries an extension list Vext whose members all exceed v; taking
// the member at position j into Vsub leaves Vext[j+1..] plus the exclusive
// neighbours of that member (neighbours above v that are neither in Vsub nor
// adjacent to it) as the next extension list.  The last two levels are the
// hot loop, run warp-parallel over all leaves at once:
//
//   prefix P = the first k-2 vertices, E = its extension list, then the
//   leaves are  (a) P + {E[j], E[l]}  for j < l          ("pair leaves")
//               (b) P + {E[j], u}     for u an exclusive neighbour of E[j]
//
// A leaf's code is the prefix code OR two table entries (the states of E[j]
// and of the last vertex to the prefix, kept in each E entry) OR the state
// of the last pair, found with one probe of the pair-state matrix (a) or read
// from the neighbour entry (b).
//
// Work units: k=3 one unit per root v; k=4 and k=5 one unit per arc position
// of the G* CSR, i.e. per (v, w1) with w1 > v.  Phase 1 runs every unit whose
// estimated work is small and splits the others into row ranges of their
// extension list, pushed to a queue that phase 2 (a second launch) drains.
#include "common.cuh"

namespace acc {

namespace {

constexpr int kCap34 = 1024;           // per-warp shared extension entries, k = 3, 4
constexpr int kCap5 = 512;             // per-warp shared entries per list, k = 5
constexpr int kGrab = 16;              // base units per atomic grab
constexpr long long kTarget = 1 << 15; // work per pushed chunk
constexpr uint32_t kDrainAt = 1u << 30;

struct Tables {
    uint32_t t2[64];   // code bits of slot k-2 from its states to the prefix slots
    uint32_t t3[64];   // code bits of slot k-1 from its states to the prefix slots
    uint32_t s2[16];   // k = 5: code bits of slot 2 from its states to slots 0, 1
    uint32_t tp[4];    // code bits of the pair (k-2, k-1) from state(x_{k-2}, x_{k-1})
    uint32_t p01[4];   // code bits of the pair (0, 1) from state(v, w1)
};

template <int K>
struct Layout {
    static constexpr int NB = K * (K - 1);
    static constexpr int NCLS = num_classes(K);
    static constexpr bool SMEM_LUT = K <= 4;
    static constexpr int CAP = K == 5 ? kCap5 : kCap34;
    static constexpr int LISTS = K == 5 ? 2 : 1;
    static constexpr size_t tables = (sizeof(Tables) + 15) & ~size_t(15);
    static constexpr size_t lut = SMEM_LUT ? (((size_t(1) << NB) * 2 + 15) & ~size_t(15)) : 0;
    static constexpr size_t pending = 16;
    static constexpr size_t hist = (K == 5 ? size_t(NCLS) * 4 : size_t(kWarpsPerBlock) * NCLS * 4 + 15) & ~size_t(15);
    static constexpr size_t ebuf = size_t(kWarpsPerBlock) * LISTS * CAP * 4;
    static constexpr size_t total = tables + lut + pending + hist + ebuf;
};

__device__ __forceinline__ uint32_t slot_bits(int K, int slot, uint32_t svec, int nprefix) {
    uint32_t out = 0;
    for (int i = 0; i < nprefix; i++) {
        const uint32_t s = (svec >> (2 * i)) & 3u;
        if (s & 1u) out |= 1u << code_bit(K, i, slot);
        if (s & 2u) out |= 1u << code_bit(K, slot, i);
    }
    return out;
}

__device__ __forceinline__ uint32_t pair_bits(int K, int a, int b, uint32_t s) {
    return ((s & 1u) << code_bit(K, a, b)) | (((s >> 1) & 1u) << code_bit(K, b, a));
}

__device__ __forceinline__ uint32_t probe(const uint32_t *__restrict__ st, long long pitch, uint32_t a, uint32_t b) {
    return (__ldg(st + (long long)a * pitch + (b >> 4)) >> ((b & 15u) << 1)) & 3u;
}

// First position of N*(x) (entries (u << 2) | s, sorted) with u > root.
__device__ __forceinline__ int first_above(const uint32_t *__restrict__ nbr, long long base, int d, uint32_t root) {
    const uint32_t key = (root + 1u) << 2;
    int lo = 0, hi = d;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(nbr + base + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int excl_scan(int x, int lane, int *total) {
    int incl = x;
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    *total = __shfl_sync(kFull, incl, kWarp - 1);
    return incl - x;
}

__device__ __forceinline__ long long incl_scan64(long long x, int lane) {
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
        const long long y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// Largest lane r with pre[r] <= t (pre non-decreasing across lanes): the row
// that flattened leaf index t falls in.
__device__ __forceinline__ int lb_search(int pre, int t) {
    int r = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const int c = __shfl_sync(kFull, pre, r + s);
        if (c <= t) r += s;
    }
    return r;
}

// Histogram sink: k <= 4 one private histogram per warp, k = 5 one per block.
template <int K>
struct Sink {
    uint32_t *hist;
    const int16_t *lut;
    unsigned long long *counts;
    uint32_t *pending;  // k = 5: block-wide increments since the last drain
    uint32_t since;     // k <= 4: this warp's increments since its last drain
    int *status;

    __device__ __forceinline__ void bump(uint32_t code) {
        const int cls = Layout<K>::SMEM_LUT ? (int)lut[code] : (int)__ldg(lut + code);
        if (cls >= 0) atomicAdd(&hist[cls], 1u);
        else set_status(status, ACC_ERR_INTERNAL);
    }

    // Called by the whole warp after each batch of at most `tot` bumps.
    __device__ __forceinline__ void after_batch(uint32_t tot, int lane) {
        if (K <= 4) {
            since += tot;
            if (since >= kDrainAt) {
                __syncwarp();
                for (int c = lane; c < Layout<K>::NCLS; c += kWarp) {
                    const uint32_t v = hist[c];
                    if (v) {
                        hist[c] = 0;
                        atomicAdd(&counts[c], (unsigned long long)v);
                    }
                }
                __syncwarp();
                since = 0;
            }
        } else {
            uint32_t old = 0;
            __threadfence_block();
            if (lane == 0) old = atomicAdd(pending, tot);
            old = __shfl_sync(kFull, old, 0);
            if (old < kDrainAt && old + tot >= kDrainAt) {
                for (int c = lane; c < Layout<K>::NCLS; c += kWarp) {
                    const uint32_t v = atomicExch(&hist[c], 0u);
                    if (v) atomicAdd(&counts[c], (unsigned long long)v);
                }
                __syncwarp();
                if (lane == 0) atomicSub(pending, old + tot);
            }
        }
    }
};

struct Scratch {
    uint32_t *buf[2];  // shared-memory lists (buf[1] only for k = 5)
    uint32_t *ovf[2];  // global overflow lists of this warp
    int cap;
};

// The last two ESU levels over extension list E[0..B) for rows [jlo, jend).
template <int K>
__device__ __forceinline__ void leaves(const EnumArgs &a, const Tables &tb, Sink<K> &sink, const uint32_t *E,
                                       int B, int jlo, int jend, const uint32_t *pm, uint32_t pcode,
                                       uint32_t root, int lane) {
    // (a) pair leaves P + {E[j], E[l]}, j < l
    for (int jb = jlo; jb < jend; jb += kWarp) {
        const int j = jb + lane;
        const bool ok = j < jend;
        const uint32_t ej = ok ? E[j] : 0u;
        const int cnt = ok ? (B - 1 - j) : 0;
        int tot;
        const int pre = excl_scan(cnt, lane, &tot);
        const uint32_t cj = pcode | tb.t2[ej & 63u];
        for (int t0 = 0; t0 < tot; t0 += kWarp) {
            const int t = t0 + lane;
            const int r = lb_search(pre, t);
            const uint32_t cr = __shfl_sync(kFull, cj, r);
            const uint32_t xr = __shfl_sync(kFull, ej, r) >> 6;
            const int pr = __shfl_sync(kFull, pre, r);
            if (t < tot) {
                const uint32_t ey = E[jb + r + 1 + (t - pr)];
                const uint32_t s = probe(a.state, a.pitch, xr, ey >> 6);
                sink.bump(cr | tb.t3[ey & 63u] | tb.tp[s]);
            }
        }
        sink.after_batch((uint32_t)tot, lane);
    }
    // (b) exclusive leaves P + {E[j], u}, u a neighbour of E[j] above the
    //     root and adjacent to no prefix vertex
    for (int jb = jlo; jb < jend; jb += kWarp) {
        const int j = jb + lane;
        uint32_t ej = 0;
        long long base = 0;
        int cnt = 0;
        if (j < jend) {
            ej = E[j];
            const uint32_t x = ej >> 6;
            const long long nb = a.nptr[x];
            const int d = a.deg[x];
            const int st = first_above(a.nbr, nb, d, root);
            base = nb + st;
            cnt = d - st;
        }
        int tot;
        const int pre = excl_scan(cnt, lane, &tot);
        const uint32_t cj = pcode | tb.t2[ej & 63u];
        for (int t0 = 0; t0 < tot; t0 += kWarp) {
            const int t = t0 + lane;
            const int r = lb_search(pre, t);
            const uint32_t cr = __shfl_sync(kFull, cj, r);
            const long long br = __shfl_sync(kFull, base, r);
            const int pr = __shfl_sync(kFull, pre, r);
            if (t < tot) {
                const uint32_t ue = __ldg(a.nbr + br + (t - pr));
                const uint32_t u = ue >> 2;
                bool excl = true;
#pragma unroll
                for (int i = 0; i < K - 2; i++) excl = excl && probe(a.state, a.pitch, pm[i], u) == 0u;
                if (excl) sink.bump(cr | tb.tp[ue & 3u]);
            }
        }
        sink.after_batch((uint32_t)tot, lane);
    }
}

// Build the list of (prefix, extension) for k >= 4 from arc position p:
// v = row of p, w1 = N*(v)[p - nptr[v]] > v; E = N*(v) after w1, then the
// exclusive neighbours of w1 (above v, not adjacent to v).  Entry:
// (x << 6) | state(v, x) | state(w1, x) << 2.  Returns B, or -1 if p is not
// a unit (its neighbour is below v).
__device__ __forceinline__ int build_level2(const EnumArgs &a, long long p, int v, uint32_t *out_w1,
                                            uint32_t *out_s01, const Scratch &sc, int which, uint32_t **E_out,
                                            int lane) {
    const long long rb = a.nptr[v];
    const int t = (int)(p - rb);
    if (t < a.lo[v]) return -1;
    const uint32_t e = __ldg(a.nbr + p);
    const uint32_t w1 = e >> 2;
    const int dv = a.deg[v], dw = a.deg[w1];
    const int A = dv - t - 1;
    const long long ub = (long long)A + dw;
    uint32_t *E = ub <= sc.cap ? sc.buf[which] : sc.ovf[which];
    for (int q = lane; q < A; q += kWarp) {
        const uint32_t xe = __ldg(a.nbr + rb + t + 1 + q);
        const uint32_t x = xe >> 2;
        E[q] = (x << 6) | (xe & 3u) | (probe(a.state, a.pitch, w1, x) << 2);
    }
    const long long wb = a.nptr[w1];
    int pos = A;
    for (int q0 = first_above(a.nbr, wb, dw, (uint32_t)v); q0 < dw; q0 += kWarp) {
        const int q = q0 + lane;
        uint32_t ue = 0;
        bool keep = false;
        if (q < dw) {
            ue = __ldg(a.nbr + wb + q);
            keep = probe(a.state, a.pitch, (uint32_t)v, ue >> 2) == 0u;
        }
        const unsigned ball = __ballot_sync(kFull, keep);
        if (keep) E[pos + __popc(ball & ((1u << lane) - 1u))] = ((ue >> 2) << 6) | ((ue & 3u) << 2);
        pos += __popc(ball);
    }
    __syncwarp();
    *out_w1 = w1;
    *out_s01 = e & 3u;
    *E_out = E;
    return pos;
}

// Split rows [0, B) with per-row work work(j) into chunks of about kTarget;
// push every chunk but the first to the queue.  Returns the end of the first
// chunk; *rest_lo is where rows the full queue could not take begin (B if
// none).
template <typename WorkFn>
__device__ int split_rows(const EnumArgs &a, uint32_t unit, int B, WorkFn work, int *rest_lo, int lane) {
    int cur = 0, first_end = -1;
    long long acc = 0;
    *rest_lo = B;
    bool full = false;
    for (int jb = 0; jb < B && !full; jb += kWarp) {
        const int j = jb + lane;
        const long long w = j < B ? work(j) : 0;
        const long long incl = incl_scan64(w, lane);
        const long long btot = __shfl_sync(kFull, incl, kWarp - 1);
        long long used = 0;
        for (;;) {
            const unsigned ball = __ballot_sync(kFull, j < B && acc + incl - used >= kTarget);
            if (!ball) {
                acc += btot - used;
                break;
            }
            const int r = __ffs(ball) - 1;
            const int end = jb + r + 1;
            if (first_end < 0) {
                first_end = end;
            } else {
                unsigned long long idx = 0;
                if (lane == 0) idx = atomicAdd(&a.info->queue_tail, 1ull);
                idx = __shfl_sync(kFull, idx, 0);
                if (idx < a.queue_cap) {
                    if (lane == 0) a.queue[idx] = make_uint4(unit, (uint32_t)cur, (uint32_t)end, 0u);
                } else {
                    *rest_lo = cur;
                    full = true;
                    break;
                }
            }
            cur = end;
            used = __shfl_sync(kFull, incl, r);
            acc = 0;
        }
    }
    if (!full && cur < B) {
        if (first_end < 0) {
            first_end = B;
        } else {
            unsigned long long idx = 0;
            if (lane == 0) idx = atomicAdd(&a.info->queue_tail, 1ull);
            idx = __shfl_sync(kFull, idx, 0);
            if (idx < a.queue_cap) {
                if (lane == 0) a.queue[idx] = make_uint4(unit, (uint32_t)cur, (uint32_t)B, 0u);
            } else {
                *rest_lo = cur;
            }
        }
    }
    if (first_end < 0) first_end = B;
    return first_end;
}

__device__ __forceinline__ int row_of(const long long *__restrict__ nptr, int n, long long p) {
    int lo = 0, hi = n - 1;  // largest v with nptr[v] <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (nptr[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int K>
__device__ void process_unit(const EnumArgs &a, const Tables &tb, Sink<K> &sink, const Scratch &sc,
                             uint32_t unit, int v, int jlo, int jhi, bool phase1, int lane) {
    if (K == 3) {
        // prefix {v}; E = neighbours of v above v, entry (x << 6) | state(v, x)
        const int dv = a.deg[v], l = a.lo[v];
        const int B = dv - l;
        if (B <= 0) return;
        uint32_t *E = B <= sc.cap ? sc.buf[0] : sc.ovf[0];
        const long long rb = a.nptr[v] + l;
        for (int q = lane; q < B; q += kWarp) {
            const uint32_t xe = __ldg(a.nbr + rb + q);
            E[q] = ((xe >> 2) << 6) | (xe & 3u);
        }
        __syncwarp();
        int rest = B;
        if (phase1) {
            const long long ub = (long long)B * (B - 1) / 2 + (long long)B * a.info->maxdeg;
            if (ub > kTarget)
                jhi = split_rows(a, unit, B, [&](int j) { return (long long)(B - 1 - j) + a.deg[E[j] >> 6] + 1; },
                                 &rest, lane);
        }
        const uint32_t pm[1] = {(uint32_t)v};
        leaves<K>(a, tb, sink, E, B, jlo, min(jhi, B), pm, 0u, (uint32_t)v, lane);
        if (rest < B) leaves<K>(a, tb, sink, E, B, rest, B, pm, 0u, (uint32_t)v, lane);
        __syncwarp();
        return;
    }
    uint32_t w1, s01, *E2;
    const int B2 = build_level2(a, unit, v, &w1, &s01, sc, 0, &E2, lane);
    if (B2 <= 0) return;
    int rest = B2;
    if (K == 4) {
        if (phase1) {
            const long long ub = (long long)B2 * (B2 - 1) / 2 + (long long)B2 * a.info->maxdeg;
            if (ub > kTarget)
                jhi = split_rows(a, unit, B2, [&](int j) { return (long long)(B2 - 1 - j) + a.deg[E2[j] >> 6] + 1; },
                                 &rest, lane);
        }
        const uint32_t pm[2] = {(uint32_t)v, w1};
        const uint32_t pcode = tb.p01[s01];
        leaves<K>(a, tb, sink, E2, B2, jlo, min(jhi, B2), pm, pcode, (uint32_t)v, lane);
        if (rest < B2) leaves<K>(a, tb, sink, E2, B2, rest, B2, pm, pcode, (uint32_t)v, lane);
        __syncwarp();
        return;
    }
    // K == 5: one more level.  Row j2 of E2 gives w2 and the list E3.
    if (phase1) {
        jhi = split_rows(a, unit, B2,
                         [&](int j) {
                             const long long b = (long long)(B2 - 1 - j) + a.deg[E2[j] >> 6];
                             return b * (b - 1) / 2 + 4 * b + 1;
                         },
                         &rest, lane);
    }
    const uint32_t pc01 = tb.p01[s01];
    for (int pass = 0; pass < 2; pass++) {
        const int r0 = pass == 0 ? jlo : rest;
        const int r1 = pass == 0 ? min(jhi, B2) : B2;
        for (int j2 = r0; j2 < r1; j2++) {
            const uint32_t e2 = E2[j2];
            const uint32_t w2 = e2 >> 6;
            const uint32_t pcode = pc01 | tb.s2[e2 & 15u];
            const int A3 = B2 - 1 - j2;
            const int dw = a.deg[w2];
            const long long ub = (long long)A3 + dw;
            uint32_t *E3 = ub <= sc.cap ? sc.buf[1] : sc.ovf[1];
            for (int q = lane; q < A3; q += kWarp) {
                const uint32_t xe = E2[j2 + 1 + q];
                const uint32_t x = xe >> 6;
                E3[q] = (x << 6) | (xe & 15u) | (probe(a.state, a.pitch, w2, x) << 4);
            }
            const long long wb = a.nptr[w2];
            int pos = A3;
            for (int q0 = first_above(a.nbr, wb, dw, (uint32_t)v); q0 < dw; q0 += kWarp) {
                const int q = q0 + lane;
                uint32_t ue = 0;
                bool keep = false;
                if (q < dw) {
                    ue = __ldg(a.nbr + wb + q);
                    const uint32_t u = ue >> 2;
                    keep = probe(a.state, a.pitch, (uint32_t)v, u) == 0u && probe(a.state, a.pitch, w1, u) == 0u;
                }
                const unsigned ball = __ballot_sync(kFull, keep);
                if (keep) E3[pos + __popc(ball & ((1u << lane) - 1u))] = ((ue >> 2) << 6) | ((ue & 3u) << 4);
                pos += __popc(ball);
            }
            __syncwarp();
            const uint32_t pm[3] = {(uint32_t)v, w1, w2};
            leaves<K>(a, tb, sink, E3, pos, 0, pos, pm, pcode, (uint32_t)v, lane);
            __syncwarp();
        }
        if (rest >= B2) break;
    }
}

template <int K>
__global__ void __launch_bounds__(kThreads, K == 5 ? 3 : 4) k_enum(EnumArgs a, int phase) {
    using L = Layout<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    Tables &tb = *reinterpret_cast<Tables *>(smem);
    int16_t *lut_s = reinterpret_cast<int16_t *>(smem + L::tables);
    uint32_t *pending = reinterpret_cast<uint32_t *>(smem + L::tables + L::lut);
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + L::tables + L::lut + L::pending);
    uint32_t *ebuf = reinterpret_cast<uint32_t *>(smem + L::tables + L::lut + L::pending + L::hist);
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;

    // tables: slot codes for every state vector, pair codes
    for (int i = tid; i < 64; i += blockDim.x) {
        tb.t2[i] = slot_bits(K, K - 2, (uint32_t)i, K - 2);
        tb.t3[i] = slot_bits(K, K - 1, (uint32_t)i, K - 2);
        if (i < 16) tb.s2[i] = K == 5 ? slot_bits(K, 2, (uint32_t)i, 2) : 0u;
        if (i < 4) {
            tb.tp[i] = pair_bits(K, K - 2, K - 1, (uint32_t)i);
            tb.p01[i] = pair_bits(K, 0, 1, (uint32_t)i);
        }
    }
    if (L::SMEM_LUT)
        for (int i = tid; i < (1 << L::NB); i += blockDim.x) lut_s[i] = a.lut[i];
    const int hist_words = K == 5 ? L::NCLS : kWarpsPerBlock * L::NCLS;
    for (int i = tid; i < hist_words; i += blockDim.x) hist[i] = 0;
    if (tid == 0) *pending = 0;
    __syncthreads();

    Sink<K> sink;
    sink.hist = K == 5 ? hist : hist + wib * L::NCLS;
    sink.lut = L::SMEM_LUT ? lut_s : a.lut;
    sink.counts = a.counts;
    sink.pending = pending;
    sink.since = 0;
    sink.status = a.status;

    Scratch sc;
    const long long gw = (long long)blockIdx.x * kWarpsPerBlock + wib;
    sc.buf[0] = ebuf + (size_t)wib * L::LISTS * L::CAP;
    sc.buf[1] = sc.buf[0] + L::CAP;
    sc.ovf[0] = a.scratch + gw * a.scratch_per_warp;
    sc.ovf[1] = sc.ovf[0] + a.scratch_per_warp / 2;
    sc.cap = L::CAP;

    if (phase == 1) {
        const long long nunits = K == 3 ? (long long)a.n : a.info->nnz;
        for (;;) {
            unsigned long long u0 = 0;
            if (lane == 0) u0 = atomicAdd(&a.info->unit_ctr, (unsigned long long)kGrab);
            u0 = __shfl_sync(kFull, u0, 0);
            if ((long long)u0 >= nunits) break;
            const long long u1 = min((long long)u0 + kGrab, nunits);
            int v = K == 3 ? 0 : row_of(a.nptr, a.n, (long long)u0);
            for (long long u = (long long)u0; u < u1; u++) {
                if (K == 3) {
                    v = (int)u;
                } else {
                    while (a.nptr[v + 1] <= u) v++;
                }
                process_unit<K>(a, tb, sink, sc, (uint32_t)u, v, 0, 0x7FFFFFFF, true, lane);
            }
        }
    } else {
        const unsigned long long tail = min(a.info->queue_tail, a.queue_cap);
        for (;;) {
            unsigned long long idx = 0;
            if (lane == 0) idx = atomicAdd(&a.info->queue_head, 1ull);
            idx = __shfl_sync(kFull, idx, 0);
            if (idx >= tail) break;
            const uint4 it = a.queue[idx];
            const int v = K == 3 ? (int)it.x : row_of(a.nptr, a.n, (long long)it.x);
            process_unit<K>(a, tb, sink, sc, it.x, v, (int)it.y, (int)it.z, false, lane);
        }
    }

    __syncthreads();
    if (K == 5) {
        for (int c = tid; c < L::NCLS; c += blockDim.x) {
            const uint32_t v = hist[c];
            if (v) atomicAdd(&a.counts[c], (unsigned long long)v);
        }
    } else {
        for (int c = tid; c < L::NCLS; c += blockDim.x) {
            unsigned long long s = 0;
            for (int w = 0; w < kWarpsPerBlock; w++) s += hist[w * L::NCLS + c];
            if (s) atomicAdd(&a.counts[c], s);
        }
    }
}

template <int K>
int blocks_per_sm() {
    static int cached = 0;
    if (cached) return cached;
    if (cudaFuncSetAttribute(k_enum<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Layout<K>::total) !=
        cudaSuccess)
        return -1;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_enum<K>, kThreads, Layout<K>::total) != cudaSuccess ||
        b < 1)
        return -1;
    cached = b;
    return b;
}

template <int K>
int launch_k(const EnumArgs &a, int num_sms, cudaStream_t s) {
    const int bps = blocks_per_sm<K>();
    if (bps < 1) return ACC_ERR_CUDA;
    const int grid = num_sms * bps;
    k_enum<K><<<grid, kThreads, Layout<K>::total, s>>>(a, 1);
    k_enum<K><<<grid, kThreads, Layout<K>::total, s>>>(a, 2);
    return cudaGetLastError() == cudaSuccess ? 2 : ACC_ERR_CUDA;
}

}  // namespace

int enum_grid_warps(int k, int num_sms) {
    int bps = k == 3 ? blocks_per_sm<3>() : (k == 4 ? blocks_per_sm<4>() : blocks_per_sm<5>());
    if (bps < 1) return ACC_ERR_CUDA;
    return num_sms * bps * kWarpsPerBlock;
}

int launch_enumerate(int k, const EnumArgs &a, int num_sms, cudaStream_t s) {
    switch (k) {
    case 3: return launch_k<3>(a, num_sms, s);
    case 4: return launch_k<4>(a, num_sms, s);
    case 5: return launch_k<5>(a, num_sms, s);
    default: return ACC_ERR_K;
    }
}

}  // namespace acc
