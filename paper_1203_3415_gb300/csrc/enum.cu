// Enumeration kernels: every connected induced k-subset exactly once,
// classified by the code -> class table and counted in shared-memory
// histograms.
//
// Which subsets: the problem of the paper (Problems Motifs-3/4/5), i.e. the
// k-sets S whose undirected version G*[S] is connected (Notation section).
// The paper counts them through per-vertex / per-edge / per-triple formulas
// over set sizes with corrections for edges among the sets.  Here ESU visits
// every connected (k-2)-prefix once; the last two levels are counted the
// paper's way (count mode, the default: pairs of extension-list members per
// pair of state-vector groups, corrected by the adjacent pairs and completed
// by the exclusive leaves found in the members' neighbour lists) or visited
// leaf by leaf (enumerate mode).  One table over all adjacency codes serves
// every class, so no multiplicity correction is needed.
//
// Exactly-once rule (ESU, Wernicke 2006, the FANMOD algorithm the paper
// cites): a set is grown from its smallest vertex v (the root).  The current
// set Vsub carries an extension list Vext whose members all exceed v; taking
// the member at position j into Vsub leaves Vext[j+1..] plus the exclusive
// neighbours of that member (neighbours above v that are neither in Vsub nor
// adjacent to it) as the next extension list.  The last two levels are the
// hot loop, run warp-parallel:
//
//   prefix P = the first k-2 vertices, E = its extension list, then the
//   leaves are  (a) P + {E[j], E[l]}  for j < l          ("pair leaves")
//               (b) P + {E[j], u}     for u an exclusive neighbour of E[j]
//
// Codes in the kernels use the state-vector layout: for tuple slot t >= 1 the
// field f_t = sum_{i<t} state(w_i, w_t) << 2i (state bit 0 = arc w_i -> w_t,
// bit 1 = arc w_t -> w_i), fields stored from the last slot (lowest bits) up
// to slot 1.  Every piece of a leaf's code is then a shifted state vector, and
// the bits that change along one extension row are the lowest ones, so the
// codes of one row hit distinct shared-memory banks of the class table.  The
// table the kernels read is the canonical-layout table with its index bits
// permuted accordingly (lut.cu), so classes are the same.
//
// Work units: k=3 one unit per root v; k=4 and k=5 one unit per arc position
// of the G* CSR, i.e. per (v, w1) with w1 > v.  Phase 1 runs every light unit
// and queues the heavy ones as row ranges of their extension list (k = 5:
// of the level-2 list, one level-3 list per row); phase 2 (a second launch)
// drains the queue.  k = 5 in the count mode scans the level-2 rows that a
// range's level-3 lists share once for all of them (count_shared_rows) and
// the lists' own rows together (count_partb_rows).
#include <math.h>

#include <type_traits>

#include "common.cuh"

namespace acc {

namespace {

// Tuning knobs (compile-time; -D overrides for sweeps).
#ifndef ACC_CAP34
#define ACC_CAP34 256
#endif
#ifndef ACC_GRAB4
#define ACC_GRAB4 2  // base units per atomic grab for k = 4 (lighter units, one hot counter)
#endif
#ifndef ACC_GRAB_SET
#define ACC_GRAB_SET 16  // base units per grab when several graphs are counted (fewer graph switches), <= 32
#endif
#ifndef ACC_GRAB
#define ACC_GRAB 1
#endif
#ifndef ACC_LIGHT
#define ACC_LIGHT (1 << 11)
#endif
#ifndef ACC_LIGHT4
#define ACC_LIGHT4 6144  // k = 4 count mode (tuned on the Chung-Lu k = 4 workload)
#endif
#ifndef ACC_TARGET
#define ACC_TARGET (1 << 12)
#endif
#ifndef ACC_TARGET5
#define ACC_TARGET5 (1 << 14)  // k = 5: longer chunks, over which the shared level-2 rows are scanned once
#endif
#ifndef ACC_UNROLL
#define ACC_UNROLL 4
#endif
#ifndef ACC_CWIN
#define ACC_CWIN 3  // count mode: 32-entry windows of the flat row scan per step (entries in flight per lane), k = 3, 4
#endif
#ifndef ACC_CWIN_P2
#define ACC_CWIN_P2 4  // the same in phase 2, whose queued chunks of heavy units run longer scans
#endif
#ifndef ACC_CWIN5
#define ACC_CWIN5 2  // the same for k = 5
#endif
#ifndef ACC_RING
#define ACC_RING 64  // count mode: rows a warp may stage for the flat scan (a power of two, at least 64), k = 3, 4
#endif
#ifndef ACC_RING5
#define ACC_RING5 64  // the same for k = 5 (its block histogram leaves less shared memory)
#endif
#ifndef ACC_COLLECT_B
#define ACC_COLLECT_B 1  // k = 5 count mode: scan the part-B rows of a tile's lists together
#endif
#ifndef ACC_SHARED_U
#define ACC_SHARED_U 2  // lists taken at a time by the shared-row scan (k = 5 count mode)
#endif
#ifndef ACC_CAP5
#define ACC_CAP5 64  // per-warp shared-memory list entries (each of two lists), k = 5
#endif
#ifndef ACC_MINB5
#define ACC_MINB5 4  // resident blocks per SM the k = 5 kernels are compiled for
#endif
#ifndef ACC_MINB34
#define ACC_MINB34 4  // resident blocks per SM the k = 3, 4 leaf kernels are compiled for
#endif
#ifndef ACC_MINB34C
#define ACC_MINB34C 4  // the same for the k = 3, 4 count-mode kernels of one graph
#endif
#ifndef ACC_LUT_SMEM34
#define ACC_LUT_SMEM34 1  // k = 3, 4: class table staged in shared memory (else read through L1)
#endif
#ifndef ACC_MINB34S
#define ACC_MINB34S 4  // the same for the k = 3, 4 count-mode kernels of a set of graphs
#endif
constexpr int kCap34 = ACC_CAP34;         // per-warp shared extension entries, k = 3, 4
constexpr int kCap5 = ACC_CAP5;           // per-warp shared entries per list, k = 5
constexpr int kGrab = ACC_GRAB;           // base units per atomic grab
constexpr long long kRowCost = 4;         // count mode: fixed work of one list row
constexpr uint32_t kDrainAt = 1u << 30;

template <int K>
struct Layout {
    static constexpr int NB = K * (K - 1);
    static constexpr int NCLS = num_classes(K);
    static constexpr bool SMEM_LUT = K <= 4 && ACC_LUT_SMEM34;
    static constexpr int CAP = K == 5 ? kCap5 : kCap34;
    static constexpr int LISTS = K == 5 ? 2 : 1;
    static constexpr int SH_PAIR = 2 * (K - 2);  // state(E[j], leaf) within the last field
    static constexpr int SH_ROW = 2 * (K - 1);   // field of slot k-2
    static constexpr size_t lut = SMEM_LUT ? (((size_t(1) << NB) * 2 + 15) & ~size_t(15)) : 0;
    static constexpr size_t pending = 16;
    // histogram words per warp (k <= 4) or block (k = 5): the classes, then a
    // trap bin that takes any add of a code without a class (never expected;
    // non-zero at the end means an internal error)
    static constexpr int HSTRIDE = NCLS + 1;
    static constexpr size_t hist = ((K == 5 ? size_t(1) : size_t(kWarpsPerBlock)) * HSTRIDE * 4 + 15) & ~size_t(15);
    static constexpr size_t ebuf = size_t(kWarpsPerBlock) * LISTS * CAP * 4;
    static constexpr int G = 1 << (2 * (K - 2));  // state vectors to the prefix: 4, 16, 64
    static constexpr size_t groups = size_t(kWarpsPerBlock) * 2 * G * 4;  // count mode: sizes + list
    // count mode: rows staged for the flat scan (a batch of 32 is staged
    // only while the ring has room for it)
    static constexpr int WIN = K == 5 ? ACC_CWIN5 : ACC_CWIN;
    static constexpr int RING = K == 5 ? ACC_RING5 : ACC_RING;
    // (k = 5: a fourth array, each row's position in its list)
    static constexpr int RING_ARRAYS = K == 5 ? 4 : 3;
    static constexpr size_t ring = size_t(kWarpsPerBlock) * RING * RING_ARRAYS * 4;
    static constexpr size_t total = lut + pending + hist + ebuf + groups + ring;
};

// Windows per step of the phase-2 scans (the queued chunks of heavy units).
template <int K>
constexpr int kWinP2 = K == 5 ? Layout<K>::WIN : ACC_CWIN_P2;

__device__ __forceinline__ uint32_t probe(const uint32_t *__restrict__ st, long long pitch, uint32_t a, uint32_t b) {
    return (__ldg(st + (long long)a * pitch + (b >> 4)) >> ((b & 15u) << 1)) & 3u;
}

// Extension-list entry: (x << 6) | states of x to the prefix vertices, two
// bits each in prefix order (at most 3 prefix vertices).
__device__ __forceinline__ uint32_t e_id(uint32_t e) { return e >> 6; }
__device__ __forceinline__ uint32_t e_sv(uint32_t e) { return e & 63u; }

// One graph of the set seen with local vertex ids.
struct GView {
    const uint32_t *state;  // the graph's pair-state block
    long long pitch;
    const long long *nptr;  // by local vertex (positions are global)
    const int *deg;
    const int *lo;
    const uint32_t *nbr;
    const uint32_t *nh;     // hashed adjacency (tables at kNhWords * nptr), or NULL
    const uint2 *rev;       // reverse positions (by global position), or NULL
    int n;
};

// One prefix vertex's adjacency as the probes read it: its dense pair-state
// row (HASH false), or its hashed table and the table's log2 bucket count.
struct PRow {
    const uint32_t *p;
    uint32_t lg;
};

template <bool HASH>
__device__ __forceinline__ PRow prow(const GView &g, uint32_t a) {
    if constexpr (HASH) return PRow{g.nh + (long long)kNhWords * g.nptr[a], nh_lg(g.deg[a])};
    else return PRow{g.state + (long long)a * g.pitch, 0u};
}

// state(a, b) for the prefix vertex a of row r.  Hashed: the bucket of b,
// then the following ones while they are full (an empty slot ends the
// search; an empty slot also reads as state 0 when b is vertex 0).
template <bool HASH>
__device__ __forceinline__ uint32_t pget(const PRow &r, uint32_t b) {
    if constexpr (HASH) {
        const uint32_t m = (1u << r.lg) - 1u;
        uint32_t k = nh_bucket(b, r.lg);
        for (uint32_t tries = 0; tries <= m; tries++, k = (k + 1u) & m) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(r.p) + k);
            if ((q.x >> 2) == b) return q.x & 3u;
            if ((q.y >> 2) == b) return q.y & 3u;
            if ((q.z >> 2) == b) return q.z & 3u;
            if ((q.w >> 2) == b) return q.w & 3u;
            if (!q.w) return 0u;  // slots fill in order: a bucket with room ends the search
        }
        return 0u;
    } else {
        return (__ldg(r.p + (b >> 4)) >> ((b & 15u) << 1)) & 3u;
    }
}

// The only graph of a single-graph count: its arrays are the kernel's own
// (global and local ids coincide).
__device__ __forceinline__ GView view_single(const EnumArgs &a) {
    GView g;
    g.state = a.state;
    g.pitch = a.gs.one.pitch;
    g.nptr = a.nptr;
    g.deg = a.deg;
    g.lo = a.lo;
    g.nbr = a.nbr;
    g.nh = reinterpret_cast<const uint32_t *>(a.nh);
    g.rev = a.rev;
    g.n = a.gs.one.n;
    return g;
}

__device__ __forceinline__ GView view_of(const EnumArgs &a, const GMeta &mt) {
    GView g;
    g.state = a.state + mt.soff;
    g.pitch = mt.pitch;
    g.nptr = a.nptr + mt.voff;
    g.deg = a.deg + mt.voff;
    g.lo = a.lo + mt.voff;
    g.nbr = a.nbr;
    g.nh = reinterpret_cast<const uint32_t *>(a.nh);
    g.rev = a.rev;
    g.n = mt.n;
    return g;
}

// First position of N*(x) (entries (u << 2) | s, sorted) with u > root.
__device__ __forceinline__ int first_above(const uint32_t *__restrict__ nbr, long long base, int d, uint32_t root) {
    const uint32_t key = (root + 1u) << 2;
    // a list wholly above the root is settled by one load
    if (d == 0 || __ldg(nbr + base) >= key) return 0;
    int lo = 1, hi = d;
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
// Each lane keeps a run of equal classes in registers (consecutive leaves of
// one extension row mostly share a class) and adds a run to shared memory
// only when the class changes.
template <int K>
struct Sink {
    uint32_t *hist;
    const int16_t *lut;
    unsigned long long *counts;
    uint32_t *pending;  // k = 5: block-wide increments since the last drain
    uint32_t since;     // increments of this warp not yet accounted
    int *status;
    int run_cls;        // this lane's current run
    uint32_t run_len;
    unsigned long long *counts_base;  // int64[B * NCLS]
    int gcur;           // graph whose counts this warp accumulates
    bool direct;        // k = 5 with several graphs: runs go straight to the int64 counts
    unsigned long long moved;  // count mode: this lane's |increments| since the last accounting
    unsigned long long scanned;  // count mode: neighbour entries this warp scanned

    // Count mode: add delta (may be negative) to class cls.  Shared counters
    // are read as signed 32-bit when drained; a delta too large for them goes
    // straight to the int64 counts.
    __device__ __forceinline__ void add(int cls, long long delta) {
        if (direct || delta >= (1ll << 28) || delta <= -(1ll << 28)) {
            if (cls < 0) set_status(status, ACC_ERR_INTERNAL);
            else atomicAdd(&counts[cls], (unsigned long long)delta);
            return;
        }
        atomicAdd(&hist[min((uint32_t)cls, (uint32_t)Layout<K>::NCLS)], (uint32_t)(int32_t)delta);
        moved += (unsigned long long)(delta < 0 ? -delta : delta);
    }

    // Count mode: add +1 or -1 to class cls (the scan's leaves and moves).
    // A code without a class (cls < 0) lands in the shared trap bin, checked
    // at the end of the kernel, so the hot loop carries no branch for it.
    __device__ __forceinline__ void add1(int cls, int delta) {
        if (direct) {
            if (cls < 0) set_status(status, ACC_ERR_INTERNAL);
            else atomicAdd(&counts[cls], (unsigned long long)(long long)delta);
        } else {
            atomicAdd(&hist[min((uint32_t)cls, (uint32_t)Layout<K>::NCLS)], (uint32_t)delta);
        }
    }

    __device__ __forceinline__ int cls_of(uint32_t code) const {
        return Layout<K>::SMEM_LUT ? (int)lut[code] : (int)__ldg(lut + code);
    }

    __device__ __forceinline__ void flush() {
        if (run_len) {
            if (run_cls < 0) set_status(status, ACC_ERR_INTERNAL);
            else if (direct) atomicAdd(&counts[run_cls], (unsigned long long)run_len);
            else atomicAdd(&hist[run_cls], run_len);
            run_len = 0;
        }
    }

    // Whole warp, between units: move to graph g (k <= 4: the warp's private
    // histogram is drained to the previous graph's counts first).
    __device__ __forceinline__ void switch_graph(int g, int lane) {
        if (g == gcur) return;
        if (K <= 4 && gcur >= 0) {
            __syncwarp();
            for (int c = lane; c < Layout<K>::NCLS; c += kWarp) {
                const int32_t v = (int32_t)hist[c];
                if (v) {
                    hist[c] = 0;
                    atomicAdd(&counts[c], (unsigned long long)(long long)v);
                }
            }
            __syncwarp();
            since = 0;
        }
        gcur = g;
        counts = counts_base + (size_t)g * Layout<K>::NCLS;
    }

    // Enumerate mode: a `valid` lane counts one leaf with adjacency code
    // `code` (into its run, added to the histogram when the class changes).
    __device__ __forceinline__ void bump(uint32_t code, bool valid) {
        if (!valid) return;
        const int cls = cls_of(code);
        if (cls == run_cls) {
            ++run_len;
        } else {
            flush();
            run_cls = cls;
            run_len = 1;
        }
    }

    // Called by the whole warp after each batch of at most `tot` bumps: keeps
    // every 32-bit shared counter below 2^32 by draining to the int64 counts.
    __device__ __forceinline__ void after_batch(uint32_t tot, int lane) {
        since += tot;
        if (K <= 4) {
            if (since >= kDrainAt) {
                flush();
                __syncwarp();
                for (int c = lane; c < Layout<K>::NCLS; c += kWarp) {
                    const int32_t v = (int32_t)hist[c];
                    if (v) {
                        hist[c] = 0;
                        atomicAdd(&counts[c], (unsigned long long)(long long)v);
                    }
                }
                __syncwarp();
                since = 0;
            }
        } else {
            if (direct || since < (1u << 20)) return;
            // account in the block-wide counter every 2^20 increments; the
            // warp that crosses 2^30 drains the block histogram (atomicExch
            // per bin, so concurrent increments are never lost)
            uint32_t old = 0;
            __threadfence_block();
            if (lane == 0) old = atomicAdd(pending, since);
            old = __shfl_sync(kFull, old, 0);
            if (old < kDrainAt && old + since >= kDrainAt) {
                for (int c = lane; c < Layout<K>::NCLS; c += kWarp) {
                    const int32_t v = (int32_t)atomicExch(&hist[c], 0u);
                    if (v) atomicAdd(&counts[c], (unsigned long long)(long long)v);
                }
                __syncwarp();
                if (lane == 0) atomicSub(pending, old + since);
            }
            since = 0;
        }
    }
};

// Count mode: fold the lanes' |increments| into the warp's accounting (whole
// warp, between batches).
template <int K>
__device__ __forceinline__ void account_moved(Sink<K> &sink, int lane) {
    unsigned long long t = sink.moved;
#pragma unroll
    for (int d = 16; d; d >>= 1) t += __shfl_xor_sync(kFull, t, d);
    sink.moved = 0;
    while (t > 0) {  // at most 2^28 per step keeps the 32-bit accounting exact
        const uint32_t step = t > (1ull << 28) ? (1u << 28) : (uint32_t)t;
        sink.after_batch(step, lane);
        t -= step;
    }
}

struct Scratch {
    uint32_t *buf[2];  // shared-memory lists (buf[1] only for k = 5)
    uint32_t *ovf[2];  // global overflow lists of this warp
    int cap;
    uint32_t *gcnt;    // count mode: group sizes and the non-empty group list
    uint32_t *ring;    // count mode: staged rows (flat start, entry offset, list entry[, list position]), RING each
    uint32_t *pb;      // k = 5 count mode: collected part-B rows (entries, then their lists' entries), global
};

// The last two ESU levels over extension list E[0..B), virtual rows
// [plo, phi).  Virtual row p joins row p and row B-1-p of the pair triangle:
// their pair counts (B-1-p and p) add up to B-1 for every p, so all virtual
// rows have the same length and a flat position maps to (row, column) with one
// comparison.  For odd B the middle row (p = B-1-p) stands alone.  pcode holds
// the code fields of the prefix slots 1..k-3.
template <int K>
__device__ __forceinline__ void leaves(const GView &g, Sink<K> &sink, const uint32_t *E, int B, int plo,
                                       int phi, const uint32_t *pm, uint32_t pcode, uint32_t root, int lane) {
    using L = Layout<K>;
    const int P = (B + 1) >> 1;
    phi = min(phi, P);
    if (plo >= phi) return;
    // (a) pair leaves P + {E[row], E[col]}, row < col.  Virtual row p,
    //     position q < B-1-p: (p, p+1+q); q >= B-1-p: (B-1-p, q+1).
    const int Lv = B - 1;
    if (Lv > 0) {
        constexpr int U = ACC_UNROLL;  // positions each lane keeps in flight
        const long long t_begin = (long long)plo * Lv, t_end = (long long)phi * Lv;
        // this lane's cursor: virtual row p, position q of flat position t0 + lane
        int p = (int)((t_begin + lane) / Lv), q = (int)((t_begin + lane) % Lv);
        for (long long t0 = t_begin; t0 < t_end; t0 += U * kWarp) {
            const long long t = t0 + lane;
            uint32_t er[U], ec[U], w[U];
            bool ok[U];
            int pu = p, qu = q;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int Lp = Lv - pu;
                const bool first = qu < Lp;
                const int row = first ? pu : Lv - pu;
                const int col = first ? pu + 1 + qu : qu + 1;
                ok[u] = t + u * kWarp < t_end && (first || 2 * pu + 1 != B);
                er[u] = ok[u] ? E[row] : 0u;
                ec[u] = ok[u] ? E[col] : 0u;
                qu += kWarp;
                while (qu >= Lv) {
                    qu -= Lv;
                    pu++;
                }
            }
            p = pu;
            q = qu;
#pragma unroll
            for (int u = 0; u < U; u++)
                w[u] = ok[u] ? __ldg(g.state + (long long)e_id(er[u]) * g.pitch + (e_id(ec[u]) >> 4)) : 0u;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const uint32_t s = (w[u] >> ((e_id(ec[u]) & 15u) << 1)) & 3u;
                sink.bump(pcode | (e_sv(er[u]) << L::SH_ROW) | e_sv(ec[u]) | (s << L::SH_PAIR), ok[u]);
            }
            sink.after_batch((uint32_t)(U * kWarp), lane);
        }
    }
    // (b) exclusive leaves P + {E[j], u}, u a neighbour of E[j] above the
    //     root and adjacent to no prefix vertex (its states to the prefix
    //     are 0).  Rows of virtual rows [plo, phi): [plo, phi) in the first
    //     half, [B-phi, B-plo) in the second.  Neighbour-list positions fit
    //     32 bits (2 |E*| < 2^32).
    const int r1lo = plo, n1 = phi - plo;
    const int r2lo = max(B - phi, P), n2 = max(0, (B - plo) - r2lo);
    const int nr = n1 + n2;
    for (int ib = 0; ib < nr; ib += kWarp) {
        const int i = ib + lane;
        uint32_t ej = 0, first = 0;
        int cnt = 0;
        if (i < nr) {
            const int j = i < n1 ? r1lo + i : r2lo + (i - n1);
            ej = E[j];
            const uint32_t x = e_id(ej);
            const long long nb = g.nptr[x];
            const int d = g.deg[x];
            const int st = first_above(g.nbr, nb, d, root);
            first = (uint32_t)(nb + st);
            cnt = d - st;
        }
        int tot;
        const int pre = excl_scan(cnt, lane, &tot);
        const uint32_t cj = pcode | (e_sv(ej) << L::SH_ROW);
        const uint32_t off = first - (uint32_t)pre;  // position of leaf t is off + t
        for (int t0 = 0; t0 < tot; t0 += kWarp) {
            const int t = t0 + lane;
            const int r = lb_search(pre, t);
            const uint32_t cr = __shfl_sync(kFull, cj, r);
            const uint32_t orow = __shfl_sync(kFull, off, r);
            bool leaf = false;
            uint32_t ue = 0;
            if (t < tot) {
                ue = __ldg(g.nbr + (orow + (uint32_t)t));
                const uint32_t u = ue >> 2;
                leaf = true;
#pragma unroll
                for (int k2 = 0; k2 < K - 2; k2++) leaf = leaf && probe(g.state, g.pitch, pm[k2], u) == 0u;
            }
            sink.bump(cr | ((ue & 3u) << L::SH_PAIR), leaf);
        }
        sink.after_batch((uint32_t)tot, lane);
    }
}

// Whether u (above the root; s[i] = state(p_i, u) to the prefix vertices
// p_0 = v, p_1 = w1, p_2 = w2) is in the prefix's extension list.  ESU builds
// every list from adjacency and vertex order alone: level 1 is N(v) above v;
// level 2 is N(v) above w1 (part A, ascending) then the neighbours of w1 above
// v not adjacent to v (part B, ascending); level 3 is level 2's list after w2
// then the neighbours of w2 above v adjacent to neither v nor w1.  So the
// states the exclusivity test reads decide membership too, and u's state
// vector (its group in the list) is those same states.  Prefix vertices
// never pass: each is adjacent to an earlier one and not above it.
template <int K>
__device__ __forceinline__ bool in_list(const uint32_t *s, uint32_t u, const uint32_t *pm, bool w2_in_a) {
    if constexpr (K == 3) {
        return s[0] != 0u;
    } else {
        const bool a = s[0] != 0u && u > pm[1];
        const bool b = s[0] == 0u && s[1] != 0u;
        if constexpr (K == 4) {
            return a || b;
        } else {
            const bool after = w2_in_a ? ((a && u > pm[2]) || b) : (b && u > pm[2]);
            return after || (s[0] == 0u && s[1] == 0u && s[2] != 0u);
        }
    }
}

// Count mode for the last two ESU levels over E[0..B), rows [jlo, jend).
// The class of a pair leaf P + {x, y} with x, y not adjacent depends only on
// the two state vectors (states to the prefix), so all such pairs are counted
// per pair of state-vector groups, |g_a| |g_b| or C(|g|, 2) of them, as the
// paper's per-vertex tables count patterns from set sizes (Table starb).
// Adjacent pairs are then moved to their own classes one by one, found in
// the neighbour lists of the list members (the paper's m / m' corrections),
// and the same scan yields the exclusive leaves P + {x, u}.  `bulk` (set for
// exactly one chunk of a list) adds the group-pair counts (count_group_pairs).
// w2_in_a (k = 5) says whether w2 lies in part A of the level-2 list.
template <int K>
__device__ __forceinline__ void count_group_pairs(Sink<K> &sink, const uint32_t *E, int B, uint32_t pcode,
                                                  uint32_t *gcnt, int lane) {
    using L = Layout<K>;
    {
        uint32_t *glist = gcnt + L::G;  // (count << 6) | group of each non-empty group (a list has < 2^26 members)
        for (int i = lane; i < L::G; i += kWarp) gcnt[i] = 0;
        __syncwarp();
        for (int q = lane; q < B; q += kWarp) atomicAdd(&gcnt[e_sv(E[q])], 1u);
        __syncwarp();
        int ng = 0;
        for (int b0 = 0; b0 < L::G; b0 += kWarp) {
            const int gi = b0 + lane;
            const uint32_t c = gi < L::G ? gcnt[gi] : 0u;
            const unsigned m = __ballot_sync(kFull, c > 0);
            if (c > 0) glist[ng + __popc(m & ((1u << lane) - 1u))] = (c << 6) | (uint32_t)gi;
            ng += __popc(m);
        }
        __syncwarp();
        // every unordered pair of members, as if not adjacent
        // pair q of the triangle ia <= ib < ng, rows of ng - ia entries
        // starting at off(ia) = ia ng - ia (ia - 1) / 2, spread over the lanes
        const int npairs = ng * (ng + 1) / 2;
        const int w = 2 * ng + 1;
        for (int q = lane; q < npairs; q += kWarp) {
            int ia = (int)(0.5f * ((float)w - sqrtf((float)(w * w - 8 * q))));
            ia = max(0, min(ia, ng - 1));
            if (ia * ng - ia * (ia - 1) / 2 > q) ia--;
            else if (ia + 1 < ng && (ia + 1) * ng - (ia + 1) * ia / 2 <= q) ia++;
            const int ib = ia + (q - (ia * ng - ia * (ia - 1) / 2));
            const uint32_t ea = glist[ia], eb = glist[ib];
            const uint32_t ga = ea & 63u, ca = ea >> 6;
            const uint32_t gb = eb & 63u, cb = eb >> 6;
            const long long pairs = ib == ia ? (long long)ca * (ca - 1) / 2 : (long long)ca * cb;
            if (pairs) sink.add(sink.cls_of(pcode | (ga << L::SH_ROW) | gb), pairs);
        }
        account_moved(sink, lane);
    }
}

// Rows j < A are neighbours of the root, E[j] the entry at position j of
// revA (the reverse positions of the root's list from that entry on): the
// part of N*(x) above the root is read there, with no search.
template <int K, bool HASH, int WN = Layout<K>::WIN>
__device__ __forceinline__ void count_leaves(const GView &g, Sink<K> &sink, const uint32_t *E, int B, int jlo,
                                             int jend, bool bulk, const uint32_t *pm, uint32_t pcode,
                                             uint32_t root, bool w2_in_a, uint32_t *gcnt, uint32_t *ring,
                                             const uint2 *revA, int A, int lane) {
    using L = Layout<K>;
    if (bulk) count_group_pairs<K>(sink, E, B, pcode, gcnt, lane);
    // neighbour scan of rows [jlo, jend): adjacent member pairs (each once,
    // from its smaller vertex) and exclusive neighbours.  The rows' entries
    // above the root form one flat sequence, cut into 32-entry windows with
    // one entry per lane, across row boundaries: rows are staged 32 at a
    // time (a lane per row) into the warp's ring as (flat start, entry
    // offset, list entry), and a window finds each lane's row from the ring
    // rows that start inside it (one OR-reduction of their start bits and a
    // population count).  Flat positions wrap modulo 2^32; only differences
    // below 2^31 are compared.  A step takes W windows.
    constexpr int W = WN;
    constexpr int RM = L::RING - 1;
    uint32_t *rS = ring, *rO = ring + L::RING, *rE = ring + 2 * L::RING;
    PRow rowp[K - 2];  // adjacency of the prefix vertices
#pragma unroll
    for (int k2 = 0; k2 < K - 2; k2++) rowp[k2] = prow<HASH>(g, pm[k2]);
    uint32_t T = 0;          // flat entries staged
    uint32_t F = 0;          // flat entries consumed
    int tail = 0, cur = -1;  // ring rows staged; last ring row starting before F
    int jb = jlo;
    const int Ae = min(A, jend);  // rows read from revA
    // stage rows while fewer than W windows are pending and the ring
    // has room for 32 more rows (the live rows are cur .. tail - 1)
    auto stage = [&]() {
        while (jb < jend && T - F < 32u * W && tail - cur + kWarp <= L::RING) {
            const int j = jb + lane;
            uint32_t ej = 0, first = 0;
            int cnt = 0;
            if (j < Ae) {
                ej = E[j];
                const uint2 r = __ldg(revA + j);
                first = r.x;
                cnt = (int)r.y;
            } else if (j < jend) {
                ej = E[j];
                const uint32_t x = e_id(ej);
                const long long nb = g.nptr[x];
                const int d = g.deg[x];
                const int st = first_above(g.nbr, nb, d, root);
                first = (uint32_t)(nb + st);
                cnt = d - st;
            }
            const unsigned nz = __ballot_sync(kFull, cnt > 0);
            int tot;
            const int pre = excl_scan(cnt, lane, &tot);
            if (cnt > 0) {
                const int slot = (tail + __popc(nz & ((1u << lane) - 1u))) & RM;
                const uint32_t sflat = T + (uint32_t)pre;
                rS[slot] = sflat;
                rO[slot] = first - sflat;
                rE[slot] = ej;
            }
            tail += __popc(nz);
            T += (uint32_t)tot;
            sink.scanned += (unsigned long long)tot;
            jb += kWarp;
        }
    };
    // the ring row of this lane's entry in the window starting at F + 32 w
    // (whole warp; windows in order)
    auto locate = [&](int w) -> int {
        const uint32_t t0 = F + 32u * w;
        // ring rows cur+1 .. cur+32 may start inside [t0, t0 + 32)
        uint32_t bit = 0;
        const int r = cur + 1 + lane;
        if (r < tail) {
            const uint32_t sd = rS[r & RM] - t0;
            if (sd < 32u) bit = 1u << sd;
        }
        const uint32_t starts = __reduce_or_sync(kFull, bit);
        const int row = cur + __popc(starts & (0xFFFFFFFFu >> (31 - lane)));
        cur += __popc(starts);
        return row & RM;
    };
    // classes of one step's leaves: an exclusive leaf P + {x, u} (u adjacent
    // to no prefix vertex) adds one to its class; an adjacent pair of list
    // members {x, u} (each once, from its smaller vertex) moves one leaf from
    // the non-adjacent class to its own.  Table reads of every window are
    // issued before any histogram add, with no branch in between.
    auto classify = [&](const auto &ue, const auto &er, const auto &ok) {
        constexpr int W = std::extent<std::remove_reference_t<decltype(ue)>>::value;
        uint32_t sv[W][K - 2];
#pragma unroll
        for (int w = 0; w < W; w++) {
            const uint32_t u = ue[w] >> 2;
#pragma unroll
            for (int k2 = 0; k2 < K - 2; k2++) sv[w][k2] = ok[w] ? pget<HASH>(rowp[k2], u) : 0u;
        }
        int add_cls[W];
        bool add[W], adj[W];
        uint32_t base[W];
#pragma unroll
        for (int w = 0; w < W; w++) {
            const uint32_t u = ue[w] >> 2, su = ue[w] & 3u;
            const uint32_t cr = pcode | (e_sv(er[w]) << L::SH_ROW);
            uint32_t mu = 0;
#pragma unroll
            for (int k2 = 0; k2 < K - 2; k2++) mu |= sv[w][k2] << (2 * k2);
            adj[w] = ok[w] && mu != 0u && u > e_id(er[w]) && in_list<K>(sv[w], u, pm, w2_in_a);
            add[w] = (ok[w] && mu == 0u) || adj[w];
            base[w] = cr | mu;
            add_cls[w] = sink.cls_of(base[w] | (su << L::SH_PAIR));
        }
#pragma unroll
        for (int w = 0; w < W; w++)
            if (add[w]) sink.add1(add_cls[w], 1);
#pragma unroll
        for (int w = 0; w < W; w++)
            if (adj[w]) sink.add1(sink.cls_of(base[w]), -1);
    };
    // one step of NW windows; FULL: all NW windows hold entries (no lane
    // masks).  The last step of a list takes only the windows it fills.
    auto step = [&](auto nw, auto full) {
        constexpr int NW = decltype(nw)::value;
        constexpr bool FULL = decltype(full)::value;
        const uint32_t pend = T - F;
        uint32_t ue[NW], er[NW];
        bool ok[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const int row = locate(w);
            ok[w] = FULL || 32u * w + lane < pend;
            er[w] = rE[row];
            const uint32_t off = rO[row];
            ue[w] = ok[w] ? __ldg(g.nbr + (off + F + 32u * w + lane)) : 0u;
        }
        classify(ue, er, ok);
        const uint32_t used = FULL || pend >= 32u * NW ? 32u * NW : pend;
        F += used;
        sink.after_batch(2u * used, lane);  // each entry moves at most two counters by one
    };
    static_assert(W >= 1 && W <= 4, "windows per step");
    for (;;) {
        stage();
        const uint32_t pend = T - F;
        if (!pend) break;
        __syncwarp();
        if (pend >= 32u * W) {
            step(std::integral_constant<int, W>{}, std::true_type{});
        } else if (pend > 32u * (W - 1)) {
            step(std::integral_constant<int, W>{}, std::false_type{});
        } else if constexpr (W >= 4) {
            if (pend > 64u) step(std::integral_constant<int, 3>{}, std::false_type{});
            else if (pend > 32u) step(std::integral_constant<int, 2>{}, std::false_type{});
            else step(std::integral_constant<int, 1>{}, std::false_type{});
        } else if constexpr (W == 3) {
            if (pend > 32u) step(std::integral_constant<int, 2>{}, std::false_type{});
            else step(std::integral_constant<int, 1>{}, std::false_type{});
        } else if constexpr (W == 2) {
            step(std::integral_constant<int, 1>{}, std::false_type{});
        }
    }
    __syncwarp();
}

// Count mode, k = 5: the last list level before the leaves.  EL (BL
// members) is the extension list of a fixed prefix P0 of k-3 vertices
// ({v, w1}: EL is the level-2 list of unit (v, w1)), entries (x << 6) |
// states of x to P0.  Member
// wl = EL[jl] extends P0 to the prefix P0 + {wl} of the two leaf levels,
// whose list EN(jl) is EL after jl (part A, with each member's state to wl
// added) followed by the neighbours of wl above v adjacent to no vertex of P0
// (part B).  Rows [r0, r1) of EL are taken here.
//
// Row j of EL (x = EL[j]) is a part-A row of every list EN(jl), jl in
// [r0, min(j, r1)), with the same neighbour entries and the same states to P0
// each time.  So each list EN(jl) is built, its group pairs counted and its
// part-B rows scanned by count_leaves, and then the shared rows are scanned
// once for all the lists: rows j in (r0, BL) are staged into the ring as one
// flat sequence of 32-entry windows (as in count_leaves, each row also
// recording j), a lane takes one entry u of a window with its states to P0,
// and the warp then walks the lists jl (wl the same for every lane): a lane
// whose row lies after jl probes wl against x and u and counts its leaf of
// list EN(jl) exactly as count_leaves would (an exclusive leaf, or the move
// of an adjacent member pair).  (For k = 4 the same sharing would need units
// of whole roots, whose level-2 lists could then no longer be split across
// warps; measured slower there, so k = 4 keeps one list per unit.)
template <int K, bool HASH>
__device__ __forceinline__ void count_shared_rows(const GView &g, Sink<K> &sink, const uint32_t *EL, int BL, int r0,
                                                  int r1, uint32_t pc0, const uint32_t *p0, const PRow *rows0,
                                                  uint32_t *ring, const uint2 *revA, int A, int lane) {
    using L = Layout<K>;
    constexpr int RM = L::RING - 1;
    constexpr int SB = 2 * (K - 3);         // bits of the states to P0
    constexpr int SHL = L::SH_ROW + 2 * (K - 2);  // field of slot k-3 (wl's states to P0)
    const uint32_t v = p0[0];
    uint32_t *rS = ring, *rO = ring + L::RING, *rE = ring + 2 * L::RING, *rJ = ring + 3 * L::RING;
    uint32_t T = 0, F = 0;   // flat entries staged, consumed
    int tail = 0, cur = -1;  // ring rows staged; last ring row starting before F
    int jb = r0 + 1;
    const int Ae = min(A, BL);  // rows read from revA (neighbours of v, as in count_leaves)
    for (;;) {
        while (jb < BL && T - F < 32u && tail - cur + kWarp <= L::RING) {
            const int j = jb + lane;
            uint32_t ej = 0, first = 0;
            int cnt = 0;
            if (j < Ae) {
                ej = EL[j];
                const uint2 r = __ldg(revA + j);
                first = r.x;
                cnt = (int)r.y;
            } else if (j < BL) {
                ej = EL[j];
                const uint32_t x = e_id(ej);
                const long long nb = g.nptr[x];
                const int d = g.deg[x];
                const int st = first_above(g.nbr, nb, d, v);
                first = (uint32_t)(nb + st);
                cnt = d - st;
            }
            const unsigned nz = __ballot_sync(kFull, cnt > 0);
            int tot;
            const int pre = excl_scan(cnt, lane, &tot);
            if (cnt > 0) {
                const int slot = (tail + __popc(nz & ((1u << lane) - 1u))) & RM;
                const uint32_t sflat = T + (uint32_t)pre;
                rS[slot] = sflat;
                rO[slot] = first - sflat;
                rE[slot] = ej;
                rJ[slot] = (uint32_t)j;
            }
            // entries scanned over all lists: cnt for each list the row is in
            unsigned long long w = (unsigned long long)cnt * (unsigned long long)max(0, min(j, r1) - r0);
#pragma unroll
            for (int d = 16; d; d >>= 1) w += __shfl_xor_sync(kFull, w, d);
            sink.scanned += w;
            tail += __popc(nz);
            T += (uint32_t)tot;
            jb += kWarp;
        }
        const uint32_t pend = T - F;
        if (!pend) break;
        __syncwarp();
        // this lane's row in the window [F, F + 32)
        uint32_t bit = 0;
        {
            const int r = cur + 1 + lane;
            if (r < tail) {
                const uint32_t sd = rS[r & RM] - F;
                if (sd < 32u) bit = 1u << sd;
            }
        }
        const uint32_t starts = __reduce_or_sync(kFull, bit);
        const int row = (cur + __popc(starts & (0xFFFFFFFFu >> (31 - lane)))) & RM;
        cur += __popc(starts);
        const bool ok = (uint32_t)lane < pend;
        const uint32_t er = rE[row];
        const int jrow = ok ? (int)rJ[row] : r0;  // lists jl < jrow take this entry
        const uint32_t ue = ok ? __ldg(g.nbr + (rO[row] + F + (uint32_t)lane)) : 0u;
        const uint32_t u = ue >> 2, su = ue & 3u, x = e_id(er);
        uint32_t s0u = 0;  // u's states to P0
#pragma unroll
        for (int k2 = 0; k2 < K - 3; k2++) s0u |= (ok ? pget<HASH>(rows0[k2], u) : 0u) << (2 * k2);
        const uint32_t s0x = er & ((1u << SB) - 1u);
        const int jmax = __reduce_max_sync(kFull, min(jrow, r1));
        // lists taken U at a time: their probes and table reads are issued
        // before any histogram add
        constexpr int U = ACC_SHARED_U;
        static_assert(kWarp % U == 0, "lists per step divide the warp");
        // the lists' entries, 32 at a time, one per lane, handed out by
        // shuffles (no dependent load of EL on each list's path)
        uint32_t elv = 0;
        for (int j0 = r0; j0 < jmax; j0 += U) {
            if (((j0 - r0) & (kWarp - 1)) == 0) elv = j0 + lane < jmax ? EL[j0 + lane] : 0u;
            int ca[U], cm[U];
            bool add[U], adj[U];
#pragma unroll
            for (int i = 0; i < U; i++) {
                const int jl = j0 + i;
                const bool act = jl < jrow && jl < jmax;
                const uint32_t el = __shfl_sync(kFull, elv, (jl - r0) & (kWarp - 1));
                const uint32_t wl = e_id(el);
                const PRow row_l = prow<HASH>(g, wl);
                const uint32_t sx = act ? pget<HASH>(row_l, x) : 0u;
                const uint32_t sw = act ? pget<HASH>(row_l, u) : 0u;
                const uint32_t cr = pc0 | ((el & ((1u << SB) - 1u)) << SHL) | ((s0x | (sx << SB)) << L::SH_ROW);
                const uint32_t mu = s0u | (sw << SB);
                uint32_t s[K - 2], pm[K - 2];
#pragma unroll
                for (int k2 = 0; k2 < K - 3; k2++) {
                    s[k2] = (s0u >> (2 * k2)) & 3u;
                    pm[k2] = p0[k2];
                }
                s[K - 3] = sw;
                pm[K - 3] = wl;
                adj[i] = act && mu != 0u && u > x && in_list<K>(s, u, pm, (el & 3u) != 0u);
                add[i] = (act && mu == 0u) || adj[i];
                ca[i] = sink.cls_of(cr | mu | (su << L::SH_PAIR));
                cm[i] = sink.cls_of(cr | mu);
            }
#pragma unroll
            for (int i = 0; i < U; i++)
                if (add[i]) sink.add1(ca[i], 1);
#pragma unroll
            for (int i = 0; i < U; i++)
                if (adj[i]) sink.add1(cm[i], -1);
            sink.after_batch(2u * U * kWarp, lane);  // each lane moves at most two counters by one per list
        }
        F += pend < 32u ? pend : 32u;
    }
    __syncwarp();
}

// Count mode, k = 5: the part-B rows that count_last_lists collected from
// several level-3 lists (pbE: the list entry of row i, (x << 6) | x's states
// to v, w1 and its list's w2; pbL: the entry EL[jl] of that list's w2), in
// one flat scan as count_leaves does for one list, with each row's own w2:
// a lane takes its row's w2 from the ring and probes it beside v and w1.
template <bool HASH>
__device__ __forceinline__ void count_partb_rows(const GView &g, Sink<5> &sink, const uint32_t *pbE,
                                                 const uint32_t *pbL, int nrows, uint32_t pc0, const uint32_t *p0,
                                                 const PRow *rows0, uint32_t *ring, int lane) {
    using L = Layout<5>;
    constexpr int W = L::WIN;
    constexpr int RM = L::RING - 1;
    const uint32_t v = p0[0];
    uint32_t *rS = ring, *rO = ring + L::RING, *rE = ring + 2 * L::RING, *rL = ring + 3 * L::RING;
    uint32_t T = 0, F = 0;   // flat entries staged, consumed
    int tail = 0, cur = -1;  // ring rows staged; last ring row starting before F
    int jb = 0;
    auto stage = [&]() {
        while (jb < nrows && T - F < 32u * W && tail - cur + kWarp <= L::RING) {
            const int j = jb + lane;
            uint32_t ej = 0, el = 0, first = 0;
            int cnt = 0;
            if (j < nrows) {
                ej = pbE[j];
                el = pbL[j];
                const uint32_t x = e_id(ej);
                const long long nb = g.nptr[x];
                const int d = g.deg[x];
                const int st = first_above(g.nbr, nb, d, v);
                first = (uint32_t)(nb + st);
                cnt = d - st;
            }
            const unsigned nz = __ballot_sync(kFull, cnt > 0);
            int tot;
            const int pre = excl_scan(cnt, lane, &tot);
            if (cnt > 0) {
                const int slot = (tail + __popc(nz & ((1u << lane) - 1u))) & RM;
                const uint32_t sflat = T + (uint32_t)pre;
                rS[slot] = sflat;
                rO[slot] = first - sflat;
                rE[slot] = ej;
                rL[slot] = el;
            }
            tail += __popc(nz);
            T += (uint32_t)tot;
            sink.scanned += (unsigned long long)tot;
            jb += kWarp;
        }
    };
    auto locate = [&](int w) -> int {
        const uint32_t t0 = F + 32u * w;
        uint32_t bit = 0;
        const int r = cur + 1 + lane;
        if (r < tail) {
            const uint32_t sd = rS[r & RM] - t0;
            if (sd < 32u) bit = 1u << sd;
        }
        const uint32_t starts = __reduce_or_sync(kFull, bit);
        const int row = cur + __popc(starts & (0xFFFFFFFFu >> (31 - lane)));
        cur += __popc(starts);
        return row & RM;
    };
    auto step = [&](auto nw, auto full) {
        constexpr int NW = decltype(nw)::value;
        constexpr bool FULL = decltype(full)::value;
        const uint32_t pend = T - F;
        uint32_t ue[NW], er[NW], el[NW];
        bool ok[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const int row = locate(w);
            ok[w] = FULL || 32u * w + lane < pend;
            er[w] = rE[row];
            el[w] = rL[row];
            const uint32_t off = rO[row];
            ue[w] = ok[w] ? __ldg(g.nbr + (off + F + 32u * w + lane)) : 0u;
        }
        uint32_t sv[NW][3];
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const uint32_t u = ue[w] >> 2;
            const PRow row_l = prow<HASH>(g, e_id(el[w]));
            sv[w][0] = ok[w] ? pget<HASH>(rows0[0], u) : 0u;
            sv[w][1] = ok[w] ? pget<HASH>(rows0[1], u) : 0u;
            sv[w][2] = ok[w] ? pget<HASH>(row_l, u) : 0u;
        }
        int add_cls[NW];
        bool add[NW], adj[NW];
        uint32_t base[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const uint32_t u = ue[w] >> 2, su = ue[w] & 3u;
            const uint32_t cr = pc0 | ((el[w] & 15u) << 14) | (e_sv(er[w]) << L::SH_ROW);
            const uint32_t mu = sv[w][0] | (sv[w][1] << 2) | (sv[w][2] << 4);
            const uint32_t pm[3] = {v, p0[1], e_id(el[w])};
            adj[w] = ok[w] && mu != 0u && u > e_id(er[w]) && in_list<5>(sv[w], u, pm, (el[w] & 3u) != 0u);
            add[w] = (ok[w] && mu == 0u) || adj[w];
            base[w] = cr | mu;
            add_cls[w] = sink.cls_of(base[w] | (su << L::SH_PAIR));
        }
#pragma unroll
        for (int w = 0; w < NW; w++)
            if (add[w]) sink.add1(add_cls[w], 1);
#pragma unroll
        for (int w = 0; w < NW; w++)
            if (adj[w]) sink.add1(sink.cls_of(base[w]), -1);
        const uint32_t used = FULL || pend >= 32u * NW ? 32u * NW : pend;
        F += used;
        sink.after_batch(2u * used, lane);  // each entry moves at most two counters by one
    };
    static_assert(W >= 1 && W <= 2, "windows per step of the part-B scan");
    for (;;) {
        stage();
        const uint32_t pend = T - F;
        if (!pend) break;
        __syncwarp();
        if (pend >= 32u * W) step(std::integral_constant<int, W>{}, std::true_type{});
        else if (pend > 32u * (W - 1)) step(std::integral_constant<int, W>{}, std::false_type{});
        else step(std::integral_constant<int, 1>{}, std::false_type{});
    }
    __syncwarp();
}

// Count mode, k = 5: rows [r0, r1) of the last list level EL (see
// count_shared_rows): each member's leaf list built, its group pairs and
// part-B rows counted by count_leaves, then the shared part-A rows.  The
// first A_el rows of EL are neighbours of v whose reverse positions start
// at revA (as for count_leaves).
template <int K, bool HASH>
__device__ __forceinline__ void count_last_lists(const GView &g, Sink<K> &sink, const Scratch &sc, const uint32_t *EL,
                                                 int BL, int r0, int r1, uint32_t pc0, const uint32_t *p0,
                                                 const PRow *rows0, const uint2 *revA, int A_el, int lane) {
    using L = Layout<K>;
    constexpr int SB = 2 * (K - 3);
    constexpr int SHL = L::SH_ROW + 2 * (K - 2);
    const uint32_t v = p0[0];
    int nb = 0;  // part-B rows collected in sc.pb
    for (int jl = r0; jl < r1; jl++) {
        const uint32_t el = EL[jl];
        const uint32_t wl = e_id(el);
        const uint32_t pcode = pc0 | ((el & ((1u << SB) - 1u)) << SHL);
        const int A = BL - 1 - jl;
        const int dw = g.deg[wl];
        const long long ub = (long long)A + dw;
        // (EL sits in buf[0] or ovf[0])
        uint32_t *EN = ub <= sc.cap ? sc.buf[1] : sc.ovf[1];
        // the list: EL after wl (with wl's states), then the neighbours of
        // wl above v adjacent to no vertex of P0, both read in one pass (the
        // neighbours at or below v skipped by their ids)
        const PRow row_l = prow<HASH>(g, wl);
        const long long wb = g.nptr[wl];
        const int nq = max(A, dw);
        int pos = A;
        for (int q0 = 0; q0 < nq; q0 += kWarp) {
            const int q = q0 + lane;
            const bool in_a = q < A;
            uint32_t xe = 0, ue = 0;
            if (in_a) xe = EL[jl + 1 + q];
            if (q < dw) ue = __ldg(g.nbr + wb + q);
            const uint32_t x = e_id(xe), u = ue >> 2;
            uint32_t sa = 0;
            bool keep = false;
            if (in_a) sa = pget<HASH>(row_l, x);
            if (q < dw && u > v) {
                keep = true;
#pragma unroll
                for (int k2 = 0; k2 < K - 3; k2++) keep = keep && pget<HASH>(rows0[k2], u) == 0u;
            }
            if (in_a) EN[q] = (x << 6) | (xe & ((1u << SB) - 1u)) | (sa << SB);
            const unsigned ball = __ballot_sync(kFull, keep);
            if (keep) EN[pos + __popc(ball & ((1u << lane) - 1u))] = (u << 6) | ((ue & 3u) << SB);
            pos += __popc(ball);
        }
        __syncwarp();
        // the group pairs of the whole list; its part-B rows are collected
        // (with the list's w2) and scanned together with those of the next
        // lists, or on their own when they alone overflow the collection
        const int nB = pos - A;
        if (!ACC_COLLECT_B || nB > kPartBRows) {
            uint32_t pm[K - 2];
#pragma unroll
            for (int k2 = 0; k2 < K - 3; k2++) pm[k2] = p0[k2];
            pm[K - 3] = wl;
            count_leaves<K, HASH>(g, sink, EN, pos, A, pos, true, pm, pcode, v, (el & 3u) != 0u, sc.gcnt, sc.ring,
                                  nullptr, 0, lane);
        } else {
            count_group_pairs<K>(sink, EN, pos, pcode, sc.gcnt, lane);
            if (nb + nB > kPartBRows) {
                count_partb_rows<HASH>(g, sink, sc.pb, sc.pb + kPartBRows, nb, pc0, p0, rows0, sc.ring, lane);
                nb = 0;
            }
            for (int q = lane; q < nB; q += kWarp) {
                sc.pb[nb + q] = EN[A + q];
                sc.pb[kPartBRows + nb + q] = el;
            }
            nb += nB;
        }
        __syncwarp();
    }
    if (nb) count_partb_rows<HASH>(g, sink, sc.pb, sc.pb + kPartBRows, nb, pc0, p0, rows0, sc.ring, lane);
    count_shared_rows<K, HASH>(g, sink, EL, BL, r0, r1, pc0, p0, rows0, sc.ring, revA, A_el, lane);
}

// Level-2 extension list of unit (v, w1), w1 at position p of N*(v): part A
// = the neighbours of v after w1 (ascending), part B = the neighbours of w1
// above v not adjacent to v (ascending), each entry (x << 6) | state(v, x) |
// state(w1, x) << 2.  Both parts are read in one pass (a lane holds one
// position of each), and the neighbours of w1 at or below v are skipped by
// their ids.  With work non-NULL it receives this lane's share of the list's
// scan work, sum over members of (degree + kRowCost), gathered with the
// probes.
template <bool HASH>
__device__ __forceinline__ int build_level2(const GView &a, long long p, int v, uint32_t w1, const Scratch &sc,
                                            uint32_t **E_out, int lane, long long *work) {
    const PRow row_v = prow<HASH>(a, (uint32_t)v), row_w1 = prow<HASH>(a, w1);
    const long long rb = a.nptr[v];
    const int t = (int)(p - rb);
    const int dv = a.deg[v], dw = a.deg[w1];
    const long long wb = a.nptr[w1];
    const int A = dv - t - 1;
    const long long ub = (long long)A + dw;
    uint32_t *E = ub <= sc.cap ? sc.buf[0] : sc.ovf[0];
    const int nq = max(A, dw);
    int pos = A;
    long long wk = 0;
    for (int q0 = 0; q0 < nq; q0 += kWarp) {
        const int q = q0 + lane;
        const bool in_a = q < A;
        uint32_t xa = 0, xb = 0;
        if (in_a) xa = __ldg(a.nbr + rb + t + 1 + q);
        if (q < dw) xb = __ldg(a.nbr + wb + q);
        const uint32_t x = xa >> 2, u = xb >> 2;
        const bool in_b = q < dw && u > (uint32_t)v;
        uint32_t sa = 0, sb = 0;
        int da = 0, db = 0;
        if (in_a) {
            sa = pget<HASH>(row_w1, x);
            if (work) da = a.deg[x];
        }
        if (in_b) {
            sb = pget<HASH>(row_v, u);
            if (work) db = a.deg[u];
        }
        if (in_a) {
            E[q] = (x << 6) | (xa & 3u) | (sa << 2);
            wk += da + kRowCost;
        }
        const bool keep = in_b && sb == 0u;
        const unsigned ball = __ballot_sync(kFull, keep);
        if (keep) {
            E[pos + __popc(ball & ((1u << lane) - 1u))] = (u << 6) | ((xb & 3u) << 2);
            wk += db + kRowCost;
        }
        pos += __popc(ball);
    }
    __syncwarp();
    if (work) *work = wk;
    *E_out = E;
    return pos;
}

// Reserve n queue slots; returns the first.
__device__ __forceinline__ unsigned long long reserve(const EnumArgs &a, unsigned long long n, int lane) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(&a.info->queue_tail, n);
    return __shfl_sync(kFull, idx, 0);
}

// Queue a heavy unit whose extension list has at most Bu entries as chunks
// of about a.target work: its Pu = ceil(Bu/2) virtual rows all carry Bu-1
// pairs (plus an allowance D per list row for exclusive leaves), so equal
// ranges of virtual rows are equal work.  Returns the first virtual row whose
// chunk did not fit the queue (Pu when all fit); the caller runs the rest.
__device__ int queue_closed_form(const EnumArgs &a, uint32_t unit, int v, long long Bu, long long D, int lane) {
    const long long Pu = (Bu + 1) / 2;
    const long long W = Pu * (Bu - 1) + Bu * D;
    long long C = (W + a.target - 1) / a.target;
    if (C > Pu) C = Pu;
    if (C < 1) C = 1;
    const unsigned long long base = reserve(a, (unsigned long long)C, lane);
    int rest = (int)Pu;
    for (long long c0 = 0; c0 < C; c0 += kWarp) {
        const long long c = c0 + lane;
        bool lost = false;
        if (c < C) {
            const uint32_t plo = (uint32_t)(c * Pu / C), phi = (uint32_t)((c + 1) * Pu / C);
            if (base + c < a.queue_cap) a.queue[base + c] = make_uint4(unit, plo, phi, (uint32_t)v);
            else lost = true;
        }
        const unsigned ball = __ballot_sync(kFull, lost);
        if (ball) {
            rest = (int)((c0 + __ffs(ball) - 1) * Pu / C);
            break;
        }
    }
    return rest;
}

// Queue rows [0, B) with per-row work work(j) as chunks of about a.target
// (two passes over the rows: count, then write).  Returns the first row the
// queue could not take (B when all fit).
template <typename WorkFn>
__device__ int queue_rows(const EnumArgs &a, uint32_t unit, int v, int B, WorkFn work, int lane) {
    unsigned long long base = 0, lim = 0;
    for (int pass = 0; pass < 2; pass++) {
        int cur = 0;
        long long acc = 0;
        unsigned long long nchunk = 0;
        for (int jb = 0; jb < B; jb += kWarp) {
            const int j = jb + lane;
            const long long w = j < B ? work(j) : 0;
            const long long incl = incl_scan64(w, lane);
            const long long btot = __shfl_sync(kFull, incl, kWarp - 1);
            long long used = 0;
            for (;;) {
                const unsigned ball = __ballot_sync(kFull, j < B && acc + incl - used >= a.target);
                if (!ball) {
                    acc += btot - used;
                    break;
                }
                const int r = __ffs(ball) - 1;
                const int end = jb + r + 1;
                if (pass == 1) {
                    if (base + nchunk >= lim) return cur;
                    if (lane == 0) a.queue[base + nchunk] = make_uint4(unit, (uint32_t)cur, (uint32_t)end, (uint32_t)v);
                }
                nchunk++;
                cur = end;
                used = __shfl_sync(kFull, incl, r);
                acc = 0;
            }
        }
        if (cur < B) {
            if (pass == 1) {
                if (base + nchunk >= lim) return cur;
                if (lane == 0) a.queue[base + nchunk] = make_uint4(unit, (uint32_t)cur, (uint32_t)B, (uint32_t)v);
            }
            nchunk++;
        }
        if (pass == 0) {
            base = reserve(a, nchunk, lane);
            lim = min(base + nchunk, a.queue_cap);
        }
    }
    return B;
}

// Sum of work(j) over rows [0, B), warp-reduced.
template <typename WorkFn>
__device__ __forceinline__ long long total_work(int B, WorkFn work, int lane) {
    long long s = 0;
    for (int j = lane; j < B; j += kWarp) s += work(j);
#pragma unroll
    for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
    return s;
}

// Run part [jlo, jhi) of one unit: virtual rows of its extension list for
// k = 3, 4, rows of the level-2 list E2 for k = 5.  In phase 1 (jlo = 0,
// jhi = all) a unit with more than a.light estimated work is queued in chunks
// instead.  D is the per-row allowance for exclusive neighbours (mean degree
// + 1); wmax bounds the count mode's work of one row (largest degree + row
// cost), so a short list skips summing its rows' work.
template <int K, bool COUNT, bool HASH, int WN = Layout<K>::WIN>
__device__ void process_unit(const EnumArgs &a, const GView &g, Sink<K> &sink, const Scratch &sc, uint32_t unit,
                             int v, int vglob, int jlo, int jhi, bool phase1, long long D, long long wmax, int lane) {
    using L = Layout<K>;
    if (K == 3 && COUNT) {
        // prefix {v}; E = neighbours of v above v; a heavy list is queued as
        // row ranges of equal scan work (the rows' neighbour counts)
        const int dv = g.deg[v], l = g.lo[v];
        const int B = dv - l;
        if (B <= 0) return;
        uint32_t *E = B <= sc.cap ? sc.buf[0] : sc.ovf[0];
        const long long rb = g.nptr[v] + l;
        for (int q = lane; q < B; q += kWarp) {
            const uint32_t xe = __ldg(g.nbr + rb + q);
            E[q] = ((xe >> 2) << 6) | (xe & 3u);
        }
        __syncwarp();
        int hi = min(jhi, B), rest = B;
        if (phase1) {
            auto work = [&](int j) { return (long long)g.deg[e_id(E[j])] + kRowCost; };
            // a list that cannot exceed the threshold even at the largest
            // degree of the set skips the sum (warp-uniform condition)
            bool heavy = false;
            if ((long long)B * wmax > a.light) heavy = total_work(B, work, lane) > a.light;
            if (heavy) {
                rest = queue_rows(a, unit, vglob, B, work, lane);
                if (rest >= B) return;
                hi = 0;
            }
        }
        const uint32_t pm[1] = {(uint32_t)v};
        // every row is a neighbour of the root, at position rb + j
        const uint2 *revA = g.rev ? g.rev + rb : nullptr;
        const int A = g.rev ? B : 0;
        if (hi > jlo)
            count_leaves<K, HASH, WN>(g, sink, E, B, jlo, hi, jlo == 0, pm, 0u, (uint32_t)v, false, sc.gcnt, sc.ring, revA,
                                  A, lane);
        if (rest < B)
            count_leaves<K, HASH, WN>(g, sink, E, B, rest, B, rest == 0, pm, 0u, (uint32_t)v, false, sc.gcnt, sc.ring,
                                  revA, A, lane);
        __syncwarp();
        return;
    }
    if (K == 3) {
        // prefix {v}; E = neighbours of v above v
        const int dv = g.deg[v], l = g.lo[v];
        const int B = dv - l;
        if (B <= 0) return;
        const int P = (B + 1) / 2;
        int hi = min(jhi, P), rest = P;
        if (phase1 && (long long)P * (B - 1) + (long long)B * D > a.light) {
            rest = queue_closed_form(a, unit, vglob, B, D, lane);
            if (rest >= P) return;
            hi = 0;
        }
        uint32_t *E = B <= sc.cap ? sc.buf[0] : sc.ovf[0];
        const long long rb = g.nptr[v] + l;
        for (int q = lane; q < B; q += kWarp) {
            const uint32_t xe = __ldg(g.nbr + rb + q);
            E[q] = ((xe >> 2) << 6) | (xe & 3u);
        }
        __syncwarp();
        const uint32_t pm[1] = {(uint32_t)v};
        leaves<K>(g, sink, E, B, jlo, hi, pm, 0u, (uint32_t)v, lane);
        if (rest < P) leaves<K>(g, sink, E, B, rest, P, pm, 0u, (uint32_t)v, lane);
        sink.flush();
        __syncwarp();
        return;
    }
    const long long rb = g.nptr[v];
    const int t = (int)(unit - rb);
    if (t < g.lo[v]) return;  // neighbour below v: not a unit
    const uint32_t e = __ldg(g.nbr + unit);
    const uint32_t w1 = e >> 2, s01 = e & 3u;
    int hi = jhi, rest = 0x7FFFFFFF;
    if (K == 4 && COUNT) {
        uint32_t *E2;
        long long wk = 0;  // this lane's share of the list's scan work (phase 1)
        const int B2 = build_level2<HASH>(g, unit, v, w1, sc, &E2, lane, phase1 ? &wk : nullptr);
        if (B2 <= 0) return;
        hi = min(hi, B2);
        rest = B2;
        if (phase1) {
            auto work = [&](int j) { return (long long)g.deg[e_id(E2[j])] + kRowCost; };
            bool heavy = false;  // as for k = 3: the sum only when it can pass the threshold
            if ((long long)B2 * wmax > a.light) {
#pragma unroll
                for (int d = 16; d; d >>= 1) wk += __shfl_xor_sync(kFull, wk, d);
                heavy = wk > a.light;
            }
            if (heavy) {
                rest = queue_rows(a, unit, vglob, B2, work, lane);
                if (rest >= B2) return;
                hi = 0;
            }
        }
        const uint32_t pm[2] = {(uint32_t)v, w1};
        const uint32_t pcode = s01 << (L::SH_ROW + 4);
        // part A of the list (the neighbours of v after w1) sits at
        // positions unit + 1 + j of v's list
        const uint2 *revA = g.rev ? g.rev + unit + 1 : nullptr;
        const int A = g.rev ? g.deg[v] - t - 1 : 0;
        if (hi > jlo)
            count_leaves<K, HASH, WN>(g, sink, E2, B2, jlo, hi, jlo == 0, pm, pcode, (uint32_t)v, false, sc.gcnt, sc.ring,
                                  revA, A, lane);
        if (rest < B2)
            count_leaves<K, HASH, WN>(g, sink, E2, B2, rest, B2, rest == 0, pm, pcode, (uint32_t)v, false, sc.gcnt,
                                  sc.ring, revA, A, lane);
        __syncwarp();
        return;
    }
    if (K == 4 && phase1) {
        long long Bu = (long long)(g.deg[v] - t - 1) + g.deg[w1];
        if (Bu > g.n - 2) Bu = g.n - 2;
        if (Bu <= 0) return;
        const long long Pu = (Bu + 1) / 2;
        if (Pu * (Bu - 1) + Bu * D > a.light) {
            rest = queue_closed_form(a, unit, vglob, Bu, D, lane);
            if (rest >= Pu) return;
            hi = 0;
        }
    }
    uint32_t *E2;
    const int B2 = build_level2<HASH>(g, unit, v, w1, sc, &E2, lane, nullptr);
    if (B2 <= 0) return;
    if (K == 4) {
        // rows of E2 are paired into virtual rows
        const int P2 = (B2 + 1) / 2;
        hi = min(hi, P2);
        rest = min(rest, P2);
        const uint32_t pm[2] = {(uint32_t)v, w1};
        const uint32_t pcode = s01 << (L::SH_ROW + 4);  // field of slot 1 sits above slot 2's
        leaves<K>(g, sink, E2, B2, jlo, hi, pm, pcode, (uint32_t)v, lane);
        if (rest < P2) leaves<K>(g, sink, E2, B2, rest, P2, pm, pcode, (uint32_t)v, lane);
        sink.flush();
        __syncwarp();
        return;
    }
    hi = min(hi, B2);
    rest = min(rest, B2);
    // K == 5: one more level.  Row j2 of E2 gives w2 and the list E3.
    if (phase1) {
        auto work = [&](int j) {
            const long long b = (long long)(B2 - 1 - j) + g.deg[e_id(E2[j])];
            return COUNT ? b * (D + 1) + 64 : b * (b - 1) / 2 + b * D + 1;
        };
        if (total_work(B2, work, lane) > a.light) {
            rest = queue_rows(a, unit, vglob, B2, work, lane);
            hi = 0;
        }
    }
    // fields: slot 1 at bit 18 (state(v, w1)), slot 2 at bit 14 (w2's states
    // to v and w1)
    const uint32_t pc01 = s01 << 18;
    const PRow row_v = prow<HASH>(g, (uint32_t)v), row_w1 = prow<HASH>(g, w1);
    if constexpr (K == 5 && COUNT) {
        const uint32_t p0[2] = {(uint32_t)v, w1};
        const PRow rows0[2] = {row_v, row_w1};
        // part A of E2 (the neighbours of v after w1) at positions unit + 1 + j
        const uint2 *revA = g.rev ? g.rev + unit + 1 : nullptr;
        const int A2 = g.rev ? g.deg[v] - t - 1 : 0;
        if (hi > jlo) count_last_lists<K, HASH>(g, sink, sc, E2, B2, jlo, hi, pc01, p0, rows0, revA, A2, lane);
        if (rest < B2) count_last_lists<K, HASH>(g, sink, sc, E2, B2, rest, B2, pc01, p0, rows0, revA, A2, lane);
        __syncwarp();
        return;
    }
    if constexpr (!COUNT) {
        for (int pass = 0; pass < 2; pass++) {
            const int r0 = pass == 0 ? jlo : rest;
            const int r1 = pass == 0 ? hi : B2;
            for (int j2 = r0; j2 < r1; j2++) {
                const uint32_t e2 = E2[j2];
                const uint32_t w2 = e_id(e2);
                const uint32_t pcode = pc01 | ((e2 & 15u) << 14);
                const int A3 = B2 - 1 - j2;
                const int dw = g.deg[w2];
                const long long ub = (long long)A3 + dw;
                uint32_t *E3 = ub <= sc.cap ? sc.buf[1] : sc.ovf[1];
                // level-3 list: the level-2 list after w2 (with w2's states),
                // then the neighbours of w2 above v adjacent to neither v nor w1,
                // both read in one pass (the neighbours at or below v skipped by
                // their ids)
                const PRow row_w2 = prow<HASH>(g, w2);
                const long long wb = g.nptr[w2];
                const int nq = max(A3, dw);
                int pos = A3;
                for (int q0 = 0; q0 < nq; q0 += kWarp) {
                    const int q = q0 + lane;
                    const bool in_a = q < A3;
                    uint32_t xe = 0, ue = 0;
                    if (in_a) xe = E2[j2 + 1 + q];
                    if (q < dw) ue = __ldg(g.nbr + wb + q);
                    const uint32_t x = e_id(xe), u = ue >> 2;
                    uint32_t sa = 0;
                    bool keep = false;
                    if (in_a) sa = pget<HASH>(row_w2, x);
                    if (q < dw && u > (uint32_t)v) keep = pget<HASH>(row_v, u) == 0u && pget<HASH>(row_w1, u) == 0u;
                    if (in_a) E3[q] = (x << 6) | (xe & 15u) | (sa << 4);
                    const unsigned ball = __ballot_sync(kFull, keep);
                    if (keep) E3[pos + __popc(ball & ((1u << lane) - 1u))] = (u << 6) | ((ue & 3u) << 4);
                    pos += __popc(ball);
                }
                __syncwarp();
                const uint32_t pm[3] = {(uint32_t)v, w1, w2};
                leaves<K>(g, sink, E3, pos, 0, (pos + 1) / 2, pm, pcode, (uint32_t)v, lane);
                __syncwarp();
            }
            if (rest >= B2) break;
        }
    }
    sink.flush();
    __syncwarp();
}

// One instantiation per phase, so each is register-allocated for its own path
// (phase 1: the unit loop, work estimates and queueing; phase 2: the queue),
// and per kind of set (SET: several graphs, each seen through its offsets;
// otherwise one graph read through the kernel's own arrays).
template <int K, bool COUNT, int PHASE, bool SET, bool HASH>
__global__ void __launch_bounds__(kThreads, K == 5 ? ACC_MINB5 : (COUNT ? (SET ? ACC_MINB34S : ACC_MINB34C) : ACC_MINB34))
    k_enum(EnumArgs a) {
    grid_dep_wait();
    using L = Layout<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    int16_t *lut_s = reinterpret_cast<int16_t *>(smem);
    uint32_t *pending = reinterpret_cast<uint32_t *>(smem + L::lut);
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + L::lut + L::pending);
    uint32_t *ebuf = reinterpret_cast<uint32_t *>(smem + L::lut + L::pending + L::hist);
    uint32_t *groups = reinterpret_cast<uint32_t *>(smem + L::lut + L::pending + L::hist + L::ebuf);
    uint32_t *rings = reinterpret_cast<uint32_t *>(smem + L::lut + L::pending + L::hist + L::ebuf + L::groups);
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    constexpr bool several = SET;
    // phase 2 with nothing queued: no table to stage, nothing to flush
    if constexpr (PHASE == 2)
        if (a.info->queue_tail == 0) return;
    // a set refused by the count bound of the degree scan is not enumerated
    // (phase 1 then queues nothing, so phase 2 returns above)
    if constexpr (PHASE == 1)
        if (a.status && *(volatile int *)a.status == ACC_ERR_OVERFLOW) return;

    if (L::SMEM_LUT)
        for (int i = tid; i < (1 << L::NB); i += blockDim.x) lut_s[i] = a.lut[i];
    const int hist_words = K == 5 ? L::HSTRIDE : kWarpsPerBlock * L::HSTRIDE;
    for (int i = tid; i < hist_words; i += blockDim.x) hist[i] = 0;
    if (tid == 0) *pending = 0;
    __syncthreads();

    Sink<K> sink;
    sink.hist = K == 5 ? hist : hist + wib * L::HSTRIDE;
    sink.lut = L::SMEM_LUT ? lut_s : a.lut;
    sink.counts_base = a.counts;
    sink.counts = a.counts;
    sink.gcur = several ? -1 : 0;
    sink.direct = K == 5 && several;
    sink.pending = pending;
    sink.since = 0;
    sink.status = a.status;
    sink.run_cls = -1;
    sink.run_len = 0;

    Scratch sc;
    const long long gw = (long long)blockIdx.x * kWarpsPerBlock + wib;
    sc.buf[0] = ebuf + (size_t)wib * L::LISTS * L::CAP;
    sc.buf[1] = sc.buf[0] + L::CAP;
    // per-warp scratch: two overflow lists, then the collected part-B rows
    sc.ovf[0] = a.scratch + gw * a.scratch_per_warp;
    sc.ovf[1] = sc.ovf[0] + (a.scratch_per_warp - 2 * kPartBRows) / 2;
    sc.pb = sc.ovf[0] + (a.scratch_per_warp - 2 * kPartBRows);
    sc.cap = L::CAP;
    sc.gcnt = groups + (size_t)wib * 2 * L::G;
    sc.ring = rings + (size_t)wib * L::RING_ARRAYS * L::RING;
    sink.moved = 0;
    sink.scanned = 0;
    const long long nnz = a.info->nnz;
    const long long NV = a.gs.NV;
    const long long D = (NV > 0 ? nnz / NV : 0) + 1;
    const long long wmax = (long long)a.info->maxdeg + kRowCost;  // largest work of one list row

    if constexpr (PHASE == 1) {
        // units: roots (k = 3) or G* arc positions (v, w1) with w1 > v
        constexpr bool ROOTS = K == 3;
        const long long nunits = ROOTS ? NV : nnz;
        const int grab = a.gs.B > 1 ? ACC_GRAB_SET : (K == 4 && !ROOTS ? ACC_GRAB4 : kGrab);
        for (;;) {
            unsigned long long u0 = 0;
            if (lane == 0) u0 = atomicAdd(&a.info->unit_ctr, (unsigned long long)grab);
            u0 = __shfl_sync(kFull, u0, 0);
            if ((long long)u0 >= nunits) break;
            const long long u1 = min((long long)u0 + grab, nunits);
            // arc units: each grabbed position's row vertex (bit 31: a
            // neighbour below the row's vertex, not a unit), one per lane
            uint32_t rows = 0;
            if (!ROOTS && u0 + lane < (unsigned long long)u1) rows = __ldg(a.src + u0 + lane);
            for (long long u = (long long)u0; u < u1; u++) {
                int vg;
                if (ROOTS) {
                    vg = (int)u;
                } else {
                    const uint32_t r = __shfl_sync(kFull, rows, (int)(u - (long long)u0));
                    if (r >> 31) continue;
                    vg = (int)r;
                }
                if constexpr (SET) {
                    const int gi = a.gs.graph_of(vg);
                    const GMeta mt = a.gs.meta(gi);
                    sink.switch_graph(gi, lane);
                    process_unit<K, COUNT, HASH>(a, view_of(a, mt), sink, sc, (uint32_t)u, vg - mt.voff, vg, 0,
                                                 0x7FFFFFFF, true, D, wmax, lane);
                } else {
                    process_unit<K, COUNT, HASH>(a, view_single(a), sink, sc, (uint32_t)u, vg, vg, 0, 0x7FFFFFFF,
                                                 true, D, wmax, lane);
                }
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
            const int vg = (int)it.w;
            if constexpr (SET) {
                const int gi = a.gs.graph_of(vg);
                const GMeta mt = a.gs.meta(gi);
                sink.switch_graph(gi, lane);
                process_unit<K, COUNT, HASH, kWinP2<K>>(a, view_of(a, mt), sink, sc, it.x, vg - mt.voff, vg,
                                                        (int)it.y, (int)it.z, false, D, wmax, lane);
            } else {
                process_unit<K, COUNT, HASH, kWinP2<K>>(a, view_single(a), sink, sc, it.x, vg, vg, (int)it.y,
                                                        (int)it.z, false, D, wmax, lane);
            }
        }
    }

    if (COUNT && lane == 0 && sink.scanned) atomicAdd(&a.info->scanned, sink.scanned);
    __syncthreads();
    // an add that found no class (never expected) is an internal error
    if (K <= 4 ? (lane == 0 && sink.hist[L::NCLS] != 0u) : (tid == 0 && hist[L::NCLS] != 0u))
        set_status(a.status, ACC_ERR_INTERNAL);
    if (several) {
        // each warp drains its own histogram to the graph it ended on
        // (k = 5 with several graphs counted straight into int64)
        if (K <= 4 && sink.gcur >= 0) {
            for (int c = lane; c < L::NCLS; c += kWarp) {
                const int32_t v = (int32_t)sink.hist[c];
                if (v) atomicAdd(&sink.counts[c], (unsigned long long)(long long)v);
            }
        }
    } else if (K == 5) {
        for (int c = tid; c < L::NCLS; c += blockDim.x) {
            const int32_t v = (int32_t)hist[c];
            if (v) atomicAdd(&a.counts[c], (unsigned long long)(long long)v);
        }
    } else {
        for (int c = tid; c < L::NCLS; c += blockDim.x) {
            long long s = 0;
            for (int w = 0; w < kWarpsPerBlock; w++) s += (int32_t)hist[w * L::HSTRIDE + c];
            if (s) atomicAdd(&a.counts[c], (unsigned long long)s);
        }
    }
}

template <int K, bool COUNT, int PHASE, bool SET, bool HASH>
int blocks_per_sm() {
    static int cached = 0;
    if (cached) return cached;
    if (cudaFuncSetAttribute(k_enum<K, COUNT, PHASE, SET, HASH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Layout<K>::total) != cudaSuccess)
        return -1;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_enum<K, COUNT, PHASE, SET, HASH>, kThreads,
                                                      Layout<K>::total) != cudaSuccess ||
        b < 1)
        return -1;
    cached = b;
    return b;
}

template <int K, bool COUNT, int PHASE, bool SET, bool HASH>
int launch_phase(const EnumArgs &a, int num_sms, cudaStream_t s, int grid_num, int grid_den) {
    const int bps = blocks_per_sm<K, COUNT, PHASE, SET, HASH>();
    if (bps < 1) return ACC_ERR_CUDA;
    int grid = (int)((long long)num_sms * bps * grid_num / grid_den);
    if (grid < num_sms) grid = num_sms;
    if (grid > num_sms * bps) grid = num_sms * bps;
    launch_pdl(k_enum<K, COUNT, PHASE, SET, HASH>, grid, kThreads, Layout<K>::total, s, a);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

template <int K, bool COUNT, bool SET, bool HASH>
int launch_ph(const EnumArgs &a, int num_sms, int phase, cudaStream_t s, int grid_num, int grid_den) {
    return phase == 1 ? launch_phase<K, COUNT, 1, SET, HASH>(a, num_sms, s, grid_num, grid_den)
                      : launch_phase<K, COUNT, 2, SET, HASH>(a, num_sms, s, grid_num, grid_den);
}

// Hashed adjacency is read by the count mode only (the enumerate mode probes
// pairs of list members, for which the dense block is kept).
template <int K, bool COUNT>
int launch_k(const EnumArgs &a, int num_sms, int phase, cudaStream_t s, int grid_num, int grid_den) {
    const bool set = a.gs.B > 1;
    if constexpr (COUNT) {
        if (a.nh)
            return set ? launch_ph<K, true, true, true>(a, num_sms, phase, s, grid_num, grid_den)
                       : launch_ph<K, true, false, true>(a, num_sms, phase, s, grid_num, grid_den);
    }
    return set ? launch_ph<K, COUNT, true, false>(a, num_sms, phase, s, grid_num, grid_den)
               : launch_ph<K, COUNT, false, false>(a, num_sms, phase, s, grid_num, grid_den);
}

// Most resident blocks per SM of any instantiation for k (sizes the per-warp
// overflow lists).
template <int K>
int bps_max() {
    const int b[12] = {blocks_per_sm<K, false, 1, false, false>(), blocks_per_sm<K, false, 2, false, false>(),
                       blocks_per_sm<K, true, 1, false, false>(),  blocks_per_sm<K, true, 2, false, false>(),
                       blocks_per_sm<K, false, 1, true, false>(),  blocks_per_sm<K, false, 2, true, false>(),
                       blocks_per_sm<K, true, 1, true, false>(),   blocks_per_sm<K, true, 2, true, false>(),
                       blocks_per_sm<K, true, 1, false, true>(),   blocks_per_sm<K, true, 2, false, true>(),
                       blocks_per_sm<K, true, 1, true, true>(),    blocks_per_sm<K, true, 2, true, true>()};
    int m = 0;
    for (int x : b) {
        if (x < 1) return -1;
        if (x > m) m = x;
    }
    return m;
}

}  // namespace

long long enum_default_light(int k, bool count_mode) { return k == 4 && count_mode ? ACC_LIGHT4 : ACC_LIGHT; }
long long enum_default_target(int k, bool count_mode) { return k == 5 && count_mode ? ACC_TARGET5 : ACC_TARGET; }

int enum_grid_warps(int k, int num_sms) {
    const int bps = k == 3 ? bps_max<3>() : (k == 4 ? bps_max<4>() : bps_max<5>());
    if (bps < 1) return ACC_ERR_CUDA;
    return num_sms * bps * kWarpsPerBlock;
}

int launch_enumerate(int k, const EnumArgs &a, int num_sms, int phase, cudaStream_t s, int grid_num, int grid_den) {
    const bool c = a.mode == 0;
    switch (k) {
    case 3: return c ? launch_k<3, true>(a, num_sms, phase, s, grid_num, grid_den)
                     : launch_k<3, false>(a, num_sms, phase, s, grid_num, grid_den);
    case 4: return c ? launch_k<4, true>(a, num_sms, phase, s, grid_num, grid_den)
                     : launch_k<4, false>(a, num_sms, phase, s, grid_num, grid_den);
    case 5: return c ? launch_k<5, true>(a, num_sms, phase, s, grid_num, grid_den)
                     : launch_k<5, false>(a, num_sms, phase, s, grid_num, grid_den);
    default: return ACC_ERR_K;
    }
}

}  // namespace acc
