"""Scenarios run against the whole library built for the host (every CUDA
source compiled with the shim and the stand-in runtime, where device memory
is host memory), through the C ABI with the Python binding's own signature
table.  Run as a child process, one scenario per call:

    python tests/emu/lib_scenarios.py <library.so> <scenario>

Each scenario compares what the library returns with the oracle and raises
on the first difference; exit status 0 means it passed.  Buffers the ABI
calls device buffers are numpy arrays here."""
import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_1203_3415_gb300 as acc  # noqa: E402  (constants, types and the signature table only)
import synth  # noqa: E402
from tests.graph_helpers import esu_scanned_entries, random_digraph  # noqa: E402

NCLS = {3: 13, 4: 199, 5: 9364}


def P(a):
    return ctypes.c_void_p(a.ctypes.data)


def csr(n, s, d):
    s, d = np.asarray(s, np.int64), np.asarray(d, np.int64)
    order = np.lexsort((d, s))
    col = np.ascontiguousarray(d[order], dtype=np.int32)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(s, minlength=n), out=rowptr[1:])
    return rowptr, col


def sync(lib):
    """Wait for the device, as a caller does before reading what an
    asynchronous call wrote (the stand-in runtime's deferred mode holds the
    work until then)."""
    lib.emu_device_synchronize()


def ok(rc, what):
    if rc != 0:
        raise AssertionError(f"{what}: returned {rc}")


class Ctx:
    def __init__(self, lib):
        self.lib = lib
        self.h = ctypes.c_void_p()
        self.bufs = {}
        ok(lib.acc_ctx_create(ctypes.byref(self.h), 0), "acc_ctx_create")

    def count(self, rowptr, col, n, k):
        # the same output buffers every call, as a caller repeating a count
        # does (the launch-graph replay recognises a repeat by its pointers)
        out, st = self.bufs.setdefault(k, (np.zeros(NCLS[k], np.int64), np.zeros(1, np.int32)))
        out[:] = -1
        st[:] = -1
        rc = self.lib.acc_motif_count(self.h, P(rowptr), P(col), n, len(col), k, None, P(out), P(st))
        sync(self.lib)  # with a status pointer the count only enqueues
        return rc, int(st[0]), out.copy()

    def stats(self):
        s = np.zeros(acc.ACC_STATS_LEN, np.int64)
        ok(self.lib.acc_motif_last_stats(self.h, P(s)), "acc_motif_last_stats")
        return s

    def close(self):
        self.lib.acc_ctx_destroy(self.h)


def graphs(seed, count, nmax):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(3, nmax))
        s, d = random_digraph(rng, n, p=float(rng.uniform(0.1, 0.4)), recip=float(rng.random()))
        out.append((n, np.asarray(s, np.int64), np.asarray(d, np.int64)))
    return out


def scenario_modes(lib):
    """Every k in every counting mode, on several graphs, on one context."""
    c = Ctx(lib)
    cases = {3: graphs(1, 3, 40), 4: graphs(2, 3, 22), 5: graphs(3, 2, 12)}
    g = synth.chung_lu(60, 200, 2.1, 30, 20, 4)
    cases[4].append((g.n, g.src, g.dst))
    for mode in (acc.ACC_MODE_COUNT, acc.ACC_MODE_ENUMERATE, acc.ACC_MODE_FORMULA, acc.ACC_MODE_AUTO):
        ok(lib.acc_ctx_set_mode(c.h, mode), "acc_ctx_set_mode")
        for k, gs in cases.items():
            for n, s, d in gs:
                rp, cl = csr(n, s, d)
                rc, st, got = c.count(rp, cl, n, k)
                want = oracle.count(n, s, d, k)
                if rc or st or got.tolist() != want.tolist():
                    raise AssertionError(f"mode {mode} k {k} n {n}: rc {rc} status {st}")
                # the count mode's work figure equals the same sum over a
                # plain ESU walk (below 1024 vertices nothing is renumbered);
                # the automatic mode takes the count mode for k = 4, 5 and the
                # formula path (no scan) for k = 3 on these small graphs
                counted = mode == acc.ACC_MODE_COUNT or (mode == acc.ACC_MODE_AUTO and k > 3)
                if counted and c.stats()[6] != esu_scanned_entries(n, s, d, k):
                    raise AssertionError(f"mode {mode} k {k} n {n}: {c.stats()[6]} entries scanned")
                if mode == acc.ACC_MODE_AUTO and k == 3 and n > 0 and c.stats()[6] != 0:
                    raise AssertionError(f"automatic mode, k 3, n {n}: not the formula path")
    # the count mode probing the hashed adjacency tables (built on the device
    # after the neighbour lists: one more kernel), with the lists built with
    # and without the dense block, and the dense block again
    ok(lib.acc_ctx_set_mode(c.h, acc.ACC_MODE_COUNT), "acc_ctx_set_mode")
    for adj in (acc.ACC_ADJ_HASH, acc.ACC_ADJ_SPARSE, acc.ACC_ADJ_DENSE, acc.ACC_ADJ_SPARSE, acc.ACC_ADJ_HASH):
        ok(lib.acc_ctx_set_adjacency(c.h, adj), "acc_ctx_set_adjacency")
        for k, gs in cases.items():
            for n, s, d in gs:
                rp, cl = csr(n, s, d)
                rc, st, got = c.count(rp, cl, n, k)
                if rc or st or got.tolist() != oracle.count(n, s, d, k).tolist():
                    raise AssertionError(f"adjacency {adj} k {k} n {n}: rc {rc} status {st}")
    if lib.acc_ctx_set_adjacency(c.h, 4) != acc.ACC_ERR_ARG:
        raise AssertionError("an unknown adjacency choice is accepted")
    if lib.acc_ctx_set_mode(c.h, 4) != acc.ACC_ERR_ARG:
        raise AssertionError("an unknown mode is accepted")
    c.close()


def scenario_repeats(lib):
    """Repeated counts replay one captured launch sequence: the same counts
    as launching one by one, also when the buffers' contents change, after a
    malformed repeat, and with launch graphs switched off."""
    replays = lib.emu_graph_launch_count
    replays.restype = ctypes.c_longlong
    c = Ctx(lib)
    # 1200 vertices: renumbered, so the sequence is 10 kernels (the build's
    # six, the reverse positions, two enumeration phases, the block clear)
    g = synth.chung_lu(1200, 2400, 2.2, 60, 20, 5)
    rp, cl = csr(g.n, g.src, g.dst)
    want = oracle.count(g.n, g.src, g.dst, 3).tolist()
    for i in range(4):
        rc, st, got = c.count(rp, cl, g.n, 3)
        if rc or st or got.tolist() != want or c.stats()[0] != 10:
            raise AssertionError(f"repeat {i}: rc {rc} status {st} launches {c.stats()[0]}")
    # a fresh context's first count leaves the pair-state buffer clean, the
    # second is remembered, the third is captured and launched, the fourth
    # replayed
    if replays() != 2:
        raise AssertionError(f"{replays()} graph launches for 4 counts")
    # 80 vertices (8 kernels: no renumbering), k = 4
    g = synth.chung_lu(80, 250, 2.1, 30, 20, 5)
    rp, cl = csr(g.n, g.src, g.dst)
    want = oracle.count(g.n, g.src, g.dst, 4).tolist()
    for i in range(3):
        rc, st, got = c.count(rp, cl, g.n, 4)
        if rc or st or got.tolist() != want or c.stats()[0] != 8:
            raise AssertionError(f"k = 4 repeat {i}: rc {rc} status {st} launches {c.stats()[0]}")
    # new arcs in the same buffers (same n and m)
    for seed in (11, 12):
        h = synth.erdos_renyi(g.n, len(cl), 10, seed)
        r2, c2 = csr(g.n, h.src, h.dst)
        rp[:] = r2
        cl[:] = c2
        rc, st, got = c.count(rp, cl, g.n, 4)
        if rc or st or got.tolist() != oracle.count(g.n, h.src, h.dst, 4).tolist():
            raise AssertionError(f"contents changed, seed {seed}")
    keep = int(cl[0])
    cl[0] = 0  # row 0's first arc becomes a self-loop
    rc, st, _ = c.count(rp, cl, g.n, 4)
    if rc != 0 or st != acc.ACC_ERR_INPUT:
        raise AssertionError(f"malformed repeat: rc {rc} status {st}")
    cl[0] = keep
    want = oracle.count(g.n, np.repeat(np.arange(g.n), np.diff(rp)), cl.astype(np.int64), 4).tolist()
    for i in range(2):
        rc, st, got = c.count(rp, cl, g.n, 4)
        if rc or st or got.tolist() != want:
            raise AssertionError(f"recovery {i}")
    before = replays()
    if before != 2 + 7:
        raise AssertionError(f"k = 4 repeats replayed {before - 2} times")
    ok(lib.acc_ctx_set_launch_graphs(c.h, 0), "acc_ctx_set_launch_graphs")
    for i in range(2):
        rc, st, got = c.count(rp, cl, g.n, 4)
        if rc or st or got.tolist() != want:
            raise AssertionError("launch graphs off")
    if replays() != before:
        raise AssertionError("a graph replayed with launch graphs off")
    c.close()


def scenario_host_and_errors(lib):
    """The host-buffer entry point, the synchronous status (NULL status
    pointer), and the host-checked argument errors."""
    c = Ctx(lib)
    n, s, d = graphs(6, 1, 30)[0]
    rp, cl = csr(n, s, d)
    for k in (3, 4):
        out = np.zeros(NCLS[k], np.int64)
        ok(lib.acc_motif_count_host(c.h, P(rp), P(cl), n, len(cl), k, P(out)), "count_host")
        if out.tolist() != oracle.count(n, s, d, k).tolist():
            raise AssertionError(f"count_host k {k}")
    bad = cl.copy()
    bad[0] = n  # target out of range
    out = np.zeros(13, np.int64)
    rc = lib.acc_motif_count(c.h, P(rp), P(bad), n, len(bad), 3, None, P(out), None)
    if rc != acc.ACC_ERR_INPUT:
        raise AssertionError(f"synchronous status: {rc}")
    if lib.acc_motif_count(c.h, P(rp), P(cl), n, len(cl), 6, None, P(out), None) != acc.ACC_ERR_K:
        raise AssertionError("k = 6 accepted")
    if lib.acc_motif_count(c.h, None, P(cl), n, len(cl), 3, None, P(out), None) != acc.ACC_ERR_ARG:
        raise AssertionError("null rowptr accepted")
    # above the size limits (the count mode takes graphs above the dense
    # block's limit, up to ACC_MAX_N_SPARSE): refused on the host, before the
    # undersized arrays passed here could be read
    if lib.acc_motif_count(c.h, P(rp), P(cl), acc.ACC_MAX_N_SPARSE + 1, len(cl), 3, None, P(out), None) != \
            acc.ACC_ERR_TOO_LARGE:
        raise AssertionError("n above the sparse limit accepted")
    ok(lib.acc_ctx_set_mode(c.h, acc.ACC_MODE_ENUMERATE), "acc_ctx_set_mode")
    if lib.acc_motif_count(c.h, P(rp), P(cl), acc.ACC_MAX_N + 1, len(cl), 3, None, P(out), None) != \
            acc.ACC_ERR_TOO_LARGE:
        raise AssertionError("n above the dense limit accepted outside the count mode")
    ok(lib.acc_ctx_set_mode(c.h, acc.ACC_MODE_COUNT), "acc_ctx_set_mode")
    # an empty graph counts nothing
    e_rp = np.zeros(5, np.int64)
    rc = lib.acc_motif_count(c.h, P(e_rp), P(np.zeros(1, np.int32)), 4, 0, 3, None, P(out), None)
    if rc or out.any():
        raise AssertionError("empty graph")
    c.close()


def _descs(gs):
    arrays = [csr(n, s, d) for n, s, d in gs]
    descs = (acc.acc_graph_desc * len(gs))()
    for i, ((n, _, _), (rp, cl)) in enumerate(zip(gs, arrays)):
        descs[i].rowptr = rp.ctypes.data
        descs[i].col = cl.ctypes.data
        descs[i].n = n
        descs[i].m = len(cl)
    return descs, arrays


def scenario_batch(lib):
    """A batch of graphs prepared once and run several times in every mode,
    then the autotuner, for k = 3, 4 and 5; each k prepared in another mode
    (a run in a mode that needs more workspace than the prepare's grows it
    first)."""
    c = Ctx(lib)
    for k, nmax, prep_mode in ((3, 30, acc.ACC_MODE_ENUMERATE), (4, 18, acc.ACC_MODE_COUNT),
                               (5, 10, acc.ACC_MODE_FORMULA)):
        gs = graphs(20 + k, 6, nmax)
        gs.insert(2, (5, np.zeros(0, np.int64), np.zeros(0, np.int64)))
        descs, keep = _descs(gs)
        ok(lib.acc_ctx_set_mode(c.h, prep_mode), "set_mode before prepare")
        ok(lib.acc_motif_batch_prepare(c.h, descs, len(gs), k, None), "batch_prepare")
        want = [oracle.count(n, s, d, k).tolist() for n, s, d in gs]
        # every mode on the same prepared batch (graph sets take each mode's
        # per-graph counting branch)
        for mode in (acc.ACC_MODE_COUNT, acc.ACC_MODE_ENUMERATE, acc.ACC_MODE_FORMULA, acc.ACC_MODE_COUNT):
            ok(lib.acc_ctx_set_mode(c.h, mode), "set_mode")
            for rep in range(2):
                out = np.full(len(gs) * NCLS[k], -1, np.int64)
                st = np.full(1, -1, np.int32)
                ok(lib.acc_motif_batch_run(c.h, None, P(out), P(st)), "batch_run")
                sync(lib)
                if st[0] != 0 or out.reshape(len(gs), -1).tolist() != want:
                    raise AssertionError(f"batch k {k} mode {mode} rep {rep}")
        if k == 4:
            light, target = ctypes.c_int64(), ctypes.c_int64()
            ms = ctypes.c_float()
            ok(lib.acc_motif_batch_autotune(c.h, None, ctypes.byref(light), ctypes.byref(target), ctypes.byref(ms)),
               "autotune")
            out = np.full(len(gs) * NCLS[k], -1, np.int64)
            ok(lib.acc_motif_batch_run(c.h, None, P(out), None), "batch_run after autotune")
            sync(lib)
            if out.reshape(len(gs), -1).tolist() != want:
                raise AssertionError("batch after autotune")
        out = np.full(len(gs) * NCLS[k], -1, np.int64)
        ok(lib.acc_motif_count_batch(c.h, descs, len(gs), k, None, P(out), None), "count_batch")
        if out.reshape(len(gs), -1).tolist() != want:
            raise AssertionError(f"count_batch k {k}")
    c.close()


def scenario_significance(lib):
    """Device randomisation (both modes, speculative and row-scanning) then
    counting the copies and Z-scores, against the oracle's copies, counts
    and Z-scores."""
    c = Ctx(lib)
    gs = graphs(30, 3, 16)
    descs, arrays = _descs(gs)
    R, q = 3, 2
    seeds = np.array([5, 6, 7], np.uint64)
    M = sum(len(cl) for _, cl in arrays)
    for mode in (acc.ACC_RAND_SWAP, acc.ACC_RAND_MUTUAL):
        for mem in (1 << 30, 0):
            ok(lib.acc_ctx_set_randomise_memory(c.h, mem), "set_randomise_memory")
            out = np.full(R * M, -1, np.int32)
            accepted = np.full(len(gs) * R, -1, np.int64)
            st = np.full(1, -1, np.int32)
            ok(lib.acc_swap_randomise(c.h, descs, len(gs), R, q, P(seeds), mode, None, P(out), P(accepted), P(st)),
               "swap_randomise")
            sync(lib)
            if st[0] != 0:
                raise AssertionError(f"randomise status {st[0]}")
            off = 0
            for g, ((n, _, _), (rp, cl)) in enumerate(zip(gs, arrays)):
                m = len(cl)
                for r in range(R):
                    want, wa = oracle.swap_randomise(n, rp, cl, q * m, int(seeds[g]) + r, mode)
                    if not np.array_equal(out[off + r * m: off + (r + 1) * m], want) or accepted[g * R + r] != wa:
                        raise AssertionError(f"copy mode {mode} mem {mem} graph {g} copy {r}")
                off += R * m
    # count the real graph and its copies as one batch, then Z-scores
    k = 3
    g0, (rp0, cl0) = gs[0], arrays[0]
    n0, m0 = g0[0], len(cl0)
    copies = [cl0] + [out[r * m0:(r + 1) * m0].copy() for r in range(R)]
    group = [(n0, np.repeat(np.arange(n0), np.diff(rp0)), cc.astype(np.int64)) for cc in copies]
    descs2, keep2 = _descs(group)
    counts = np.zeros((R + 1) * NCLS[k], np.int64)
    ok(lib.acc_motif_count_batch(c.h, descs2, R + 1, k, None, P(counts), None), "count_batch copies")
    z = np.zeros(NCLS[k], np.float64)
    ok(lib.acc_motif_zscores(P(counts), 1, R + 1, k, None, P(z)), "zscores")
    sync(lib)
    cnt = counts.reshape(R + 1, -1)
    want = oracle.zscores(cnt[0], cnt[1:])
    if not np.array_equal(z, want, equal_nan=True):
        raise AssertionError("zscores")
    c.close()


def scenario_server(lib):
    """The request server: resident graphs, requests of every k, both
    policies, polled and drained; every finished request's counts equal the
    oracle's."""
    srv = ctypes.c_void_p()
    ok(lib.acc_server_create(ctypes.byref(srv), 0, 3, 1 << 30), "server_create")
    gs = graphs(40, 4, 20)
    arrays = [csr(n, s, d) for n, s, d in gs]
    ids = []
    for (n, _, _), (rp, cl) in zip(gs, arrays):
        gid = ctypes.c_int32()
        ok(lib.acc_server_add_graph(srv, P(rp), P(cl), n, len(cl), ctypes.byref(gid)), "add_graph")
        ids.append(gid.value)
    ok(lib.acc_server_reserve(srv), "reserve")
    for policy in (acc.ACC_SERVE_FIFO, acc.ACC_SERVE_SHORTEST):
        ok(lib.acc_server_set_policy(srv, policy, 0.5), "set_policy")
        reqs = []
        for i, gid in enumerate(ids):
            for k in (3, 4, 5) if i < 2 else (3, 4):
                rid = ctypes.c_int64()
                ok(lib.acc_server_submit(srv, gid, k, ctypes.byref(rid)), "submit")
                reqs.append((rid.value, i, k))
        running, queued = ctypes.c_int32(), ctypes.c_int32()
        ok(lib.acc_server_progress(srv, ctypes.byref(running), ctypes.byref(queued)), "progress")
        ok(lib.acc_server_drain(srv), "drain")
        for rid, i, k in reqs:
            state = ctypes.c_int32()
            out = np.zeros(NCLS[k], np.int64)
            lat = ctypes.c_double()
            ok(lib.acc_server_poll(srv, rid, ctypes.byref(state), P(out), ctypes.byref(lat)), "poll")
            n, s, d = gs[i]
            if state.value != acc.ACC_REQ_DONE or out.tolist() != oracle.count(n, s, d, k).tolist():
                raise AssertionError(f"request {rid} graph {i} k {k}: state {state.value}")
    lib.acc_server_destroy(srv)
    # request errors: a malformed graph, and a graph whose workspace can
    # never fit the budget
    srv = ctypes.c_void_p()
    ok(lib.acc_server_create(ctypes.byref(srv), 0, 2, 1 << 30), "server_create")
    rp, cl = np.array([0, 1, 2, 2, 2], np.int64), np.array([1, 1], np.int32)  # self-loop 1 -> 1
    gid, rid, state = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    ok(lib.acc_server_add_graph(srv, P(rp), P(cl), 4, 2, ctypes.byref(gid)), "add_graph")
    ok(lib.acc_server_submit(srv, gid.value, 3, ctypes.byref(rid)), "submit")
    ok(lib.acc_server_drain(srv), "drain")
    ok(lib.acc_server_poll(srv, rid.value, ctypes.byref(state), None, None), "poll")
    if state.value != acc.ACC_ERR_INPUT:
        raise AssertionError(f"malformed request: state {state.value}")
    if lib.acc_server_submit(srv, 99, 3, ctypes.byref(rid)) != acc.ACC_ERR_ARG:
        raise AssertionError("unknown graph id accepted")
    if lib.acc_server_set_policy(srv, 7, 0.0) != acc.ACC_ERR_ARG:
        raise AssertionError("unknown policy accepted")
    lib.acc_server_destroy(srv)
    g = synth.chung_lu(3000, 9000, 2.2, 100, 10, 3)
    rp, cl = csr(g.n, g.src, g.dst)
    ok(lib.acc_server_create(ctypes.byref(srv), 0, 1, 1 << 16), "server_create")
    ok(lib.acc_server_add_graph(srv, P(rp), P(cl), g.n, len(cl), ctypes.byref(gid)), "add_graph")
    ok(lib.acc_server_submit(srv, gid.value, 4, ctypes.byref(rid)), "submit")
    ok(lib.acc_server_drain(srv), "drain")
    ok(lib.acc_server_poll(srv, rid.value, ctypes.byref(state), None, None), "poll")
    if state.value != acc.ACC_ERR_NOMEM:
        raise AssertionError(f"request over the budget: state {state.value}")
    lib.acc_server_destroy(srv)


def scenario_misc_api(lib):
    """The small entry points: error strings, class counts, prepare, the
    schedule, timing, statistics, options and their argument checks."""
    lib.acc_strerror.restype = ctypes.c_char_p
    for code in range(0, -10, -1):
        if not lib.acc_strerror(code):
            raise AssertionError(f"no message for {code}")
    if [lib.acc_motif_num_classes(k) for k in (3, 4, 5)] != [13, 199, 9364]:
        raise AssertionError("num_classes")
    c = Ctx(lib)
    for k in (3, 4, 5):
        ok(lib.acc_motif_prepare(c.h, k, None), f"prepare k {k}")
    if lib.acc_motif_prepare(c.h, 7, None) != acc.ACC_ERR_K:
        raise AssertionError("prepare k = 7 accepted")
    light, target = ctypes.c_int64(), ctypes.c_int64()
    ok(lib.acc_ctx_set_schedule(c.h, 777, 3333), "set_schedule")
    ok(lib.acc_ctx_get_schedule(c.h, ctypes.byref(light), ctypes.byref(target)), "get_schedule")
    if (light.value, target.value) != (777, 3333):
        raise AssertionError("schedule round trip")
    n, s, d = graphs(70, 1, 30)[0]
    rp, cl = csr(n, s, d)
    want = oracle.count(n, s, d, 4).tolist()
    ok(lib.acc_ctx_set_timing(c.h, 1), "set_timing")
    rc, st, got = c.count(rp, cl, n, 4)
    if rc or st or got.tolist() != want:
        raise AssertionError("count with schedule and timing")
    ms = np.zeros(4, np.float32)
    ok(lib.acc_motif_last_timing(c.h, P(ms)), "last_timing")
    if (ms < 0).any():
        raise AssertionError(f"negative stage times {ms}")
    st7 = c.stats()
    if st7[0] < 7 or st7[3] != len({(min(a, b), max(a, b)) for a, b in zip(s.tolist(), d.tolist())}):
        raise AssertionError(f"stats {st7}")
    ok(lib.acc_ctx_set_timing(c.h, 0), "set_timing off")
    ok(lib.acc_ctx_set_schedule(c.h, 0, 0), "schedule back to the default")
    for bad in (lambda: lib.acc_ctx_set_mode(c.h, 9), lambda: lib.acc_ctx_set_randomise_memory(c.h, -1),
                lambda: lib.acc_ctx_set_schedule(c.h, -5, 10)):
        if bad() != acc.ACC_ERR_ARG:
            raise AssertionError("a bad option was accepted")
    rc, st, got = c.count(rp, cl, n, 4)
    if rc or st or got.tolist() != want:
        raise AssertionError("count after the options")
    c.close()


def scenario_fuzz(lib, seed=2024, ops=60):
    """A seeded random sequence of calls on one context: counts (fresh and
    repeated on the same buffers, so launch graphs are captured, replayed and
    dropped), batches, randomisation, mode, schedule and launch-graph
    switches, over graphs of 0 to 40 vertices; every result against the
    oracle."""
    rng = np.random.default_rng(seed)
    c = Ctx(lib)
    held = None  # (n, s, d, rowptr, col) kept for repeats
    mode_names = (acc.ACC_MODE_COUNT, acc.ACC_MODE_ENUMERATE, acc.ACC_MODE_FORMULA)

    def draw(nmax):
        n = int(rng.integers(0, nmax + 1))
        if n == 0:
            return 0, np.zeros(0, np.int64), np.zeros(0, np.int64)
        s, d = random_digraph(rng, n, p=float(rng.uniform(0.0, 0.5)), recip=float(rng.random()))
        return n, np.asarray(s, np.int64), np.asarray(d, np.int64)

    for i in range(ops):
        op = rng.choice(["count", "repeat", "repeat", "batch", "randomise", "mode", "schedule", "graphs"])
        if op in ("count", "repeat"):
            if op == "count" or held is None:
                n, s, d = draw(40)
                held = (n, s, d, *csr(n, s, d))
            n, s, d, rp, cl = held
            k = int(rng.choice([3, 4] if n > 12 else [3, 4, 5]))
            rc, st, got = c.count(rp, cl, n, k)
            if rc or st or got.tolist() != oracle.count(n, s, d, k).tolist():
                raise AssertionError(f"op {i} {op}: n {n} k {k} rc {rc} status {st}")
        elif op == "batch":
            gs = [draw(16) for _ in range(int(rng.integers(1, 5)))]
            k = int(rng.choice([3, 4]))
            descs, keep = _descs(gs)
            out = np.full(len(gs) * NCLS[k], -1, np.int64)
            ok(lib.acc_motif_count_batch(c.h, descs, len(gs), k, None, P(out), None), f"op {i} batch")
            if out.reshape(len(gs), -1).tolist() != [oracle.count(n, s, d, k).tolist() for n, s, d in gs]:
                raise AssertionError(f"op {i} batch")
        elif op == "randomise":
            gs = [draw(20) for _ in range(int(rng.integers(1, 3)))]
            descs, arrays = _descs(gs)
            R, q = int(rng.integers(1, 3)), int(rng.integers(0, 3))
            mode = int(rng.integers(0, 2))
            seeds = rng.integers(0, 1 << 62, size=len(gs)).astype(np.uint64)
            M = sum(len(cl) for _, cl in arrays)
            out = np.full(max(1, R * M), -1, np.int32)
            accd = np.full(len(gs) * R, -1, np.int64)
            ok(lib.acc_swap_randomise(c.h, descs, len(gs), R, q, P(seeds), mode, None, P(out), P(accd), None),
               f"op {i} randomise")
            off = 0
            for g, ((n, _, _), (rp, cl)) in enumerate(zip(gs, arrays)):
                m = len(cl)
                for r in range(R):
                    want, wa = oracle.swap_randomise(n, rp, cl, q * m, int(seeds[g]) + r, mode)
                    if not np.array_equal(out[off + r * m: off + (r + 1) * m], want) or accd[g * R + r] != wa:
                        raise AssertionError(f"op {i} randomise graph {g} copy {r}")
                off += R * m
        elif op == "mode":
            ok(lib.acc_ctx_set_mode(c.h, int(rng.choice(mode_names))), f"op {i} mode")
        elif op == "schedule":
            light, target = (0, 0) if rng.random() < 0.3 else (int(rng.integers(1, 5000)), int(rng.integers(1, 5000)))
            ok(lib.acc_ctx_set_schedule(c.h, light, target), f"op {i} schedule")
        else:
            ok(lib.acc_ctx_set_launch_graphs(c.h, int(rng.integers(0, 2))), f"op {i} graphs")
    c.close()


def scenario_tables(lib):
    """The class table through the context (copy, classify, class codes) and
    the allocation-free build, against the oracle's table."""
    c = Ctx(lib)
    for k in (3, 4, 5):
        cls, codes = oracle.table(k)
        t = np.zeros(1 << (k * (k - 1)), np.int16)
        ok(lib.acc_motif_copy_table(c.h, k, P(t)), "copy_table")
        if not np.array_equal(t, np.asarray(cls, np.int16)):
            raise AssertionError(f"copy_table k {k}")
        for ci in (0, NCLS[k] // 2, NCLS[k] - 1):
            code = ctypes.c_uint32()
            ok(lib.acc_motif_class_code(c.h, k, ci, ctypes.byref(code)), "class_code")
            back = ctypes.c_int32()
            ok(lib.acc_motif_classify_code(c.h, k, code.value, ctypes.byref(back)), "classify_code")
            if code.value != codes[ci] or back.value != ci:
                raise AssertionError(f"class {ci} k {k}")
        st = np.zeros(1 << (k * (k - 1)), np.int16)
        sc = np.zeros(NCLS[k], np.uint32)
        ok(lib.acc_motif_build_table_static(k, None, P(st), P(sc)), "build_table_static")
        if not np.array_equal(st, t) or not np.array_equal(sc, np.asarray(codes, np.uint32)):
            raise AssertionError(f"static table k {k}")
    c.close()


def scenario_captured_pipeline(lib):
    """The significance step captured by the caller into one graph on its
    own stream (global capture mode: an allocation, a free, a synchronous
    copy or a wait inside would fail the capture) and replayed: R copies of
    each base graph randomised, the bases and copies counted as one
    prepared batch, Z-scores; every replay equals the oracle's copies,
    counts and Z-scores."""
    for f in (lib.emu_stream_create, lib.emu_capture_end):
        f.restype = ctypes.c_void_p
    lib.emu_capture_begin.argtypes = [ctypes.c_void_p]
    lib.emu_capture_end.argtypes = [ctypes.c_void_p]
    lib.emu_graph_replay.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    c = Ctx(lib)
    s = lib.emu_stream_create()
    k, R, q = 3, 3, 2
    bases = graphs(50, 3, 24)
    descs, arrays = _descs(bases)
    G = len(bases)
    seeds = np.array([100 + g for g in range(G)], np.uint64)
    M = sum(len(cl) for _, cl in arrays)
    out = np.zeros(R * M, np.int32)
    accepted = np.zeros(G * R, np.int64)
    status = np.zeros(1, np.int32)
    counts = np.zeros(G * (R + 1) * NCLS[k], np.int64)
    z = np.zeros(G * NCLS[k], np.float64)

    def randomise():
        ok(lib.acc_swap_randomise(c.h, descs, G, R, q, P(seeds), acc.ACC_RAND_SWAP, s, P(out), P(accepted),
                                  P(status)), "swap_randomise")

    # eager: randomise once, then lay out the batch (each base, then its copies)
    randomise()
    sync(lib)
    batch, off = [], 0
    for (n, _, _), (rp, cl) in zip(bases, arrays):
        m = len(cl)
        batch.append((rp, cl, n))
        batch.extend((rp, out[off + r * m: off + (r + 1) * m], n) for r in range(R))
        off += R * m
    bdesc = (acc.acc_graph_desc * len(batch))()
    for i, (rp, cl, n) in enumerate(batch):
        bdesc[i].rowptr, bdesc[i].col, bdesc[i].n, bdesc[i].m = rp.ctypes.data, cl.ctypes.data, n, len(cl)
    ok(lib.acc_motif_batch_prepare(c.h, bdesc, len(batch), k, s), "batch_prepare")

    def step():
        randomise()
        ok(lib.acc_motif_batch_run(c.h, s, P(counts), P(status)), "batch_run")
        ok(lib.acc_motif_zscores(P(counts), G, R + 1, k, s, P(z)), "zscores")

    step()  # eager once more, as a warm-up
    sync(lib)
    ok(lib.emu_capture_begin(s), "capture begin")
    step()
    ex = lib.emu_capture_end(s)
    if not ex:
        raise AssertionError("the step could not be captured")
    # expected values, from the oracle alone
    want_out, want_acc, want_counts = [], [], []
    for g, ((n, _, _), (rp, cl)) in enumerate(zip(bases, arrays)):
        m = len(cl)
        src = np.repeat(np.arange(n), np.diff(rp))
        want_counts.append(oracle.count(n, src, cl.astype(np.int64), k))
        for r in range(R):
            cp, a = oracle.swap_randomise(n, rp, cl, q * m, int(seeds[g]) + r, acc.ACC_RAND_SWAP)
            want_out.append(cp)
            want_acc.append(a)
            want_counts.append(oracle.count(n, src, cp.astype(np.int64), k))
    want_counts = np.array(want_counts)
    want_z = np.concatenate([oracle.zscores(want_counts[g * (R + 1)], want_counts[g * (R + 1) + 1:(g + 1) * (R + 1)])
                             for g in range(G)])
    for rep in range(2):
        out[:] = -1
        accepted[:] = -1
        counts[:] = -1
        z[:] = 0
        status[:] = -1
        ok(lib.emu_graph_replay(ex, s), "graph replay")
        sync(lib)
        if status[0] != 0:
            raise AssertionError(f"replay {rep}: status {status[0]}")
        if not np.array_equal(out, np.concatenate(want_out)) or accepted.tolist() != want_acc:
            raise AssertionError(f"replay {rep}: copies")
        if not np.array_equal(counts.reshape(len(batch), -1), want_counts):
            raise AssertionError(f"replay {rep}: counts")
        if not np.array_equal(z, want_z, equal_nan=True):
            raise AssertionError(f"replay {rep}: Z-scores")
    c.close()


def scenario_injected_failures(lib):
    """Failure detection without a device fault: the n-th allocation, kernel
    launch, copy or graph launch of a call fails.  The call returns
    ACC_ERR_NOMEM (allocation) or ACC_ERR_CUDA (the others), and the same
    context then counts correctly.  Counts are failed at every point they
    reach on a fresh context (tables and workspace made), on the call that
    captures the launch graph (third count of a context) and on one that
    replays it; a batch and the randomiser are failed at a spread of
    points."""
    lib.emu_inject.argtypes = [ctypes.c_int, ctypes.c_longlong]
    expect = {0: acc.ACC_ERR_NOMEM, 1: acc.ACC_ERR_CUDA, 2: acc.ACC_ERR_CUDA, 3: acc.ACC_ERR_CUDA}
    g = synth.chung_lu(40, 120, 2.1, 20, 20, 9)
    rp, cl = csr(g.n, g.src, g.dst)
    want = oracle.count(g.n, g.src, g.dst, 3).tolist()
    tripped = {}
    for before in (0, 2, 3):  # counts made before the failing one
        for kind in (0, 1, 2, 3):
            for n in range(1, 80):
                c = Ctx(lib)
                for _ in range(before):
                    c.count(rp, cl, g.n, 3)
                lib.emu_inject(kind, n)
                rc, st, got = c.count(rp, cl, g.n, 3)
                lib.emu_inject(kind, 0)
                if rc == 0:
                    if st != 0 or got.tolist() != want:
                        raise AssertionError(f"kind {kind} n {n}: wrong counts without an error")
                    c.close()
                    break  # the call makes fewer than n such calls
                if rc != expect[kind]:
                    raise AssertionError(f"after {before} kind {kind} n {n}: returned {rc}")
                tripped[(before, kind)] = n
                for _ in range(2):
                    rc, st, got = c.count(rp, cl, g.n, 3)
                    if rc or st or got.tolist() != want:
                        raise AssertionError(f"after {before} kind {kind} n {n}: not usable after the failure")
                c.close()
    # every kind fails a fresh count; launches fail the capturing count; the
    # graph launch fails the capturing and the replaying count
    for key in [(0, 0), (0, 1), (0, 2), (2, 1), (2, 3), (3, 3)]:
        if key not in tripped:
            raise AssertionError(f"no failure injected for {key}: {sorted(tripped)}")
    spread = (1, 2, 3, 5, 8, 13, 21, 34)
    gs = graphs(60, 3, 14)
    descs, arrays = _descs(gs)
    bwant = [oracle.count(n, s, d, 3).tolist() for n, s, d in gs]
    for kind in (0, 1, 2):
        for n in spread:
            c = Ctx(lib)
            out = np.zeros(len(gs) * 13, np.int64)
            lib.emu_inject(kind, n)
            rc = lib.acc_motif_count_batch(c.h, descs, len(gs), 3, None, P(out), None)
            lib.emu_inject(kind, 0)
            ok(lib.acc_motif_count_batch(c.h, descs, len(gs), 3, None, P(out), None), "batch after a failure")
            if out.reshape(len(gs), -1).tolist() != bwant:
                raise AssertionError(f"batch kind {kind} n {n}")
            c.close()
            if rc == 0:
                break
            if rc != expect[kind]:
                raise AssertionError(f"batch kind {kind} n {n}: returned {rc}")
    R, seeds = 2, np.array([3, 4, 5], np.uint64)
    rwant = np.concatenate([oracle.swap_randomise(n, rp_, cl_, 2 * len(cl_), int(seeds[g]) + r)[0]
                            for g, ((n, _, _), (rp_, cl_)) in enumerate(zip(gs, arrays)) for r in range(R)])
    M = len(rwant) // R
    for kind in (0, 1, 2):
        for n in spread:
            c = Ctx(lib)
            out = np.zeros(R * M, np.int32)
            accd = np.zeros(len(gs) * R, np.int64)
            lib.emu_inject(kind, n)
            rc = lib.acc_swap_randomise(c.h, descs, len(gs), R, 2, P(seeds), acc.ACC_RAND_SWAP, None, P(out),
                                        P(accd), None)
            lib.emu_inject(kind, 0)
            ok(lib.acc_swap_randomise(c.h, descs, len(gs), R, 2, P(seeds), acc.ACC_RAND_SWAP, None, P(out), P(accd),
                                      None), "randomise after a failure")
            if not np.array_equal(out, rwant):
                raise AssertionError(f"randomise kind {kind} n {n}")
            c.close()
            if rc == 0:
                break
            if rc != expect[kind]:
                raise AssertionError(f"randomise kind {kind} n {n}: returned {rc}")


if __name__ == "__main__":
    lib = acc.declare(ctypes.CDLL(sys.argv[1]))
    globals()["scenario_" + sys.argv[2]](lib)
    print("ok")
