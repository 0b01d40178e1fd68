"""Serving form: requests admitted by free slots and device memory, running
concurrently on the GPU, give exactly the counts they give alone (tolerance
0: int64 histograms), and every served result equals the CPU oracle's counts
(stored by tests/golden/make_golden.py --serving for the test pool, or
computed here)."""
import hashlib
import os

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays
from tests.graph_helpers import serving_test_pool

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "serving_pool.txt")


@pytest.fixture(scope="module")
def acc():
    import torch  # noqa: F401
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    return p


def pool():
    return serving_test_pool()


def stored_pool_counts(graphs):
    """{(graph index, k): (N_k, counts sha256)} of the oracle's counts of the
    test pool, after checking that the generator still makes the same graphs."""
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    want = {}
    for gi, k, n, m, gsha, total, csha in rows:
        g = graphs[int(gi)]
        assert (g.n, g.m, synth.graph_digest(g)) == (int(n), int(m), gsha), "generator drifted from the stored graphs"
        want[(int(gi), int(k))] = (int(total), csha)
    return want


def digest(counts):
    return hashlib.sha256(np.ascontiguousarray(counts, dtype="<i8").tobytes()).hexdigest()


def to_dev(g):
    import torch
    r, c = g.csr()
    return torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()


def requests(n_graphs, count, seed):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, n_graphs)), int(rng.choice([3, 3, 4, 4, 5]))) for _ in range(count)]


def test_mix_equals_alone(acc):
    graphs = pool()
    stored = stored_pool_counts(graphs)
    dev = [to_dev(g) for g in graphs]
    reqs = requests(len(graphs), 48, 11)
    counter = acc.Counter(0)
    alone = {}
    for gi, k in set(reqs):
        alone[(gi, k)] = counter.count(dev[gi][0], dev[gi][1], graphs[gi].n, k).cpu().numpy()
    counter.close()
    # every request's count alone equals the oracle's (stored), k = 5 and the
    # largest graphs included
    for key, counts in alone.items():
        assert (int(counts.sum()), digest(counts)) == stored[key], key
    srv = acc.Server(0, slots=4, mem_budget_bytes=48 << 30)
    ids = [srv.add_graph(r, c, g.n) for (r, c), g in zip(dev, graphs)]
    srv.reserve()
    rids = [srv.submit(ids[gi], k) for gi, k in reqs]  # all at once: they queue and overlap
    most = 0
    while True:
        running, queued = srv.progress()
        most = max(most, running)
        if running == 0 and queued == 0:
            break
    assert most >= 2  # several requests were on the device together
    srv.drain()
    for rid, (gi, k) in zip(rids, reqs):
        st, counts, lat = srv.poll(rid)
        assert st == acc.ACC_REQ_DONE and lat >= 0.0
        assert counts.tolist() == alone[(gi, k)].tolist(), (gi, k)
        assert (int(counts.sum()), digest(counts)) == stored[(gi, k)], (gi, k)
    srv.close()


def test_memory_admission_serialises(acc):
    graphs = [synth.chung_lu(n, 4 * n, 2.2, 120, 10, 7100 + n) for n in (6000, 5600, 5800, 6000)]
    dev = [to_dev(g) for g in graphs]
    want = [oracle.count(g.n, g.src, g.dst, 4, threads=oracle.max_threads()) for g in graphs]
    # a budget that holds one such workspace (~0.4 GB) but not two
    srv = acc.Server(0, slots=4, mem_budget_bytes=int(0.6e9))
    ids = [srv.add_graph(r, c, g.n) for (r, c), g in zip(dev, graphs)]
    rids = [srv.submit(i, 4) for i in ids]
    while True:
        running, queued = srv.progress()
        assert running <= 1
        if running == 0 and queued == 0:
            break
    for rid, w in zip(rids, want):
        st, counts, _ = srv.poll(rid)
        assert st == acc.ACC_REQ_DONE and counts.tolist() == w.tolist()
    srv.close()


def test_request_errors(acc):
    import torch
    srv = acc.Server(0, slots=2, mem_budget_bytes=8 << 30)
    r, c = csr_arrays(4, [0, 1], [1, 1])  # self-loop 1 -> 1
    bad = srv.add_graph(torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), 4)
    rid = srv.submit(bad, 3)
    srv.drain()
    assert srv.poll(rid)[0] == acc.ACC_ERR_INPUT
    srv.close()
    # a graph whose workspace can never fit the budget
    g = synth.chung_lu(20000, 80000, 2.2, 200, 10, 3)
    rr, cc = to_dev(g)
    srv = acc.Server(0, slots=1, mem_budget_bytes=1 << 20)
    gid = srv.add_graph(rr, cc, g.n)
    rid = srv.submit(gid, 4)
    srv.drain()
    assert srv.poll(rid)[0] == acc.ACC_ERR_NOMEM
    srv.close()


@pytest.mark.parametrize("policy", ["shortest", "fifo"])
def test_admission_policy_order(acc, policy):
    """One slot, three large requests then a small one: shortest-first runs
    the small one as soon as the slot frees, FIFO runs it last; the counts
    are the same either way."""
    graphs = pool()
    big, small = graphs[7], graphs[4]
    (rb, cb), (rs, cs) = to_dev(big), to_dev(small)
    srv = acc.Server(0, slots=1, mem_budget_bytes=16 << 30)
    if policy == "fifo":
        srv.set_policy(acc.ACC_SERVE_FIFO)
    gb, gs = srv.add_graph(rb, cb, big.n), srv.add_graph(rs, cs, small.n)
    srv.reserve()
    bigs = [srv.submit(gb, 5) for _ in range(3)]
    s = srv.submit(gs, 3)
    while srv.poll(s)[0] != acc.ACC_REQ_DONE:
        pass
    last_big_state = srv.poll(bigs[2])[0]
    if policy == "fifo":
        assert last_big_state == acc.ACC_REQ_DONE
    else:
        assert last_big_state == acc.ACC_REQ_QUEUED
    srv.drain()
    stored = stored_pool_counts(graphs)
    for rid in bigs:
        st, counts, _ = srv.poll(rid)
        assert st == acc.ACC_REQ_DONE
        assert (int(counts.sum()), digest(counts)) == stored[(7, 5)]
    assert srv.poll(s)[1].tolist() == oracle.count(small.n, small.src, small.dst, 3).tolist()
    with pytest.raises(acc.MotifError):
        srv.set_policy(7)
    srv.close()
