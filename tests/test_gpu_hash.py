"""GPU parity of the count mode probing hashed adjacency tables instead of
the dense pair-state block, with the lists built from the dense block
(ACC_ADJ_HASH) or without it (ACC_ADJ_SPARSE): the same int64 counts as the
CPU oracle on random, power-law, hub and closed-form graphs, graph sets, the
full-size workloads (stored oracle counts), graphs above the automatic
choice's threshold and a million-vertex graph above the dense block's
limit."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays, gpu_count
from tests.graph_helpers import complete_bidirected, directed_path, out_star, random_digraph

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", params=["hash", "sparse"])
def counter(request):
    import torch  # noqa: F401
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    c = p.Counter(0)
    c.set_adjacency(p.ACC_ADJ_HASH if request.param == "hash" else p.ACC_ADJ_SPARSE)
    yield c
    c.close()


@pytest.mark.parametrize("k", [3, 4, 5])
def test_random_small_graphs(counter, k):
    rng = np.random.default_rng(3100 + k)
    for _ in range(30):
        n = int(rng.integers(1, {3: 40, 4: 26, 5: 16}[k]))
        s, d = random_digraph(rng, n, p=float(rng.random()), recip=float(rng.random()))
        assert gpu_count(counter, n, s, d, k).tolist() == oracle.count(n, s, d, k).tolist(), (k, n)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_power_law_and_hubs(counter, k):
    nmax = 3000 if k < 5 else 1200
    cases = [synth.chung_lu(nmax, 4 * nmax, 2.2, 150, 10, 3200 + k),
             synth.regulatory(nmax // 2, 3 * nmax // 2, nmax // 40, 2.0, 100, 3, 33)]
    for g in cases:
        assert gpu_count(counter, g.n, g.src, g.dst, k).tolist() == \
            oracle.count(g.n, g.src, g.dst, k, threads=oracle.max_threads()).tolist()
    L = {3: 3000, 4: 600, 5: 90}[k]
    n, s, d = L + 1, *out_star(L)
    assert gpu_count(counter, n, s, d, k).tolist() == oracle.count(n, s, d, k).tolist()
    n = {3: 40, 4: 24, 5: 14}[k]
    s, d = complete_bidirected(n)
    assert gpu_count(counter, n, s, d, k).tolist() == oracle.count(n, s, d, k).tolist()
    s, d = directed_path(700)
    assert gpu_count(counter, 700, s, d, k).tolist() == oracle.count(700, s, d, k).tolist()


def test_graph_sets(counter):
    import torch
    rng = np.random.default_rng(3300)
    graphs = []
    for i in range(10):
        n = int(rng.integers(0, 50))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 2, recip=float(rng.random()))
        graphs.append((n, s, d))
    g = synth.chung_lu(2000, 8000, 2.3, 120, 10, 3301)
    graphs.append((g.n, g.src, g.dst))
    dev = []
    for n, s, d in graphs:
        r, c = csr_arrays(n, s, d)
        dev.append((torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), n))
    for k in (3, 4, 5):
        counter.prepare_batch(dev, k)
        got = counter.run_batch().cpu().numpy()
        for i, (n, s, d) in enumerate(graphs):
            assert got[i].tolist() == oracle.count(n, s, d, k, threads=oracle.max_threads()).tolist(), (k, i)


@pytest.mark.parametrize("name,make,k", [("er_n1000_m5000_k3", synth.er_k3, 3),
                                         ("chung_lu_n20000_m100000_k4", synth.chung_lu_k4, 4),
                                         ("regulatory_n5000_m15000_k5", synth.regulatory_k5, 5)])
def test_full_size_workloads(counter, name, make, k):
    from tests.golden.golden_io import read_counts
    hdr, want = read_counts(os.path.join(GOLDEN, name + ".txt"))
    g = make()
    assert synth.graph_digest(g) in hdr["graph"]
    assert np.array_equal(gpu_count(counter, g.n, g.src, g.dst, k), want)


def test_automatic_choice_by_size():
    """By default a 50000-vertex graph is counted at k = 5 with hashed tables
    (one more kernel than the dense run) and at k = 4 with the dense block;
    the counts are the dense block's either way."""
    import paper_1203_3415_gb300 as p
    g = synth.chung_lu(50000, 100000, 2.2, 60, 10, 3400)
    auto, dense = p.Counter(0), p.Counter(0)
    dense.set_adjacency(p.ACC_ADJ_DENSE)
    for k, extra in ((5, 1), (4, 0)):
        a = gpu_count(auto, g.n, g.src, g.dst, k)
        na = auto.last_stats()["launches"]
        d = gpu_count(dense, g.n, g.src, g.dst, k)
        nd = dense.last_stats()["launches"]
        assert a.tolist() == d.tolist() and na == nd + extra, k
    auto.close()
    dense.close()


def test_hub_rows_above_the_warp_sort():
    """A hub with 5000 out-neighbours, repeated arcs and in-arcs: its raw row
    (both directions, repeats) takes the sparse build's block sort (k = 3:
    the build is the same for every k, and the oracle would visit the hub's
    2e10 four-vertex sets one by one)."""
    import paper_1203_3415_gb300 as p
    rng = np.random.default_rng(3500)
    n = 6000
    outs = rng.permutation(np.arange(1, n))[:5000]
    ins = rng.permutation(np.arange(1, n))[:800]
    s = np.concatenate([np.zeros(5000 + 700, np.int64), ins, rng.integers(1, n, 3000)])
    d = np.concatenate([outs, outs[:700], np.zeros(800, np.int64), rng.integers(1, n, 3000)])
    keep = s != d
    s, d = s[keep].astype(np.int32), d[keep].astype(np.int32)
    c = p.Counter(0)
    c.set_adjacency(p.ACC_ADJ_SPARSE)
    assert gpu_count(c, n, s, d, 3).tolist() == oracle.count(n, s, d, 3, threads=oracle.max_threads()).tolist()
    c.close()


def test_million_vertices_above_the_dense_limit():
    """A sparse directed Chung-Lu graph with 10^6 vertices (above ACC_MAX_N,
    whose dense block would take 250 GB) counts in the count mode, through
    the sparse build, with the oracle's counts for k = 3 and 4 (stored by
    tests/golden/make_golden.py --million); the other modes refuse it."""
    import hashlib
    import paper_1203_3415_gb300 as p
    from tests.golden.make_golden import million_vertex_graph
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "million_vertices.txt"))
            if ln.strip() and not ln.startswith("#")]
    g = million_vertex_graph()
    assert g.n > p.ACC_MAX_N
    c = p.Counter(0)
    for k, n, m, gsha, total, csha in rows:
        assert (g.n, g.m, synth.graph_digest(g)) == (int(n), int(m), gsha), "generator drifted from the stored graph"
        got = gpu_count(c, g.n, g.src, g.dst, int(k))
        assert int(got.sum()) == int(total), k
        assert hashlib.sha256(np.ascontiguousarray(got, dtype="<i8").tobytes()).hexdigest() == csha, k
    c.set_mode(p.ACC_MODE_ENUMERATE)
    with pytest.raises(p.MotifError) as e:
        gpu_count(c, g.n, g.src, g.dst, 3)
    assert e.value.code == p.ACC_ERR_TOO_LARGE
    c.close()
