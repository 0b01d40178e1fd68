"""GPU parity of the k = 3 formula path (ACC_MODE_FORMULA: the paper's
per-vertex set-size formulas with triangle corrections, Thm teo3 / Algorithm
s3 / Table starb): the 13 class counts equal the oracle's, element by
element, on the same seeded inputs as the enumeration's tests."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays, gpu_count
from tests.graph_helpers import complete_bidirected, directed_cycle, directed_path, random_digraph, \
    transitive_tournament

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def counter():
    import torch  # noqa: F401
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    c = p.Counter(0)
    c.set_mode(p.ACC_MODE_FORMULA)
    yield c
    c.close()


def test_random_graphs(counter):
    rng = np.random.default_rng(3003)
    for trial in range(60):
        n = int(rng.integers(3, 64))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 2, recip=float(rng.random()))
        assert gpu_count(counter, n, s, d, 3).tolist() == oracle.count(n, s, d, 3).tolist(), (trial, n)


@pytest.mark.parametrize("n,m,seed", [(4000, 24000, 11), (1500, 12000, 12), (30000, 90000, 13)])
def test_power_law(counter, n, m, seed):
    g = synth.chung_lu(n, m, 2.2, 200, 10, seed)
    assert gpu_count(counter, g.n, g.src, g.dst, 3).tolist() == \
        oracle.count(g.n, g.src, g.dst, 3, threads=oracle.max_threads()).tolist()


def test_star_example_and_closed_forms(counter):
    from tests.test_oracle_pins import star_graph
    n, s, d = star_graph()
    got = gpu_count(counter, n, s, d, 3)
    assert sorted(got[got > 0].tolist()) == [6, 6, 10, 16, 20, 20]  # Fig. star
    for n, (s, d) in [(9, complete_bidirected(9)), (40, directed_path(40)), (30, directed_cycle(30)),
                      (12, transitive_tournament(12))]:
        assert gpu_count(counter, n, s, d, 3).tolist() == oracle.count(n, s, d, 3).tolist()
    z = np.zeros(0, dtype=np.int32)
    assert gpu_count(counter, 0, z, z, 3).sum() == 0
    assert gpu_count(counter, 50, z, z, 3).sum() == 0


def test_full_size_k3_workload(counter):
    from tests.golden.golden_io import read_counts
    import os
    hdr, expect = read_counts(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                           "er_n1000_m5000_k3.txt"))
    g = synth.er_k3()
    assert f"sha256={synth.graph_digest(g)}" in hdr["graph"]
    assert gpu_count(counter, g.n, g.src, g.dst, 3).tolist() == expect.tolist()


def test_batch_and_mode_agreement(counter):
    import torch
    import paper_1203_3415_gb300 as p
    rng = np.random.default_rng(77)
    graphs = []
    for _ in range(10):
        n = int(rng.integers(0, 300))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 3, recip=float(rng.random()))
        graphs.append((n, s, d))
    g = synth.chung_lu(2500, 10000, 2.2, 120, 10, 14)
    graphs.append((g.n, g.src, g.dst))
    dev = []
    for n, s, d in graphs:
        r, c = csr_arrays(n, s, d)
        dev.append((torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), n))
    counter.prepare_batch(dev, 3)
    got = counter.run_batch().cpu().numpy()
    for i, (n, s, d) in enumerate(graphs):
        assert got[i].tolist() == oracle.count(n, s, d, 3).tolist(), i
    # k = 5 in this mode runs the per-triple formulas
    h = synth.chung_lu(600, 2400, 2.2, 60, 10, 15)
    assert gpu_count(counter, h.n, h.src, h.dst, 5).tolist() == \
        oracle.count(h.n, h.src, h.dst, 5, threads=oracle.max_threads()).tolist()
    with pytest.raises(p.MotifError):
        counter.set_mode(4)  # no such mode (3 is the automatic one)


def test_automatic_mode_takes_both_paths():
    """ACC_MODE_AUTO: k = 3 on graphs of at most 16384 vertices runs the
    formula path (no neighbour entries scanned), larger k = 3 graphs and
    every k = 4 count run the count mode (entries scanned); the counts equal
    the oracle's in both branches."""
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    c = p.Counter(0)
    c.set_mode(p.ACC_MODE_AUTO)
    try:
        small = synth.chung_lu(4000, 24000, 2.2, 200, 10, 21)
        assert gpu_count(c, small.n, small.src, small.dst, 3).tolist() == \
            oracle.count(small.n, small.src, small.dst, 3).tolist()
        assert c.last_stats()["scanned_entries"] == 0
        big = synth.chung_lu(20000, 80000, 2.2, 300, 10, 22)
        assert gpu_count(c, big.n, big.src, big.dst, 3).tolist() == \
            oracle.count(big.n, big.src, big.dst, 3, threads=oracle.max_threads()).tolist()
        assert c.last_stats()["scanned_entries"] > 0
        h = synth.chung_lu(1500, 6000, 2.2, 100, 10, 23)
        assert gpu_count(c, h.n, h.src, h.dst, 4).tolist() == \
            oracle.count(h.n, h.src, h.dst, 4, threads=oracle.max_threads()).tolist()
        assert c.last_stats()["scanned_entries"] > 0
    finally:
        c.close()
