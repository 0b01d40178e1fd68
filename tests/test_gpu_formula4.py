"""GPU parity of the k = 4 formula path (ACC_MODE_FORMULA: the paper's
per-edge formulas over the 15 neighbour sets of an edge with linked-pair
corrections and the final division by each pattern's multiplicity, Thm
lema4d / Cor coro:a / Algorithm mine / Fact correction): the 199 class counts
equal the oracle's, element by element."""
import os

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
    rng = np.random.default_rng(4004)
    for trial in range(60):
        n = int(rng.integers(2, 64))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 2, recip=float(rng.random()))
        assert gpu_count(counter, n, s, d, 4).tolist() == oracle.count(n, s, d, 4).tolist(), (trial, n)


@pytest.mark.parametrize("n,m,seed", [(3000, 15000, 21), (1200, 9000, 22), (20000, 60000, 23)])
def test_power_law(counter, n, m, seed):
    g = synth.chung_lu(n, m, 2.2, 300, 10, seed)
    assert gpu_count(counter, g.n, g.src, g.dst, 4).tolist() == \
        oracle.count(g.n, g.src, g.dst, 4, threads=oracle.max_threads()).tolist()


def test_closed_forms_and_degenerate_graphs(counter):
    for n, (s, d) in [(9, complete_bidirected(9)), (40, directed_path(40)), (30, directed_cycle(30)),
                      (12, transitive_tournament(12))]:
        assert gpu_count(counter, n, s, d, 4).tolist() == oracle.count(n, s, d, 4).tolist()
    # out-star with 40 leaves: C(40, 3) out-stars, one hub edge per 4-set
    s = np.zeros(40, np.int32)
    d = np.arange(1, 41, dtype=np.int32)
    got = gpu_count(counter, 41, s, d, 4)
    assert got.sum() == 9880 and got.tolist() == oracle.count(41, s, d, 4).tolist()
    z = np.zeros(0, dtype=np.int32)
    assert gpu_count(counter, 0, z, z, 4).sum() == 0
    assert gpu_count(counter, 50, z, z, 4).sum() == 0
    assert gpu_count(counter, 2, np.array([0], np.int32), np.array([1], np.int32), 4).sum() == 0


def test_full_size_k4_workload(counter):
    from tests.golden.golden_io import read_counts
    hdr, expect = read_counts(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                           "chung_lu_n20000_m100000_k4.txt"))
    g = synth.chung_lu_k4()
    assert f"sha256={synth.graph_digest(g)}" in hdr["graph"]
    assert gpu_count(counter, g.n, g.src, g.dst, 4).tolist() == expect.tolist()


def test_batch(counter):
    import torch
    rng = np.random.default_rng(78)
    graphs = []
    for _ in range(10):
        n = int(rng.integers(0, 200))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 3, recip=float(rng.random()))
        graphs.append((n, s, d))
    g = synth.chung_lu(2500, 10000, 2.2, 120, 10, 24)
    graphs.append((g.n, g.src, g.dst))
    dev = []
    for n, s, d in graphs:
        r, c = csr_arrays(n, s, d)
        dev.append((torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), n))
    counter.prepare_batch(dev, 4)
    got = counter.run_batch().cpu().numpy()
    for i, (n, s, d) in enumerate(graphs):
        assert got[i].tolist() == oracle.count(n, s, d, 4).tolist(), i
