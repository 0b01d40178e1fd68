"""GPU parity of the k = 5 formula path (ACC_MODE_FORMULA: the paper's
per-triple formulas over the 63 neighbour sets of a connected 3-set with
linked-pair corrections and the final division by each pattern's
multiplicity, Lemma lema5d / Algorithm fived / Algorithm partfive): the 9364
class counts equal the oracle's, element by element."""
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
    rng = np.random.default_rng(5005)
    for trial in range(40):
        n = int(rng.integers(2, 40))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 2, recip=float(rng.random()))
        assert gpu_count(counter, n, s, d, 5).tolist() == oracle.count(n, s, d, 5).tolist(), (trial, n)


@pytest.mark.parametrize("n,m,seed", [(600, 2400, 31), (2000, 6000, 32)])
def test_power_law(counter, n, m, seed):
    g = synth.chung_lu(n, m, 2.2, 80, 10, seed)
    assert gpu_count(counter, g.n, g.src, g.dst, 5).tolist() == \
        oracle.count(g.n, g.src, g.dst, 5, threads=oracle.max_threads()).tolist()


def test_closed_forms_and_degenerate_graphs(counter):
    for n, (s, d) in [(8, complete_bidirected(8)), (30, directed_path(30)), (20, directed_cycle(20)),
                      (9, transitive_tournament(9))]:
        assert gpu_count(counter, n, s, d, 5).tolist() == oracle.count(n, s, d, 5).tolist()
    # out-star with 12 leaves: C(12, 4) out-stars
    s = np.zeros(12, np.int32)
    d = np.arange(1, 13, dtype=np.int32)
    got = gpu_count(counter, 13, s, d, 5)
    assert got.sum() == 495 and got.tolist() == oracle.count(13, s, d, 5).tolist()
    z = np.zeros(0, dtype=np.int32)
    assert gpu_count(counter, 0, z, z, 5).sum() == 0
    assert gpu_count(counter, 50, z, z, 5).sum() == 0


def test_full_size_k5_workload(counter):
    from tests.golden.golden_io import read_counts
    hdr, expect = read_counts(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                           "regulatory_n5000_m15000_k5.txt"))
    g = synth.regulatory_k5()
    assert f"sha256={synth.graph_digest(g)}" in hdr["graph"]
    assert gpu_count(counter, g.n, g.src, g.dst, 5).tolist() == expect.tolist()


def test_batch(counter):
    import torch
    rng = np.random.default_rng(79)
    graphs = []
    for _ in range(8):
        n = int(rng.integers(0, 60))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 3, recip=float(rng.random()))
        graphs.append((n, s, d))
    g = synth.chung_lu(500, 2000, 2.2, 60, 10, 33)
    graphs.append((g.n, g.src, g.dst))
    dev = []
    for n, s, d in graphs:
        r, c = csr_arrays(n, s, d)
        dev.append((torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), n))
    counter.prepare_batch(dev, 5)
    got = counter.run_batch().cpu().numpy()
    for i, (n, s, d) in enumerate(graphs):
        assert got[i].tolist() == oracle.count(n, s, d, 5).tolist(), i
