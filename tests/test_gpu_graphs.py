"""GPU checks of the launch-graph replay of repeated counts
(acc_ctx_set_launch_graphs): a repeated count replays one captured CUDA graph
and must give exactly what launching the kernels one by one gives, also when
the buffers' contents change between repeats, when a repeat is malformed,
and when the mode or schedule changes."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays
from tests.graph_helpers import random_digraph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acc():
    import torch  # noqa: F401
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    return p


def dev_graph(n, s, d):
    import torch
    r, c = csr_arrays(n, s, d)
    return torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()


def test_repeats_equal_one_by_one(acc):
    import torch
    g = synth.chung_lu(3000, 12000, 2.2, 150, 10, 81)
    want = oracle.count(g.n, g.src, g.dst, 4, threads=oracle.max_threads())
    r, c = dev_graph(g.n, g.src, g.dst)
    cnt = acc.Counter(0)
    out = torch.zeros(199, dtype=torch.int64, device="cuda")
    for _ in range(5):
        out.zero_()
        cnt.count(r, c, g.n, 4, counts=out)
        assert out.cpu().numpy().tolist() == want.tolist()
        assert cnt.last_stats()["launches"] == 10
    cnt.set_launch_graphs(False)
    out.zero_()
    cnt.count(r, c, g.n, 4, counts=out)
    assert out.cpu().numpy().tolist() == want.tolist()
    cnt.close()


def test_contents_change_between_repeats(acc):
    import torch
    n, m = 1500, 6000
    cnt = acc.Counter(0)
    out = torch.zeros(199, dtype=torch.int64, device="cuda")
    g = synth.erdos_renyi(n, m, 10, 90)
    r, c = dev_graph(n, g.src, g.dst)
    for seed in (90, 91, 92, 93):
        g = synth.erdos_renyi(n, m, 10, seed)  # exactly m arcs: same buffers, new arcs
        rr, cc = csr_arrays(n, g.src, g.dst)
        r.copy_(torch.from_numpy(rr))
        c.copy_(torch.from_numpy(cc))
        cnt.count(r, c, n, 4, counts=out)
        assert out.cpu().numpy().tolist() == oracle.count(n, g.src, g.dst, 4).tolist(), seed
        # fewer than 8192 arcs: no reverse positions, so one launch fewer
        # than the 12000-arc graph of the test above
        assert cnt.last_stats()["launches"] == 9
    cnt.close()


def test_malformed_repeat_and_recovery(acc):
    import torch
    g = synth.chung_lu(2000, 8000, 2.2, 120, 10, 83)
    want = oracle.count(g.n, g.src, g.dst, 3)
    r, c = dev_graph(g.n, g.src, g.dst)
    cnt = acc.Counter(0)
    out = torch.zeros(13, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        cnt.count(r, c, g.n, 3, counts=out, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and out.cpu().numpy().tolist() == want.tolist()
    good = int(c[0].item())
    c[0] = 0  # row 0's first arc becomes a self-loop
    cnt.count(r, c, g.n, 3, counts=out, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == acc.ACC_ERR_INPUT
    c[0] = good
    for _ in range(2):
        cnt.count(r, c, g.n, 3, counts=out, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and out.cpu().numpy().tolist() == want.tolist()
    cnt.close()


def test_alternating_graphs_modes_and_schedules(acc):
    import torch
    rng = np.random.default_rng(84)
    graphs = []
    for n in (300, 1200, 2500):
        s, d = random_digraph(rng, n, p=6.0 / n, recip=0.2)
        graphs.append((n, s, d, *dev_graph(n, s, d)))
    want = {(i, k): oracle.count(n, s, d, k).tolist() for i, (n, s, d, _, _) in enumerate(graphs) for k in (3, 4)}
    cnt = acc.Counter(0)
    for rep in range(3):
        for mode in (acc.ACC_MODE_COUNT, acc.ACC_MODE_ENUMERATE, acc.ACC_MODE_FORMULA):
            cnt.set_mode(mode)
            for i, (n, s, d, r, c) in enumerate(graphs):
                for k in (3, 4):
                    got = cnt.count(r, c, n, k).cpu().numpy().tolist()
                    assert got == want[(i, k)], (rep, mode, i, k)
        cnt.set_schedule(512 * (rep + 1), 1024 * (rep + 1))
    cnt.close()


def test_host_entry_point_repeats(acc):
    g = synth.chung_lu(2500, 10000, 2.2, 120, 10, 85)
    rowptr, col = g.csr()
    want = oracle.count(g.n, g.src, g.dst, 4, threads=oracle.max_threads()).tolist()
    cnt = acc.Counter(0)
    for _ in range(4):
        assert cnt.count_host(rowptr, col, g.n, 4).tolist() == want
    cnt.close()
