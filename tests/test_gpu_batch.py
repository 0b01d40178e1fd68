"""GPU parity of the batched form: many graphs per launch sequence, per-graph
int64 histograms equal to the oracle's, Z-scores equal bit for bit to the
oracle's formula, and CUDA-graph replay of a prepared batch."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays
from tests.graph_helpers import complete_bidirected, directed_path, random_digraph

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", params=[0, 1], ids=["count_mode", "enumerate_mode"])
def counter(request):
    import torch  # noqa: F401
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    c = p.Counter(0)
    c.set_mode(request.param)
    yield c
    c.close()


def to_device(graphs):
    import torch
    out = []
    for n, s, d in graphs:
        rowptr, col = csr_arrays(n, s, d)
        out.append((torch.from_numpy(rowptr).cuda(), torch.from_numpy(col).cuda(), n))
    return out


def mixed_graphs(seed):
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(14):
        n = int(rng.integers(0, 60))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 2, recip=float(rng.random()))
        graphs.append((n, s, d))
    graphs.append((12, *complete_bidirected(12)))
    graphs.append((500, *directed_path(500)))
    g = synth.chung_lu(1500, 6000, 2.2, 120, 10, seed)
    graphs.append((g.n, g.src, g.dst))
    graphs.append((0, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    return graphs


@pytest.mark.parametrize("k", [3, 4, 5])
def test_batch_equals_oracle(counter, k):
    graphs = mixed_graphs(50 + k)
    dev = to_device(graphs)
    counter.prepare_batch(dev, k)
    got = counter.run_batch().cpu().numpy()
    for i, (n, s, d) in enumerate(graphs):
        assert got[i].tolist() == oracle.count(n, s, d, k, threads=oracle.max_threads()).tolist(), i
    # a second run of the same prepared batch gives the same counts
    again = counter.run_batch().cpu().numpy()
    assert np.array_equal(got, again)


def test_batch_single_graph_and_singles_agree(counter):
    import torch
    g = synth.chung_lu(3000, 12000, 2.2, 150, 10, 61)
    dev = to_device([(g.n, g.src, g.dst)])
    counter.prepare_batch(dev, 4)
    got = counter.run_batch().cpu().numpy()[0]
    single = counter.count(dev[0][0], dev[0][1], g.n, 4).cpu().numpy()
    assert got.tolist() == single.tolist()
    # a malformed member (self-loop) sets the batch status
    good = (5, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    bad = (5, np.array([0, 1], np.int32), np.array([1, 1], np.int32))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gb = to_device([good, bad])  # alive until the run is done
    counter.prepare_batch(gb, 3)
    counter.run_batch(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == -2


def test_batch_autotune_keeps_counts(counter):
    graphs = mixed_graphs(70)
    dev = to_device(graphs)
    counter.prepare_batch(dev, 4)
    try:
        light, target, ms = counter.autotune_batch()
        assert (light, target) == counter.schedule() and ms > 0.0
        got = counter.run_batch().cpu().numpy()
        for i, (n, s, d) in enumerate(graphs):
            assert got[i].tolist() == oracle.count(n, s, d, 4).tolist(), i
    finally:
        counter.set_schedule(0, 0)


def small_ensemble(b, n_rand):
    base = synth.batch_base(b)
    return [base] + [synth.batch_randomisation(base, b, i) for i in range(n_rand)]


def test_zscores_match_oracle_bitwise(counter):
    import torch
    R = 12
    groups = [small_ensemble(1, R), small_ensemble(3, R)]
    flat = [g for grp in groups for g in grp]
    dev = to_device([(g.n, g.src, g.dst) for g in flat])
    counter.prepare_batch(dev, 4)
    counts = counter.run_batch()
    z = counter.zscores(counts, len(groups), R + 1, 4).cpu().numpy()
    host = counts.cpu().numpy()
    for gi, grp in enumerate(groups):
        block = host[gi * (R + 1):(gi + 1) * (R + 1)]
        for j, g in enumerate(grp):
            assert block[j].tolist() == oracle.count(g.n, g.src, g.dst, 4, threads=oracle.max_threads()).tolist()
        want = oracle.zscores(block[0], block[1:])
        assert np.array_equal(np.isnan(want), np.isnan(z[gi]))
        ok = ~np.isnan(want)
        assert np.array_equal(want[ok].view(np.int64), z[gi][ok].view(np.int64))
    torch.cuda.synchronize()


def test_batch_replays_in_cuda_graph(counter):
    import torch
    graphs = [small_ensemble(1, 6)[i] for i in range(7)]
    dev = to_device([(g.n, g.src, g.dst) for g in graphs])
    s = torch.cuda.Stream()
    counts = torch.zeros((len(graphs), 199), dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(s):
        counter.prepare_batch(dev, 4, stream=s)
        counter.run_batch(counts=counts, status=status, stream=s)  # warm-up, sizes the workspace
    torch.cuda.synchronize()
    eager = counts.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        counter.run_batch(counts=counts, status=status, stream=s)
    for _ in range(2):
        counts.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(counts, eager)
        assert int(status.item()) == 0


def test_full_batch_against_stored_oracle_counts(counter):
    """The batched k=4 workload: 8 bases x 501 graphs in one prepared batch."""
    import hashlib
    import torch
    path = os.path.join(GOLDEN, "batch_k4.txt")
    if not os.path.exists(path):
        pytest.skip("stored batch expectations not written")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    all_graphs, per_base = [], []
    for b in range(synth.BATCH_BASES):
        grp = small_ensemble(b, synth.BATCH_RANDOMISATIONS)
        per_base.append(len(grp))
        all_graphs.extend(grp)
    dev = to_device([(g.n, g.src, g.dst) for g in all_graphs])
    counter.prepare_batch(dev, 4)
    counts = counter.run_batch()
    z = counter.zscores(counts, synth.BATCH_BASES, synth.BATCH_RANDOMISATIONS + 1, 4).cpu().numpy()
    host = counts.cpu().numpy()
    off = 0
    for b, row in enumerate(rows):
        block = host[off:off + per_base[b]]
        off += per_base[b]
        h = hashlib.sha256()
        for g in all_graphs[b * per_base[b]:(b + 1) * per_base[b]]:
            h.update(synth.graph_digest(g).encode())
        assert h.hexdigest() == row[3], "generator drifted from the stored graphs"
        assert hashlib.sha256(np.ascontiguousarray(block, dtype="<i8").tobytes()).hexdigest() == row[4], b
        assert int(block.sum()) == int(row[5])
        want = np.array([float.fromhex(x) for x in row[6:]])
        assert np.array_equal(np.isnan(want), np.isnan(z[b]))
        ok = ~np.isnan(want)
        assert np.array_equal(want[ok].view(np.int64), z[b][ok].view(np.int64))
    del dev
    torch.cuda.synchronize()


def test_prepare_waits_for_an_enqueued_run(counter):
    """prepare(A), an asynchronous run of A on a non-blocking stream, then
    prepare(B) on the same stream: the run of A still reads A's descriptors,
    so the second prepare must not overwrite them under it."""
    import torch
    ga = [synth.chung_lu(n, 4 * n, 2.2, 150, 10, 900 + n) for n in (4000, 2500, 3000)]
    gb = [synth.chung_lu(n, 5 * n, 2.2, 100, 10, 950 + n) for n in (300, 200, 600, 100)]
    da = to_device([(g.n, g.src, g.dst) for g in ga])
    db = to_device([(g.n, g.src, g.dst) for g in gb])
    s = torch.cuda.Stream()  # non-blocking with respect to the legacy stream
    ca = torch.zeros((len(ga), 199), dtype=torch.int64, device="cuda")
    cb = torch.zeros((len(gb), 199), dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(s):
        counter.prepare_batch(da, 4, stream=s)
        counter.run_batch(counts=ca, status=st, stream=s)  # enqueued only
        counter.prepare_batch(db, 4, stream=s)
        counter.run_batch(counts=cb, status=st, stream=s)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    for i, g in enumerate(ga):
        assert ca[i].cpu().numpy().tolist() == oracle.count(g.n, g.src, g.dst, 4, threads=oracle.max_threads()).tolist(), i
    for i, g in enumerate(gb):
        assert cb[i].cpu().numpy().tolist() == oracle.count(g.n, g.src, g.dst, 4).tolist(), i


def test_mode_changed_between_prepare_and_run():
    """A batch prepared in the enumerate mode and run in the count mode (and
    back): the run first grows the workspace the count mode needs (its
    reverse positions, for a set of at least 8192 arcs), and every mode gives
    the oracle's counts."""
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    graphs = []
    for seed in (91, 92, 93):
        g = synth.chung_lu(2000, 8000, 2.2, 120, 10, seed)
        graphs.append((g.n, g.src, g.dst))
    want = [oracle.count(n, s, d, 4, threads=oracle.max_threads()).tolist() for n, s, d in graphs]
    c = p.Counter(0)
    try:
        c.set_mode(p.ACC_MODE_ENUMERATE)
        dev = to_device(graphs)
        c.prepare_batch(dev, 4)
        for mode in (p.ACC_MODE_COUNT, p.ACC_MODE_ENUMERATE, p.ACC_MODE_FORMULA, p.ACC_MODE_AUTO):
            c.set_mode(mode)
            got = c.run_batch().cpu().numpy()
            assert got.tolist() == want, mode
    finally:
        c.close()
