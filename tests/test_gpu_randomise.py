"""GPU parity of the randomised copies (acc_swap_randomise): every copy equal,
element by element, to the oracle's copy for the same seed, in both modes,
and the whole significance step on the device (copies, batched count,
Z-scores) equal to the stored expectations of the batched workload."""
import hashlib
import os

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays
from tests.graph_helpers import complete_bidirected, random_digraph

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def counter():
    import torch  # noqa: F401
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    c = p.Counter(0)  # its first call is a randomisation (no count has sized its workspace)
    yield c
    c.close()


def to_device(graphs):
    import torch
    out = []
    for n, s, d in graphs:
        rowptr, col = csr_arrays(n, s, d)
        out.append((torch.from_numpy(rowptr).cuda(), torch.from_numpy(col).cuda(), n))
    return out


def check_against_oracle(graphs, dev, R, seeds, q, mode, out, acc):
    out = out.cpu().numpy()
    acc = acc.cpu().numpy()
    off = 0
    for g, ((n, s, d), (rowptr, col, _)) in enumerate(zip(graphs, dev)):
        rp, cl = rowptr.cpu().numpy(), col.cpu().numpy()
        m = len(cl)
        for r in range(R):
            want, want_acc = oracle.swap_randomise(n, rp, cl, q * m, seeds[g] + r, mode)
            got = out[off + r * m: off + (r + 1) * m]
            assert np.array_equal(got, want), (g, r)
            assert acc[g, r] == want_acc, (g, r)
        off += R * m


def mixed(seed):
    rng = np.random.default_rng(seed)
    graphs = []
    for _ in range(10):
        n = int(rng.integers(2, 80))
        s, d = random_digraph(rng, n, p=float(rng.uniform(0.01, 0.6)), recip=float(rng.random()))
        graphs.append((n, s, d))
    # hub rows longer than the entries a half-warp reads at once (64)
    g = synth.chung_lu(3000, 15000, 2.1, 400, 20, seed)
    graphs.append((g.n, g.src, g.dst))
    graphs.append((12, *complete_bidirected(12)))
    graphs.append((3, np.array([0], np.int32), np.array([1], np.int32)))  # one arc: nothing to swap
    graphs.append((4, np.zeros(0, np.int32), np.zeros(0, np.int32)))     # no arcs
    return graphs


@pytest.mark.parametrize("mode,bitmaps", [(0, True), (0, False), (1, True), (1, False)],
                         ids=["swap_speculative", "swap_row_scan", "mutual_speculative", "mutual_row_scan"])
def test_copies_equal_oracle(counter, mode, bitmaps):
    graphs = mixed(70 + mode + 2 * bitmaps)
    dev = to_device(graphs)
    R = 5
    seeds = [1_000 * (g + 1) + 17 for g in range(len(graphs))]
    counter.set_randomise_memory(16 << 30 if bitmaps else 0)
    try:
        out, acc = counter.randomise(dev, R, seeds, attempts_per_arc=3, mode=mode)
    finally:
        counter.set_randomise_memory(16 << 30)
    check_against_oracle(graphs, dev, R, seeds, 3, mode, out, acc)


def test_attempt_counts_and_seeds_near_wraparound(counter):
    graphs = mixed(91)[:4]
    dev = to_device(graphs)
    seeds = [2**64 - 2, 0, 2**63, 12345]
    for q in (0, 1, 7):
        out, acc = counter.randomise(dev, 3, seeds, attempts_per_arc=q)
        check_against_oracle(graphs, dev, 3, [x % 2**64 for x in seeds], q, 0, out, acc)
        if q == 0:
            assert int(acc.sum().item()) == 0


def test_large_graph_with_hubs(counter):
    g = synth.chung_lu_k4()  # n=20000, m=100000, rows up to 500 arcs
    graphs = [(g.n, g.src, g.dst)]
    dev = to_device(graphs)
    for mode, limit in ((0, 16 << 30), (0, 0), (1, 16 << 30), (1, 0)):
        counter.set_randomise_memory(limit)
        out, acc = counter.randomise(dev, 2, [42], attempts_per_arc=3, mode=mode)
        check_against_oracle(graphs, dev, 2, [42], 3, mode, out, acc)
    counter.set_randomise_memory(16 << 30)


def test_async_status_and_empty_calls(counter):
    import torch
    import paper_1203_3415_gb300 as p
    graphs = mixed(5)[:3]
    dev = to_device(graphs)
    st = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    out, acc = counter.randomise(dev, 2, [9, 8, 7], status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_against_oracle(graphs, dev, 2, [9, 8, 7], 3, 0, out, acc)
    # no graphs, no copies
    counter.randomise([], 4, [])
    o2, a2 = counter.randomise(dev, 0, [1, 2, 3])
    assert a2.numel() == 0
    with pytest.raises(p.MotifError):
        counter.randomise(dev, 1, [1, 2, 3], mode=2)
    with pytest.raises(p.MotifError):
        counter.randomise(dev, 1, [1, 2, 3], attempts_per_arc=-1)


@pytest.mark.parametrize("bad", ["self_loop", "target_range", "rowptr"])
def test_malformed_graph_is_an_input_error(counter, bad):
    import torch
    import paper_1203_3415_gb300 as p
    rowptr = np.array([0, 2, 3, 4], np.int64)
    col = np.array([1, 2, 2, 0], np.int32)
    if bad == "self_loop":
        col[2] = 1
    elif bad == "target_range":
        col[3] = 3
    else:
        rowptr[1] = 5
    good = to_device([(4, np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32))])
    t = (torch.from_numpy(rowptr).cuda(), torch.from_numpy(col).cuda(), 3)
    with pytest.raises(p.MotifError) as e:
        counter.randomise(good + [t], 2, [1, 2])
    assert e.value.code == p.ACC_ERR_INPUT
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    counter.randomise([t], 2, [1], status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == p.ACC_ERR_INPUT
    # the context stays usable
    out, acc = counter.randomise(good, 1, [3], attempts_per_arc=0)
    assert out[:3].cpu().tolist() == [1, 2, 3]
    out, acc = counter.randomise(good, 2, [3])
    check_against_oracle([(4, np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32))], good, 2, [3], 3, 0,
                         out, acc)


def test_significance_step_matches_stored_batch(counter):
    """8 Chung-Lu bases x 500 copies randomised on the device, counted as one
    batch of 4008 graphs and scored: equal to the oracle's stored counts and
    Z-scores for the batched workload."""
    import torch
    path = os.path.join(GOLDEN, "batch_k4.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    bases = [synth.batch_base(b) for b in range(synth.BATCH_BASES)]
    dev = [(torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), g.n) for g in bases for r, c in [g.csr()]]
    R = synth.BATCH_RANDOMISATIONS
    seeds = [1_000_000 * (b + 1) for b in range(len(bases))]
    counts, z, out = counter.significance(dev, 4, R, seeds, attempts_per_arc=3)
    host = counts.cpu().numpy()
    zh = z.cpu().numpy()
    for b, row in enumerate(rows):
        assert int(row[1]) == bases[b].n and int(row[2]) == bases[b].m
        digest = hashlib.sha256(np.ascontiguousarray(host[b], dtype="<i8").tobytes()).hexdigest()
        assert digest == row[4], b
        assert int(host[b].sum()) == int(row[5])
        want = np.array([float.fromhex(x) for x in row[6:]])
        same = (zh[b] == want) | (np.isnan(zh[b]) & np.isnan(want))
        assert same.all(), b
    # the copies themselves: the generator's graph digests
    cps = counter.copies(dev, R, out)
    for b in (1, 4):
        h = hashlib.sha256()
        for g in [bases[b]] + [synth.Graph(bases[b].n, np.repeat(np.arange(bases[b].n, dtype=np.int32),
                                                                  np.diff(bases[b].csr()[0])),
                                           c.cpu().numpy(), "") for _, c, _ in cps[b]]:
            h.update(synth.graph_digest(g).encode())
        assert h.hexdigest() == rows[b][3], b
