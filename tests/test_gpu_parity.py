"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Integer histograms, so the bar is bit-exact int64 equality everywhere.  Cases:
the code -> class table byte for byte; seeded random digraphs of all densities
and reciprocities; medium power-law graphs spanning many work units and chunk
splits; hub-heavy closed forms that force the global overflow lists and the
heavy-unit queue; edge cases (empty, tiny, repeated arcs, unsorted rows,
isolated vertices); malformed input; the host-buffer entry point; and the
full-size workloads against stored oracle counts.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import csr_arrays, gpu_count
from tests.graph_helpers import (complete_bidirected, directed_cycle, directed_path, esu_scanned_entries, in_star,
                                 out_star, random_digraph, transitive_tournament)

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


def threads():
    return max(1, oracle.max_threads())


@pytest.mark.parametrize("k", [3, 4, 5])
def test_table_matches_oracle(counter, k):
    cls, ccode = oracle.table(k)
    gpu = counter.table(k)
    assert gpu.dtype == np.int16 and gpu.shape == cls.shape
    assert (gpu.astype(np.int32) == cls).all()
    for c in range(0, len(ccode), max(1, len(ccode) // 97)):
        assert counter.class_code(k, c) == int(ccode[c])
        assert counter.classify_code(k, int(ccode[c])) == c


@pytest.mark.parametrize("k", [3, 4, 5])
def test_random_small_graphs(counter, k):
    rng = np.random.default_rng(1000 + k)
    for trial in range(40):
        n = int(rng.integers(k, 48))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 2, recip=float(rng.random()))
        assert gpu_count(counter, n, s, d, k).tolist() == oracle.count(n, s, d, k).tolist(), (trial, n)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_scanned_entries_stat(counter, k):
    """The count mode's work figure (neighbour entries scanned by the last two
    levels) equals the same sum taken over a plain ESU walk."""
    if counter.mode != 0:
        pytest.skip("count mode only")
    rng = np.random.default_rng(2000 + k)
    for trial in range(6):
        n = int(rng.integers(k, 160 if k < 5 else 70))
        s, d = random_digraph(rng, n, p=float(rng.random()) ** 2 * 0.5, recip=float(rng.random()))
        gpu_count(counter, n, s, d, k)
        assert counter.last_stats()["scanned_entries"] == esu_scanned_entries(n, s, d, k), (trial, n)


@pytest.mark.parametrize("k,n,m,seed", [(3, 4000, 24000, 11), (4, 3000, 12000, 12), (5, 1200, 3000, 13)])
def test_medium_power_law(counter, k, n, m, seed):
    g = synth.chung_lu(n, m, 2.2, 150, 10, seed)
    expect = oracle.count(g.n, g.src, g.dst, k, threads=threads())
    got = gpu_count(counter, g.n, g.src, g.dst, k)
    assert got.tolist() == expect.tolist()
    assert expect.sum() > 10 ** 5  # spans many work units


@pytest.mark.parametrize("k", [3, 4, 5])
def test_regulatory_small(counter, k):
    g = synth.regulatory(1500, 3000, 60, 2.0, 80, 3, 77)
    expect = oracle.count(g.n, g.src, g.dst, k, threads=threads())
    assert gpu_count(counter, g.n, g.src, g.dst, k).tolist() == expect.tolist()


@pytest.mark.parametrize("k,leaves", [(3, 3000), (4, 1500), (5, 260)])
def test_hub_stars_closed_form(counter, k, leaves):
    # one hub, id 0, so every k-set is rooted at it: extension lists far above
    # the shared-memory capacity and heavy units split across the queue
    for make, arcs in [(out_star, [(0, i) for i in range(1, k)]), (in_star, [(i, 0) for i in range(1, k)])]:
        s, d = make(leaves)
        got = gpu_count(counter, leaves + 1, s, d, k)
        c = oracle.classify(k, oracle.code_of_arcs(k, arcs))
        assert got[c] == math.comb(leaves, k - 1) and got.sum() == got[c]
    # the same star with the hub as the largest id
    s, d = out_star(leaves)
    perm = np.roll(np.arange(leaves + 1), -1)
    got = gpu_count(counter, leaves + 1, perm[s], perm[d], k)
    assert got.sum() == math.comb(leaves, k - 1)


@pytest.mark.parametrize("k,n", [(3, 400), (4, 200), (5, 70)])
def test_dense_closed_forms(counter, k, n):
    s, d = complete_bidirected(n)
    got = gpu_count(counter, n, s, d, k)
    full = oracle.classify(k, (1 << (k * (k - 1))) - 1)
    assert got[full] == math.comb(n, k) and got.sum() == got[full]
    s, d = transitive_tournament(n)
    got = gpu_count(counter, n, s, d, k)
    tt = oracle.classify(k, oracle.code_of_arcs(k, [(i, j) for i in range(k) for j in range(i + 1, k)]))
    assert got[tt] == math.comb(n, k) and got.sum() == got[tt]


@pytest.mark.parametrize("k", [3, 4, 5])
def test_paths_and_cycles(counter, k):
    path_cls = oracle.classify(k, oracle.code_of_arcs(k, [(i, i + 1) for i in range(k - 1)]))
    for n in (k, k + 1, 1000, 10007):
        s, d = directed_path(n)
        got = gpu_count(counter, n, s, d, k)
        assert got[path_cls] == n - k + 1 and got.sum() == n - k + 1
    s, d = directed_cycle(10007)
    got = gpu_count(counter, 10007, s, d, k)
    assert got[path_cls] == 10007 and got.sum() == 10007


def test_star_example(counter):
    # Fig. star of the paper: 16/20/20/6/6/10, total 78
    from tests.test_oracle_pins import star_graph
    n, s, d = star_graph()
    got = gpu_count(counter, n, s, d, 3)
    assert got.tolist() == oracle.count(n, s, d, 3).tolist()
    assert sorted(got[got > 0].tolist()) == [6, 6, 10, 16, 20, 20]


@pytest.mark.parametrize("k", [3, 4, 5])
def test_edge_cases(counter, k):
    import torch
    z = np.zeros(0, dtype=np.int32)
    assert gpu_count(counter, 0, z, z, k).sum() == 0
    assert gpu_count(counter, 100, z, z, k).sum() == 0
    s, d = complete_bidirected(k - 1)
    assert gpu_count(counter, k - 1, s, d, k).sum() == 0
    # repeated arcs and unsorted rows count once; isolated vertices add nothing
    rng = np.random.default_rng(5)
    s, d = random_digraph(rng, 30, 0.3, 0.4)
    base = oracle.count(30, s, d, k)
    s2, d2 = np.concatenate([s, s[:20]]), np.concatenate([d, d[:20]])
    rowptr, col = csr_arrays(30, s2, d2)
    for v in range(30):  # reverse each row
        col[rowptr[v]:rowptr[v + 1]] = col[rowptr[v]:rowptr[v + 1]][::-1].copy()
    out = counter.count(torch.from_numpy(rowptr).cuda(), torch.from_numpy(col).cuda(), 30, k)
    assert out.cpu().numpy().tolist() == base.tolist()
    assert gpu_count(counter, 45, s, d, k).tolist() == base.tolist()


@pytest.mark.parametrize("k", [3, 4])
def test_repeated_arcs_relabelled_and_buffer_reuse(counter, k):
    """Graphs above the renumbering threshold with repeated arcs and reversed
    rows, interleaved with other sizes and a malformed call on one context:
    each call must see an all-zero pair-state buffer."""
    import torch
    import paper_1203_3415_gb300 as p
    g = synth.chung_lu(1500, 6000, 2.2, 120, 10, 71)
    s2 = np.concatenate([g.src, g.src[::3], g.dst[:50]])
    d2 = np.concatenate([g.dst, g.dst[::3], g.src[:50]])  # repeats, plus 50 reverse arcs
    rowptr, col = csr_arrays(g.n, s2, d2)
    for v in range(g.n):
        col[rowptr[v]:rowptr[v + 1]] = col[rowptr[v]:rowptr[v + 1]][::-1].copy()
    want = oracle.count(g.n, s2, d2, k, threads=oracle.max_threads())
    r_dev, c_dev = torch.from_numpy(rowptr).cuda(), torch.from_numpy(col).cuda()
    assert counter.count(r_dev, c_dev, g.n, k).cpu().numpy().tolist() == want.tolist()
    h = synth.chung_lu(3000, 9000, 2.2, 150, 10, 72)
    assert gpu_count(counter, h.n, h.src, h.dst, k).tolist() == \
        oracle.count(h.n, h.src, h.dst, k, threads=oracle.max_threads()).tolist()
    bad_r, bad_c = csr_arrays(1200, [0, 1], [1, 1])  # self-loop
    with pytest.raises(p.MotifError):
        counter.count(torch.from_numpy(bad_r).cuda(), torch.from_numpy(bad_c).cuda(), 1200, k)
    assert counter.count(r_dev, c_dev, g.n, k).cpu().numpy().tolist() == want.tolist()


def test_large_graph_paths(counter):
    """n = 40000: the renumbering without the shared-memory histogram, the
    tiled degree scan and three occupancy words per row."""
    g = synth.chung_lu(40000, 160000, 2.2, 300, 10, 73)
    want = oracle.count(g.n, g.src, g.dst, 3, threads=oracle.max_threads())
    assert gpu_count(counter, g.n, g.src, g.dst, 3).tolist() == want.tolist()


@pytest.mark.parametrize("k", [3, 4, 5])
def test_schedules_give_identical_counts(counter, k):
    """Every unit heavy and cut into one-unit tiles (the queue overflows and
    units finish their own rows), every unit light, and mixtures: the
    schedule moves work between warps, never the counts."""
    import paper_1203_3415_gb300 as p
    n, m = {3: (3000, 15000), 4: (2000, 8000), 5: (800, 2400)}[k]
    g = synth.chung_lu(n, m, 2.2, 150, 10, 90 + k)
    want = oracle.count(g.n, g.src, g.dst, k, threads=threads()).tolist()
    try:
        for light, target in [(1, 1), (1, 64), (1 << 40, 1 << 40), (64, 1 << 40), (0, 0)]:
            counter.set_schedule(light, target)
            assert gpu_count(counter, g.n, g.src, g.dst, k).tolist() == want, (light, target)
        with pytest.raises(p.MotifError):
            counter.set_schedule(-1, 0)
    finally:
        counter.set_schedule(0, 0)


def test_graph_above_131072_vertices(counter):
    """n = 140000 (a 4.9 GB pair-state block): 64-bit offsets and the
    renumbering and scan paths for large sets."""
    g = synth.chung_lu(140000, 420000, 2.2, 300, 10, 74)
    want = oracle.count(g.n, g.src, g.dst, 3, threads=oracle.max_threads())
    assert gpu_count(counter, g.n, g.src, g.dst, 3).tolist() == want.tolist()


def test_malformed_input(counter):
    import torch
    import paper_1203_3415_gb300 as p
    good_r, good_c = csr_arrays(5, [0, 1, 2], [1, 2, 3])
    cases = []
    r, c = good_r.copy(), good_c.copy(); c[1] = 1; cases.append((r, c))         # self-loop 1 -> 1
    r, c = good_r.copy(), good_c.copy(); c[2] = 5; cases.append((r, c))         # target out of range
    r, c = good_r.copy(), good_c.copy(); c[0] = -3; cases.append((r, c))        # negative target
    r, c = good_r.copy(), good_c.copy(); r[2], r[3] = r[3], r[2]; cases.append((r, c))  # rowptr decreasing
    r, c = good_r.copy(), good_c.copy(); r[-1] = 2; cases.append((r, c))        # rowptr[n] != m
    for r, c in cases:
        with pytest.raises(p.MotifError) as e:
            counter.count(torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), 5, 3)
            torch.cuda.synchronize()
        assert e.value.code == p.ACC_ERR_INPUT
        # asynchronous form: the status word carries the error
        st = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        counter.count(torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda(), 5, 3, status=st)
        assert int(st.item()) == p.ACC_ERR_INPUT
    # host-checked errors
    rr = torch.from_numpy(good_r).cuda()
    cc = torch.from_numpy(good_c).cuda()
    assert p.acc_motif_count(counter.ctx, rr.data_ptr(), cc.data_ptr(), 5, 3, 6, 0, rr.data_ptr(), None) == p.ACC_ERR_K
    # above the size limit (the count mode builds graphs above the dense
    # block's limit without it, up to ACC_MAX_N_SPARSE vertices): refused on
    # the host, before the undersized arrays passed here could be read
    too_many = p.ACC_MAX_N_SPARSE + 1 if counter.mode == p.ACC_MODE_COUNT else p.ACC_MAX_N + 1
    assert p.acc_motif_count(counter.ctx, rr.data_ptr(), cc.data_ptr(), too_many, 3, 3, 0, rr.data_ptr(),
                             None) == p.ACC_ERR_TOO_LARGE
    assert p.acc_motif_count(counter.ctx, 0, cc.data_ptr(), 5, 3, 3, 0, rr.data_ptr(), None) == p.ACC_ERR_ARG
    # a good graph after the errors still counts
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = counter.count(rr, cc, 5, 3, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(out.sum().item()) == 2


@pytest.mark.parametrize("k", [3, 4, 5])
def test_host_entry_point(counter, k):
    g = synth.chung_lu(2000, 8000, 2.3, 120, 10, 21)
    rowptr, col = g.csr()
    got = counter.count_host(rowptr, col, g.n, k)
    assert got.tolist() == gpu_count(counter, g.n, g.src, g.dst, k).tolist()


def test_nonblocking_stream(counter):
    import torch
    g = synth.chung_lu(3000, 12000, 2.2, 150, 10, 31)
    expect = oracle.count(g.n, g.src, g.dst, 4, threads=threads())
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = gpu_count(counter, g.n, g.src, g.dst, 4, stream=s)
    assert got.tolist() == expect.tolist()


def read_golden(name):
    from tests.golden.golden_io import read_counts
    return read_counts(os.path.join(GOLDEN, name + ".txt"))


@pytest.mark.parametrize("name,make,k", [
    ("er_n1000_m5000_k3", synth.er_k3, 3),
    ("chung_lu_n20000_m100000_k4", synth.chung_lu_k4, 4),
    ("regulatory_n5000_m15000_k5", synth.regulatory_k5, 5),
])
def test_full_size_workloads(counter, name, make, k):
    hdr, expect = read_golden(name)
    g = make()
    assert f"sha256={synth.graph_digest(g)}" in hdr["graph"], "generator drifted from the stored graph"
    got = gpu_count(counter, g.n, g.src, g.dst, k)
    assert got.tolist() == expect.tolist()
    # a property that holds at any size: relabelling the vertices changes nothing
    perm = np.random.default_rng(9).permutation(g.n).astype(np.int32)
    got2 = gpu_count(counter, g.n, perm[g.src], perm[g.dst], k)
    assert got2.tolist() == expect.tolist()


def test_workspace_reuse_across_sizes(counter):
    a = synth.chung_lu(500, 2000, 2.2, 60, 10, 41)
    b = synth.chung_lu(3000, 9000, 2.2, 100, 10, 42)
    ea = oracle.count(a.n, a.src, a.dst, 4)
    for _ in range(2):
        assert gpu_count(counter, a.n, a.src, a.dst, 4).tolist() == ea.tolist()
        gpu_count(counter, b.n, b.src, b.dst, 5)
        gpu_count(counter, b.n, b.src, b.dst, 3)


def test_count_bound_guard(counter):
    """The overflow guard: an out-star with 50000 leaves at k = 5 has a
    degree bound of about 6.5e18 > 2^62, so it is refused with
    ACC_ERR_OVERFLOW (synchronously and through the status word) without
    being enumerated; at k = 4 its bound (about 8.3e13) passes and the count
    is the closed form C(50000, 3) in the out-star class (count mode; the
    enumerate mode would visit all 2e13 leaves).  The context then counts a
    small graph correctly."""
    import torch
    import paper_1203_3415_gb300 as p
    L = 50000
    r, c = csr_arrays(L + 1, np.zeros(L, np.int32), np.arange(1, L + 1, dtype=np.int32))
    rr, cc = torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()
    with pytest.raises(p.MotifError) as e:
        counter.count(rr, cc, L + 1, 5)
    assert e.value.code == p.ACC_ERR_OVERFLOW
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    counter.count(rr, cc, L + 1, 5, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == p.ACC_ERR_OVERFLOW
    if counter.mode == p.ACC_MODE_COUNT:
        got = counter.count(rr, cc, L + 1, 4).cpu().numpy()
        n, s, d = 4, *out_star(3)
        want_cls = int(np.flatnonzero(oracle.count(n, s, d, 4))[0])
        assert int(got.sum()) == math.comb(L, 3) and int(got[want_cls]) == math.comb(L, 3)
    assert gpu_count(counter, 5, [0, 1, 2], [1, 2, 3], 3).tolist() == oracle.count(5, [0, 1, 2], [1, 2, 3], 3).tolist()
