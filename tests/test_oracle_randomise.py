"""Pins of the oracle's randomised copies (the random ensemble of the
significance step, Implementation section, steps i and iii).

The oracle scans CSR rows for membership; the input generator's own
double-edge swap (synth.c) keeps its arcs in a hash set.  The two were written
separately, so equal outputs for the same stream pin the oracle's draws,
reject rules and updates; the invariants below pin what every copy must keep
whatever the draws.
"""
import numpy as np
import pytest

from tests.graph_helpers import random_digraph


def csr(n, s, d):
    order = np.lexsort((d, s))
    col = np.ascontiguousarray(d[order], dtype=np.int32)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(s, minlength=n), out=rowptr[1:])
    return rowptr, col


def arcs_of(rowptr, col):
    n = len(rowptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    return src, col.astype(np.int64)


def check_simple(n, rowptr, col):
    s, d = arcs_of(rowptr, col)
    assert (s != d).all(), "self-loop"
    assert ((d >= 0) & (d < n)).all()
    key = s * n + d
    assert len(np.unique(key)) == len(key), "repeated arc"
    return s, d, key


def mutual_profile(n, rowptr, col):
    """Per vertex: single out-arcs, single in-arcs, mutual neighbours."""
    s, d, key = check_simple(n, rowptr, col)
    mutual = np.isin(d * n + s, key)
    return (np.bincount(s[~mutual], minlength=n), np.bincount(d[~mutual], minlength=n),
            np.bincount(s[mutual], minlength=n))


def test_splitmix_first_draw(syn):
    # SplitMix64 from state 0: the first output is 0xE220A8397B1DCDAF
    assert syn.SplitMix64(0).next() == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("seed", [1, 7, 1_000_000, 2**63 + 5])
def test_mode0_equals_generator_hash_set_swaps(orc, syn, seed):
    rng = np.random.default_rng(seed % 1000)
    n = 60
    s, d = random_digraph(rng, n, p=0.08, recip=0.3)
    rowptr, col = csr(n, s, d)
    src, _ = arcs_of(rowptr, col)
    g = syn.Graph(n, src.astype(np.int32), col.copy())
    for attempts in [0, 1, 5, 3 * len(col)]:
        want, acc_want = syn.swap_randomise(g, attempts, seed)
        got, acc = orc.swap_randomise(n, rowptr, col, attempts, seed)
        assert acc == acc_want
        assert np.array_equal(got, want.dst)
        assert np.array_equal(want.src, src)


def test_mode0_equals_generator_on_a_batch_base(orc, syn):
    base = syn.batch_base(1)
    rowptr, col = base.csr()
    assert np.array_equal(col, base.dst)  # the base lists its arcs in CSR order
    for i in range(3):
        want = syn.batch_randomisation(base, 1, i)
        got, acc = orc.swap_randomise(base.n, rowptr, col, 3 * base.m, 2_000_000 + i)
        assert np.array_equal(got, want.dst)
        assert acc > base.m


@pytest.mark.parametrize("mode", [0, 1])
def test_copies_keep_degrees_and_stay_simple(orc, mode):
    rng = np.random.default_rng(11 + mode)
    for trial in range(6):
        n = int(rng.integers(2, 90))
        s, d = random_digraph(rng, n, p=float(rng.uniform(0.02, 0.5)), recip=float(rng.random()))
        rowptr, col = csr(n, s, d)
        out, acc = orc.swap_randomise(n, rowptr, col, 4 * len(col) + 3, 99 + trial, mode)
        check_simple(n, rowptr, out)
        assert np.array_equal(np.bincount(out, minlength=n), np.bincount(col, minlength=n))
        if mode == 1:
            for a, b in zip(mutual_profile(n, rowptr, col), mutual_profile(n, rowptr, out)):
                assert np.array_equal(a, b)
        assert 0 <= acc <= 4 * len(col) + 3


def test_mode1_mutual_pairs_move_as_pairs(orc):
    # two mutual pairs and nothing else: every copy is a perfect matching of
    # {0, 1, 2, 3} by mutual pairs, and all three matchings occur
    s = np.array([0, 1, 2, 3], np.int32)
    d = np.array([1, 0, 3, 2], np.int32)
    rowptr, col = csr(4, s, d)
    seen = set()
    for seed in range(64):
        out, _ = orc.swap_randomise(4, rowptr, col, 7, seed, 1)
        partner = {v: int(out[v]) for v in range(4)}  # one out-arc per vertex
        assert all(partner[partner[v]] == v for v in range(4))
        seen.add(tuple(sorted({tuple(sorted((v, partner[v]))) for v in range(4)})))
    assert seen == {((0, 1), (2, 3)), ((0, 2), (1, 3)), ((0, 3), (1, 2))}


def test_mode1_single_arcs_stay_single(orc):
    # a directed 6-cycle plus one mutual pair: single arcs never gain a reverse
    s = np.array([0, 1, 2, 3, 4, 5, 6, 7], np.int32)
    d = np.array([1, 2, 3, 4, 5, 0, 7, 6], np.int32)
    rowptr, col = csr(8, s, d)
    accepted = 0
    for seed in range(20):
        out, acc = orc.swap_randomise(8, rowptr, col, 50, seed, 1)
        ss, dd, key = check_simple(8, rowptr, out)
        assert int(np.isin(dd * 8 + ss, key).sum()) == 2
        accepted += acc
    assert accepted > 0


def test_mode0_on_mode_invariant_cases(orc):
    # a complete bidirected graph has no legal swap; one arc has nothing to swap with
    n = 5
    s, d = np.nonzero(~np.eye(n, dtype=bool))
    rowptr, col = csr(n, s.astype(np.int32), d.astype(np.int32))
    for mode in (0, 1):
        out, acc = orc.swap_randomise(n, rowptr, col, 200, 3, mode)
        assert acc == 0 and np.array_equal(out, col)
    rowptr1 = np.array([0, 1, 1], np.int64)
    col1 = np.array([1], np.int32)
    out, acc = orc.swap_randomise(2, rowptr1, col1, 10, 3)
    assert acc == 0 and out.tolist() == [1]
    out, acc = orc.swap_randomise(0, np.zeros(1, np.int64), np.zeros(0, np.int32), 10, 3)
    assert acc == 0 and len(out) == 0


def test_stored_batch_graphs_are_the_generators(syn):
    # the stored batch expectations were written from the oracle's copies; the
    # input generator's own copies of base 1 (500 of them) hash the same
    import hashlib
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_k4.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    base = syn.batch_base(1)
    h = hashlib.sha256()
    for g in [base] + [syn.batch_randomisation(base, 1, i) for i in range(syn.BATCH_RANDOMISATIONS)]:
        h.update(syn.graph_digest(g).encode())
    assert h.hexdigest() == rows[1][3]
