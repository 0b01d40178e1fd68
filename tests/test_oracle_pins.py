"""Pins for the oracle's counters against what the paper and the mathematics fix.

* the paper's star example (Fig. star, Section "Counting isomorphic patterns of
  size 3"): 16/20/20/6/6/10 open 3-patterns around the centre;
* Table starb (Theorem teo3): the 13 per-vertex k=3 formulas, summed over all
  vertices with the closed (triangle) lines divided by 3 (Algorithm s3), must
  equal the enumeration on random digraphs;
* Table ept (Theorem teo4u) with the multiplicity correction of Fact
  correction (1/3/3/4/5/6) on all-bidirected graphs, for k=4;
* closed forms: complete bidirected graphs, directed paths and cycles,
  transitive tournaments, out- and in-stars;
* brute force over every k-subset on tiny graphs (all densities and
  reciprocities), and invariants (relabelling, arc reversal, disjoint union,
  isolated vertices) on graphs too large for brute force.
"""
import math

import numpy as np
import pytest

from tests.graph_helpers import (bidirected, complete_bidirected, directed_cycle, directed_path,
                                 in_star, out_star, random_digraph, relabel, transitive_tournament)


def cls_of(orc, k, arcs):
    c = orc.classify(k, orc.code_of_arcs(k, arcs))
    assert c >= 0
    return c


def bi(a, b):
    return [(a, b), (b, a)]


# ---------------------------------------------------------------------------
# The paper's star example
# ---------------------------------------------------------------------------

def star_graph():
    """Fig. star: centre v_c with n_a = 4 bidirected, n_b = 4 out- and n_c = 5
    in-neighbours (read from the figure's drawing: 5 arcs into the centre, 4
    out of it, 4 drawn with both arrow ends)."""
    src, dst = [], []
    leaf = 1
    for _ in range(4):  # A: bidirected
        src += [0, leaf]; dst += [leaf, 0]; leaf += 1
    for _ in range(4):  # B: centre -> leaf
        src += [0]; dst += [leaf]; leaf += 1
    for _ in range(5):  # C: leaf -> centre
        src += [leaf]; dst += [0]; leaf += 1
    return leaf, np.array(src), np.array(dst)


def test_star_example(orc):
    n, s, d = star_graph()
    counts = orc.count(n, s, d, 3)
    expect = np.zeros(13, dtype=np.int64)
    # the six patterns and frequencies printed beside Fig. star
    expect[cls_of(orc, 3, bi(0, 1) + [(0, 2)])] += 4 * 4          # o<->o->o : n_a n_b
    expect[cls_of(orc, 3, bi(0, 1) + [(2, 0)])] += 4 * 5          # o<->o<-o : n_a n_c
    expect[cls_of(orc, 3, [(1, 0), (0, 2)])] += 4 * 5             # o->o->o  : n_b n_c
    expect[cls_of(orc, 3, bi(0, 1) + bi(0, 2))] += math.comb(4, 2)  # o<->o<->o
    expect[cls_of(orc, 3, [(0, 1), (0, 2)])] += math.comb(4, 2)   # o<-o->o
    expect[cls_of(orc, 3, [(1, 0), (2, 0)])] += math.comb(5, 2)   # o->o<-o
    assert counts.tolist() == expect.tolist()
    assert counts.sum() == math.comb(13, 2) == 78
    assert (orc.count_bruteforce(n, s, d, 3) == counts).all()


# ---------------------------------------------------------------------------
# Table starb (Theorem teo3, Algorithm s3)
# ---------------------------------------------------------------------------

# patterns of Table starb, lines 1..13, as arcs over slots 0..2 (slot 0 is the
# centre of the open lines); the closed lines are read from the drawings
STARB_PATTERNS = [
    bi(0, 1) + [(0, 2)],                  # 1  o<->o->o
    bi(0, 1) + [(2, 0)],                  # 2  o<->o<-o
    [(1, 0), (0, 2)],                     # 3  o->o->o
    bi(0, 1) + bi(0, 2),                  # 4  o<->o<->o
    [(0, 1), (0, 2)],                     # 5  o<-o->o
    [(1, 0), (2, 0)],                     # 6  o->o<-o
    bi(0, 1) + bi(1, 2) + bi(2, 0),       # 7  all bidirected
    [(1, 0), (2, 1), (0, 2)],             # 8  directed cycle
    [(0, 1), (2, 1)] + bi(0, 2),          # 9
    [(1, 0), (2, 1)] + bi(0, 2),          # 10
    bi(0, 1) + bi(1, 2) + [(2, 0)],       # 11
    [(1, 0), (1, 2)] + bi(0, 2),          # 12
    [(1, 0), (1, 2), (0, 2)],             # 13 transitive triangle
]


def starb_counts(n, src, dst):
    """Table starb summed over v; closed lines divided by 3 (Algorithm s3).

    The variables of Table vars come from a plain scan over each vertex's
    neighbour pairs: A = bidirected, B = out-only, C = in-only neighbours;
    m_xy counts one-way arcs from set x to set y, m'_xy bidirected pairs
    between x and y (within one set when x = y)."""
    A = np.zeros((n, n), dtype=bool)
    A[src, dst] = True
    total = np.zeros(14, dtype=np.int64)
    for v in range(n):
        nb = {}
        for u in range(n):
            if u == v:
                continue
            if A[v, u] and A[u, v]:
                nb[u] = "a"
            elif A[v, u]:
                nb[u] = "b"
            elif A[u, v]:
                nb[u] = "c"
        cnt = {t: sum(1 for x in nb.values() if x == t) for t in "abc"}
        m = {(x, y): 0 for x in "abc" for y in "abc"}
        mp = {(x, y): 0 for x in "abc" for y in "abc"}
        us = sorted(nb)
        for i, x in enumerate(us):
            for y in us[i + 1:]:
                tx, ty = nb[x], nb[y]
                if A[x, y] and A[y, x]:
                    mp[(tx, ty)] += 1
                    if tx != ty:
                        mp[(ty, tx)] += 1
                elif A[x, y]:
                    m[(tx, ty)] += 1
                elif A[y, x]:
                    m[(ty, tx)] += 1
        na, nbb, nc = cnt["a"], cnt["b"], cnt["c"]
        c2 = lambda x: x * (x - 1) // 2
        line = [0,
                na * nbb - m["a", "b"] - m["b", "a"] - mp["a", "b"],
                na * nc - m["a", "c"] - m["c", "a"] - mp["a", "c"],
                nbb * nc - m["b", "c"] - m["c", "b"] - mp["b", "c"],
                c2(na) - m["a", "a"] - mp["a", "a"],
                c2(nbb) - m["b", "b"] - mp["b", "b"],
                c2(nc) - m["c", "c"] - mp["c", "c"],
                mp["a", "a"],
                m["b", "c"],
                m["a", "b"] + mp["c", "c"],
                m["b", "a"] + m["a", "c"] + mp["c", "b"],
                mp["a", "b"] + mp["a", "c"] + m["a", "a"],
                m["c", "a"] + mp["b", "b"],
                m["c", "b"] + m["b", "b"] + m["c", "c"]]
        total += np.array(line, dtype=np.int64)
    for ln in range(7, 14):
        assert total[ln] % 3 == 0
        total[ln] //= 3
    return total[1:]


def test_starb_patterns_are_the_13_classes(orc):
    classes = [cls_of(orc, 3, p) for p in STARB_PATTERNS]
    assert sorted(classes) == list(range(13))


@pytest.mark.parametrize("seed", range(6))
def test_starb_formula_matches_enumeration(orc, seed):
    rng = np.random.default_rng(100 + seed)
    n = 40
    s, d = random_digraph(rng, n, p=[0.05, 0.1, 0.2, 0.3, 0.15, 0.25][seed],
                          recip=[0.0, 0.1, 0.3, 0.5, 0.9, 1.0][seed])
    lines = starb_counts(n, s, d)
    counts = orc.count(n, s, d, 3)
    expect = np.zeros(13, dtype=np.int64)
    for ln, pat in enumerate(STARB_PATTERNS):
        expect[cls_of(orc, 3, pat)] += lines[ln]
    assert counts.tolist() == expect.tolist()


# ---------------------------------------------------------------------------
# Table ept (Theorem teo4u) and Fact correction on all-bidirected graphs
# ---------------------------------------------------------------------------

def ept_counts(n, edges):
    """Undirected 4-pattern counts by Table ept summed over edges, divided by the
    multiplicities of Fact correction.  Order: P4, tailed triangle, S3, C4,
    K4 minus an edge, K4."""
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b); adj[b].add(a)
    tot = np.zeros(6, dtype=np.int64)
    und = {(min(a, b), max(a, b)) for a, b in edges}
    for u, v in und:
        Z = (adj[u] & adj[v]) - {u, v}
        X = adj[u] - Z - {v}
        Y = adj[v] - Z - {u}
        def mm(P, Q):
            if P is Q:
                return sum(1 for a in P for b in adj[a] if b in P) // 2
            return sum(1 for a in P for b in adj[a] if b in Q)
        nx, ny, nz = len(X), len(Y), len(Z)
        mxx, myy, mzz = mm(X, X), mm(Y, Y), mm(Z, Z)
        mxy, mxz, myz = mm(X, Y), mm(X, Z), mm(Y, Z)
        c2 = lambda x: x * (x - 1) // 2
        tot += np.array([nx * ny - mxy,
                         (nx + ny) * nz - mxz - myz + mxx + myy,
                         c2(nx) + c2(ny) - mxx - myy,
                         mxy,
                         c2(nz) + mxz + myz - mzz,
                         mzz], dtype=np.int64)
    div = np.array([1, 3, 3, 4, 5, 6], dtype=np.int64)
    assert (tot % div == 0).all()
    return tot // div


EPT_PATTERNS = [
    bi(0, 1) + bi(1, 2) + bi(2, 3),                      # P4
    bi(0, 1) + bi(1, 2) + bi(2, 0) + bi(2, 3),           # tailed triangle
    bi(0, 1) + bi(0, 2) + bi(0, 3),                      # S3 (claw)
    bi(0, 1) + bi(1, 2) + bi(2, 3) + bi(3, 0),           # C4
    bi(0, 1) + bi(1, 2) + bi(2, 3) + bi(3, 0) + bi(0, 2),  # K4 minus an edge
    bi(0, 1) + bi(1, 2) + bi(2, 3) + bi(3, 0) + bi(0, 2) + bi(1, 3),  # K4
]


@pytest.mark.parametrize("seed", range(4))
def test_ept_formula_matches_enumeration(orc, seed):
    rng = np.random.default_rng(200 + seed)
    n = 30
    p = [0.1, 0.2, 0.35, 0.5][seed]
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    s, d = bidirected(edges)
    counts = orc.count(n, s, d, 4)
    expect = np.zeros(199, dtype=np.int64)
    for val, pat in zip(ept_counts(n, edges), EPT_PATTERNS):
        expect[cls_of(orc, 4, pat)] += val
    assert counts.tolist() == expect.tolist()


def test_all_bidirected_hits_21_classes_at_k5(orc):
    # undirected connected 5-vertex graphs: 21 (Section on undirected k=5)
    rng = np.random.default_rng(7)
    n = 14
    hit = set()
    for p in (0.25, 0.4, 0.6):
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        s, d = bidirected(edges)
        hit |= set(np.nonzero(orc.count(n, s, d, 5))[0].tolist())
    assert len(hit) == 21


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [3, 4, 5])
def test_complete_bidirected(orc, k):
    n = 9
    s, d = complete_bidirected(n)
    counts = orc.count(n, s, d, k)
    full = orc.classify(k, (1 << (k * (k - 1))) - 1)
    assert counts[full] == math.comb(n, k)
    assert counts.sum() == math.comb(n, k)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_directed_path_and_cycle(orc, k):
    path_cls = cls_of(orc, k, [(i, i + 1) for i in range(k - 1)])
    n = 57
    s, d = directed_path(n)
    counts = orc.count(n, s, d, k)
    assert counts[path_cls] == n - k + 1 and counts.sum() == n - k + 1
    s, d = directed_cycle(n)
    counts = orc.count(n, s, d, k)
    assert counts[path_cls] == n and counts.sum() == n


@pytest.mark.parametrize("k", [3, 4, 5])
def test_transitive_tournament(orc, k):
    n = 11
    s, d = transitive_tournament(n)
    counts = orc.count(n, s, d, k)
    tt = cls_of(orc, k, [(i, j) for i in range(k) for j in range(i + 1, k)])
    assert counts[tt] == math.comb(n, k) and counts.sum() == math.comb(n, k)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_stars(orc, k):
    leaves = 12
    s, d = out_star(leaves)
    counts = orc.count(leaves + 1, s, d, k)
    cls = cls_of(orc, k, [(0, i) for i in range(1, k)])
    assert counts[cls] == math.comb(leaves, k - 1) and counts.sum() == math.comb(leaves, k - 1)
    s, d = in_star(leaves)
    counts = orc.count(leaves + 1, s, d, k)
    cls = cls_of(orc, k, [(i, 0) for i in range(1, k)])
    assert counts[cls] == math.comb(leaves, k - 1) and counts.sum() == math.comb(leaves, k - 1)


# ---------------------------------------------------------------------------
# Brute force and invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [3, 4, 5])
def test_enumeration_equals_bruteforce(orc, k):
    rng = np.random.default_rng(300 + k)
    for trial in range(60):
        n = int(rng.integers(k, 15))
        s, d = random_digraph(rng, n, p=float(rng.random()), recip=float(rng.random()))
        assert orc.count(n, s, d, k).tolist() == orc.count_bruteforce(n, s, d, k).tolist()


@pytest.mark.parametrize("k", [3, 4, 5])
def test_empty_and_tiny(orc, k):
    z = np.zeros(0, dtype=np.int32)
    assert orc.count(0, z, z, k).sum() == 0
    assert orc.count(k - 1, *complete_bidirected(k - 1), k).sum() == 0
    assert orc.count(50, z, z, k).sum() == 0


def test_self_loop_rejected(orc):
    with pytest.raises(ValueError):
        orc.count(3, [0, 1], [1, 1], 3)


def test_repeated_arcs_collapse(orc):
    s, d = directed_path(8)
    s2, d2 = np.concatenate([s, s]), np.concatenate([d, d])
    for k in (3, 4, 5):
        assert orc.count(8, s2, d2, k).tolist() == orc.count(8, s, d, k).tolist()


def reverse_class_map(orc, k):
    """Class of the reversed digraph for each class (arcs i->j become j->i)."""
    _, ccode = orc.table(k)
    out = []
    for c in ccode:
        c = int(c)
        arcs = [(j, i) for i in range(k) for j in range(k)
                if i != j and (c >> orc.code_bit(k, i, j)) & 1]
        out.append(cls_of(orc, k, arcs))
    return np.array(out)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_invariants(orc, k):
    rng = np.random.default_rng(400 + k)
    n = 70
    s, d = random_digraph(rng, n, p=0.06, recip=0.2)
    base = orc.count(n, s, d, k)
    # relabelling
    perm = rng.permutation(n)
    s2, d2 = relabel(perm, s, d)
    assert orc.count(n, s2, d2, k).tolist() == base.tolist()
    # reversing every arc maps class c to rev(c)
    rev = reverse_class_map(orc, k)
    rc = orc.count(n, d, s, k)
    assert rc[rev].tolist() == base.tolist()
    # disjoint union with a second graph adds the histograms
    s3, d3 = random_digraph(rng, 40, p=0.1, recip=0.5)
    other = orc.count(40, s3, d3, k)
    su = np.concatenate([s, s3 + n]); du = np.concatenate([d, d3 + n])
    assert orc.count(n + 40, su, du, k).tolist() == (base + other).tolist()
    # isolated vertices change nothing
    assert orc.count(n + 5, s, d, k).tolist() == base.tolist()
    # root ranges partition the count
    parts = orc.count(n, s, d, k, roots=(0, 30)) + orc.count(n, s, d, k, roots=(30, n))
    assert parts.tolist() == base.tolist()
    # threads do not change the result
    assert orc.count(n, s, d, k, threads=4).tolist() == base.tolist()


# ---------------------------------------------------------------------------
# Z-scores (step iii of the motif pipeline; population deviation reading)
# ---------------------------------------------------------------------------

def test_zscores_closed_form(orc):
    rand = np.array([[1, 7], [2, 7], [3, 7], [4, 7]], dtype=np.int64)
    real = np.array([5, 9], dtype=np.int64)
    z = orc.zscores(real, rand)
    # mean 2.5, population variance 1.25: Z = 2.5 / sqrt(1.25) = sqrt(5)
    assert abs(z[0] - math.sqrt(5.0)) <= 4e-16 * math.sqrt(5.0)
    assert math.isnan(z[1])  # zero deviation
    rand = np.array([[10], [20]], dtype=np.int64)
    assert orc.zscores(np.array([15]), rand)[0] == 0.0
    assert orc.zscores(np.array([25]), rand)[0] == 2.0


def test_sorted_list_arc_test_equals_bit_matrix(orc):
    """The oracle's two arc tests (dense bit matrix; binary search in sorted
    out-lists, used above 65536 vertices) give the same counts: on random
    digraphs with repeated arcs, on the closed forms, and on the brute force
    over all k-subsets."""
    rng = np.random.default_rng(4400)
    try:
        cases = []
        for _ in range(40):
            n = int(rng.integers(1, 22))
            s, d = random_digraph(rng, n, p=float(rng.random()), recip=float(rng.random()))
            if len(s):  # repeated arcs
                j = rng.integers(0, len(s), size=len(s) // 3 + 1)
                s, d = np.concatenate([s, s[j]]), np.concatenate([d, d[j]])
            cases.append((n, s, d))
        dense = [[orc.count(n, s, d, k).tolist() for k in (3, 4, 5)] for n, s, d in cases]
        orc.set_dense_max(0)
        for (n, s, d), want in zip(cases, dense):
            assert [orc.count(n, s, d, k).tolist() for k in (3, 4, 5)] == want
            if n <= 12:
                assert orc.count(n, s, d, 4).tolist() == orc.count_bruteforce(n, s, d, 4).tolist()
        s, d = complete_bidirected(9)
        assert int(orc.count(9, s, d, 5).sum()) == math.comb(9, 5)
        s, d = directed_path(30)
        assert int(orc.count(30, s, d, 4).sum()) == 27
    finally:
        orc.set_dense_max(65536)
