"""Pins for the oracle's code -> class table (canonical labelling by brute force).

Each check rests on something other than the oracle itself: the class counts the
paper prints (Problems Motifs-3/4/5: 13, 199 and 9364 connected classes), the
labelled connected digraph counts from the component recurrence, the orbit-
stabiliser identity, and invariance under relabelling.
"""
import itertools
import math

import numpy as np
import pytest


@pytest.mark.parametrize("k,expected", [(3, 13), (4, 199), (5, 9364)])
def test_class_counts_match_paper(orc, k, expected):
    # Problems Motifs-3/4/5 (Background, "Problem statement"): 13, 199 and 9364
    # isomorphism classes of connected k-vertex digraphs.
    cls, ccode = orc.table(k)
    assert len(ccode) == expected
    assert cls.max() == expected - 1
    assert np.all(np.diff(ccode.astype(np.int64)) > 0)  # ascending canonical codes


def connected_labelled(k):
    """Labelled weakly connected digraphs on k vertices, by the component of vertex 1.

    d(j) = 2^(j(j-1)) digraphs on j labelled vertices; c(k) = d(k) minus those
    where vertex 1 lies in a component of size j < k:
        c(k) = d(k) - sum_{j<k} C(k-1, j-1) c(j) d(k-j).
    """
    d = lambda j: 2 ** (j * (j - 1))
    c = {1: 1}
    for n in range(2, k + 1):
        c[n] = d(n) - sum(math.comb(n - 1, j - 1) * c[j] * d(n - j) for j in range(1, n))
    return c[k]


@pytest.mark.parametrize("k", [3, 4, 5])
def test_labelled_connected_codes(orc, k):
    cls, _ = orc.table(k)
    assert int((cls >= 0).sum()) == connected_labelled(k)
    # the same numbers as a literal check of the recurrence: 54, 3834, 1027080
    assert connected_labelled(k) == {3: 54, 4: 3834, 5: 1027080}[k]


@pytest.mark.parametrize("k", [3, 4, 5])
def test_orbit_stabiliser(orc, k):
    # every class is an orbit of k!/|Aut| labelled codes; the orbits tile the
    # connected codes exactly once
    cls, ccode = orc.table(k)
    total = sum(math.factorial(k) // orc.automorphisms(k, int(c)) for c in ccode)
    assert total == int((cls >= 0).sum())
    sizes = np.bincount(cls[cls >= 0], minlength=len(ccode))
    for i, c in enumerate(ccode[:: max(1, len(ccode) // 200)]):
        j = int(np.searchsorted(ccode, c))
        assert sizes[j] == math.factorial(k) // orc.automorphisms(k, int(c))


@pytest.mark.parametrize("k,total", [(3, 16), (4, 218)])
def test_all_digraph_classes(orc, k, total):
    # unlabelled digraphs on 3 and 4 vertices, connected or not, number 16
    # and 218; the 3 disconnected 3-vertex ones (no arc, one arc, one
    # bidirected pair) plus the paper's 13 connected ones give 16.
    canon = {orc.canonical(k, c) for c in range(1 << (k * (k - 1)))}
    assert len(canon) == total


def test_three_vertex_classes_by_hand(orc):
    # the 13 connected 3-vertex digraphs: 6 with two linked pairs (each pair
    # one of ->, <-, <->, arranged around a centre) and 7 triangles
    # (Table starb lists 6 open and 7 closed patterns).
    cls, ccode = orc.table(3)
    open_, closed = 0, 0
    for c in ccode:
        pairs = 0
        for i, j in [(0, 1), (0, 2), (1, 2)]:
            if (c >> orc.code_bit(3, i, j)) & 1 or (c >> orc.code_bit(3, j, i)) & 1:
                pairs += 1
        open_ += pairs == 2
        closed += pairs == 3
    assert (open_, closed) == (6, 7)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_table_is_relabelling_invariant(orc, k):
    cls, ccode = orc.table(k)
    rng = np.random.default_rng(10 + k)
    nbits = k * (k - 1)
    perms = list(itertools.permutations(range(k)))
    for _ in range(400):
        code = int(rng.integers(0, 1 << nbits))
        p = perms[int(rng.integers(0, len(perms)))]
        assert cls[code] == cls[orc.permute(k, code, p)]
    # a canonical code is the minimum of its orbit
    for c in ccode[:: max(1, len(ccode) // 50)]:
        c = int(c)
        assert all(orc.permute(k, c, p) >= c for p in perms)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_disconnected_codes_have_no_class(orc, k):
    cls, _ = orc.table(k)
    assert cls[0] == -1  # no arcs
    # a digraph with one isolated slot (slot k-1 untouched) is disconnected
    code = 0
    for i in range(k - 1):
        for j in range(k - 1):
            if i != j:
                code |= 1 << orc.code_bit(k, i, j)
    assert cls[code] == -1
    assert cls[(1 << (k * (k - 1))) - 1] >= 0  # complete bidirected digraph
