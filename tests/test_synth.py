"""The seeded generators: determinism and the structural properties of each workload."""
import math

import numpy as np
import pytest


def simple(g):
    s, d = g.src.astype(np.int64), g.dst.astype(np.int64)
    assert (s != d).all(), "self-loop"
    assert ((s >= 0) & (s < g.n) & (d >= 0) & (d < g.n)).all()
    key = s * g.n + d
    assert len(np.unique(key)) == len(key), "repeated arc"
    rev = d * g.n + s
    return int(np.isin(rev, key).sum())  # arcs whose reverse is present


def test_deterministic(syn):
    a, b = syn.er_k3(), syn.er_k3()
    assert syn.graph_digest(a) == syn.graph_digest(b)
    c = syn.erdos_renyi(1000, 5000, 10, 2)
    assert syn.graph_digest(a) != syn.graph_digest(c)


def test_det_log_exp(syn):
    for x in [1e-300, 1e-5, 0.3, 1.0, 2.0, 7.5, 1e5, 1e300]:
        assert abs(syn.det_log(x) - math.log(x)) <= 4e-16 * max(1.0, abs(math.log(x)))
    for y in [-700.0, -20.0, -1.0, 0.0, 0.5, 3.0, 40.0, 700.0]:
        assert abs(syn.det_exp(y) - math.exp(y)) <= 4e-16 * math.exp(y)


def test_er_k3(syn):
    g = syn.er_k3()
    assert (g.n, g.m) == (1000, 5000)
    assert simple(g) == 500  # 250 reciprocal pairs = 10% of arcs


def test_chung_lu_k4(syn):
    g = syn.chung_lu_k4()
    assert (g.n, g.m) == (20000, 100000)
    assert simple(g) == 10000
    assert np.bincount(g.src, minlength=g.n).max() <= 500
    assert np.bincount(g.dst, minlength=g.n).max() <= 500


def test_regulatory_k5(syn):
    g = syn.regulatory_k5()
    assert (g.n, g.m) == (5000, 15000)
    assert simple(g) == 450  # 225 reciprocal pairs = 3% of arcs
    out = np.bincount(g.src, minlength=g.n)
    assert out.max() <= 200 + 1  # hub cap, plus at most one reciprocated arc
    assert (out >= 20).sum() <= 250


def test_swap_randomise_preserves_degrees(syn):
    base = syn.batch_base(1)
    r, acc = syn.swap_randomise(base, 3 * base.m, 12345)
    simple(r)
    assert acc > base.m  # most attempts accepted on a sparse graph
    for a, b in [(base.src, r.src), (base.dst, r.dst)]:
        assert (np.bincount(a, minlength=base.n) == np.bincount(b, minlength=base.n)).all()
    assert syn.graph_digest(r) != syn.graph_digest(base)


def test_batch_sizes(syn):
    sizes = syn.batch_base_sizes()
    assert len(sizes) == 8 and sizes[:3] == [2000, 500, 5000]
    assert all(500 <= n <= 5000 for n in sizes)


def test_serving_stream(syn):
    specs = syn.serving_pool_specs()
    assert len(specs) == 64
    assert all(100 <= n <= 50000 and 4 * n - 1 <= m <= 10 * n + 1 for n, m, _ in specs)
    reqs = syn.serving_requests()
    assert 3500 < len(reqs) < 4500
    ks = np.array([k for _, _, k in reqs])
    assert abs((ks == 3).mean() - 0.5) < 0.05 and abs((ks == 5).mean() - 0.15) < 0.05


def test_csr(syn):
    g = syn.er_k3()
    rowptr, col = g.csr()
    assert rowptr[0] == 0 and rowptr[-1] == g.m
    for v in (0, 17, 999):
        row = col[rowptr[v]:rowptr[v + 1]]
        assert (np.diff(row) > 0).all()
        assert sorted(row.tolist()) == sorted(g.dst[g.src == v].tolist())
