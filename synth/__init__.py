"""Seeded synthetic directed graphs for the motif counter's tests and bench.

Input preparation only: this module draws arc lists and converts them to CSR.
It holds none of the counting arithmetic, so the CPU oracle and the CUDA path
can both consume its output without sharing any of the method's code.

The generators live in ``synth.c`` (SplitMix64 streams, deterministic log/exp
built from IEEE basic operations) so that a seed gives the same graph on x86-64
and on aarch64.  ``graph_digest`` hashes the sorted arc list so a test can tell
that it holds the same graph a stored expectation was computed on.

Workload recipes (the shapes the counter is measured on):

* ``er_k3``        directed Erdos-Renyi, n=1000, m=5000, 10% of arcs in
                   reciprocal pairs, seed 1 (k=3 case).
* ``chung_lu_k4``  directed Chung-Lu, n=20000, m=100000, Pareto density
                   exponent 2.2 for out- and in-weights, degrees capped at 500,
                   10% reciprocal, seed 2 (k=4 case).
* ``regulatory_k5`` n=5000, m=15000, 250 hubs (5%) with Pareto(2.0) out-degrees
                   capped at 200, uniform targets, 3% reciprocal, seed 3 (k=5).
* ``batch_k4``     8 directed Chung-Lu base graphs (exponent 2.3, m=4n,
                   n in [500, 5000] log-uniform with both ends), each with 500
                   degree-preserving randomisations of 3m swap attempts
                   (arcs drawn by their position in the base's out-CSR,
                   copy i of base b seeded 10^6 (b+1) + i).
* ``serving_pool`` 64 directed Chung-Lu graphs (exponent 2.2, cap 200),
                   n log-uniform in [100, 50000], mean out-degree in [4, 10],
                   plus a Poisson request stream at 200 req/s.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_synth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library next to it (gcc, no fused FMA)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i32p = ctypes.POINTER(ctypes.c_int32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.synth_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, i32p, i32p]
    lib.synth_er.restype = ctypes.c_int
    lib.synth_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_uint64, i32p, i32p]
    lib.synth_chung_lu.restype = ctypes.c_int
    lib.synth_regulatory.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p, i32p]
    lib.synth_regulatory.restype = ctypes.c_int
    lib.synth_swap_randomise.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int64,
                                         ctypes.c_uint64, i32p, i32p]
    lib.synth_swap_randomise.restype = ctypes.c_int64
    lib.synth_log.argtypes = [ctypes.c_double]
    lib.synth_log.restype = ctypes.c_double
    lib.synth_exp.argtypes = [ctypes.c_double]
    lib.synth_exp.restype = ctypes.c_double
    lib.synth_splitmix_next.argtypes = [u64p]
    lib.synth_splitmix_next.restype = ctypes.c_uint64
    lib.synth_splitmix_unit.argtypes = [u64p]
    lib.synth_splitmix_unit.restype = ctypes.c_double
    lib.synth_splitmix_below.argtypes = [u64p, ctypes.c_uint64]
    lib.synth_splitmix_below.restype = ctypes.c_uint64
    _lib = lib
    return lib


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


@dataclass
class Graph:
    """A simple directed graph as an arc list over vertices 0..n-1."""
    n: int
    src: np.ndarray  # int32[m]
    dst: np.ndarray  # int32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def csr(self):
        """Out-CSR: int64 rowptr[n+1] and int32 col[m], rows sorted by target."""
        return arcs_to_csr(self.n, self.src, self.dst)


def arcs_to_csr(n: int, src: np.ndarray, dst: np.ndarray):
    order = np.lexsort((dst, src))
    col = np.ascontiguousarray(dst[order], dtype=np.int32)
    counts = np.bincount(src, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, col


def graph_digest(g: Graph) -> str:
    """SHA-256 of the sorted arc list (n, then (src, dst) pairs as int32 LE)."""
    order = np.lexsort((g.dst, g.src))
    pairs = np.stack([g.src[order], g.dst[order]], axis=1).astype("<i4")
    h = hashlib.sha256()
    h.update(np.int64(g.n).astype("<i8").tobytes())
    h.update(pairs.tobytes())
    return h.hexdigest()


class SplitMix64:
    """The same SplitMix64 stream as synth.c, for Python-side draws."""

    def __init__(self, seed: int):
        self._state = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next(self) -> int:
        return int(_load().synth_splitmix_next(ctypes.byref(self._state)))

    def unit(self) -> float:
        return float(_load().synth_splitmix_unit(ctypes.byref(self._state)))

    def below(self, bound: int) -> int:
        return int(_load().synth_splitmix_below(ctypes.byref(self._state), bound))


def det_log(x: float) -> float:
    return float(_load().synth_log(x))


def det_exp(x: float) -> float:
    return float(_load().synth_exp(x))


def _alloc(m: int):
    return np.empty(m, dtype=np.int32), np.empty(m, dtype=np.int32)


def erdos_renyi(n: int, m: int, recip_pct: int, seed: int) -> Graph:
    src, dst = _alloc(m)
    rc = _load().synth_er(n, m, recip_pct, seed, _i32p(src), _i32p(dst))
    if rc != 0:
        raise ValueError(f"synth_er failed ({rc}) for n={n} m={m}")
    return Graph(n, src, dst, f"er_n{n}_m{m}_s{seed}")


def chung_lu(n: int, m: int, exponent: float, cap: int, recip_pct: int, seed: int) -> Graph:
    src, dst = _alloc(m)
    rc = _load().synth_chung_lu(n, m, exponent, cap, recip_pct, seed, _i32p(src), _i32p(dst))
    if rc != 0:
        raise ValueError(f"synth_chung_lu failed ({rc}) for n={n} m={m}")
    return Graph(n, src, dst, f"cl_n{n}_m{m}_s{seed}")


def regulatory(n: int, m: int, n_hubs: int, exponent: float, cap: int, recip_pct: int,
               seed: int) -> Graph:
    src, dst = _alloc(m)
    rc = _load().synth_regulatory(n, m, n_hubs, exponent, cap, recip_pct, seed,
                                  _i32p(src), _i32p(dst))
    if rc != 0:
        raise ValueError(f"synth_regulatory failed ({rc}) for n={n} m={m}")
    return Graph(n, src, dst, f"reg_n{n}_m{m}_s{seed}")


def swap_randomise(g: Graph, attempts: int, seed: int) -> tuple[Graph, int]:
    """Degree-preserving double-edge-swap randomisation of ``g``."""
    src, dst = _alloc(g.m)
    acc = _load().synth_swap_randomise(g.n, g.m, _i32p(np.ascontiguousarray(g.src)),
                                       _i32p(np.ascontiguousarray(g.dst)), attempts, seed,
                                       _i32p(src), _i32p(dst))
    if acc < 0:
        raise MemoryError("synth_swap_randomise failed")
    return Graph(g.n, src, dst, f"{g.name}_swap{seed}"), int(acc)


# ----------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------

def er_k3() -> Graph:
    """k=3 workload: directed Erdos-Renyi n=1000, m=5000, 10% reciprocal, seed 1."""
    g = erdos_renyi(1000, 5000, 10, 1)
    g.name = "er_n1000_m5000"
    return g


def chung_lu_k4() -> Graph:
    """k=4 workload: directed Chung-Lu n=20000, m=100000, exponent 2.2, cap 500, seed 2."""
    g = chung_lu(20000, 100000, 2.2, 500, 10, 2)
    g.name = "chung_lu_n20000_m100000"
    return g


def regulatory_k5() -> Graph:
    """k=5 workload: 250 Pareto(2.0) hubs capped at 200, n=5000, m=15000, 3%, seed 3."""
    g = regulatory(5000, 15000, 250, 2.0, 200, 3, 3)
    g.name = "regulatory_n5000_m15000"
    return g


def log_uniform_int(rng: SplitMix64, lo: int, hi: int) -> int:
    a, b = det_log(float(lo)), det_log(float(hi))
    v = int(det_exp(a + rng.unit() * (b - a)) + 0.5)
    return min(max(v, lo), hi)


BATCH_BASES = 8
BATCH_RANDOMISATIONS = 500


def batch_base_sizes() -> list[int]:
    """Vertex counts of the 8 base graphs: 2000, 500, 5000, then 5 log-uniform draws."""
    rng = SplitMix64(100)
    sizes = [2000, 500, 5000]
    while len(sizes) < BATCH_BASES:
        sizes.append(log_uniform_int(rng, 500, 5000))
    return sizes


def csr_order(g: Graph) -> Graph:
    """The same graph with its arcs listed in out-CSR order (by source, then
    target), so that arc e of the list is position e of ``g.csr()``."""
    order = np.lexsort((g.dst, g.src))
    return Graph(g.n, np.ascontiguousarray(g.src[order]), np.ascontiguousarray(g.dst[order]), g.name)


def batch_base(b: int) -> Graph:
    """Base graph b of the batch, arcs in out-CSR order: the swaps of its
    randomisations pick arcs by CSR position."""
    n = batch_base_sizes()[b]
    g = csr_order(chung_lu(n, 4 * n, 2.3, min(500, n // 2), 10, 100 + b))
    g.name = f"batch_base{b}_n{n}"
    return g


def batch_randomisation(base: Graph, b: int, i: int) -> Graph:
    """Randomisation i of base graph b: 3m swap attempts, seed 10^6 (b+1) + i."""
    g, _ = swap_randomise(base, 3 * base.m, 1_000_000 * (b + 1) + i)
    g.name = f"batch_base{b}_rand{i}"
    return g


def batch_k4(n_bases: int = BATCH_BASES, n_rand: int = BATCH_RANDOMISATIONS) -> list[list[Graph]]:
    """[[base, rand_0, ..., rand_{R-1}] for each base graph]."""
    out = []
    for b in range(n_bases):
        base = batch_base(b)
        out.append([base] + [batch_randomisation(base, b, i) for i in range(n_rand)])
    return out


SERVING_POOL = 64


def serving_pool_specs(pool: int = SERVING_POOL, seed: int = 5):
    """(n, m, seed) of each resident graph of the serving workload."""
    rng = SplitMix64(seed)
    specs = []
    for g in range(pool):
        n = log_uniform_int(rng, 100, 50000)
        d = 4.0 + 6.0 * rng.unit()
        m = int(n * d + 0.5)
        specs.append((n, m, 1000 * seed + g))
    return specs


def serving_graph(spec) -> Graph:
    n, m, s = spec
    g = chung_lu(n, m, 2.2, 200, 10, s)
    g.name = f"serve_n{n}_m{m}_s{s}"
    return g


def serving_requests(duration_s: float = 20.0, rate: float = 200.0, pool: int = SERVING_POOL,
                     seed: int = 5):
    """Poisson arrivals: list of (t_arrival_s, graph_id, k), k in {3:50%, 4:35%, 5:15%}."""
    rng = SplitMix64(seed * 7919 + 1)
    t = 0.0
    out = []
    while True:
        t += -det_log(1.0 - rng.unit()) / rate
        if t >= duration_s:
            break
        gid = rng.below(pool)
        u = rng.unit()
        k = 3 if u < 0.50 else (4 if u < 0.85 else 5)
        out.append((t, gid, k))
    return out
