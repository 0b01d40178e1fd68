"""CPU oracle for exact connected induced k-subgraph counting (k = 3, 4, 5).

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, links or runs anything in this directory; only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg do.  It
shares no code with the CUDA path.

``oracle.c`` holds the arithmetic: the adjacency-code convention, brute-force
canonical forms (minimum over all k! relabellings), the code -> class table,
the all-subsets counter for tiny graphs, the ESU enumeration counter, the
Z-score formula and the randomised copies (double-edge swaps, with or without
keeping mutual arcs mutual).  This module compiles it with gcc and wraps it with ctypes.

Every function follows the problem statement of the paper (Problems
Motifs-3/4/5, Background section): count the connected induced subgraphs of
size k of a directed graph, grouped by isomorphism class (13/199/9364 classes),
with connectivity taken in the undirected version G* (Notation section).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None
_tables: dict[int, tuple[np.ndarray, np.ndarray]] = {}

NUM_CLASSES = {3: 13, 4: 199, 5: 9364}


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP when the compiler has it)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC], check=True,
                       stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i32p = ctypes.POINTER(ctypes.c_int32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.oracle_num_classes.argtypes = [ctypes.c_int]
    lib.oracle_code_connected.argtypes = [ctypes.c_int, ctypes.c_uint32]
    lib.oracle_permute_code.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_permute_code.restype = ctypes.c_uint32
    lib.oracle_canonical_code.argtypes = [ctypes.c_int, ctypes.c_uint32]
    lib.oracle_canonical_code.restype = ctypes.c_uint32
    lib.oracle_automorphisms.argtypes = [ctypes.c_int, ctypes.c_uint32]
    lib.oracle_build_table.argtypes = [ctypes.c_int, i32p, u32p, ctypes.c_int]
    lib.oracle_count_bruteforce.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int,
                                            u32p, ctypes.c_int, i64p]
    lib.oracle_count_esu.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int, i32p,
                                     ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, i64p]
    lib.oracle_max_threads.argtypes = []
    lib.oracle_zscores.argtypes = [ctypes.c_int, ctypes.c_int, i64p, i64p, f64p]
    lib.oracle_swap_randomise.argtypes = [ctypes.c_int32, ctypes.c_int64, i64p, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int32)]
    lib.oracle_swap_randomise.restype = ctypes.c_int64
    lib.oracle_zscores.restype = None
    lib.oracle_set_dense_max.argtypes = [ctypes.c_int32]
    lib.oracle_set_dense_max.restype = None
    _lib = lib
    return lib


def set_dense_max(n: int) -> None:
    """Graphs of at most n vertices keep the arc test in a dense bit matrix,
    larger ones in sorted out-neighbour lists (default 65536; the counts are
    the same either way)."""
    _load().oracle_set_dense_max(n)


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def code_bit(k: int, i: int, j: int) -> int:
    """Bit of the adjacency code that records the arc from tuple slot i to slot j."""
    return i * (k - 1) + (j - (1 if j > i else 0))


def connected(k: int, code: int) -> bool:
    return bool(_load().oracle_code_connected(k, code))


def permute(k: int, code: int, perm) -> int:
    arr = (ctypes.c_int * k)(*perm)
    return int(_load().oracle_permute_code(k, code, arr))


def canonical(k: int, code: int) -> int:
    return int(_load().oracle_canonical_code(k, code))


def automorphisms(k: int, code: int) -> int:
    return int(_load().oracle_automorphisms(k, code))


def table(k: int) -> tuple[np.ndarray, np.ndarray]:
    """(class_of_code int32[2^(k(k-1))] with -1 for disconnected codes,
    class_code uint32[K] ascending canonical codes).  Cached per process."""
    if k in _tables:
        return _tables[k]
    ncodes = 1 << (k * (k - 1))
    cls = np.empty(ncodes, dtype=np.int32)
    ccode = np.empty(16384, dtype=np.uint32)
    nclass = _load().oracle_build_table(k, _p(cls, ctypes.c_int32), _p(ccode, ctypes.c_uint32), 16384)
    if nclass < 0:
        raise RuntimeError(f"oracle_build_table failed for k={k}")
    _tables[k] = (cls, ccode[:nclass].copy())
    return _tables[k]


def classify(k: int, code: int) -> int:
    """Class index of an adjacency code (-1 if its digraph is disconnected)."""
    return int(table(k)[0][code])


def code_of_arcs(k: int, arcs) -> int:
    """Adjacency code of a k-vertex digraph given as arcs over slots 0..k-1."""
    code = 0
    for a, b in arcs:
        code |= 1 << code_bit(k, a, b)
    return code


def _arcs(src, dst):
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    return s, d


def count_bruteforce(n: int, src, dst, k: int) -> np.ndarray:
    """Counts over all C(n, k) subsets, each canonicalised directly."""
    s, d = _arcs(src, dst)
    _, ccode = table(k)
    counts = np.zeros(len(ccode), dtype=np.int64)
    rc = _load().oracle_count_bruteforce(n, len(s), _p(s, ctypes.c_int32), _p(d, ctypes.c_int32), k,
                                         _p(ccode, ctypes.c_uint32), len(ccode), _p(counts, ctypes.c_int64))
    if rc != 0:
        raise ValueError(f"oracle_count_bruteforce failed ({rc})")
    return counts


def count(n: int, src, dst, k: int, threads: int = 1, roots: tuple[int, int] | None = None) -> np.ndarray:
    """Counts by ESU enumeration; ``roots=(lo, hi)`` keeps the k-sets whose
    smallest vertex lies in [lo, hi)."""
    s, d = _arcs(src, dst)
    cls, ccode = table(k)
    counts = np.zeros(len(ccode), dtype=np.int64)
    lo, hi = (0, n) if roots is None else roots
    rc = _load().oracle_count_esu(n, len(s), _p(s, ctypes.c_int32), _p(d, ctypes.c_int32), k,
                                  _p(cls, ctypes.c_int32), len(ccode), lo, hi, threads,
                                  _p(counts, ctypes.c_int64))
    if rc != 0:
        raise ValueError(f"oracle_count_esu failed ({rc})")
    return counts


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def zscores(real: np.ndarray, rand: np.ndarray) -> np.ndarray:
    """Z-scores of ``real`` (int64[K]) against ``rand`` (int64[R, K])."""
    real = np.ascontiguousarray(real, dtype=np.int64)
    rand = np.ascontiguousarray(rand, dtype=np.int64)
    R, K = rand.shape
    z = np.empty(K, dtype=np.float64)
    _load().oracle_zscores(K, R, _p(real, ctypes.c_int64), _p(rand, ctypes.c_int64), _p(z, ctypes.c_double))
    return z


def swap_randomise(n: int, rowptr, col, attempts: int, seed: int, mode: int = 0) -> tuple[np.ndarray, int]:
    """Randomised copy of the out-CSR graph (rowptr, col): the copy's targets
    in the positions of ``col`` and the number of accepted swaps.  mode 0:
    double-edge swaps; mode 1: swaps that keep mutual arcs mutual."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    out = np.empty(len(col), dtype=np.int32)
    acc = _load().oracle_swap_randomise(n, len(col), _p(rowptr, ctypes.c_int64), _p(col, ctypes.c_int32),
                                        attempts, seed & 0xFFFFFFFFFFFFFFFF, mode, _p(out, ctypes.c_int32))
    if acc < 0:
        raise ValueError("oracle_swap_randomise: invalid argument")
    return out, int(acc)
