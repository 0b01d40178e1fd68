"""The library's own kernel source, run on the CPU.

tests/emu/shim.h stands in for the CUDA constructs the kernels use: a thread
per lane and a 32-thread barrier for every warp collective, so a lane that
skips a collective its warp reaches hangs the warp and the driver reports
it.  The kernels' code is cut from the CUDA sources between fixed anchors
and compiled with g++ together with the library's own internal headers; the
results are compared with the oracle (copies, k = 3, 4, 5 formula counts) or with
the lists a plain host loop writes (neighbour-list fill).  This checks the
kernels' logic and warp discipline without a GPU; the GPU tests check the
compiled kernels."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle
import synth
from tests.graph_helpers import random_digraph

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1203_3415_gb300", "csrc")
EMU = os.path.join(HERE, "emu")


def _region(src, start, end):
    a = src.index(start)
    b = src.index(end, a)
    return src[a:b]


def _function(src, head):
    a = src.index(head)
    return src[a:src.index("\n}\n", a) + 3]


@pytest.fixture(scope="session")
def emu_bins(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("emu")
    rand = open(os.path.join(CSRC, "randomise.cu")).read()
    open(out / "rand_kernels.inc", "w").write(_region(rand, "constexpr int kRandThreads", "}  // namespace\n"))
    f4 = open(os.path.join(CSRC, "formula4.cu")).read()
    open(out / "f4_kernels.inc", "w").write(_region(f4, "constexpr int kF4Classes", "}  // namespace\n"))
    f3 = open(os.path.join(CSRC, "formula3.cu")).read()
    open(out / "f3_kernels.inc", "w").write(_region(f3, "constexpr int kF3Classes", "}  // namespace\n"))
    f5 = open(os.path.join(CSRC, "formula5.cu")).read()
    open(out / "f5_kernels.inc", "w").write(_region(f5, "constexpr int kF5Classes", "}  // namespace\n"))
    graph = open(os.path.join(CSRC, "graph.cu")).read()
    open(out / "fill_kernels.inc", "w").write(
        _function(graph, "__device__ __forceinline__ int warp_excl_scan") + "\n" +
        _function(graph, "__global__ void k_fill("))
    bins = {}
    for name in ("emu_rand", "emu_f4", "emu_f35", "emu_fill"):
        exe = out / name
        cmd = ["g++", "-std=c++20", "-O1", "-pthread", "-w", "-I", str(out), "-I", EMU, "-I",
               os.path.join(EMU, "fake"), "-I", CSRC, "-o", str(exe), os.path.join(EMU, name + ".cpp")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode and "barrier" in r.stderr:
            pytest.skip("the host compiler has no C++20 <barrier>")
        assert r.returncode == 0, r.stderr[-3000:]
        bins[name] = str(exe)
    bins["dir"] = out
    return bins


def csr(n, s, d):
    order = np.lexsort((d, s))
    col = np.ascontiguousarray(np.asarray(d)[order], dtype=np.int32)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(np.asarray(s, np.int64), minlength=n), out=rowptr[1:])
    return rowptr, col


def _run(exe, inp, out, tmp):
    ip, op = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
    open(ip, "wb").write(inp)
    r = subprocess.run([exe, ip, op], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return open(op, "rb").read() if out else r.stdout


@pytest.mark.parametrize("mode,use_bits", [(0, 1), (0, 0), (1, 1), (1, 0)],
                         ids=["swap_speculative", "swap_row_scan", "mutual_speculative", "mutual_row_scan"])
def test_randomiser_kernels_equal_oracle(emu_bins, mode, use_bits):
    rng = np.random.default_rng(500 + 2 * mode + use_bits)
    graphs = []
    for _ in range(3):
        n = int(rng.integers(4, 30))
        s, d = random_digraph(rng, n, p=float(rng.uniform(0.1, 0.5)), recip=float(rng.random()))
        graphs.append((n, *csr(n, s, d)))
    graphs.append((4, np.zeros(5, np.int64), np.zeros(0, np.int32)))  # no arcs
    R, q = 2, 2
    seeds = [7 + 1000 * g for g in range(len(graphs))]
    buf = struct.pack("<5i", len(graphs), R, q, mode, use_bits)
    for (n, rp, cl), sd in zip(graphs, seeds):
        buf += struct.pack("<iqQ", n, len(cl), sd) + rp.astype("<i8").tobytes() + cl.astype("<i4").tobytes()
    raw = _run(emu_bins["emu_rand"], buf, True, emu_bins["dir"])
    M = sum(len(cl) for _, _, cl in graphs)
    status = struct.unpack("<i", raw[:4])[0]
    out = np.frombuffer(raw[4:4 + 4 * R * M], "<i4")
    acc = np.frombuffer(raw[4 + 4 * R * M:], "<i8").reshape(len(graphs), R)
    assert status == 0
    off = 0
    for g, (n, rp, cl) in enumerate(graphs):
        m = len(cl)
        for r in range(R):
            want, wa = oracle.swap_randomise(n, rp, cl, q * m, seeds[g] + r, mode)
            assert np.array_equal(out[off + r * m: off + (r + 1) * m], want), (g, r)
            assert acc[g, r] == wa, (g, r)
        off += R * m


def _gstar(n, s, d):
    """Pair-state block, sorted G* lists with states, degrees, below-counts."""
    pitch = ((n + 15) // 16 + 3) & ~3
    S = np.zeros((n, n), np.uint8)
    for a, b in zip(np.asarray(s).tolist(), np.asarray(d).tolist()):
        S[a, b] |= 1
        S[b, a] |= 2
    st = np.zeros(n * pitch, np.uint32)
    nptr, deg, lo, nbr = [0], [], [], []
    for v in range(n):
        us = np.nonzero(S[v])[0]
        for u in us:
            st[v * pitch + (u >> 4)] |= np.uint32(int(S[v, u]) << ((u & 15) * 2))
        deg.append(len(us))
        lo.append(int((us < v).sum()))
        nbr += [(int(u) << 2) | int(S[v, u]) for u in us]
        nptr.append(len(nbr))
    return pitch, st, np.array(nptr, np.int64), np.array(deg, np.int32), np.array(lo, np.int32), \
        np.array(nbr, np.uint32)


def test_k4_formula_kernels_equal_oracle(emu_bins):
    rng = np.random.default_rng(44)
    cases = []
    for _ in range(3):
        n = int(rng.integers(5, 22))
        cases.append((n, *random_digraph(rng, n, p=float(rng.uniform(0.1, 0.5)), recip=float(rng.random()))))
    g = synth.chung_lu(40, 120, 2.1, 15, 20, 5)
    cases.append((g.n, g.src, g.dst))
    cls, cc = oracle.table(4)
    for n, s, d in cases:
        pitch, st, nptr, deg, lo, nbr = _gstar(n, s, d)
        buf = struct.pack("<3q", n, pitch, len(nbr)) + st.tobytes() + nptr.astype("<i8").tobytes() + \
            deg.astype("<i4").tobytes() + lo.astype("<i4").tobytes() + nbr.astype("<u4").tobytes() + \
            np.asarray(cls, "<i2").tobytes() + np.asarray(cc, "<u4").tobytes()
        vals = [int(x) for x in _run(emu_bins["emu_f4"], buf, False, emu_bins["dir"]).split()]
        assert vals[0] == 0
        assert vals[1:] == oracle.count(n, s, d, 4).tolist(), n


@pytest.mark.parametrize("k", [3, 5])
def test_k3_k5_formula_kernels_equal_oracle(emu_bins, k):
    rng = np.random.default_rng(30 + k)
    cases = []
    for _ in range(3):
        n = int(rng.integers(4, 40 if k == 3 else 14))
        cases.append((n, *random_digraph(rng, n, p=float(rng.uniform(0.1, 0.5)), recip=float(rng.random()))))
    if k == 3:
        g = synth.chung_lu(200, 800, 2.1, 40, 20, 6)
        cases.append((g.n, g.src, g.dst))
    cls, cc = oracle.table(k)
    for n, s, d in cases:
        pitch, st, nptr, deg, lo, nbr = _gstar(n, s, d)
        buf = struct.pack("<4q", k, n, pitch, len(nbr)) + st.tobytes() + nptr.astype("<i8").tobytes() + \
            deg.astype("<i4").tobytes() + lo.astype("<i4").tobytes() + nbr.astype("<u4").tobytes() + \
            np.asarray(cls, "<i2").tobytes() + np.asarray(cc, "<u4").tobytes()
        vals = [int(x) for x in _run(emu_bins["emu_f35"], buf, False, emu_bins["dir"]).split()]
        assert vals[0] == 0
        assert vals[1:] == oracle.count(n, s, d, k).tolist(), (k, n)


@pytest.mark.parametrize("rw", [1, 4, 32])
def test_fill_kernel_writes_sorted_lists(emu_bins, rw):
    rng = np.random.default_rng(60 + rw)
    # 600 vertices: two 32-word chunks per row, so a warp's rows can hold more
    # marked chunks than lanes and a row's chunks can straddle two rounds
    for n in ((int(rng.integers(1, 120)),) if rw == 1 else (int(rng.integers(1, 200)), 600)):
        s, d = random_digraph(rng, n, p=min(0.3, 8.0 / max(n, 1)), recip=0.3)
        pitch, st, nptr, deg, lo, nbr = _gstar(n, s, d)
        occ_w = max(1, ((pitch + 31) // 32 + 31) // 32)
        occ = np.zeros(n * occ_w, np.uint32)
        for v in range(n):
            for wd in np.nonzero(st[v * pitch:(v + 1) * pitch])[0]:
                ch = int(wd) // 32
                occ[v * occ_w + ch // 32] |= np.uint32(1 << (ch % 32))
        buf = struct.pack("<4q", n, pitch, occ_w, rw) + st.tobytes() + occ.tobytes() + nptr.astype("<i8").tobytes()
        got = np.frombuffer(_run(emu_bins["emu_fill"], buf, True, emu_bins["dir"]), "<u4")
        assert np.array_equal(got, nbr), (n, rw)
