"""The library's own CUDA source, run on the CPU.

tests/emu/shim.h stands in for the CUDA constructs the kernels use: a fiber
per GPU thread, a barrier of the warp's 32 lanes for every warp collective
and of the block's threads for __syncthreads, so a lane that skips a
collective its warp reaches leaves the warp waiting, which the shim reports
as a hang.  Kernel launches are rewritten into host calls and the sources
compiled with g++ against the library's own internal headers and a
stand-in CUDA runtime (tests/emu/fake/cuda_runtime.h).

Kernel by kernel: the randomiser, the k = 3, 4, 5 formula paths and the
Z-scores through their launchers; the enumeration kernels (both modes,
light, heavy and queue-full schedules, single graphs and graph sets, and
with tiny shared-memory lists and drain threshold so their overflow lists
and drain run on small graphs); the neighbour-list fill; the whole graph
builder (against a plain construction, and on malformed inputs under the
address sanitizer); the class-table builder (against the oracle's table).
Results are compared with the oracle or with what a plain host loop writes.

End to end: the whole library built for the host runs through its C ABI
(tests/emu/lib_scenarios.py), under the address sanitizer, also under other
lane and block orders, with device work deferred until the host waits for
it, and with injected allocation, launch, copy and graph-launch failures.

This checks the kernels' logic, their warp and block discipline and the
host orchestration without a GPU; the GPU tests check the compiled
kernels."""
import os
import re
import shutil
import struct
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from tests.graph_helpers import random_digraph, out_star, complete_bidirected, directed_path

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


def _launches_to_calls(src):
    """Every `kernel<<<grid, block, smem, stream>>>(args);` of a CUDA source as
    `emu_launch(grid, block, smem, stream, [&] { kernel(args); });`, and its
    dynamic shared arrays as the launch's buffer."""
    out, i = [], 0
    while True:
        a = src.find("<<<", i)
        if a < 0:
            break
        name_start = a
        if src[name_start - 1] == ">":  # template arguments: back to their '<'
            depth = 0
            while True:
                name_start -= 1
                depth += {">": 1, "<": -1}.get(src[name_start], 0)
                if depth == 0:
                    break
        while name_start > 0 and (src[name_start - 1].isalnum() or src[name_start - 1] == "_"):
            name_start -= 1
        b = src.index(">>>(", a)
        depth, c = 1, b + 4
        while depth:
            depth += {"(": 1, ")": -1}.get(src[c], 0)
            c += 1
        assert src[c] == ";", src[a:c + 1]
        out.append(src[i:name_start])
        out.append("emu_launch(%s, [=] { %s(%s); })" % (src[a + 3:b], src[name_start:a], src[b + 4:c - 1]))
        i = c
    out.append(src[i:])
    src = "".join(out)
    # the same for launch_pdl(kernel, grid, block, smem, stream, args...)
    out, i = [], 0
    while True:
        a = src.find("launch_pdl(", i)
        if a < 0:
            break
        j = a + len("launch_pdl(")
        k = j
        while src[k].isalnum() or src[k] == "_":
            k += 1
        if src[k] == "<":  # template arguments of the kernel
            depth = 0
            while True:
                depth += {"<": 1, ">": -1}.get(src[k], 0)
                k += 1
                if depth == 0:
                    break
        kernel = src[j:k]
        parts, depth, start, c = [], 0, k + 1, k + 1
        assert src[k] == ",", src[a:k + 20]
        while True:
            ch = src[c]
            if ch in "([{":
                depth += 1
            elif ch in ")]}":
                if depth == 0:
                    parts.append(src[start:c])
                    break
                depth -= 1
            elif ch == "," and depth == 0:
                parts.append(src[start:c])
                start = c + 1
            c += 1
        assert src[c + 1] == ";", src[a:c + 2]
        cfg, args = parts[:4], parts[4:]
        out.append(src[i:a])
        out.append("emu_launch(%s, [=] { %s(%s); })" % (",".join(cfg), kernel, ",".join(args)))
        i = c + 1
    out.append(src[i:])
    src = "".join(out)
    src = re.sub(r"extern __shared__ (?:__align__\(\d+\) )?([\w ]+?) (\w+)\[\];",
                 r"\1 *\2 = reinterpret_cast<\1 *>(emu_dyn_smem);", src)
    assert "extern __shared__" not in src
    return src


@pytest.fixture(scope="session")
def emu_bins(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("emu")
    rand = open(os.path.join(CSRC, "randomise.cu")).read()
    open(out / "rand_all.inc", "w").write(_launches_to_calls(rand.split('#include "randomise.cuh"\n', 1)[1]))
    # the formula paths whole, kernels and launchers
    for kk in (3, 4, 5):
        src = open(os.path.join(CSRC, "formula%d.cu" % kk)).read()
        open(out / ("f%d_all.inc" % kk), "w").write(_launches_to_calls(src.split('#include "formula.cuh"\n', 1)[1]))
    graph = open(os.path.join(CSRC, "graph.cu")).read()
    open(out / "fill_kernels.inc", "w").write(
        _function(graph, "__device__ __forceinline__ int warp_excl_scan") + "\n" +
        _function(graph, "__global__ void k_fill("))
    en = open(os.path.join(CSRC, "enum.cu")).read()
    region = _region(en, "// Tuning knobs", "template <int K, bool COUNT, int PHASE, bool SET, bool HASH>\nint blocks_per_sm")
    # the kernels' dynamic shared memory becomes a static host buffer; the
    # histogram drain threshold becomes a compile-time parameter
    for old, new in (("extern __shared__ __align__(16) unsigned char smem[];", "unsigned char *smem = emu_smem;"),
                     ("constexpr uint32_t kDrainAt = 1u << 30;", "constexpr uint32_t kDrainAt = EMU_DRAIN_AT;")):
        assert region.count(old) == 1, old
        region = region.replace(old, new)
    open(out / "enum_kernels.inc", "w").write(region)
    lut = open(os.path.join(CSRC, "lut.cu")).read()
    open(out / "relayout.inc", "w").write(_function(lut, "template <int K>\n__global__ void k_relayout("))
    # the graph builder whole, kernels and launcher: each <<<...>>> launch
    # becomes emu_launch, the dynamic shared arrays its buffer; a copy of the
    # internal header with small single-block limits, so that the tiled
    # degree scan and the histogram renumbering run on small sets
    bdir = out / "build"
    bdir.mkdir()
    open(bdir / "graph_kernels.inc", "w").write(_launches_to_calls(
        open(os.path.join(CSRC, "graph.cu")).read().split('#include "common.cuh"\n', 1)[1]))
    common = open(os.path.join(CSRC, "common.cuh")).read()
    for old, new in (('#include "../../include/acc_motif.h"',
                      '#include "' + os.path.join(ROOT, "include", "acc_motif.h") + '"'),
                     ("constexpr long long kScanSingleMax = 1 << 15;", "constexpr long long kScanSingleMax = 2048;"),
                     ("constexpr int kRelabelSmemMax = 1 << 15;", "constexpr int kRelabelSmemMax = 2048;")):
        assert common.count(old) == 1, old
        common = common.replace(old, new)
    open(bdir / "common.cuh", "w").write(common)
    # the same with a count limit of 10^4, for the overflow guard on small graphs
    gdir = out / "guard"
    gdir.mkdir()
    old = "constexpr double kCountLimit = 4611686018427387904.0;  // 2^62"
    assert common.count(old) == 1, old
    open(gdir / "common.cuh", "w").write(common.replace(old, "constexpr double kCountLimit = 10000.0;"))
    open(gdir / "graph_kernels.inc", "w").write(open(bdir / "graph_kernels.inc").read())
    z_src = open(os.path.join(CSRC, "batch.cu")).read().split('#include "common.cuh"\n', 1)[1]
    open(out / "z_all.inc", "w").write(_launches_to_calls(z_src))
    # the class-table builder (kernels and launch_build_lut)
    lut_src = open(os.path.join(CSRC, "lut.cu")).read().split('#include "common.cuh"\n', 1)[1]
    open(out / "lut_all.inc", "w").write(_launches_to_calls(lut_src.split("// Allocation-free table build.")[0]))
    # (binary, source, extra flags): the enumeration kernels as built, and
    # with tiny shared-memory lists and drain threshold so that the overflow
    # lists and the histogram drain run on small graphs
    targets = [(n, n, []) for n in ("emu_rand", "emu_f4", "emu_fill")]
    targets += [("emu_f3", "emu_f35", ["-DEMU_K=3"]), ("emu_f5", "emu_f35", ["-DEMU_K=5"])]
    targets += [("emu_enum", "emu_enum", ["-DEMU_DRAIN_AT=(1u<<30)"]),
                ("emu_enum_small", "emu_enum", ["-DEMU_DRAIN_AT=256u", "-DACC_CAP34=16", "-DACC_CAP5=8",
                                                    "-DACC_PARTB_ROWS=8"]),
                ("emu_build", "emu_build", ["-I", str(bdir), "-fsanitize=address", "-DEMU_LANE_STACK=65536"]),
                ("emu_build_guard", "emu_build", ["-I", str(gdir), "-DEMU_LANE_STACK=65536"]),
                ("emu_lut", "emu_lut", ["-O2"]),
                ("emu_z", "emu_z", ["-ffp-contract=off"])]
    procs = []
    for name, src, extra in targets:
        exe = out / name
        cmd = ["g++", "-std=c++20", "-O1", "-pthread", "-w", *extra, "-I", str(out), "-I", EMU, "-I",
               os.path.join(EMU, "fake"), "-I", CSRC, "-o", str(exe), os.path.join(EMU, src + ".cpp")]
        procs.append((name, exe, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    bins = {}
    for name, exe, pr in procs:
        _, err = pr.communicate()
        if pr.returncode and "barrier" in err:
            pytest.skip("the host compiler has no C++20 <barrier>")
        assert pr.returncode == 0, err[-3000:]
        bins[name] = str(exe)
    bins["dir"] = out
    return bins


def csr(n, s, d):
    order = np.lexsort((d, s))
    col = np.ascontiguousarray(np.asarray(d)[order], dtype=np.int32)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(np.asarray(s, np.int64), minlength=n), out=rowptr[1:])
    return rowptr, col


def _width():
    return max(1, min(8, (os.cpu_count() or 2) - 1))


def _run(exe, inp, out, tmp):
    return _run_many(exe, [inp], out, tmp)[0]


def _run_many(exe, inps, out, tmp):
    """Run the emulator once per input, one process per core at most (each
    runs its lanes as fibers on one host thread); outputs in input order."""
    width = _width()
    res, running, nxt = [None] * len(inps), [], 0
    while nxt < len(inps) or running:
        while nxt < len(inps) and len(running) < width:
            ip, op = os.path.join(tmp, "in%d.bin" % nxt), os.path.join(tmp, "out%d.bin" % nxt)
            open(ip, "wb").write(inps[nxt])
            pr = subprocess.Popen([exe, ip, op], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
            running.append((nxt, op, pr))
            nxt += 1
        i, op, pr = running.pop(0)
        so, se = pr.communicate(timeout=600)
        assert pr.returncode == 0, se[-2000:]
        res[i] = open(op, "rb").read() if out else so
    return res


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
    else:
        # 2500 vertices: the prefix of C(deg, 2) runs over three 1024-vertex
        # tiles with its carry
        g = synth.erdos_renyi(2500, 1500, 10, 7)
        cases.append((g.n, g.src, g.dst))
    cls, cc = oracle.table(k)
    for n, s, d in cases:
        pitch, st, nptr, deg, lo, nbr = _gstar(n, s, d)
        buf = struct.pack("<4q", k, n, pitch, len(nbr)) + st.tobytes() + nptr.astype("<i8").tobytes() + \
            deg.astype("<i4").tobytes() + lo.astype("<i4").tobytes() + nbr.astype("<u4").tobytes() + \
            np.asarray(cls, "<i2").tobytes() + np.asarray(cc, "<u4").tobytes()
        vals = [int(x) for x in _run(emu_bins["emu_f%d" % k], buf, False, emu_bins["dir"]).split()]
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


def _enum_input(k, graphs, mode, light=2048, target=4096, blocks=2, qcap=1 << 16):
    """Emulator input for counting a set of graphs [(n, src, dst)]."""
    cls, _ = oracle.table(k)
    dims, st, nptr, deg, lo, nbr = [], [], [np.zeros(1, np.int64)], [], [], []
    base = 0
    for n, s, d in graphs:
        pitch, st_g, nptr_g, deg_g, lo_g, nbr_g = _gstar(n, s, d)
        dims.append((n, pitch, len(nbr_g)))
        st.append(st_g)
        nptr.append(nptr_g[1:] + base)
        base += len(nbr_g)
        deg.append(deg_g)
        lo.append(lo_g)
        nbr.append(nbr_g)
    buf = struct.pack("<7q", k, len(graphs), mode, light, target, blocks, qcap)
    buf += b"".join(struct.pack("<3q", *x) for x in dims)
    buf += np.concatenate(st).astype("<u4").tobytes() + np.concatenate(nptr).astype("<i8").tobytes() + \
        np.concatenate(deg).astype("<i4").tobytes() + np.concatenate(lo).astype("<i4").tobytes() + \
        np.concatenate(nbr).astype("<u4").tobytes() + np.asarray(cls, "<i2").tobytes()
    return buf


def _enum_many(exe, tmp, k, jobs):
    """Run [(graphs, kwargs)] through the enumeration kernels: per job
    (status, chunks queued, entries scanned, counts per graph)."""
    outs = _run_many(exe, [_enum_input(k, g, **kw) for g, kw in jobs], False, tmp)
    ncls = {3: 13, 4: 199, 5: 9364}[k]
    res = []
    for (graphs, _), o in zip(jobs, outs):
        vals = [int(x) for x in o.split()]
        res.append((vals[0], vals[1], vals[2],
                    [vals[3 + g * ncls: 3 + (g + 1) * ncls] for g in range(len(graphs))]))
    return res


def _enum_cases(rng, k, count, nmax):
    cases = []
    for _ in range(count):
        n = int(rng.integers(3, nmax))
        cases.append((n, *random_digraph(rng, n, p=float(rng.uniform(0.1, 0.5)), recip=float(rng.random()))))
    return cases


# (light, target, queue capacity): every unit light; every unit heavy and cut
# into one-row chunks; every unit heavy with a queue of 3 chunks, so most
# heavy units run their unqueued rows in phase 1
SCHEDULES = {"light": (1 << 30, 1 << 30, 1 << 16), "heavy": (0, 1, 1 << 16), "queue_full": (0, 1, 3)}


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("mode", [0, 1, 2], ids=["count", "enumerate", "count_hashed"])
@pytest.mark.parametrize("sched", list(SCHEDULES))
def test_enumeration_kernels_equal_oracle(emu_bins, k, mode, sched):
    light, target, qcap = SCHEDULES[sched]
    rng = np.random.default_rng(700 + 10 * k + mode)
    cases = _enum_cases(rng, k, 3, {3: 40, 4: 24, 5: 13}[k])
    cases.append((5, np.array([0, 1, 2, 3], np.int64), np.array([1, 2, 3, 4], np.int64)))  # a directed path
    cases.append((6, np.zeros(0, np.int64), np.zeros(0, np.int64)))  # no arcs
    most = 0
    jobs = [([c], dict(mode=mode, light=light, target=target, qcap=qcap)) for c in cases]
    for (n, s, d), (status, queued, scanned, counts) in zip(cases, _enum_many(emu_bins["emu_enum"],
                                                                                emu_bins["dir"], k, jobs)):
        got = counts[0]
        assert status == 0
        assert got == oracle.count(n, s, d, k).tolist(), (k, mode, sched, n)
        if mode == 1:
            assert scanned == 0
        most = max(most, queued)
    # chunks reserved (past the capacity too when the queue is full)
    if sched == "light":
        assert most == 0
    elif k > 3:
        assert most > (3 if sched == "queue_full" else 0)


def _by_degree(n, s, d):
    """The same graph renumbered by descending G* degree, as the library's
    builder does (hubs become roots); counts do not change."""
    s, d = np.asarray(s, np.int64), np.asarray(d, np.int64)
    und = set(zip(np.minimum(s, d).tolist(), np.maximum(s, d).tolist()))
    deg = np.zeros(n, np.int64)
    for a, b in und:
        deg[a] += 1
        deg[b] += 1
    new = np.empty(n, np.int64)
    new[np.argsort(-deg, kind="stable")] = np.arange(n)
    return new[s], new[d]


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("mode", [0, 1, 2], ids=["count", "enumerate", "count_hashed"])
def test_enumeration_overflow_lists_and_drain(emu_bins, k, mode):
    """Shared-memory lists of 16 entries (8 for k = 5) and a histogram drained
    every 256 increments: hub graphs send the extension lists to the per-warp
    overflow buffers and the counts through the drain."""
    if k == 5:
        gs = [synth.chung_lu(18, 38, 2.1, 11, 20, 40 + mode)]
    elif k == 4:
        gs = [synth.chung_lu(40, 110, 2.1, 26, 20, 34 + mode)]
    else:
        gs = [synth.chung_lu(70, 260, 2.1, 45, 20, 33 + mode), synth.regulatory(60, 200, 6, 2.1, 40, 10, 9)]
    jobs, want = [], []
    for g in gs:
        s, d = _by_degree(g.n, g.src, g.dst)
        for light, target in ((1 << 30, 1 << 30), (64, 64)):
            jobs.append(([(g.n, s, d)], dict(mode=mode, light=light, target=target)))
            want.append(oracle.count(g.n, g.src, g.dst, k).tolist())
    for (status, _, _, got), w, (_, kw) in zip(_enum_many(emu_bins["emu_enum_small"], emu_bins["dir"], k, jobs),
                                               want, jobs):
        assert status == 0
        assert got[0] == w, (k, kw)


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("mode", [0, 1, 2], ids=["count", "enumerate", "count_hashed"])
def test_enumeration_kernels_on_graph_sets(emu_bins, k, mode):
    """Several graphs in one launch pair (the batched form): units of every
    graph interleave in the warps' grabs, each graph's counts stay apart."""
    rng = np.random.default_rng(800 + 10 * k + mode)
    graphs = _enum_cases(rng, k, 4, {3: 24, 4: 14, 5: 10}[k])
    graphs.insert(2, (7, np.zeros(0, np.int64), np.zeros(0, np.int64)))
    want = [oracle.count(n, s, d, k).tolist() for n, s, d in graphs]
    jobs = [(graphs, dict(mode=mode, light=light, target=target, blocks=3, qcap=qcap))
            for light, target, qcap in SCHEDULES.values()]
    for (status, _, _, got), (_, kw) in zip(_enum_many(emu_bins["emu_enum"], emu_bins["dir"], k, jobs), jobs):
        assert status == 0
        assert got == want, (k, kw)


def _err_input():
    import re
    hdr = open(os.path.join(ROOT, "include", "acc_motif.h")).read()
    return int(re.search(r"#define\s+ACC_ERR_INPUT\s+\(?(-?\d+)\)?", hdr).group(1))


def _build_many(bins, jobs, binary="emu_build", guard_k=0, sparse=False):
    """Run the graph builder over [(graphs, relabel, num_sms)], graphs a list
    of (n, rowptr, col): per job, the two builds' records."""
    inps = []
    for graphs, relabel, num_sms in jobs:
        buf = struct.pack("<3q", int(relabel) + 2 * int(sparse) + 256 * guard_k, num_sms, len(graphs))
        buf += b"".join(struct.pack("<2q", n, len(cl)) for n, _, cl in graphs)
        for n, rp, cl in graphs:
            buf += np.asarray(rp, "<i8").tobytes() + np.asarray(cl, "<i4").tobytes()
        inps.append(buf)
    names = ("head", "label", "deg", "lo", "nptr", "nbr", "state", "occ", "clean", "src", "rev")
    res = []
    for o in _run_many(bins[binary], inps, True, bins["dir"]):
        raw = np.frombuffer(o, "<i8")
        recs, i = [], 0
        while i < len(raw):
            recs.append(raw[i + 1:i + 1 + raw[i]])
            i += 1 + raw[i]
        assert len(recs) == 2 * len(names)
        res.append([dict(zip(names, recs[j * len(names):(j + 1) * len(names)])) for j in range(2)])
    return res


def _check_build(r, graphs, relabel, sparse=False):
    """The builder's records against a plain construction: per graph, the
    renumbering orders vertices by descending (clamped) out- plus in-degree
    and is a permutation; the pair states, degrees, below-counts, neighbour
    lists (positions over the whole set), each entry's row (bit 31: a
    neighbour below the row's vertex) and occupancy bits are those of the
    renumbered graph (the sparse build keeps no pair states or bits); the
    reverse positions give, for the entry v -> x, the part of x's list above
    v (first position, length)."""
    status, _, nnz, maxdeg, zeroed = r["head"].tolist()
    assert status == 0 and zeroed == 1 and r["clean"][0] == 1
    voff, base = 0, 0
    st_all, nptr_all, deg_all, lo_all, nbr_all, occ_all = [], [np.zeros(1, np.int64)], [], [], [], []
    occ_w = max(1, ((((max([n for n, _, _ in graphs] + [0]) + 15) // 16) + 31) // 32 + 31) // 32)
    for n, rp, cl in graphs:
        src = np.repeat(np.arange(n), np.diff(np.asarray(rp, np.int64)))
        dst = np.asarray(cl, np.int64)
        new = np.arange(n)
        if relabel:
            lab = r["label"][voff:voff + n] - voff
            assert sorted(lab.tolist()) == list(range(n))
            key = np.minimum(np.bincount(src, minlength=n) + np.bincount(dst, minlength=n), max(n - 1, 0))
            inv = np.empty(n, np.int64)
            inv[lab] = np.arange(n)
            assert np.all(np.diff(key[inv]) <= 0)
            new = lab
        pitch, st, nptr, deg, lo, nbr = _gstar(n, new[src], new[dst])
        st_all.append(st)
        nptr_all.append(nptr[1:] + base)
        base += len(nbr)
        deg_all.append(deg)
        lo_all.append(lo)
        nbr_all.append(nbr)
        occ = np.zeros(n * occ_w, np.int64)
        for v in range(n):
            for wd in np.nonzero(st[v * pitch:(v + 1) * pitch])[0]:
                ch = int(wd) // 32
                occ[v * occ_w + ch // 32] |= 1 << (ch % 32)
        occ_all.append(occ)
        voff += n
    cat = lambda xs: np.concatenate(xs).astype(np.int64) if xs else np.zeros(0, np.int64)  # noqa: E731
    if sparse:
        assert len(r["state"]) == 0 and len(r["occ"]) == 0
    else:
        assert np.array_equal(r["state"], cat(st_all))
        assert np.array_equal(r["occ"], cat(occ_all))
    assert np.array_equal(r["deg"], cat(deg_all)) and np.array_equal(r["lo"], cat(lo_all))
    assert np.array_equal(r["nptr"], cat(nptr_all)) and np.array_equal(r["nbr"], cat(nbr_all))
    assert nnz == base and maxdeg == (int(max(d.max(initial=0) for d in deg_all)) if deg_all else 0)
    # row of each entry: global vertex, bit 31 for a neighbour below it
    nptr_cat, nbr_cat = cat(nptr_all), cat(nbr_all)
    want_src = np.zeros(len(nbr_cat), np.int64)
    voff = 0
    for n, _, _ in graphs:
        for v in range(n):
            b, e = nptr_cat[voff + v], nptr_cat[voff + v + 1]
            want_src[b:e] = (voff + v) | np.where((nbr_cat[b:e] >> 2) < v, 1 << 31, 0)
        voff += n
    assert np.array_equal(r["src"], want_src)
    want_rev = np.zeros((len(nbr_cat), 2), np.int64)
    voff = 0
    for n, _, _ in graphs:
        for v in range(n):
            for p in range(nptr_cat[voff + v], nptr_cat[voff + v + 1]):
                x = voff + (int(nbr_cat[p]) >> 2)
                row = (nbr_cat[nptr_cat[x]:nptr_cat[x + 1]] >> 2).tolist()
                i = row.index(v)  # the lists are symmetric
                want_rev[p] = (nptr_cat[x] + i + 1, len(row) - i - 1)
        voff += n
    assert np.array_equal(r["rev"], want_rev.reshape(-1))


def _raw_csr(n, s, d, rng):
    """An out-CSR with the rows' arcs in random order (repeats kept)."""
    s, d = np.asarray(s, np.int64), np.asarray(d, np.int64)
    order = np.lexsort((rng.random(len(s)), s))
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(s, minlength=n), out=rp[1:])
    return n, rp, d[order].astype(np.int32)


@pytest.mark.parametrize("sparse", [False, True], ids=["dense", "sparse"])
@pytest.mark.parametrize("relabel", [False, True], ids=["as_given", "renumbered"])
def test_graph_builder_equals_plain_construction(emu_bins, relabel, sparse):
    """The whole builder (zeroing, renumbering, ingest, degree scan, fill,
    then the clear) on the host, built with 2048-vertex single-block limits:
    one small graph (one-block scan, shared-memory renumbering), and a set
    of 5270 vertices with two graphs over 2048 (tiled scan over two tiles,
    histogram renumbering), an empty graph and repeated and mutual arcs."""
    rng = np.random.default_rng(900 + relabel)
    n = 300
    s, d = random_digraph(rng, n, p=0.02, recip=0.3)
    small = [_raw_csr(n, s, d, rng)]
    big = []
    for n in (50, 2500, 0, 120, 2600):
        s, d = random_digraph(rng, n, p=min(0.1, 3.0 / max(n, 1)), recip=0.3) if n else ([], [])
        s, d = np.asarray(s, np.int64), np.asarray(d, np.int64)
        if len(s):  # repeat some arcs
            k = rng.integers(0, len(s), size=len(s) // 10)
            s, d = np.concatenate([s, s[k]]), np.concatenate([d, d[k]])
        big.append(_raw_csr(n, s, d, rng))
    jobs = [(small, relabel, 1), (big, relabel, 2)]
    if sparse:
        # rows longer than the warp sort's 2048 raw entries take the block
        # sort: a hub with 3000 out-arcs, 600 of them repeated, and 500 in-arcs
        rng2 = np.random.default_rng(950 + relabel)
        n = 4000
        outs = rng2.permutation(np.arange(1, n))[:3000]
        s = np.concatenate([np.zeros(3000 + 600, np.int64), rng2.permutation(np.arange(1, n))[:500]])
        d = np.concatenate([outs, outs[:600], np.zeros(500, np.int64)])
        jobs.append(([_raw_csr(n, s, d, rng)], relabel, 2))
    for (graphs, _, _), builds in zip(jobs, _build_many(emu_bins, jobs, sparse=sparse)):
        for r in builds:
            _check_build(r, graphs, relabel, sparse)


def test_graph_builder_reports_malformed_input(emu_bins):
    """Self-loops, targets out of range, rows out of order or outside the
    arcs, and arcs of a graph without vertices set ACC_ERR_INPUT; the clear
    still leaves the pair-state buffer all zero (the build runs under the
    address sanitizer, so nothing is read or written out of bounds either)."""
    err = _err_input()
    ok_rp, ok_col = np.array([0, 2, 3, 4], np.int64), np.array([1, 2, 2, 0], np.int32)
    bad = [
        (3, ok_rp, np.array([1, 2, 2, 2], np.int32)),   # self-loop 2 -> 2
        (3, ok_rp, np.array([1, 3, 2, 0], np.int32)),   # target n
        (3, ok_rp, np.array([1, -1, 2, 0], np.int32)),  # negative target
        (3, np.array([0, 3, 2, 4], np.int64), ok_col),  # rowptr decreasing
        (3, np.array([1, 2, 3, 4], np.int64), ok_col),  # rowptr[0] != 0
        (3, np.array([0, 2, 3, 3], np.int64), ok_col),  # rowptr[n] != m
        (3, np.array([0, 2, 3, 9], np.int64), ok_col),  # rowptr past m
    ]
    empty_with_arcs = (0, np.array([0], np.int64), np.array([0], np.int32))
    jobs = [([case], True, 1) for case in bad] + [([(3, ok_rp, ok_col), case], True, 1) for case in bad]
    jobs.append(([(3, ok_rp, ok_col), empty_with_arcs], False, 1))
    good = [(3, ok_rp, ok_col)]
    jobs.append((good, True, 1))
    for sparse in (False, True):
        res = _build_many(emu_bins, jobs, sparse=sparse)
        for (graphs, _, _), builds in zip(jobs[:-1], res[:-1]):
            for r in builds:
                assert r["head"][0] == err, graphs
                assert r["clean"][0] == 1
        for r in res[-1]:
            _check_build(r, good, True, sparse)


def test_count_bound_guard(emu_bins):
    """The degree scan's overflow guard, built with a count limit of 10^4, on
    one-block scans and on tiled scans (sets above this build's 2048-vertex
    single-block limit).  A set holding a graph whose exact count (oracle)
    exceeds the limit must be refused with ACC_ERR_OVERFLOW, since the guard
    is an upper bound; a set whose graphs have at most C(n, k) <= 10^4
    k-subsets must pass, by the bound's C(n, k) cap; a directed path passes
    too (its bound is sum d^2 / 2 ~ 2n at k = 5: every factor D - 1 is 1)."""
    overflow = -5
    star = (31, *out_star(30))           # N_5 = C(30, 4) = 27405
    k12 = (12, *complete_bidirected(12))  # C(12, 4) = 495, C(12, 5) = 792
    rng = np.random.default_rng(77)
    cases = [([star], 5, True), ([k12], 4, False), ([k12], 5, False),
             ([(2000, *directed_path(2000))], 5, False),
             ([(2500, *directed_path(2500)), star], 5, True),
             ([k12] * 200, 4, False), ([k12] * 200 + [star], 5, True)]
    for graphs, k, refused in cases:
        exact = [int(oracle.count(n, s, d, k).sum()) for n, s, d in graphs]
        if refused:
            assert max(exact) > 10000
        jobs = [([_raw_csr(n, s, d, rng) for n, s, d in graphs], True, 2)]
        (builds,) = _build_many(emu_bins, jobs, binary="emu_build_guard", guard_k=k)
        for r in builds:
            assert r["head"][0] == (overflow if refused else 0), (k, [g[0] for g in graphs])


def _sv_to_canonical(k):
    """Canonical code of every state-vector layout code: field f_t (slots
    t = k-1 in the lowest bits up to t = 1) holds state(w_i, w_t) at bits
    2i, 2i+1 for i < t; state bit 0 is the arc w_i -> w_t, bit 1 the arc
    w_t -> w_i; the arc from slot i to slot j is canonical bit
    i (k-1) + j - [j > i]."""
    cp = np.arange(1 << (k * (k - 1)), dtype=np.int64)
    c = np.zeros_like(cp)
    off = 0
    bit = lambda i, j: i * (k - 1) + j - (1 if j > i else 0)  # noqa: E731
    for t in range(k - 1, 0, -1):
        for i in range(t):
            st = (cp >> (off + 2 * i)) & 3
            c |= (st & 1) << bit(i, t)
            c |= (st >> 1) << bit(t, i)
        off += 2 * t
    return c


@pytest.mark.parametrize("k", [3, 4, 5])
def test_table_builder_equals_oracle_table(emu_bins, k):
    """The device table builder (canonical code per adjacency code, class
    ranks, the table and its kernel layout) run on the host: the table and
    the class codes equal the oracle's, the relayout permutes it as the
    enumeration kernels read it."""
    raw = _run(emu_bins["emu_lut"], struct.pack("<q", k), True, emu_bins["dir"])
    ncodes = 1 << (k * (k - 1))
    rc = struct.unpack("<q", raw[:8])[0]
    lut = np.frombuffer(raw[8:8 + 2 * ncodes], "<i2")
    lut_sv = np.frombuffer(raw[8 + 2 * ncodes:8 + 4 * ncodes], "<i2")
    cc = np.frombuffer(raw[8 + 4 * ncodes:], "<u4")
    assert rc == 4  # four launches
    cls, codes = oracle.table(k)
    assert np.array_equal(lut, np.asarray(cls, np.int16))
    assert np.array_equal(cc, np.asarray(codes, np.uint32))
    assert np.array_equal(lut_sv, lut[_sv_to_canonical(k)])


def test_zscore_kernel_equals_oracle_bitwise(emu_bins):
    """Z-scores of groups of counts (real graph first, then its copies) from
    the device kernel's source equal the oracle's bit for bit, NaN where the
    copies' counts do not vary."""
    rng = np.random.default_rng(950)
    groups, size, K = 5, 40, 13
    counts = rng.integers(0, 1 << 40, size=(groups, size, K), dtype=np.int64)
    counts[1, :, 3] = 77                       # no spread: NaN
    counts[2, 1:, 5] = 9                       # no spread among the copies
    counts[3, :, :] = rng.integers(0, 3, size=(size, K))  # small integers
    buf = struct.pack("<3q", groups, size, K) + counts.astype("<i8").tobytes()
    raw = _run(emu_bins["emu_z"], buf, True, emu_bins["dir"])
    assert struct.unpack("<q", raw[:8])[0] == 1
    z = np.frombuffer(raw[8:], "<f8").reshape(groups, K)
    for g in range(groups):
        want = oracle.zscores(counts[g, 0], counts[g, 1:])
        assert np.array_equal(z[g], want, equal_nan=True), g  # exact values, NaN in the same places
    assert np.isnan(z[1, 3]) and np.isnan(z[2, 5])


LIB_SCENARIOS = ("modes", "repeats", "host_and_errors", "batch", "significance", "captured_pipeline", "server",
                 "tables", "injected_failures", "misc_api", "fuzz")
# (scenario, EMU_SCHED, EMU_DEFER): the scenarios that run every kernel,
# again with the lanes resumed and the blocks run in reverse and in
# pseudo-random orders, and with the device's work deferred until the host
# waits for it
LIB_RUNS = [(s, 0, 0) for s in LIB_SCENARIOS] + \
    [("modes", 1, 0), ("modes", 7777, 0), ("batch", 1, 0), ("batch", 4242, 0), ("captured_pipeline", 1, 0),
     ("captured_pipeline", 31337, 0), ("server", 99, 0), ("fuzz", 5150, 0)] + \
    [(s, 0, 1) for s in ("modes", "repeats", "host_and_errors", "batch", "significance", "captured_pipeline",
                         "server", "misc_api", "fuzz")]


@pytest.fixture(scope="session")
def emu_lib_results(tmp_path_factory):
    """Build the whole library for the host (every CUDA source with its
    launches rewritten, the shim and the stand-in runtime; address-sanitized
    with exact-size device allocations where the compiler can) as one shared
    library, then run every scenario of tests/emu/lib_scenarios.py against it
    in child processes, one per core at most: {(scenario, schedule): (exit
    status, output)}."""
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("emulib")
    units = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith(".cu"):
            src = '#include "shim.h"\n' + _launches_to_calls(open(os.path.join(CSRC, name)).read())
            open(out / (name[:-3] + ".cpp"), "w").write(src)
            units.append(str(out / (name[:-3] + ".cpp")))
    units.append(os.path.join(EMU, "emu_rt.cpp"))
    # under the address sanitizer when the compiler has it, with every device
    # allocation exactly its requested size: any access past a buffer fails
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    # (64 KiB lane stacks: the sanitizer clears a lane's whole stack shadow
    # at every switch)
    san = ["-fsanitize=address", "-DEMU_EXACT_ALLOC", "-DEMU_LANE_STACK=65536"] \
        if os.path.isabs(asan) and os.path.exists(asan) else []
    procs = []
    for i, u in enumerate(units):
        # (every count-mode set builds the reverse positions, however small)
        cmd = ["g++", "-std=c++20", "-O1", "-fPIC", "-pthread", "-w", *san, "-DACC_REV_MIN_ARCS=0", "-I", EMU, "-I",
               os.path.join(EMU, "fake"), "-I", CSRC, "-c", u, "-o", str(out / ("u%d.o" % i))]
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for pr in procs:
        _, err = pr.communicate()
        assert pr.returncode == 0, err[-3000:]
    so = str(out / "libacc_emu.so")
    r = subprocess.run(["g++", "-shared", "-pthread", *san[:1], "-o", so] +
                       [str(out / ("u%d.o" % i)) for i in range(len(units))], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ)
    if san:  # the interpreter is not instrumented: load the runtime first
        env["LD_PRELOAD"] = asan
        env["ASAN_OPTIONS"] = "detect_leaks=0"
    width = _width()
    results, running, todo = {}, [], list(LIB_RUNS)
    while todo or running:
        while todo and len(running) < width:
            name = todo.pop(0)
            env["EMU_SCHED"] = str(name[1])
            env["EMU_DEFER"] = str(name[2])
            pr = subprocess.Popen([sys.executable, os.path.join(EMU, "lib_scenarios.py"), so, name[0]], cwd=ROOT,
                                  env=dict(env), stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
            running.append((name, pr))
        name, pr = running.pop(0)
        try:
            so_out, _ = pr.communicate(timeout=900)
        except subprocess.TimeoutExpired:
            pr.kill()
            so_out, _ = pr.communicate()
        results[name] = (pr.returncode, so_out)
    return results


@pytest.mark.parametrize("scenario", LIB_RUNS,
                         ids=lambda r: r[0] + ("-sched%d" % r[1] if r[1] else "") + ("-deferred" if r[2] else ""))
def test_library_on_the_host(emu_lib_results, scenario):
    """The library's C ABI end to end on the host: counts in every mode, the
    launch-graph replay of repeated counts, the host-buffer entry point and
    argument errors, batches and the autotuner, randomisation and Z-scores,
    the significance step captured by the caller and replayed, the request
    server, and the class tables, each against the oracle; the scenarios
    that run every kernel also under other lane and block orders (a race
    check: every order is a valid GPU schedule)."""
    rc, output = emu_lib_results[scenario]
    assert rc == 0, output[-3000:]
