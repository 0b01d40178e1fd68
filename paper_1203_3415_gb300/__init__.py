"""Python binding of libaccmotif.so, the GB300 connected-k-subgraph counter.

Argument marshalling only: every function below forwards to the C ABI entry
point of the same name (declared in include/acc_motif.h); all the work runs in
the library's CUDA kernels.  There is no CPU fallback: if the library is not
built, the first call raises ImportError.

The ``Counter`` class is a convenience around one context for callers holding
PyTorch CUDA tensors (PyTorch provides device memory and streams only).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaccmotif.so")

ACC_OK = 0
ACC_ERR_K = -1
ACC_ERR_INPUT = -2
ACC_ERR_NOMEM = -3
ACC_ERR_TIMEOUT = -4
ACC_ERR_OVERFLOW = -5
ACC_ERR_CUDA = -6
ACC_ERR_ARG = -7
ACC_ERR_TOO_LARGE = -8
ACC_ERR_INTERNAL = -9
ACC_MAX_N = 524288
ACC_MAX_N_SPARSE = 67108864
ACC_STATS_LEN = 7

NUM_CLASSES = {3: 13, 4: 199, 5: 9364}

# every symbol include/acc_motif.h declares, in declaration order
EXPORTS = (
    "acc_strerror", "acc_motif_num_classes", "acc_ctx_create", "acc_ctx_destroy", "acc_motif_prepare",
    "acc_motif_count", "acc_motif_count_host", "acc_motif_batch_prepare", "acc_motif_batch_run",
    "acc_motif_count_batch", "acc_motif_zscores", "acc_swap_randomise", "acc_ctx_set_randomise_memory", "acc_ctx_set_launch_graphs", "acc_motif_class_code", "acc_motif_classify_code",
    "acc_motif_copy_table", "acc_motif_last_stats", "acc_ctx_set_timing", "acc_motif_last_timing",
    "acc_motif_build_table_static", "acc_ctx_set_mode", "acc_server_create", "acc_server_destroy", "acc_server_add_graph",
    "acc_server_reserve", "acc_server_submit", "acc_server_progress", "acc_server_poll", "acc_server_drain",
    "acc_server_set_policy", "acc_ctx_set_schedule", "acc_ctx_get_schedule", "acc_motif_batch_autotune",
    "acc_ctx_set_adjacency",
)
ACC_REQ_QUEUED, ACC_REQ_RUNNING, ACC_REQ_DONE = 0, 1, 2
ACC_SERVE_FIFO, ACC_SERVE_SHORTEST = 0, 1
ACC_MODE_COUNT, ACC_MODE_ENUMERATE, ACC_MODE_FORMULA, ACC_MODE_AUTO = 0, 1, 2, 3
ACC_ADJ_AUTO, ACC_ADJ_DENSE, ACC_ADJ_HASH, ACC_ADJ_SPARSE = 0, 1, 2, 3
ACC_RAND_SWAP, ACC_RAND_MUTUAL = 0, 1


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run paper_1203_3415_gb300.build.build() "
                          f"(the counter has no CPU fallback)")
    return declare(ctypes.CDLL(LIB_PATH))


def declare(lib):
    """Set the argument and result types of every entry point of the C ABI
    on a loaded library handle; returns it."""
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.acc_strerror.argtypes = [ctypes.c_int]
    lib.acc_strerror.restype = ctypes.c_char_p
    lib.acc_motif_num_classes.argtypes = [ctypes.c_int]
    lib.acc_ctx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.acc_ctx_destroy.argtypes = [vp]
    lib.acc_ctx_destroy.restype = None
    lib.acc_motif_prepare.argtypes = [vp, ctypes.c_int, vp]
    lib.acc_motif_count.argtypes = [vp, vp, vp, i32, i64, ctypes.c_int, vp, vp, vp]
    lib.acc_motif_count_host.argtypes = [vp, vp, vp, i32, i64, ctypes.c_int, vp]
    lib.acc_motif_batch_prepare.argtypes = [vp, vp, i32, ctypes.c_int, vp]
    lib.acc_motif_batch_run.argtypes = [vp, vp, vp, vp]
    lib.acc_motif_count_batch.argtypes = [vp, vp, i32, ctypes.c_int, vp, vp, vp]
    lib.acc_motif_zscores.argtypes = [vp, i32, i32, ctypes.c_int, vp, vp]
    lib.acc_swap_randomise.argtypes = [vp, vp, i32, i32, i64, vp, ctypes.c_int, vp, vp, vp, vp]
    lib.acc_ctx_set_randomise_memory.argtypes = [vp, i64]
    lib.acc_ctx_set_launch_graphs.argtypes = [vp, ctypes.c_int]
    lib.acc_motif_class_code.argtypes = [vp, ctypes.c_int, i32, ctypes.POINTER(ctypes.c_uint32)]
    lib.acc_motif_classify_code.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(i32)]
    lib.acc_motif_copy_table.argtypes = [vp, ctypes.c_int, vp]
    lib.acc_motif_last_stats.argtypes = [vp, vp]
    lib.acc_ctx_set_timing.argtypes = [vp, ctypes.c_int]
    lib.acc_ctx_set_mode.argtypes = [vp, ctypes.c_int]
    lib.acc_ctx_set_adjacency.argtypes = [vp, ctypes.c_int]
    lib.acc_motif_last_timing.argtypes = [vp, vp]
    lib.acc_motif_build_table_static.argtypes = [ctypes.c_int, vp, vp, vp]
    lib.acc_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i32, i64]
    lib.acc_server_destroy.argtypes = [vp]
    lib.acc_server_destroy.restype = None
    lib.acc_server_add_graph.argtypes = [vp, vp, vp, i32, i64, ctypes.POINTER(i32)]
    lib.acc_server_reserve.argtypes = [vp]
    lib.acc_server_submit.argtypes = [vp, i32, ctypes.c_int, ctypes.POINTER(i64)]
    lib.acc_server_progress.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.acc_server_poll.argtypes = [vp, i64, ctypes.POINTER(i32), vp, ctypes.POINTER(ctypes.c_double)]
    lib.acc_server_drain.argtypes = [vp]
    lib.acc_server_set_policy.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    lib.acc_ctx_set_schedule.argtypes = [vp, i64, i64]
    lib.acc_ctx_get_schedule.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.acc_motif_batch_autotune.argtypes = [vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                             ctypes.POINTER(ctypes.c_float)]
    return lib


_lib_handle = None


def _L():
    """The loaded library; raises ImportError when it is not built."""
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = _load()
    return _lib_handle


class MotifError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {acc_strerror(code)} ({code})" if what else f"{acc_strerror(code)} ({code})")


def _check(rc: int, what: str) -> int:
    if rc != ACC_OK:
        raise MotifError(rc, what)
    return rc


# ---------------------------------------------------------------------------
# C ABI, one function per entry point (pointers as Python ints)
# ---------------------------------------------------------------------------

def acc_strerror(code: int) -> str:
    return _L().acc_strerror(code).decode()


def acc_motif_num_classes(k: int) -> int:
    return _L().acc_motif_num_classes(k)


def acc_ctx_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(_L().acc_ctx_create(ctypes.byref(h), device), "acc_ctx_create")
    return h.value


def acc_ctx_destroy(ctx: int) -> None:
    _L().acc_ctx_destroy(ctx)


def acc_motif_prepare(ctx: int, k: int, stream: int = 0) -> int:
    return _L().acc_motif_prepare(ctx, k, stream)


def acc_motif_count(ctx: int, d_rowptr: int, d_col: int, n: int, m: int, k: int, stream: int,
                    d_counts: int, d_status: int | None) -> int:
    return _L().acc_motif_count(ctx, d_rowptr, d_col, n, m, k, stream, d_counts, d_status)


def acc_motif_count_host(ctx: int, h_rowptr: int, h_col: int, n: int, m: int, k: int, h_counts: int) -> int:
    return _L().acc_motif_count_host(ctx, h_rowptr, h_col, n, m, k, h_counts)


class acc_graph_desc(ctypes.Structure):
    """One graph of a batch: device rowptr (int64[n+1]) and col (int32[m])."""
    _fields_ = [("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("m", ctypes.c_int64)]


def acc_motif_batch_prepare(ctx: int, h_graphs, B: int, k: int, stream: int) -> int:
    return _L().acc_motif_batch_prepare(ctx, ctypes.cast(h_graphs, ctypes.c_void_p), B, k, stream)


def acc_motif_batch_run(ctx: int, stream: int, d_counts: int, d_status: int | None) -> int:
    return _L().acc_motif_batch_run(ctx, stream, d_counts, d_status)


def acc_motif_count_batch(ctx: int, h_graphs, B: int, k: int, stream: int, d_counts: int,
                          d_status: int | None) -> int:
    return _L().acc_motif_count_batch(ctx, ctypes.cast(h_graphs, ctypes.c_void_p), B, k, stream, d_counts,
                                      d_status)


def acc_motif_zscores(d_counts: int, groups: int, group_size: int, k: int, stream: int, d_z: int) -> int:
    return _L().acc_motif_zscores(d_counts, groups, group_size, k, stream, d_z)


def acc_swap_randomise(ctx: int, h_graphs, G: int, R: int, attempts_per_arc: int, h_seeds, mode: int,
                       stream: int, d_out: int, d_accepted: int | None, d_status: int | None) -> int:
    return _L().acc_swap_randomise(ctx, ctypes.cast(h_graphs, ctypes.c_void_p), G, R, attempts_per_arc,
                                   ctypes.cast(h_seeds, ctypes.c_void_p), mode, stream, d_out, d_accepted,
                                   d_status)


def acc_ctx_set_launch_graphs(ctx: int, on: int) -> int:
    return _L().acc_ctx_set_launch_graphs(ctx, on)


def acc_ctx_set_randomise_memory(ctx: int, nbytes: int) -> int:
    return _L().acc_ctx_set_randomise_memory(ctx, nbytes)


def acc_motif_class_code(ctx: int, k: int, cls: int) -> int:
    out = ctypes.c_uint32()
    _check(_L().acc_motif_class_code(ctx, k, cls, ctypes.byref(out)), "acc_motif_class_code")
    return out.value


def acc_motif_classify_code(ctx: int, k: int, code: int) -> int:
    out = ctypes.c_int32()
    _check(_L().acc_motif_classify_code(ctx, k, code, ctypes.byref(out)), "acc_motif_classify_code")
    return out.value


def acc_motif_copy_table(ctx: int, k: int, h_table: int) -> int:
    return _L().acc_motif_copy_table(ctx, k, h_table)


def acc_motif_last_stats(ctx: int, h_stats: int) -> int:
    return _L().acc_motif_last_stats(ctx, h_stats)


def acc_ctx_set_mode(ctx: int, mode: int) -> int:
    return _L().acc_ctx_set_mode(ctx, mode)


def acc_ctx_set_adjacency(ctx: int, adjacency: int) -> int:
    return _L().acc_ctx_set_adjacency(ctx, adjacency)


def acc_ctx_set_timing(ctx: int, on: int) -> int:
    return _L().acc_ctx_set_timing(ctx, on)


def acc_motif_last_timing(ctx: int, h_ms: int) -> int:
    return _L().acc_motif_last_timing(ctx, h_ms)


def acc_motif_build_table_static(k: int, stream: int, d_table: int, d_class_code: int) -> int:
    """Table build that allocates nothing (working memory is a fixed array in
    the library); for callers that cannot allocate device memory."""
    return _L().acc_motif_build_table_static(k, stream, d_table, d_class_code)


def acc_server_create(device: int, slots: int, mem_budget_bytes: int) -> int:
    h = ctypes.c_void_p()
    _check(_L().acc_server_create(ctypes.byref(h), device, slots, mem_budget_bytes), "acc_server_create")
    return h.value


def acc_server_destroy(srv: int) -> None:
    _L().acc_server_destroy(srv)


def acc_server_add_graph(srv: int, d_rowptr: int, d_col: int, n: int, m: int) -> int:
    gid = ctypes.c_int32()
    _check(_L().acc_server_add_graph(srv, d_rowptr, d_col, n, m, ctypes.byref(gid)), "acc_server_add_graph")
    return gid.value


def acc_server_reserve(srv: int) -> int:
    return _L().acc_server_reserve(srv)


def acc_server_submit(srv: int, graph_id: int, k: int) -> int:
    rid = ctypes.c_int64()
    _check(_L().acc_server_submit(srv, graph_id, k, ctypes.byref(rid)), "acc_server_submit")
    return rid.value


def acc_server_progress(srv: int):
    run, q = ctypes.c_int32(), ctypes.c_int32()
    _check(_L().acc_server_progress(srv, ctypes.byref(run), ctypes.byref(q)), "acc_server_progress")
    return run.value, q.value


def acc_server_poll(srv: int, request_id: int, h_counts: int | None = None):
    """(state, latency_s) of a request; h_counts receives the counts when done."""
    st, lat = ctypes.c_int32(), ctypes.c_double()
    _check(_L().acc_server_poll(srv, request_id, ctypes.byref(st), h_counts, ctypes.byref(lat)), "acc_server_poll")
    return st.value, lat.value


def acc_server_drain(srv: int) -> int:
    return _L().acc_server_drain(srv)


def acc_server_set_policy(srv: int, policy: int, aging_s: float) -> int:
    return _L().acc_server_set_policy(srv, policy, aging_s)


def acc_ctx_set_schedule(ctx: int, light: int, target: int) -> int:
    return _L().acc_ctx_set_schedule(ctx, light, target)


def acc_ctx_get_schedule(ctx: int):
    """(light, target) in effect."""
    light, target = ctypes.c_int64(), ctypes.c_int64()
    _check(_L().acc_ctx_get_schedule(ctx, ctypes.byref(light), ctypes.byref(target)), "acc_ctx_get_schedule")
    return light.value, target.value


def acc_motif_batch_autotune(ctx: int, stream: int):
    """(light, target, ms) chosen for the prepared batch."""
    light, target, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_float()
    _check(_L().acc_motif_batch_autotune(ctx, stream, ctypes.byref(light), ctypes.byref(target), ctypes.byref(ms)),
           "acc_motif_batch_autotune")
    return light.value, target.value, ms.value


class Server:
    """Request server with continuous batching (see include/acc_motif.h)."""

    def __init__(self, device: int = 0, slots: int = 4, mem_budget_bytes: int = 64 << 30):
        self.srv = acc_server_create(device, slots, mem_budget_bytes)
        self._graphs = []  # keeps the device tensors alive
        self._k = {}

    def add_graph(self, rowptr, col, n: int) -> int:
        self._graphs.append((rowptr, col))
        return acc_server_add_graph(self.srv, rowptr.data_ptr(), col.data_ptr() if col.numel() else 0, n,
                                    col.numel())

    def reserve(self):
        _check(acc_server_reserve(self.srv), "acc_server_reserve")

    def set_policy(self, policy: int, aging_s: float = 1.0):
        """ACC_SERVE_SHORTEST (default) or ACC_SERVE_FIFO admission order."""
        _check(acc_server_set_policy(self.srv, policy, aging_s), "acc_server_set_policy")

    def submit(self, graph_id: int, k: int) -> int:
        rid = acc_server_submit(self.srv, graph_id, k)
        self._k[rid] = k
        return rid

    def progress(self):
        return acc_server_progress(self.srv)

    def poll(self, rid: int):
        """(state, counts or None, latency_s)."""
        import numpy as np
        out = np.zeros(NUM_CLASSES[self._k[rid]], dtype=np.int64)
        st, lat = acc_server_poll(self.srv, rid, out.ctypes.data)
        return st, (out if st == ACC_REQ_DONE else None), lat

    def drain(self):
        _check(acc_server_drain(self.srv), "acc_server_drain")

    def close(self):
        if self.srv:
            acc_server_destroy(self.srv)
            self.srv = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Convenience wrapper for PyTorch tensors
# ---------------------------------------------------------------------------

class Counter:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        self.mode = ACC_MODE_COUNT
        self.ctx = acc_ctx_create(device)

    def close(self):
        if self.ctx:
            acc_ctx_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prepare(self, k: int, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(acc_motif_prepare(self.ctx, k, s.cuda_stream), "acc_motif_prepare")

    def count(self, rowptr, col, n: int, k: int, counts=None, status=None, stream=None):
        """Counts of the graph given as CUDA tensors rowptr (int64[n+1]) and col
        (int32[m]).  Returns the int64 counts tensor.  With ``status`` (a CUDA
        int32 tensor of one element) the call does not wait; else it waits and
        raises MotifError on any error."""
        import torch
        assert rowptr.dtype == torch.int64 and col.dtype == torch.int32
        assert rowptr.is_cuda and col.is_cuda and rowptr.is_contiguous() and col.is_contiguous()
        s = stream if stream is not None else torch.cuda.current_stream(rowptr.device)
        if counts is None:
            counts = torch.empty(NUM_CLASSES[k], dtype=torch.int64, device=rowptr.device)
        rc = acc_motif_count(self.ctx, rowptr.data_ptr(), col.data_ptr() if col.numel() else 0, n,
                             col.numel(), k, s.cuda_stream, counts.data_ptr(),
                             status.data_ptr() if status is not None else None)
        _check(rc, "acc_motif_count")
        return counts

    def count_host(self, rowptr, col, n: int, k: int, counts=None):
        """Counts from host arrays (numpy or CPU tensors; pinned is fastest)."""
        import numpy as np
        rowptr_np = np.ascontiguousarray(rowptr, dtype=np.int64) if not hasattr(rowptr, "data_ptr") else None
        col_np = np.ascontiguousarray(col, dtype=np.int32) if not hasattr(col, "data_ptr") else None
        rp = rowptr_np.ctypes.data if rowptr_np is not None else rowptr.data_ptr()
        cp = col_np.ctypes.data if col_np is not None else col.data_ptr()
        m = len(col_np) if col_np is not None else col.numel()
        if counts is None:
            counts = np.zeros(NUM_CLASSES[k], dtype=np.int64)
        hp = counts.ctypes.data if isinstance(counts, np.ndarray) else counts.data_ptr()
        _check(acc_motif_count_host(self.ctx, rp, cp if m else 0, n, m, k, hp), "acc_motif_count_host")
        return counts

    def prepare_batch(self, graphs, k: int, stream=None):
        """Prepare a batch from a list of (rowptr, col, n) CUDA tensors; the
        tensors must stay alive until the last run_batch."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        descs = (acc_graph_desc * max(1, len(graphs)))()
        for i, (rowptr, col, n) in enumerate(graphs):
            assert rowptr.dtype == torch.int64 and col.dtype == torch.int32 and rowptr.is_cuda and col.is_cuda
            descs[i].rowptr = rowptr.data_ptr()
            descs[i].col = col.data_ptr() if col.numel() else 0
            descs[i].n = n
            descs[i].m = col.numel()
        self._batch = (len(graphs), k, descs)
        _check(acc_motif_batch_prepare(self.ctx, descs, len(graphs), k, s.cuda_stream), "acc_motif_batch_prepare")

    def run_batch(self, counts=None, status=None, stream=None):
        """Counts of the prepared batch as an int64 [B, num_classes] tensor."""
        import torch
        B, k, _ = self._batch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        if counts is None:
            counts = torch.empty((B, NUM_CLASSES[k]), dtype=torch.int64, device=f"cuda:{self.device}")
        _check(acc_motif_batch_run(self.ctx, s.cuda_stream, counts.data_ptr(),
                                   status.data_ptr() if status is not None else None), "acc_motif_batch_run")
        return counts

    def zscores(self, counts, groups: int, group_size: int, k: int, stream=None):
        """Z-scores [groups, num_classes] of counts [groups * group_size, num_classes]."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        z = torch.empty((groups, NUM_CLASSES[k]), dtype=torch.float64, device=counts.device)
        _check(acc_motif_zscores(counts.data_ptr(), groups, group_size, k, s.cuda_stream, z.data_ptr()),
               "acc_motif_zscores")
        return z

    def randomise(self, graphs, R: int, seeds, attempts_per_arc: int = 3, mode: int = ACC_RAND_SWAP,
                  out=None, accepted=None, status=None, stream=None):
        """R randomised copies of each graph of ``graphs`` ((rowptr, col, n)
        CUDA tensors) by acc_swap_randomise; copy r of graph g uses the stream
        seeded seeds[g] + r.  Returns (out, accepted): out is the int32 tensor
        of every copy's targets (graph g's copies from R * (m_0 + ... +
        m_{g-1}), copy r at that start + r * m_g), accepted int64 [G, R]."""
        import torch
        G = len(graphs)
        dev = graphs[0][0].device if G else torch.device("cuda", self.device)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        descs = (acc_graph_desc * max(1, G))()
        total = 0
        for i, (rowptr, col, n) in enumerate(graphs):
            assert rowptr.dtype == torch.int64 and col.dtype == torch.int32 and rowptr.is_cuda and col.is_cuda
            descs[i].rowptr = rowptr.data_ptr()
            descs[i].col = col.data_ptr() if col.numel() else 0
            descs[i].n = n
            descs[i].m = col.numel()
            total += col.numel()
        seeds_arr = (ctypes.c_uint64 * max(1, G))(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in seeds][:G])
        if out is None:
            out = torch.empty(max(1, R * total), dtype=torch.int32, device=dev)
        if accepted is None:
            accepted = torch.empty((G, R), dtype=torch.int64, device=dev)
        rc = acc_swap_randomise(self.ctx, descs, G, R, attempts_per_arc, seeds_arr, mode, s.cuda_stream,
                                out.data_ptr(), accepted.data_ptr() if accepted.numel() else None,
                                status.data_ptr() if status is not None else None)
        _check(rc, "acc_swap_randomise")
        return out, accepted

    def set_launch_graphs(self, on: bool):
        """Replay one CUDA graph for repeated counts (default on)."""
        _check(acc_ctx_set_launch_graphs(self.ctx, 1 if on else 0), "acc_ctx_set_launch_graphs")

    def set_randomise_memory(self, nbytes: int):
        """Bytes the copies' adjacency bitmaps may take (0: scan rows)."""
        _check(acc_ctx_set_randomise_memory(self.ctx, nbytes), "acc_ctx_set_randomise_memory")

    @staticmethod
    def copies(graphs, R: int, out):
        """The copies in ``out`` (from randomise) as [(rowptr, col, n), ...]
        per graph: R views sharing the graph's rowptr."""
        res, off = [], 0
        for rowptr, col, n in graphs:
            m = col.numel()
            res.append([(rowptr, out[off + r * m: off + (r + 1) * m], n) for r in range(R)])
            off += R * m
        return res

    def significance(self, graphs, k: int, R: int, seeds, attempts_per_arc: int = 3,
                     mode: int = ACC_RAND_SWAP, stream=None):
        """The significance step on the device: R randomised copies of each
        graph, the real graphs and their copies counted as one batch, and the
        Z-scores of each real graph against its copies.  Returns (counts
        int64 [G, 1 + R, num_classes], z float64 [G, num_classes], out)."""
        import torch
        G = len(graphs)
        out, _ = self.randomise(graphs, R, seeds, attempts_per_arc, mode, stream=stream)
        batch = []
        for g, cps in zip(graphs, self.copies(graphs, R, out)):
            batch.append(g)
            batch.extend(cps)
        self.prepare_batch(batch, k, stream=stream)
        counts = self.run_batch(stream=stream)
        z = self.zscores(counts, G, R + 1, k, stream=stream)
        return counts.view(G, R + 1, NUM_CLASSES[k]), z, out

    def table(self, k: int):
        import numpy as np
        out = np.empty(1 << (k * (k - 1)), dtype=np.int16)
        _check(acc_motif_copy_table(self.ctx, k, out.ctypes.data), "acc_motif_copy_table")
        return out

    def class_code(self, k: int, cls: int) -> int:
        return acc_motif_class_code(self.ctx, k, cls)

    def classify_code(self, k: int, code: int) -> int:
        return acc_motif_classify_code(self.ctx, k, code)

    def set_mode(self, mode: int):
        """ACC_MODE_COUNT (default) or ACC_MODE_ENUMERATE; same counts."""
        _check(acc_ctx_set_mode(self.ctx, mode), "acc_ctx_set_mode")
        self.mode = mode

    def set_adjacency(self, adjacency: int):
        """ACC_ADJ_AUTO (default), ACC_ADJ_DENSE, ACC_ADJ_HASH or ACC_ADJ_SPARSE; same counts."""
        _check(acc_ctx_set_adjacency(self.ctx, adjacency), "acc_ctx_set_adjacency")

    def set_schedule(self, light: int = 0, target: int = 0):
        """Enumeration work schedule (0: default); see acc_ctx_set_schedule."""
        _check(acc_ctx_set_schedule(self.ctx, light, target), "acc_ctx_set_schedule")

    def schedule(self):
        """(light, target) in effect."""
        return acc_ctx_get_schedule(self.ctx)

    def autotune_batch(self, stream=None):
        """Pick the fastest schedule for the prepared batch: (light, target, ms)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return acc_motif_batch_autotune(self.ctx, s.cuda_stream)

    def set_timing(self, on: bool = True):
        _check(acc_ctx_set_timing(self.ctx, 1 if on else 0), "acc_ctx_set_timing")

    def last_timing(self):
        """(build_ms, enumerate_ms, phase1_ms, phase2_ms) of the last count
        (timing must be on)."""
        import numpy as np
        out = np.zeros(4, dtype=np.float32)
        _check(acc_motif_last_timing(self.ctx, out.ctypes.data), "acc_motif_last_timing")
        return tuple(float(x) for x in out)

    def last_stats(self):
        import numpy as np
        out = np.zeros(ACC_STATS_LEN, dtype=np.int64)
        _check(acc_motif_last_stats(self.ctx, out.ctypes.data), "acc_motif_last_stats")
        return {"launches": int(out[0]), "units": int(out[1]), "chunks": int(out[2]),
                "undirected_edges": int(out[3]), "max_degree": int(out[4]), "blocks": int(out[5]),
                "scanned_entries": int(out[6])}
