// The emulation's globals for the library built whole for the host (the
// harness binaries define their own), and a counter the tests read.
#include "shim.h"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;

// CUDA graphs launched so far (each replay of a captured launch sequence)
extern "C" long long emu_graph_launch_count() { return emu_graph_launches; }

// A caller's own stream and capture, as a framework capturing the library's
// calls into a CUDA graph does (global mode: every unsafe call refused).
extern "C" void *emu_stream_create() {
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    return s;
}
extern "C" int emu_capture_begin(void *s) {
    return cudaStreamBeginCapture(static_cast<cudaStream_t>(s), cudaStreamCaptureModeGlobal);
}
// ends the capture; the instantiated graph, or null when the capture failed
extern "C" void *emu_capture_end(void *s) {
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(static_cast<cudaStream_t>(s), &g) != cudaSuccess) return nullptr;
    cudaGraphExec_t e = nullptr;
    const bool ok = cudaGraphInstantiate(&e, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    return ok ? e : nullptr;
}
extern "C" int emu_graph_replay(void *e, void *s) {
    return cudaGraphLaunch(static_cast<cudaGraphExec_t>(e), static_cast<cudaStream_t>(s));
}

// Failure injection: the n-th allocation (kind 0), kernel launch (1), copy
// or set (2) or graph launch (3) from now fails; n = 0 clears it.
extern "C" void emu_inject(int kind, long long n) {
    (kind == 0 ? emu_fail_malloc : kind == 1 ? emu_fail_launch : kind == 2 ? emu_fail_copy : emu_fail_graph) = n;
}

// Wait for all queued work (deferred mode), as cudaDeviceSynchronize.
extern "C" void emu_device_synchronize() { emu_flush_all(); }
