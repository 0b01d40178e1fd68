// Host stand-in for the CUDA runtime, enough for the library's sources to
// compile and run on the host in the kernel emulation tests.  "Device"
// memory is host memory; every stream runs its work at once, in order,
// except while it is being captured, when kernel launches, copies, memsets
// and event records are kept (by value, as a launch keeps its arguments)
// and a launch of the graph made from them runs them in the same order.
// As on the device, a capture refuses the calls it cannot hold: waiting on
// the captured stream, and, while any capture in the global mode is open,
// allocating, freeing, synchronous copies and sets, and waits on anything.
// Events read the host clock.  For failure tests, emu_fail_* make the n-th
// allocation, kernel launch, copy or graph launch from now fail as the
// device would report it (a launch error is returned by the next cudaGetLastError; a
// failure inside a capture invalidates the capture).
#pragma once
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <functional>
#include <map>
#include <vector>

typedef int cudaError_t;
#define cudaSuccess 0
#define cudaErrorNotReady 600
#define cudaErrorInvalidValue 1
#define cudaErrorStreamCaptureUnsupported 900

struct EmuStream {
    bool capturing = false;
    bool global = false;   // captured in the global mode
    bool invalid = false;  // an operation failed while captured
    std::vector<std::function<void()>> rec;
    std::vector<std::function<void()>> pending;  // deferred mode: work not yet run
};
inline int emu_global_captures = 0;  // captures open in the global mode
inline long long emu_fail_malloc = 0, emu_fail_launch = 0, emu_fail_copy = 0, emu_fail_graph = 0;
inline cudaError_t emu_last_error = 0;  // returned (and cleared) by cudaGetLastError
// true when this call is the one a countdown selects
inline bool emu_trip(long long &countdown) { return countdown > 0 && --countdown == 0; }

#define EMU_REFUSE_IN_CAPTURE \
    if (emu_global_captures > 0) return cudaErrorStreamCaptureUnsupported
typedef EmuStream *cudaStream_t;
inline void emu_spoil(cudaStream_t s) {
    if (s && s->capturing) s->invalid = true;
}
struct EmuEvent {
    double t = 0.0;
    bool done = true;           // the work before its record has run
    EmuStream *s = nullptr;     // the stream it was recorded on
};
typedef EmuEvent *cudaEvent_t;
struct EmuGraph {
    std::vector<std::function<void()>> ops;
};
typedef EmuGraph *cudaGraph_t;
typedef EmuGraph *cudaGraphExec_t;

enum cudaMemcpyKind { cudaMemcpyHostToHost, cudaMemcpyHostToDevice, cudaMemcpyDeviceToHost, cudaMemcpyDeviceToDevice,
                      cudaMemcpyDefault };
enum cudaStreamCaptureMode { cudaStreamCaptureModeGlobal, cudaStreamCaptureModeThreadLocal,
                             cudaStreamCaptureModeRelaxed };
enum cudaDeviceAttr { cudaDevAttrMultiProcessorCount = 16 };
enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize = 8 };
#define cudaStreamNonBlocking 1
#define cudaEventDisableTiming 2

// streaming multiprocessors the emulated device reports
#ifndef EMU_NUM_SMS
#define EMU_NUM_SMS 2
#endif

// Deferred mode (environment variable EMU_DEFER=1): work waits in its
// stream's queue until something waits for that stream (a stream, event or
// device synchronisation, a blocking copy or set on the null stream, a
// free), as on the device, where it runs behind the host.  A host read of a
// result before such a wait then sees the buffer as it was.  Streams are
// run in the order they are waited on: the library orders work on several
// streams only through such waits.
inline bool emu_defer() {
    static const bool v = [] {
        const char *e = std::getenv("EMU_DEFER");
        return e && e[0] == '1';
    }();
    return v;
}
inline EmuStream emu_null_stream;  // the legacy stream's queue
inline std::vector<EmuStream *> &emu_streams() {
    static std::vector<EmuStream *> v;
    return v;
}
inline EmuStream *emu_queue(cudaStream_t s) { return s ? s : &emu_null_stream; }
inline void emu_flush(cudaStream_t s) {
    EmuStream *q = emu_queue(s);
    while (!q->pending.empty()) {
        std::vector<std::function<void()>> ops;
        ops.swap(q->pending);
        for (auto &op : ops) op();
    }
}
inline void emu_flush_all() {
    emu_flush(nullptr);
    for (size_t i = 0; i < emu_streams().size(); i++) emu_flush(emu_streams()[i]);
}

// run op now (deferred mode: queue it), or keep it when s is being captured
inline void emu_submit(cudaStream_t s, std::function<void()> op) {
    if (s && s->capturing) s->rec.push_back(std::move(op));
    else if (emu_defer()) emu_queue(s)->pending.push_back(std::move(op));
    else op();
}

inline cudaError_t cudaGetLastError() {
    const cudaError_t e = emu_last_error;
    emu_last_error = cudaSuccess;
    return e;
}
inline cudaError_t cudaPeekAtLastError() { return emu_last_error; }
inline const char *cudaGetErrorString(cudaError_t) { return "emulated"; }
template <class T> inline cudaError_t cudaFuncSetAttribute(T, cudaFuncAttribute, int) { return cudaSuccess; }
template <class T> inline cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int *b, T, int, size_t) {
    *b = 1;
    return cudaSuccess;
}
inline cudaError_t cudaSetDevice(int d) { return d == 0 ? cudaSuccess : cudaErrorInvalidValue; }
inline cudaError_t cudaGetDevice(int *d) {
    *d = 0;
    return cudaSuccess;
}
inline cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr, int) {
    *v = EMU_NUM_SMS;
    return cudaSuccess;
}
inline cudaError_t cudaDeviceSynchronize() {
    EMU_REFUSE_IN_CAPTURE;
    emu_flush_all();
    return cudaSuccess;
}
inline cudaError_t cudaMemGetInfo(size_t *free_b, size_t *total_b) {
    *free_b = size_t(8) << 30;
    *total_b = size_t(16) << 30;
    return cudaSuccess;
}

// Allocations are 256-byte aligned, as the device's; with EMU_EXACT_ALLOC
// (address-sanitizer builds) they have exactly the requested size, so a
// read or write past the end of a buffer is caught.
template <class T> inline cudaError_t cudaMalloc(T **p, size_t bytes) {
    EMU_REFUSE_IN_CAPTURE;
    if (emu_trip(emu_fail_malloc)) {
        *p = nullptr;
        return 2;  // out of memory
    }
#ifdef EMU_EXACT_ALLOC
    void *q = nullptr;
    if (posix_memalign(&q, 256, bytes ? bytes : 1)) q = nullptr;
    *p = static_cast<T *>(q);
#else
    *p = static_cast<T *>(std::aligned_alloc(256, (bytes + 255) / 256 * 256 + 256));
#endif
    return *p ? cudaSuccess : 2;
}
inline cudaError_t cudaFree(void *p) {
    EMU_REFUSE_IN_CAPTURE;
    emu_flush_all();  // a free waits for the device
    std::free(p);
    return cudaSuccess;
}
// pinned host allocations (start -> bytes): copies to and from them are
// asynchronous; copies to and from other (pageable) host memory wait, as on
// the device
inline std::map<uintptr_t, size_t> &emu_pinned() {
    static std::map<uintptr_t, size_t> m;
    return m;
}
inline bool emu_is_pinned(const void *p) {
    auto &m = emu_pinned();
    auto it = m.upper_bound((uintptr_t)p);
    if (it == m.begin()) return false;
    --it;
    return (uintptr_t)p < it->first + it->second;
}
template <class T> inline cudaError_t cudaMallocHost(T **p, size_t bytes) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) emu_pinned()[(uintptr_t)*p] = bytes ? bytes : 1;
    return e;
}
inline cudaError_t cudaFreeHost(void *p) {
    emu_pinned().erase((uintptr_t)p);
    return cudaFree(p);
}
template <class T> inline cudaError_t cudaGetSymbolAddress(void **p, T &sym) {
    *p = static_cast<void *>(&sym);
    return cudaSuccess;
}

inline cudaError_t cudaMemcpy(void *d, const void *s, size_t n, cudaMemcpyKind) {
    EMU_REFUSE_IN_CAPTURE;
    if (emu_trip(emu_fail_copy)) return cudaErrorInvalidValue;
    emu_flush(nullptr);  // blocking: after the null stream's work
    if (n) std::memmove(d, s, n);
    return cudaSuccess;
}
inline cudaError_t cudaMemcpyAsync(void *d, const void *s, size_t n, cudaMemcpyKind kind, cudaStream_t st) {
    if (emu_trip(emu_fail_copy)) {
        emu_spoil(st);
        return cudaErrorInvalidValue;
    }
    const bool pageable = (kind == cudaMemcpyHostToDevice && !emu_is_pinned(s)) ||
                          (kind == cudaMemcpyDeviceToHost && !emu_is_pinned(d));
    if (emu_defer() && pageable && !(st && st->capturing)) {
        emu_flush(st);  // a pageable copy waits for the stream and completes before returning
        if (n) std::memmove(d, s, n);
        return cudaSuccess;
    }
    emu_submit(st, [=] {
        if (n) std::memmove(d, s, n);
    });
    return cudaSuccess;
}
inline cudaError_t cudaMemset(void *p, int v, size_t n) {
    EMU_REFUSE_IN_CAPTURE;
    emu_flush(nullptr);
    std::memset(p, v, n);
    return cudaSuccess;
}
inline cudaError_t cudaMemsetAsync(void *p, int v, size_t n, cudaStream_t st) {
    if (emu_trip(emu_fail_copy)) {
        emu_spoil(st);
        return cudaErrorInvalidValue;
    }
    emu_submit(st, [=] { std::memset(p, v, n); });
    return cudaSuccess;
}

inline cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned) {
    *s = new EmuStream;
    emu_streams().push_back(*s);
    return cudaSuccess;
}
inline cudaError_t cudaStreamDestroy(cudaStream_t s) {
    emu_flush(s);  // its work still completes
    auto &v = emu_streams();
    for (size_t i = 0; i < v.size(); i++)
        if (v[i] == s) {
            v.erase(v.begin() + (long)i);
            break;
        }
    delete s;
    return cudaSuccess;
}
inline cudaError_t cudaStreamSynchronize(cudaStream_t s) {
    EMU_REFUSE_IN_CAPTURE;
    if (s && s->capturing) return cudaErrorStreamCaptureUnsupported;
    emu_flush(s);
    return cudaSuccess;
}
inline cudaError_t cudaStreamBeginCapture(cudaStream_t s, cudaStreamCaptureMode mode) {
    if (!s || s->capturing) return cudaErrorInvalidValue;
    s->capturing = true;
    s->global = mode != cudaStreamCaptureModeRelaxed;
    emu_global_captures += s->global;
    s->rec.clear();
    return cudaSuccess;
}
enum cudaStreamCaptureStatus { cudaStreamCaptureStatusNone, cudaStreamCaptureStatusActive,
                               cudaStreamCaptureStatusInvalidated };
inline cudaError_t cudaStreamIsCapturing(cudaStream_t s, cudaStreamCaptureStatus *st) {
    *st = s && s->capturing ? (s->invalid ? cudaStreamCaptureStatusInvalidated : cudaStreamCaptureStatusActive)
                            : cudaStreamCaptureStatusNone;
    return cudaSuccess;
}
inline cudaError_t cudaStreamEndCapture(cudaStream_t s, cudaGraph_t *g) {
    if (!s || !s->capturing) return cudaErrorInvalidValue;
    s->capturing = false;
    emu_global_captures -= s->global;
    s->global = false;
    if (s->invalid) {  // as the device: a capture that saw a failure gives no graph
        s->invalid = false;
        s->rec.clear();
        *g = nullptr;
        return 901;
    }
    *g = new EmuGraph{std::move(s->rec)};
    s->rec.clear();
    return cudaSuccess;
}
inline cudaError_t cudaGraphInstantiate(cudaGraphExec_t *e, cudaGraph_t g, unsigned long long) {
    *e = new EmuGraph(*g);
    return cudaSuccess;
}
inline long long emu_graph_launches = 0;  // graphs launched so far (read by the tests)
inline cudaError_t cudaGraphLaunch(cudaGraphExec_t e, cudaStream_t s) {
    if (emu_trip(emu_fail_graph)) return cudaErrorInvalidValue;
    emu_graph_launches++;
    for (auto &op : e->ops) emu_submit(s, op);
    return cudaSuccess;
}
inline cudaError_t cudaGraphDestroy(cudaGraph_t g) {
    delete g;
    return cudaSuccess;
}
inline cudaError_t cudaGraphExecDestroy(cudaGraphExec_t e) {
    delete e;
    return cudaSuccess;
}

inline double emu_now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
inline cudaError_t cudaEventCreate(cudaEvent_t *e) {
    *e = new EmuEvent;
    return cudaSuccess;
}
inline cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned) { return cudaEventCreate(e); }
inline cudaError_t cudaEventDestroy(cudaEvent_t e) {
    if (!e->done) emu_flush(e->s);  // its record still runs
    delete e;
    return cudaSuccess;
}
inline cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s) {
    if (!(s && s->capturing)) {
        e->done = false;
        e->s = s;
    }
    emu_submit(s, [=] {
        e->t = emu_now_ms();
        e->done = true;
    });
    return cudaSuccess;
}
// not ready the first time the work before it is still queued; the device
// runs that work meanwhile
inline cudaError_t cudaEventQuery(cudaEvent_t e) {
    if (e->done) return cudaSuccess;
    emu_flush(e->s);
    return cudaErrorNotReady;
}
inline cudaError_t cudaEventSynchronize(cudaEvent_t e) {
    EMU_REFUSE_IN_CAPTURE;
    if (!e->done) emu_flush(e->s);
    return cudaSuccess;
}
inline cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t a, cudaEvent_t b) {
    *ms = (float)(b->t - a->t);
    return cudaSuccess;
}
