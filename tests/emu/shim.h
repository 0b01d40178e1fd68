// CPU stand-ins for the CUDA constructs the library's kernels use, so that a
// kernel's own source can run on the host: one host thread per lane (from a
// pool of persistent threads), every
// warp collective (shuffles, ballot, match, reduce, __syncwarp) a barrier of
// the 32 lane threads, and atomics on std::atomic_ref.  A lane that skips a
// collective its warp reaches leaves the others waiting at the barrier,
// which the driver reports as a hang.  Shared arrays are static: one block
// runs at a time, either one warp after another (run_warps, for kernels
// whose blocks never synchronise across warps) or all its threads at once
// (run_blocks / emu_launch, where __syncthreads is a barrier of the block's
// threads and a thread that returns leaves it, as an exited GPU thread no
// longer holds a block barrier back).
#pragma once
#include <algorithm>
#include <atomic>
#include <barrier>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <semaphore>
#include <thread>
#include <vector>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __restrict__
#define __launch_bounds__(...)
#define __shared__ static
using std::max;
using std::min;

struct int4 { int x, y, z, w; };
struct uint4 { unsigned x, y, z, w; };
inline int4 make_int4(int a, int b, int c, int d) { return {a, b, c, d}; }
inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return {a, b, c, d}; }
struct dim { unsigned x; };
extern thread_local dim threadIdx, blockIdx;
extern dim blockDim, gridDim;
struct WarpCtx { std::barrier<> *bar; uint64_t slot[32]; };
extern thread_local WarpCtx *tw;
// the block barrier of the running thread (null under run_warps)
inline thread_local std::barrier<> *tblk = nullptr;

template <class T> inline T __ldg(const T *p) { return *p; }
inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
inline int lane_() { return threadIdx.x & 31; }
inline void wsync() { tw->bar->arrive_and_wait(); }
inline void __syncwarp(unsigned = 0xffffffffu) { wsync(); }
inline void __syncthreads() {
    if (tblk) tblk->arrive_and_wait();
    else wsync();
}
template <class T> inline T exch(T v, int src) {
    wsync();
    tw->slot[lane_()] = (uint64_t)(int64_t)v;
    wsync();
    T r = (T)(int64_t)tw->slot[src & 31];
    wsync();
    return r;
}
template <class T> inline T __shfl_xor_sync(unsigned, T v, int d) { return exch(v, lane_() ^ d); }
template <class T> inline T __shfl_sync(unsigned, T v, int src) { return exch(v, src); }
template <class T> inline T __shfl_up_sync(unsigned, T v, int d) {
    T r = exch(v, lane_() >= d ? lane_() - d : lane_());
    return r;
}
inline unsigned __ballot_sync(unsigned, int p) {
    wsync();
    tw->slot[lane_()] = p ? 1 : 0;
    wsync();
    unsigned r = 0;
    for (int i = 0; i < 32; i++) r |= (tw->slot[i] ? 1u : 0u) << i;
    wsync();
    return r;
}
inline int __any_sync(unsigned m, int p) { return __ballot_sync(m, p) != 0; }
inline unsigned __match_any_sync(unsigned, int v) {
    wsync();
    tw->slot[lane_()] = (uint64_t)(uint32_t)v;
    wsync();
    unsigned r = 0;
    for (int i = 0; i < 32; i++) r |= (tw->slot[i] == (uint64_t)(uint32_t)v ? 1u : 0u) << i;
    wsync();
    return r;
}
inline int __reduce_max_sync(unsigned, int v) {
    wsync();
    tw->slot[lane_()] = (uint64_t)(int64_t)v;
    wsync();
    int r = (int)(int64_t)tw->slot[0];
    for (int i = 1; i < 32; i++) r = std::max(r, (int)(int64_t)tw->slot[i]);
    wsync();
    return r;
}
// IEEE double operations rounded to nearest, as the CUDA names define them;
// the host's own double arithmetic is that (compiled without contraction)
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dsub_rn(double a, double b) { return a - b; }
inline double __dmul_rn(double a, double b) { return a * b; }
inline double __ddiv_rn(double a, double b) { return a / b; }
inline double __dsqrt_rn(double a) { return std::sqrt(a); }
inline double __ll2double_rn(long long a) { return (double)a; }
inline int __ffs(int x) { return x ? __builtin_ctz((unsigned)x) + 1 : 0; }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
// position of the offset-th (1-based) set bit of mask at or above base
inline unsigned __fns(unsigned mask, unsigned base, int offset) {
    int c = 0;
    for (unsigned i = base; i < 32; i++)
        if ((mask >> i) & 1u && ++c == offset) return i;
    return 0xffffffffu;
}
inline unsigned atomicOr(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_or(v); }
inline unsigned atomicAnd(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_and(v); }
inline int atomicAdd(int *p, int v) { return std::atomic_ref<int>(*p).fetch_add(v); }
inline unsigned atomicAdd(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_add(v); }
inline unsigned atomicSub(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_sub(v); }
inline unsigned atomicExch(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).exchange(v); }
inline void __threadfence_block() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) {
    return std::atomic_ref<unsigned long long>(*p).fetch_add(v);
}
inline int atomicMax(int *p, int v) {
    std::atomic_ref<int> r(*p);
    int old = r.load();
    while (old < v && !r.compare_exchange_weak(old, v)) {
    }
    return old;
}
inline int atomicCAS(int *p, int c, int v) {
    std::atomic_ref<int>(*p).compare_exchange_strong(c, v);
    return c;
}

// Persistent host threads that play the lanes: run(n, job) has threads
// 0..n-1 call job(i) once each and waits for them; false when they have not
// all returned within the limit (a lane left a collective).  Threads are
// created once and reused, so a launch costs no thread creation.
struct LanePool {
    struct Worker {
        std::binary_semaphore go{0};
    };
    std::vector<std::unique_ptr<Worker>> ws;
    std::function<void(int)> job;
    std::mutex m;
    std::condition_variable fin;
    int remaining = 0;
    void loop(Worker *w, int id) {
        for (;;) {
            w->go.acquire();  // only the threads a run needs are woken
            job(id);
            std::lock_guard<std::mutex> lk(m);
            if (--remaining == 0) fin.notify_all();
        }
    }
    bool run(int n, std::function<void(int)> j, int limit_s) {
        while ((int)ws.size() < n) {
            ws.emplace_back(new Worker);
            Worker *w = ws.back().get();
            const int id = (int)ws.size() - 1;
            std::thread([this, w, id] { loop(w, id); }).detach();
        }
        job = std::move(j);
        {
            std::lock_guard<std::mutex> lk(m);
            remaining = n;
        }
        for (int i = 0; i < n; i++) ws[i]->go.release();
        std::unique_lock<std::mutex> lk(m);
        return fin.wait_for(lk, std::chrono::seconds(limit_s), [&] { return remaining == 0; });
    }
};
inline LanePool *lane_pool() {
    static LanePool *p = new LanePool;  // never destroyed: its threads outlive main
    return p;
}

// Run f() as blocks x (threads / 32) warps, one warp at a time; exits the
// process when a warp does not finish within the limit.
template <class F> bool run_warps(int blocks, int threads, F f, int limit_s = 120) {
    blockDim.x = threads;
    gridDim.x = blocks;
    for (int b = 0; b < blocks; b++)
        for (int w = 0; w < threads / 32; w++) {
            std::barrier<> bar(32);
            WarpCtx ctx;
            ctx.bar = &bar;
            const bool ok = lane_pool()->run(32, [&](int l) {
                threadIdx.x = w * 32 + l;
                blockIdx.x = b;
                tw = &ctx;
                tblk = nullptr;
                f();
            }, limit_s);
            if (!ok) {
                fprintf(stderr, "warp %d of block %d did not finish\n", w, b);
                std::_Exit(3);
            }
        }
    return true;
}

// Run f() as `blocks` blocks of `threads` threads, one block at a time, all
// threads of a block at once; exits the process when a block does not
// finish within the limit.
template <class F> bool run_blocks(int blocks, int threads, F f, int limit_s = 120) {
    blockDim.x = threads;
    gridDim.x = blocks;
    const int nw = (threads + 31) / 32;
    for (int b = 0; b < blocks; b++) {
        std::barrier<> block_bar(threads);
        std::vector<std::unique_ptr<std::barrier<>>> wbar;
        std::vector<WarpCtx> ctx(nw);
        for (int w = 0; w < nw; w++) {
            wbar.emplace_back(new std::barrier<>(std::min(32, threads - 32 * w)));
            ctx[w].bar = wbar.back().get();
        }
        const bool ok = lane_pool()->run(threads, [&](int t) {
            threadIdx.x = t;
            blockIdx.x = b;
            tw = &ctx[t / 32];
            tblk = &block_bar;
            f();
            block_bar.arrive_and_drop();
            tblk = nullptr;
        }, limit_s);
        if (!ok) {
            fprintf(stderr, "block %d did not finish\n", b);
            std::_Exit(3);
        }
    }
    return true;
}

// Stand-in for a kernel launch <<<grid, block, dynamic smem, stream>>>: the
// dynamic shared memory is emu_dyn_smem (zeroed, at least `smem` bytes).
inline std::vector<uint64_t> emu_dyn_buf;
inline unsigned char *emu_dyn_smem = nullptr;
template <class F> void emu_launch(long long grid, long long block, size_t smem, void *, F f) {
    emu_dyn_buf.assign(smem / 8 + 2, 0);
    emu_dyn_smem = reinterpret_cast<unsigned char *>(emu_dyn_buf.data());
    run_blocks((int)grid, (int)block, f);
}
