// CPU stand-ins for the CUDA constructs the library's kernels use, so that a
// kernel's own source can run on the host.  Every GPU thread is a fiber
// (ucontext) on the calling host thread; every warp collective (shuffles,
// ballot, match, reduce, __syncwarp) is a barrier of the warp's 32 lanes and
// __syncthreads one of the block's threads, and a fiber runs until it
// reaches a barrier or returns, so lanes interleave only at collectives (a
// valid GPU schedule, the same on every run).  A lane that skips a
// collective its warp reaches leaves the others waiting with nothing left
// to run, which is reported as a hang at once.  A thread that returns
// leaves its block's barrier, as an exited GPU thread no longer holds
// __syncthreads back.  Blocks run one at a time, either as one warp after
// another (run_warps, for kernels whose blocks never synchronise across
// warps) or whole (run_blocks / emu_launch); shared arrays are static.
#pragma once
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <ucontext.h>
#include <vector>

#include <cuda_runtime.h>  // the host stand-in (streams, capture)

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __restrict__
#define __launch_bounds__(...)
#define __shared__ static
#define __align__(n) __attribute__((aligned(n)))
using std::max;
using std::min;

struct int4 { int x, y, z, w; };
struct uint2 { unsigned x, y; };
struct uint4 { unsigned x, y, z, w; };
inline uint2 make_uint2(unsigned a, unsigned b) { return {a, b}; }
inline int4 make_int4(int a, int b, int c, int d) { return {a, b, c, d}; }
inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return {a, b, c, d}; }
struct dim { unsigned x; };
extern thread_local dim threadIdx, blockIdx;
extern dim blockDim, gridDim;
// A barrier of a fixed group of lanes: a warp, or a block's threads.
struct Bar {
    int expected = 0, arrived = 0;
};
struct WarpCtx {
    Bar *bar;
    uint64_t slot[32];
};
extern thread_local WarpCtx *tw;
// the block barrier of the running lane (null under run_warps)
inline thread_local Bar *tblk = nullptr;

// One GPU thread: its fiber, ids and barriers, and what it waits on.
struct Lane {
    ucontext_t ctx;
    int tid = 0, bid = 0;
    WarpCtx *warp = nullptr;
    Bar *block = nullptr;
    int state = 0;  // 0 runnable, 1 waiting at wbar, 2 returned
    Bar *wbar = nullptr;
};
struct FiberSched {
    ucontext_t main;
    std::vector<Lane> lanes;
    std::vector<std::unique_ptr<char[]>> stacks;
    int cur = -1;
    std::function<void()> *job = nullptr;
};
inline FiberSched &fsched() {
    static FiberSched s;
    return s;
}
#ifndef EMU_LANE_STACK
#define EMU_LANE_STACK (256 * 1024)
#endif
constexpr size_t kLaneStack = EMU_LANE_STACK;  // bytes of stack per lane

// The order in which runnable lanes are resumed and blocks are run, from the
// environment variable EMU_SCHED: 0 (or unset) ascending, 1 descending,
// n >= 2 pseudo-random orders drawn from seed n.  Every order is a schedule
// the GPU may take, so no result may depend on it: running the same work
// under several orders is a race check.
inline unsigned long long emu_sched() {
    static const unsigned long long v = [] {
        const char *e = std::getenv("EMU_SCHED");
        return e ? std::strtoull(e, nullptr, 10) : 0ull;
    }();
    return v;
}
inline std::vector<int> emu_order(int n) {
    static unsigned long long draws = 0;
    std::vector<int> o(n);
    for (int i = 0; i < n; i++) o[i] = i;
    const unsigned long long mode = emu_sched();
    if (mode == 1) {
        std::reverse(o.begin(), o.end());
    } else if (mode >= 2) {
        unsigned long long x = mode * 0x9E3779B97F4A7C15ull + ++draws;
        for (int i = n - 1; i > 0; i--) {  // Fisher-Yates with SplitMix64 draws
            x += 0x9E3779B97F4A7C15ull;
            unsigned long long z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            std::swap(o[i], o[(int)(z % (unsigned long long)(i + 1))]);
        }
    }
    return o;
}

inline void bar_release(Bar *b) {
    b->arrived = 0;
    for (auto &l : fsched().lanes)
        if (l.state == 1 && l.wbar == b) {
            l.state = 0;
            l.wbar = nullptr;
        }
}
inline void bar_wait(Bar *b) {
    FiberSched &s = fsched();
    if (++b->arrived >= b->expected) {
        bar_release(b);
        return;
    }
    Lane &l = s.lanes[s.cur];
    l.state = 1;
    l.wbar = b;
    swapcontext(&l.ctx, &s.main);
}
// a lane that returns leaves the group
inline void bar_drop(Bar *b) {
    b->expected--;
    if (b->arrived > 0 && b->arrived >= b->expected) bar_release(b);
}
inline void lane_entry() {
    FiberSched &s = fsched();
    (*s.job)();
    Lane &l = s.lanes[s.cur];
    if (l.block) bar_drop(l.block);
    l.state = 2;  // returning resumes the scheduler (uc_link)
}
// Run job() once on each of n lanes set up by init(lane, i), switching to a
// lane only when the one running waits or returns; false when lanes are
// left waiting with none runnable (a collective some lane never reaches).
template <class Init> bool run_lanes(int n, std::function<void()> job, Init init) {
    FiberSched &s = fsched();
    while ((int)s.stacks.size() < n) s.stacks.emplace_back(new char[kLaneStack]);
    s.lanes.assign(n, Lane{});
    s.job = &job;
    for (int i = 0; i < n; i++) {
        Lane &l = s.lanes[i];
        init(l, i);
        getcontext(&l.ctx);
        l.ctx.uc_stack.ss_sp = s.stacks[i].get();
        l.ctx.uc_stack.ss_size = kLaneStack;
        l.ctx.uc_link = &s.main;
        makecontext(&l.ctx, lane_entry, 0);
    }
    bool ok = true;
    for (;;) {
        bool ran = false, left = false;
        for (int i : emu_order(n)) {
            Lane &l = s.lanes[i];
            if (l.state == 2) continue;
            left = true;
            if (l.state != 0) continue;
            s.cur = i;
            threadIdx.x = l.tid;
            blockIdx.x = l.bid;
            tw = l.warp;
            tblk = l.block;
            swapcontext(&s.main, &l.ctx);
            ran = true;
        }
        if (!left) break;
        if (!ran) {
            ok = false;
            break;
        }
    }
    s.cur = -1;
    tblk = nullptr;
    return ok;
}

template <class T> inline T __ldg(const T *p) { return *p; }
inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
inline int lane_() { return threadIdx.x & 31; }
inline void wsync() { bar_wait(tw->bar); }
inline void __syncwarp(unsigned = 0xffffffffu) { wsync(); }
inline void __syncthreads() {
    if (tblk) bar_wait(tblk);
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
inline unsigned __reduce_or_sync(unsigned, unsigned v) {
    wsync();
    tw->slot[lane_()] = (uint64_t)v;
    wsync();
    unsigned r = 0;
    for (int i = 0; i < 32; i++) r |= (unsigned)tw->slot[i];
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
inline float atomicAdd(float *p, float v) { return std::atomic_ref<float>(*p).fetch_add(v); }
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
inline unsigned atomicCAS(unsigned *p, unsigned c, unsigned v) {
    std::atomic_ref<unsigned>(*p).compare_exchange_strong(c, v);
    return c;
}
inline int atomicCAS(int *p, int c, int v) {
    std::atomic_ref<int>(*p).compare_exchange_strong(c, v);
    return c;
}

// Run f() as blocks x (threads / 32) warps, one warp at a time; exits the
// process when a warp's lanes wait at a collective some lane never reaches.
template <class F> bool run_warps(int blocks, int threads, F f) {
    blockDim.x = threads;
    gridDim.x = blocks;
    for (int b : emu_order(blocks))
        for (int w = 0; w < threads / 32; w++) {
            Bar bar;
            bar.expected = 32;
            WarpCtx ctx{};
            ctx.bar = &bar;
            const bool ok = run_lanes(32, [&] { f(); }, [&](Lane &l, int i) {
                l.tid = w * 32 + i;
                l.bid = b;
                l.warp = &ctx;
            });
            if (!ok) {
                fprintf(stderr, "warp %d of block %d did not finish\n", w, b);
                std::_Exit(3);
            }
        }
    return true;
}

// Run f() as `blocks` blocks of `threads` threads, one block at a time, all
// threads of a block together; exits the process on a hang as above.
template <class F> bool run_blocks(int blocks, int threads, F f) {
    blockDim.x = threads;
    gridDim.x = blocks;
    const int nw = (threads + 31) / 32;
    std::vector<Bar> wbar(nw);
    std::vector<WarpCtx> ctx(nw);
    for (int b : emu_order(blocks)) {
        Bar block_bar;
        block_bar.expected = threads;
        for (int w = 0; w < nw; w++) {
            wbar[w] = Bar{};
            wbar[w].expected = std::min(32, threads - 32 * w);
            ctx[w].bar = &wbar[w];
        }
        const bool ok = run_lanes(threads, [&] { f(); }, [&](Lane &l, int t) {
            l.tid = t;
            l.bid = b;
            l.warp = &ctx[t / 32];
            l.block = &block_bar;
        });
        if (!ok) {
            fprintf(stderr, "block %d did not finish\n", b);
            std::_Exit(3);
        }
    }
    return true;
}

// Stand-in for a kernel launch <<<grid, block, dynamic smem, stream>>> (kept
// by value while the stream is being captured): the dynamic shared memory is
// emu_dyn_smem (zeroed, at least `smem` bytes).
inline std::vector<uint64_t> emu_dyn_buf;
inline unsigned char *emu_dyn_smem = nullptr;
template <class F> void emu_launch(long long grid, long long block, size_t smem, cudaStream_t s, F f) {
    if (emu_trip(emu_fail_launch)) {  // the launch is refused: nothing runs
        emu_last_error = 98;
        emu_spoil(s);
        return;
    }
    emu_submit(s, [=] {
        emu_dyn_buf.assign(smem / 8 + 2, 0);
        emu_dyn_smem = reinterpret_cast<unsigned char *>(emu_dyn_buf.data());
        run_blocks((int)grid, (int)block, f);
    });
}
