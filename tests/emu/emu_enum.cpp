// Runs the enumeration kernels (source extracted from csrc/enum.cu into
// enum_kernels.inc, the class-table relayout from csrc/lut.cu into
// relayout.inc) on the host over a G* build given as input, the way the
// library launches them: phase 1 (light units whole, heavy units queued),
// then phase 2 (the queue drained).  Input: k n pitch nnz maxdeg mode light
// target blocks queue_cap (int64 each), state[n * pitch], nptr[n + 1],
// deg[n], lo[n], nbr[nnz] and the canonical code -> class table
// (2^(k(k-1)) int16).  Output: status, chunks queued, entries scanned, the
// counts.  Blocks run one warp each, one after another, so the kernels'
// shared memory is one static buffer.
#include "shim.h"
#include "common.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
alignas(16) static unsigned char emu_smem[1 << 18];
namespace acc {
namespace lutk {
#include "relayout.inc"
}  // namespace lutk
namespace en {
#include "enum_kernels.inc"
}  // namespace en
}  // namespace acc
using acc::EnumArgs;

template <class T> static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

template <int K, bool COUNT>
static void run(EnumArgs a, int blocks) {
    static_assert(acc::en::Layout<K>::total <= sizeof(emu_smem));
    run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 1>(a); });
    run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 2>(a); });
}

template <int K>
static void relayout(const int16_t *lut, int16_t *lut_sv) {
    // one thread per layout code; no collectives, so the host thread runs them
    blockDim.x = 256;
    for (uint32_t cp = 0; cp < (1u << (K * (K - 1))); cp++) {
        blockIdx.x = cp / 256;
        threadIdx.x = cp % 256;
        acc::lutk::k_relayout<K>(lut, lut_sv);
    }
}

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long h[10];
    if (!rd(f, h, 10)) return 2;
    const long long k = h[0], n = h[1], pitch = h[2], nnz = h[3], maxdeg = h[4], mode = h[5];
    const int blocks = (int)h[8];
    const int ncls = k == 3 ? 13 : (k == 4 ? 199 : 9364);
    const size_t ncode = (size_t)1 << (k * (k - 1));
    std::vector<uint32_t> st(n * pitch + 1);
    std::vector<long long> nptr(n + 1);
    std::vector<int> deg(n + 1), lo(n + 1);
    std::vector<uint32_t> nbr(nnz + 1);
    std::vector<int16_t> lut(ncode), lut_sv(ncode);
    if (!rd(f, st.data(), n * pitch) || !rd(f, nptr.data(), n + 1) || !rd(f, deg.data(), n) || !rd(f, lo.data(), n) ||
        !rd(f, nbr.data(), nnz) || !rd(f, lut.data(), ncode))
        return 2;
    fclose(f);
    if (k == 3) relayout<3>(lut.data(), lut_sv.data());
    else if (k == 4) relayout<4>(lut.data(), lut_sv.data());
    else relayout<5>(lut.data(), lut_sv.data());

    acc::GraphInfo info{};
    info.nnz = nnz;
    info.maxdeg = (int)maxdeg;
    // per-warp overflow lists as the host sizes them: 2 (n + 32) rounded up
    const long long spw = 2 * ((n + 32 + 31) & ~31LL);
    std::vector<uint32_t> scratch((size_t)spw * blocks * acc::kWarpsPerBlock + 1);
    std::vector<uint4> queue((size_t)h[9] + 1);
    std::vector<unsigned long long> counts(ncls, 0);
    int status = 0;

    EnumArgs a{};
    a.state = st.data();
    a.deg = deg.data();
    a.lo = lo.data();
    a.nptr = nptr.data();
    a.nbr = nbr.data();
    a.lut = lut_sv.data();
    a.gs.B = 1;
    a.gs.NV = n;
    a.gs.M = nnz / 2;
    a.gs.one.n = (int)n;
    a.gs.one.pitch = pitch;
    a.max_n = (int)n;
    a.info = &info;
    a.queue = queue.data();
    a.queue_cap = (unsigned long long)h[9];
    a.scratch = scratch.data();
    a.scratch_per_warp = spw;
    a.mode = (int)mode;
    a.light = h[6];
    a.target = h[7];
    a.counts = counts.data();
    a.status = &status;
    const bool count = mode == 0;
    if (n > 0) {
        if (k == 3) count ? run<3, true>(a, blocks) : run<3, false>(a, blocks);
        else if (k == 4) count ? run<4, true>(a, blocks) : run<4, false>(a, blocks);
        else count ? run<5, true>(a, blocks) : run<5, false>(a, blocks);
    }
    printf("%d %llu %llu", status, info.queue_tail, info.scanned);
    for (int i = 0; i < ncls; i++) printf(" %llu", counts[i]);
    printf("\n");
    return 0;
}
