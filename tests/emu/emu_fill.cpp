// Runs the neighbour-list fill (source extracted from csrc/graph.cu into
// fill_kernels.inc) on the host.  Input: n pitch occ_w rw, state[n * pitch],
// occ[n * occ_w], nptr[n + 1].  Output: the nptr[n] list entries.
#include "shim.h"
#include "common.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
namespace acc {
namespace {
#include "fill_kernels.inc"
}  // namespace
}  // namespace acc
using acc::GSet;

template <class T> static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long n, pitch, occ_w, rw;
    if (!rd(f, &n, 1) || !rd(f, &pitch, 1) || !rd(f, &occ_w, 1) || !rd(f, &rw, 1)) return 2;
    std::vector<uint32_t> st(n * pitch + 8);
    std::vector<uint32_t> occ(n * occ_w + 1);
    std::vector<long long> nptr(n + 1);
    if (!rd(f, st.data(), n * pitch) || !rd(f, occ.data(), n * occ_w) || !rd(f, nptr.data(), n + 1)) return 2;
    fclose(f);
    GSet gs{};
    gs.B = 1;
    gs.NV = n;
    gs.one.n = (int)n;
    gs.one.pitch = pitch;
    std::vector<uint32_t> out(nptr[n] + 1, 0xEEEEEEEEu);
    run_warps(2, 64, [&] {
        acc::k_fill(gs, st.data(), occ.data(), (int)occ_w, nptr.data(), out.data(), nullptr, (int)rw);
    });
    FILE *o = fopen(argv[2], "wb");
    fwrite(out.data(), 4, nptr[n], o);
    fclose(o);
    return 0;
}
