// Runs the k = 3 or k = 5 formula kernels (source extracted from
// csrc/formula3.cu and csrc/formula5.cu into f3_kernels.inc / f5_kernels.inc)
// on the host over a G* build given as input: k n pitch nnz, state[n *
// pitch], nptr[n + 1], deg[n], lo[n], nbr[nnz], the code -> class table
// (2^(k(k-1)) int16) and the class codes.  Output: status and the counts.
#include "shim.h"
#include "common.cuh"
#include "formula.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
namespace acc {
namespace f3 {
#include "f3_kernels.inc"
}  // namespace f3
namespace f5 {
#include "f5_kernels.inc"
}  // namespace f5
}  // namespace acc
using acc::GSet;

template <class T> static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long k, n, pitch, nnz;
    if (!rd(f, &k, 1) || !rd(f, &n, 1) || !rd(f, &pitch, 1) || !rd(f, &nnz, 1)) return 2;
    const int ncls = k == 3 ? 13 : 9364;
    const size_t ncode = (size_t)1 << (k * (k - 1));
    std::vector<uint32_t> st(n * pitch + 1);
    std::vector<long long> nptr(n + 1);
    std::vector<int> deg(n + 1), lo(n + 1);
    std::vector<uint32_t> nbr(nnz + 1);
    std::vector<int16_t> lut(ncode);
    std::vector<uint32_t> cc(ncls);
    if (!rd(f, st.data(), n * pitch) || !rd(f, nptr.data(), n + 1) || !rd(f, deg.data(), n) || !rd(f, lo.data(), n) ||
        !rd(f, nbr.data(), nnz) || !rd(f, lut.data(), ncode) || !rd(f, cc.data(), ncls))
        return 2;
    fclose(f);
    GSet gs{};
    gs.B = 1;
    gs.NV = n;
    gs.M = nnz;
    gs.one.n = (int)n;
    gs.one.pitch = pitch;
    std::vector<unsigned long long> counts(ncls, 0);
    int status = 0;
    if (k == 3) {
        run_warps(3, 32, [&] {
            acc::f3::k_formula3(gs, st.data(), nptr.data(), deg.data(), lo.data(), nbr.data(), lut.data(),
                                counts.data(), &status);
        });
    } else {
        // the prefix of C(deg, 2) the one-block prefix kernel writes
        std::vector<long long> pre(n + 1, 0);
        for (long long v = 0; v < n; v++) pre[v + 1] = pre[v] + (long long)deg[v] * (deg[v] - 1) / 2;
        run_warps(3, 32, [&] {
            acc::f5::k_formula5(gs, st.data(), nptr.data(), deg.data(), nbr.data(), lut.data(), pre.data(),
                                counts.data(), &status);
        });
        blockDim.x = 1;
        gridDim.x = 1;
        threadIdx.x = 0;
        blockIdx.x = 0;
        acc::f5::k_formula5_divide(counts.data(), ncls, cc.data(), &status);
    }
    printf("%d", status);
    for (int i = 0; i < ncls; i++) printf(" %llu", counts[i]);
    printf("\n");
    return 0;
}
