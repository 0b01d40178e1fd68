// Runs the k = 3 or k = 5 formula path (csrc/formula3.cu or csrc/formula5.cu,
// kernels and launcher, each launch turned into emu_launch; source in
// f3_all.inc / f5_all.inc, chosen by EMU_K) on the host over a G* build given
// as input: k n pitch nnz, state[n * pitch], nptr[n + 1], deg[n], lo[n],
// nbr[nnz], the code -> class table (2^(k(k-1)) int16) and the class codes.
// Output: status and the counts.
#include "shim.h"
#include "common.cuh"
#include "formula.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
#if EMU_K == 3
#include "f3_all.inc"
#else
#include "f5_all.inc"
#endif
using acc::GSet;

template <class T> static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long k, n, pitch, nnz;
    if (!rd(f, &k, 1) || !rd(f, &n, 1) || !rd(f, &pitch, 1) || !rd(f, &nnz, 1)) return 2;
    if (k != EMU_K) return 2;
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
#if EMU_K == 3
    const int rc = acc::launch_formula3(gs, st.data(), nptr.data(), deg.data(), lo.data(), nbr.data(), lut.data(),
                                        counts.data(), &status, 1, nullptr);
#else
    std::vector<long long> pre(n + 1, -1);  // written by the launcher's prefix kernel
    const int rc = acc::launch_formula5(gs, st.data(), nptr.data(), deg.data(), nbr.data(), lut.data(), cc.data(),
                                        pre.data(), counts.data(), &status, 1, nullptr);
#endif
    if (rc < 0) return 4;
    printf("%d", status);
    for (int i = 0; i < ncls; i++) printf(" %llu", counts[i]);
    printf("\n");
    return 0;
}
