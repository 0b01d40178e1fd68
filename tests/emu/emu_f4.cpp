// Runs the k = 4 formula path (csrc/formula4.cu, kernels and launch_formula4,
// each launch turned into emu_launch; source in f4_all.inc) on the host over
// a G* build given as input: n pitch nnz,
// state[n * pitch], nptr[n + 1], deg[n], lo[n], nbr[nnz], the code -> class
// table (4096 int16) and the class codes (199 uint32).  Output: status and
// the 199 counts.
#include "shim.h"
#include "common.cuh"
#include "formula.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
#include "f4_all.inc"
using acc::GSet;
using acc::GraphInfo;

template <class T> static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long n, pitch, nnz;
    if (!rd(f, &n, 1) || !rd(f, &pitch, 1) || !rd(f, &nnz, 1)) return 2;
    std::vector<uint32_t> st(n * pitch + 1);
    std::vector<long long> nptr(n + 1);
    std::vector<int> deg(n + 1), lo(n + 1);
    std::vector<uint32_t> nbr(nnz + 1);
    std::vector<int16_t> lut(4096);
    std::vector<uint32_t> cc(199);
    if (!rd(f, st.data(), n * pitch) || !rd(f, nptr.data(), n + 1) || !rd(f, deg.data(), n) || !rd(f, lo.data(), n) ||
        !rd(f, nbr.data(), nnz) || !rd(f, lut.data(), 4096) || !rd(f, cc.data(), 199))
        return 2;
    fclose(f);
    GSet gs{};
    gs.B = 1;
    gs.NV = n;
    gs.M = nnz;
    gs.one.n = (int)n;
    gs.one.pitch = pitch;
    GraphInfo info{};
    info.nnz = nnz;
    std::vector<unsigned long long> counts(199, 0);
    int status = 0;
    const int rc = acc::launch_formula4(gs, st.data(), nptr.data(), deg.data(), lo.data(), nbr.data(), lut.data(),
                                        cc.data(), &info, counts.data(), &status, 1, nullptr);
    if (rc < 0) return 4;
    printf("%d", status);
    for (int i = 0; i < 199; i++) printf(" %llu", counts[i]);
    printf("\n");
    return 0;
}
