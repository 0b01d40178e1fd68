// Runs the randomiser (csrc/randomise.cu, kernels and launch_randomise, each
// launch turned into emu_launch; source in rand_all.inc) on the host.  Input:
// G R q mode use_bits, then per graph n m seed rowptr[n+1] col[m]; use_bits 0
// withholds the bitmaps (and the mutual mode's reverse positions), which
// selects the row-scan kernels.  Output: status, the copies, accepted counts.
#include "shim.h"
#include "common.cuh"
#include "randomise.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
#include "rand_all.inc"
using acc::RGraph;

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    int G, R, q, mode, use_bits;
    if (fread(&G, 4, 1, f) != 1 || fread(&R, 4, 1, f) != 1 || fread(&q, 4, 1, f) != 1 ||
        fread(&mode, 4, 1, f) != 1 || fread(&use_bits, 4, 1, f) != 1)
        return 2;
    std::vector<std::vector<long long>> rp(G);
    std::vector<std::vector<int>> cl(G);
    std::vector<RGraph> metas(G);
    long long M = 0, NV = 0, bwords = 0;
    for (int g = 0; g < G; g++) {
        int n;
        long long m;
        unsigned long long seed;
        if (fread(&n, 4, 1, f) != 1 || fread(&m, 8, 1, f) != 1 || fread(&seed, 8, 1, f) != 1) return 2;
        rp[g].resize(n + 1);
        cl[g].resize(m + 1);
        if (fread(rp[g].data(), 8, n + 1, f) != (size_t)(n + 1) || fread(cl[g].data(), 4, m, f) != (size_t)m) return 2;
        RGraph &rg = metas[g];
        memset(&rg, 0, sizeof(rg));
        rg.rowptr = rp[g].data();
        rg.col = cl[g].data();
        rg.m = m;
        rg.n = n;
        rg.moff = M;
        rg.ooff = M * R;
        rg.attempts = (long long)q * m;
        rg.seed = seed;
        rg.voff = (int)NV;
        rg.bw = (int)((((long long)n + 31) / 32 + 3) & ~3ll);
        rg.boff = bwords;
        M += m;
        NV += n;
        bwords += (long long)n * rg.bw * R;
    }
    fclose(f);
    std::vector<int4> rows(M + 1);
    std::vector<int> out(R * M + 1, -7), rpart(M + 1, -5), pts(R * M + 1, -6);
    std::vector<uint32_t> bits(bwords + 64, 0xdeadbeefu);
    std::vector<long long> accepted((size_t)G * R + 1, -1);
    int status = 0;
    const int rc = acc::launch_randomise(metas.data(), G, R, M, NV, mode, rows.data(), out.data(),
                                         use_bits ? bits.data() : nullptr, use_bits ? rpart.data() : nullptr,
                                         use_bits ? pts.data() : nullptr, accepted.data(), &status, 1, nullptr);
    if (rc < 0) return 4;
    FILE *o = fopen(argv[2], "wb");
    fwrite(&status, 4, 1, o);
    fwrite(out.data(), 4, R * M, o);
    fwrite(accepted.data(), 8, G * R, o);
    fclose(o);
    return 0;
}
