// Runs the Z-score path (csrc/batch.cu, kernel and launch_zscores, the launch
// turned into emu_launch; source in z_all.inc) on the host.  Input (int64):
// groups group_size K, then counts[groups][group_size][K].  Output: the
// launcher's return value (int64) and the groups x K Z-scores (double).
#include "shim.h"
#include "common.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
#include "z_all.inc"

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long h[3];
    if (fread(h, 8, 3, f) != 3) return 2;
    const size_t n = (size_t)(h[0] * h[1] * h[2]);
    std::vector<long long> counts(n + 1);
    if (fread(counts.data(), 8, n, f) != n) return 2;
    fclose(f);
    std::vector<double> z((size_t)(h[0] * h[2]) + 1, -1.0);
    const long long rc = acc::launch_zscores(counts.data(), (int)h[0], (int)h[1], (int)h[2], z.data(), nullptr);
    FILE *o = fopen(argv[2], "wb");
    fwrite(&rc, 8, 1, o);
    fwrite(z.data(), 8, (size_t)(h[0] * h[2]), o);
    fclose(o);
    return 0;
}
