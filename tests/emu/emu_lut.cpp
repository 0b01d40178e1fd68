// Runs the class-table builder (csrc/lut.cu: k_canon, k_rank_scan, k_finish,
// k_relayout through launch_build_lut, each launch turned into emu_launch;
// source in lut_all.inc) on the host for one k given on the command line's
// input file (int64 k).  Output: the launcher's return value, then the
// code -> class table and its state-vector relayout (int16 each, 2^(k(k-1))
// entries) and the class codes (uint32, one per class).
#include "shim.h"
#include "common.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
#include "lut_all.inc"

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long k = 0;
    if (fread(&k, 8, 1, f) != 1) return 2;
    fclose(f);
    const size_t ncodes = (size_t)1 << acc::code_bits((int)k);
    const int ncls = acc::num_classes((int)k);
    std::vector<uint32_t> canon(ncodes), class_code(ncls, 0xFFFFFFFFu);
    std::vector<int> rank((size_t)acc::rank_ints((int)k));
    std::vector<int16_t> lut(ncodes, 0x5555), lut_sv(ncodes, 0x5555);
    const long long rc = acc::launch_build_lut((int)k, canon.data(), rank.data(), lut.data(), class_code.data(),
                                               lut_sv.data(), nullptr);
    FILE *o = fopen(argv[2], "wb");
    fwrite(&rc, 8, 1, o);
    fwrite(lut.data(), 2, ncodes, o);
    fwrite(lut_sv.data(), 2, ncodes, o);
    fwrite(class_code.data(), 4, ncls, o);
    fclose(o);
    return 0;
}
