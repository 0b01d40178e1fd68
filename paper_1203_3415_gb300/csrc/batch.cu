// Significance of the class counts of a real graph against randomised
// copies (step iii of the motif pipeline, Implementation section: compare
// the frequencies with those of an ensemble of random graphs; the paper names
// the step but gives no formula).
//
// Z_c = (N_c(real) - mu_c) / sigma_c over the R randomisations of a group,
// mu_c = S1 / R with S1 the exact int64 sum, sigma_c the population deviation
// sqrt(sum_i (N_ic - mu_c)^2 / R) accumulated in increasing i, NaN when
// sigma_c = 0.  Every operation is an explicitly rounded IEEE double
// operation (no fused multiply-add), so the result is reproducible bit for
// bit by any IEEE double implementation that follows the same sequence.
#include <math.h>

#include "common.cuh"

namespace acc {

namespace {

// Thread per (group, class).  counts is [groups][group_size][K]; entry 0 of
// each group is the real graph, entries 1..group_size-1 its randomisations.
__global__ void k_zscores(const long long *__restrict__ counts, int groups, int group_size, int K, double *z) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)groups * K) return;
    const int g = (int)(idx / K), c = (int)(idx % K);
    const long long *base = counts + (long long)g * group_size * K;
    const int R = group_size - 1;
    long long s1 = 0;
    for (int i = 1; i <= R; i++) s1 += base[(long long)i * K + c];
    const double rr = (double)R;
    const double mu = __ddiv_rn(__ll2double_rn(s1), rr);
    double m2 = 0.0;
    for (int i = 1; i <= R; i++) {
        const double d = __dsub_rn(__ll2double_rn(base[(long long)i * K + c]), mu);
        m2 = __dadd_rn(m2, __dmul_rn(d, d));
    }
    const double sd = __dsqrt_rn(__ddiv_rn(m2, rr));
    const double num = __dsub_rn(__ll2double_rn(base[c]), mu);
    z[idx] = sd == 0.0 ? nan("") : __ddiv_rn(num, sd);
}

}  // namespace

int launch_zscores(const long long *counts, int groups, int group_size, int K, double *z, cudaStream_t s) {
    const long long total = (long long)groups * K;
    if (total == 0) return 0;
    const int threads = 256;
    k_zscores<<<(int)((total + threads - 1) / threads), threads, 0, s>>>(counts, groups, group_size, K, z);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

}  // namespace acc
