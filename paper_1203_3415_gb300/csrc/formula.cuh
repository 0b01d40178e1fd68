// Declarations of the formula paths (the paper's per-vertex, per-edge and
// per-triple set-size formulas for k = 3, 4, 5).
#pragma once

#include "common.cuh"

namespace acc {

// formula3.cu: k = 3 counts by the per-vertex formulas (one launch).
int launch_formula3(const GSet &gs, const uint32_t *state, const long long *nptr, const int *deg, const int *lo,
                    const uint32_t *nbr, const int16_t *lut, unsigned long long *counts, int *status, int num_sms,
                    cudaStream_t s);
// formula4.cu: k = 4 counts by the per-edge formulas, then the division by
// each class's multiplicity (two launches).
int launch_formula4(const GSet &gs, const uint32_t *state, const long long *nptr, const int *deg, const int *lo,
                    const uint32_t *nbr, const int16_t *lut, const uint32_t *class_code, const GraphInfo *info,
                    unsigned long long *counts, int *status, int num_sms, cudaStream_t s);
// formula5.cu: k = 5 counts by the per-triple formulas (pre: NV + 1 values of
// scratch), then the division by each class's multiplicity (three launches).
int launch_formula5(const GSet &gs, const uint32_t *state, const long long *nptr, const int *deg, const uint32_t *nbr,
                    const int16_t *lut, const uint32_t *class_code, long long *pre, unsigned long long *counts,
                    int *status, int num_sms, cudaStream_t s);
}  // namespace acc
