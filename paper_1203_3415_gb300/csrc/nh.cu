// Hashed adjacency: the neighbour entries of every vertex in a small
// open-addressing table, so that the count-mode probes of a large graph read
// a structure of 32 bytes per neighbour entry (L2-resident) instead of the
// dense n x n pair-state block.
//
// The paper tests adjacency "in O(1)" by hashing (its k=4 and k=5 complexity
// discussion); the dense block serves that role for graphs whose block stays
// in L2, and these tables for the rest.  Layout and hash: common.cuh
// (kNhWords, nh_lg, nh_bucket).
#include "common.cuh"

namespace acc {

namespace {

// Thread per neighbour entry: insert it into its row's table (atomicCAS on
// the slots of its bucket, then of the following buckets).  The row's table
// has 2^lg buckets of four slots and at most 2^lg <= 2 deg entries fit the
// kNhWords * deg words of the row's region.
__global__ void k_nh_fill(const long long *__restrict__ nptr, const int *__restrict__ deg,
                          const uint32_t *__restrict__ nbr, const uint32_t *__restrict__ src,
                          const GraphInfo *__restrict__ info, uint32_t *nh) {
    grid_dep_wait();
    const long long nnz = info->nnz;
    for (long long pos = blockIdx.x * (long long)blockDim.x + threadIdx.x; pos < nnz;
         pos += (long long)gridDim.x * blockDim.x) {
        const uint32_t p = src[pos] & 0x7FFFFFFFu;
        const uint32_t e = nbr[pos];
        const uint32_t lg = nh_lg(deg[p]);
        const uint32_t mask = (1u << lg) - 1u;
        uint32_t *tab = nh + (long long)kNhWords * nptr[p];
        uint32_t b = nh_bucket(e >> 2, lg);
        for (uint32_t tries = 0; tries <= mask; tries++, b = (b + 1u) & mask) {
            bool done = false;
            for (int j = 0; j < 4 && !done; j++) done = atomicCAS(tab + 4 * b + j, 0u, e) == 0u;
            if (done) break;
        }
    }
}

}  // namespace

int launch_nh_build(const long long *nptr, const int *deg, const uint32_t *nbr, const uint32_t *src,
                    const GraphInfo *info, long long max_entries, uint32_t *nh, int num_sms, cudaStream_t s) {
    if (max_entries <= 0) return 0;
    if (cudaMemsetAsync(nh, 0, (size_t)max_entries * kNhWords * sizeof(uint32_t), s) != cudaSuccess)
        return ACC_ERR_CUDA;
    long long grid = (max_entries + 255) / 256;
    if (grid > (long long)num_sms * 16) grid = (long long)num_sms * 16;
    launch_pdl(k_nh_fill, (int)grid, 256, 0, s, nptr, deg, nbr, src, info, nh);
    return cudaGetLastError() == cudaSuccess ? 1 : ACC_ERR_CUDA;
}

}  // namespace acc
