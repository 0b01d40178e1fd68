// Code -> class table, built on the device once per k.
//
// The paper classifies without isomorphism tests by hard-coding, per local
// structure, which histogram slot each configuration feeds (pattern
// matrices of the k=4 and k=5 sections, "precomputed" once and reused).
// Here the same role is played by one table over all 2^(k(k-1)) adjacency
// codes: code -> class of the digraph it describes, -1 if that digraph is not
// weakly connected.  A code's class is the rank (ascending) of its canonical
// code (minimum over the k! vertex orders) among the canonical codes of
// connected digraphs.  k = 5: 2^20 codes x 120 orders, a few ms on the GPU.
#include "common.cuh"

namespace acc {

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
// Codes per block of the canonicalisation (and of its block-local ranks); at
// most kRankBlock blocks (2^20 codes), so one block scans the block counts.
constexpr int kRankBlock = 1024;

// True when the launch just enqueued was accepted; a refused launch's error
// is cleared, and the caller launches nothing that would read its output.
bool launch_ok() {
    if (cudaPeekAtLastError() == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

template <int K>
struct Fact { static constexpr int v = K * Fact<K - 1>::v; };
template <>
struct Fact<0> { static constexpr int v = 1; };

// Thread per code: weak connectivity, then the minimum code over all vertex
// orders.  A code's bits for the arcs out of vertex i form one row of k-1
// bits (bit i (k-1) + t for the arc to the t-th other vertex), so the image
// of a code under order p is the OR over i of img[p][i][row i]: one table
// load per vertex instead of one per set bit.  Each block builds img (dest
// [p][b] is where order p sends code bit b) and also ranks the canonical
// codes among its own kRankBlock codes (rank_local) and writes how many it
// holds (block_count); k_rank_scan turns the block counts into offsets, so
// rank(c) = rank_local[c] + block_off[c / kRankBlock].
template <int K>
__global__ void __launch_bounds__(kRankBlock) k_canon(uint32_t *canon, int *rank_local, int *block_count) {
    constexpr int NB = K * (K - 1);
    constexpr int NP = Fact<K>::v;
    constexpr int R = 1 << (K - 1);  // values of one vertex's row
    constexpr uint32_t NCODES = 1u << NB;
    __shared__ uint8_t dest[NP][NB];
    __shared__ uint32_t img[NP][K][R];
    __shared__ int warp_off[kRankBlock / 32];
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        // decode order p from the factorial number system
        int pool[K], pi[K], r = p;
        for (int i = 0; i < K; i++) pool[i] = i;
        int left = K;
        for (int i = 0; i < K; i++) {
            int f = 1;
            for (int j = 2; j < left; j++) f *= j;
            const int q = r / f;
            r -= q * f;
            pi[i] = pool[q];
            for (int j = q; j < left - 1; j++) pool[j] = pool[j + 1];
            left--;
        }
        for (int i = 0; i < K; i++)
            for (int j = 0; j < K; j++)
                if (i != j) dest[p][code_bit(K, i, j)] = (uint8_t)code_bit(K, pi[i], pi[j]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NP * K * R; e += blockDim.x) {
        const int p = e / (K * R), i = (e / R) % K, row = e % R;
        uint32_t out = 0;
        for (int t = 0; t < K - 1; t++)
            if ((row >> t) & 1) out |= 1u << dest[p][i * (K - 1) + t];
        img[p][i][row] = out;
    }
    __syncthreads();
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t best = kNone;
    if (c < NCODES) {
        uint32_t adj[K];
        for (int i = 0; i < K; i++) adj[i] = 0;
        for (int i = 0; i < K; i++)
            for (int j = 0; j < K; j++)
                if (i != j && ((c >> code_bit(K, i, j)) & 1u)) {
                    adj[i] |= 1u << j;
                    adj[j] |= 1u << i;
                }
        uint32_t reach = 1;
        for (int it = 0; it < K; it++) {
            uint32_t nxt = reach;
            for (int i = 0; i < K; i++)
                if ((reach >> i) & 1u) nxt |= adj[i];
            reach = nxt;
        }
        if (reach == (1u << K) - 1u) {
            int row[K];
#pragma unroll
            for (int i = 0; i < K; i++) row[i] = (int)((c >> (i * (K - 1))) & (R - 1u));
            best = c;
            for (int p = 0; p < NP; p++) {
                uint32_t out = 0;
#pragma unroll
                for (int i = 0; i < K; i++) out |= img[p][i][row[i]];
                best = min(best, out);
            }
        }
        canon[c] = best;
    }
    // block-local exclusive rank of the canonical codes (ascending code)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned ball = __ballot_sync(kFull, best == c);
    if (lane == 0) warp_off[wid] = __popc(ball);
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        const int x = lane < nw ? warp_off[lane] : 0;
        int incl = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane < nw) warp_off[lane] = incl - x;
        if (lane == 31) block_count[blockIdx.x] = incl;
    }
    __syncthreads();
    if (c < NCODES) rank_local[c] = warp_off[wid] + __popc(ball & ((1u << lane) - 1u));
}

// One block: exclusive prefix sums of the nb <= kRankBlock block counts.
__global__ void __launch_bounds__(kRankBlock) k_rank_scan(const int *__restrict__ block_count, int nb,
                                                          int *block_off) {
    __shared__ int warp_sum[kRankBlock / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int x = t < nb ? block_count[t] : 0;
    int incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        const int ws = lane < nw ? warp_sum[lane] : 0;
        int wi = ws;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < nw) warp_sum[lane] = wi - ws;
    }
    __syncthreads();
    if (t < nb) block_off[t] = warp_sum[wid] + incl - x;
}

__global__ void k_finish(const uint32_t *__restrict__ canon, const int *__restrict__ rank_local,
                         const int *__restrict__ block_off, uint32_t ncodes, int ncls, int16_t *lut,
                         uint32_t *class_code) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncodes) return;
    const uint32_t cc = canon[c];
    // a rank at or above the class count would be a canonicalisation bug:
    // mark it (-2) for the host check instead of writing out of range
    const int r = cc == kNone ? -1 : rank_local[cc] + block_off[cc / kRankBlock];
    lut[c] = (int16_t)(r >= ncls ? -2 : r);
    if (cc == c && r < ncls) class_code[r] = c;
}

// canon, rank, finish: the class table and class codes of k into lut and
// class_code; rank holds rank_ints(k) ints.  Returns the launches made.
int launch_table(int k, uint32_t *canon, int *rank, int16_t *lut, uint32_t *class_code, cudaStream_t s) {
    const uint32_t ncodes = 1u << code_bits(k);
    const int nb = (int)((ncodes + kRankBlock - 1) / kRankBlock);
    int *block_count = rank + ncodes, *block_off = block_count + kRankBlock;
    switch (k) {
    case 3: k_canon<3><<<nb, kRankBlock, 0, s>>>(canon, rank, block_count); break;
    case 4: k_canon<4><<<nb, kRankBlock, 0, s>>>(canon, rank, block_count); break;
    case 5: k_canon<5><<<nb, kRankBlock, 0, s>>>(canon, rank, block_count); break;
    default: return ACC_ERR_K;
    }
    if (!launch_ok()) return ACC_ERR_CUDA;
    k_rank_scan<<<1, kRankBlock, 0, s>>>(block_count, nb, block_off);
    if (!launch_ok()) return ACC_ERR_CUDA;
    const int threads = 256;
    const int grid = (int)((ncodes + threads - 1) / threads);
    k_finish<<<grid, threads, 0, s>>>(canon, rank, block_off, ncodes, num_classes(k), lut, class_code);
    if (!launch_ok()) return ACC_ERR_CUDA;
    return 3;
}

// The same table indexed in the state-vector layout the enumeration kernels
// use: field f_t = sum_{i<t} state(w_i, w_t) << 2i for slots t = k-1 (lowest
// bits) down to 1 (highest), state bit 0 = arc w_i -> w_t, bit 1 = arc
// w_t -> w_i.  Thread per layout code: map it to the canonical code, copy
// that code's class.
template <int K>
__global__ void k_relayout(const int16_t *__restrict__ lut, int16_t *lut_sv) {
    const uint32_t cp = blockIdx.x * blockDim.x + threadIdx.x;
    if (cp >= (1u << (K * (K - 1)))) return;
    uint32_t c = 0;
    int off = 0;
    for (int t = K - 1; t >= 1; t--) {
        for (int i = 0; i < t; i++) {
            const uint32_t st = (cp >> (off + 2 * i)) & 3u;
            if (st & 1u) c |= 1u << code_bit(K, i, t);
            if (st & 2u) c |= 1u << code_bit(K, t, i);
        }
        off += 2 * t;
    }
    lut_sv[cp] = lut[c];
}

}  // namespace

int rank_ints(int k) { return (1 << code_bits(k)) + 2 * kRankBlock; }

int launch_build_lut(int k, uint32_t *canon, int *rank, int16_t *lut, uint32_t *class_code, int16_t *lut_sv,
                     cudaStream_t s) {
    const uint32_t ncodes = 1u << code_bits(k);
    const int rc = launch_table(k, canon, rank, lut, class_code, s);
    if (rc < 0) return rc;
    const int threads = 256;
    const int grid = (int)((ncodes + threads - 1) / threads);
    switch (k) {
    case 3: k_relayout<3><<<grid, threads, 0, s>>>(lut, lut_sv); break;
    case 4: k_relayout<4><<<grid, threads, 0, s>>>(lut, lut_sv); break;
    default: k_relayout<5><<<grid, threads, 0, s>>>(lut, lut_sv); break;
    }
    return cudaGetLastError() == cudaSuccess ? rc + 1 : ACC_ERR_CUDA;
}

}  // namespace acc

// ---------------------------------------------------------------------------
// Allocation-free table build.
//
// Some callers cannot allocate device memory at the point where they need the
// table: code running under a strict memory budget that hands out every byte
// up front, a framework that owns the device allocator, or a stream being
// captured into a CUDA graph (where a cudaMalloc would break the capture).
// acc_motif_build_table_static serves them: the caller passes the output
// buffers, and the working memory comes from the fixed array below, which is
// part of the library image (every GPU that loads the library holds these
// 8 MiB and 8 KiB until the process exits).
// ---------------------------------------------------------------------------

#include <mutex>

namespace acc {
namespace {

// Canonical code (first 2^20 words), then the block-local rank of every
// adjacency code of the largest supported k (5: 2^20 codes) followed by the
// per-block counts and offsets of the rank (2 kRankBlock words).
constexpr size_t kStaticCodes = size_t(1) << 20;
static __device__ __align__(256) uint32_t g_table_scratch[2 * kStaticCodes + 2 * kRankBlock];

constexpr int kMaxDevices = 64;
uint32_t *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_table_scratch on the current device (in host code the
// symbol name is only a stand-in, not an address).  It is looked up again on
// every call made outside a stream capture, so a module reloaded after a
// cudaDeviceReset is followed; a call made while `s` is being captured reuses
// the address an earlier call on the device found (a capture is no place to
// load a module), and fails if there was none.
int static_scratch(cudaStream_t s, uint32_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ACC_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (capturing) {
        if (!g_scratch_addr[dev]) return ACC_ERR_CUDA;
    } else {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_table_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ACC_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_addr[dev];
    return ACC_OK;
}

}  // namespace
}  // namespace acc

extern "C" ACC_API int acc_motif_build_table_static(int k, void *stream, int16_t *d_table,
                                                    uint32_t *d_class_code) {
    using namespace acc;
    if (k < 3 || k > 5) return ACC_ERR_K;
    if (!d_table || !d_class_code) return ACC_ERR_ARG;
    const uint32_t ncodes = 1u << code_bits(k);
    if (ncodes > kStaticCodes) return ACC_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *scratch = nullptr;
    const int rc = static_scratch(s, &scratch);
    if (rc) return rc;
    // every scratch word the kernels read is written earlier in the same
    // call, so nothing carries over from the previous call and nothing has to
    // be cleared
    uint32_t *canon = scratch;
    int *rank = reinterpret_cast<int *>(scratch + kStaticCodes);
    const int n = launch_table(k, canon, rank, d_table, d_class_code, s);
    return n < 0 ? n : ACC_OK;
}
