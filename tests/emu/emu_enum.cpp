// Runs the enumeration kernels (source extracted from csrc/enum.cu into
// enum_kernels.inc, the class-table relayout from csrc/lut.cu into
// relayout.inc) on the host over the G* build of a set of B graphs given as
// input, the way the library launches them: phase 1 (light units whole,
// heavy units queued), then phase 2 (the queue drained).  Input (int64
// unless noted): k B mode (0 count, 1 enumerate, 2 count on hashed adjacency)
// light target blocks queue_cap, then n pitch nnz of
// each graph, then the set's arrays: state (the graphs' blocks one after
// another), nptr[NV + 1] (positions over the whole set), deg[NV], lo[NV]
// (int32), nbr (uint32, local ids) and the canonical code -> class table
// (2^(k(k-1)) int16).  Output: status, chunks queued, entries scanned, the
// B x classes counts.  Blocks run one warp each, one after another, so the
// kernels' shared memory is one static buffer.
#include "shim.h"
#include "common.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
alignas(16) static unsigned char emu_smem[1 << 18];
namespace acc {
namespace lutk {
#include "relayout.inc"
}  // namespace lutk
namespace en {
#include "enum_kernels.inc"
}  // namespace en
}  // namespace acc
using acc::EnumArgs;

template <class T> static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

template <int K, bool COUNT>
static void run(EnumArgs a, int blocks) {
    static_assert(acc::en::Layout<K>::total <= sizeof(emu_smem));
    // the instantiation the library launches: one graph or a set of several,
    // dense or hashed adjacency (count mode)
    if constexpr (COUNT) {
        if (a.nh) {
            if (a.gs.B > 1) {
                run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 1, true, true>(a); });
                run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 2, true, true>(a); });
            } else {
                run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 1, false, true>(a); });
                run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 2, false, true>(a); });
            }
            return;
        }
    }
    if (a.gs.B > 1) {
        run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 1, true, false>(a); });
        run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 2, true, false>(a); });
    } else {
        run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 1, false, false>(a); });
        run_warps(blocks, 32, [&] { acc::en::k_enum<K, COUNT, 2, false, false>(a); });
    }
}

template <int K>
static void relayout(const int16_t *lut, int16_t *lut_sv) {
    // one thread per layout code; no collectives, so the host thread runs them
    blockDim.x = 256;
    for (uint32_t cp = 0; cp < (1u << (K * (K - 1))); cp++) {
        blockIdx.x = cp / 256;
        threadIdx.x = cp % 256;
        acc::lutk::k_relayout<K>(lut, lut_sv);
    }
}

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long h[7];
    if (!rd(f, h, 7)) return 2;
    const long long k = h[0], B = h[1], mode = h[2];
    const int blocks = (int)h[5];
    const int ncls = k == 3 ? 13 : (k == 4 ? 199 : 9364);
    const size_t ncode = (size_t)1 << (k * (k - 1));
    std::vector<acc::GMeta> meta(B);
    long long NV = 0, words = 0, nnz = 0, max_n = 0;
    for (long long g = 0; g < B; g++) {
        long long d[3];
        if (!rd(f, d, 3)) return 2;
        meta[g] = acc::GMeta{};
        meta[g].n = (int)d[0];
        meta[g].pitch = d[1];
        meta[g].voff = (int)NV;
        meta[g].soff = words;
        NV += d[0];
        words += d[0] * d[1];
        nnz += d[2];
        max_n = std::max(max_n, d[0]);
    }
    std::vector<uint32_t> st(words + 1);
    std::vector<long long> nptr(NV + 1);
    std::vector<int> deg(NV + 1), lo(NV + 1), gid(NV + 1);
    std::vector<uint32_t> nbr(nnz + 1);
    std::vector<int16_t> lut(ncode), lut_sv(ncode);
    if (!rd(f, st.data(), words) || !rd(f, nptr.data(), NV + 1) || !rd(f, deg.data(), NV) || !rd(f, lo.data(), NV) ||
        !rd(f, nbr.data(), nnz) || !rd(f, lut.data(), ncode))
        return 2;
    fclose(f);
    for (long long g = 0; g < B; g++)
        for (int v = 0; v < meta[g].n; v++) gid[meta[g].voff + v] = (int)g;
    if (k == 3) relayout<3>(lut.data(), lut_sv.data());
    else if (k == 4) relayout<4>(lut.data(), lut_sv.data());
    else relayout<5>(lut.data(), lut_sv.data());

    acc::GraphInfo info{};
    info.nnz = nnz;
    info.maxdeg = 0;
    for (long long v = 0; v < NV; v++) info.maxdeg = std::max(info.maxdeg, deg[v]);
    // per-warp scratch as the host sizes it: two overflow lists of max_n + 32
    // entries rounded up, then the k = 5 count mode's collected part-B rows
    const long long spw = 2 * ((max_n + 32 + 31) & ~31LL) + 2 * acc::kPartBRows;
    std::vector<uint32_t> scratch((size_t)spw * blocks * acc::kWarpsPerBlock + 1);
    std::vector<uint4> queue((size_t)h[6] + 1);
    std::vector<unsigned long long> counts((size_t)B * ncls, 0);
    int status = 0;

    // row of each entry, bit 31 for a neighbour below the row's vertex (the
    // first lo[v] entries of a sorted row), as the neighbour-list fill writes it
    std::vector<uint32_t> src(nnz + 1);
    for (long long v = 0; v < NV; v++)
        for (long long p = nptr[v]; p < nptr[v + 1]; p++)
            src[p] = (uint32_t)v | (p - nptr[v] < lo[v] ? 0x80000000u : 0u);

    // mode 2: the count mode probing hashed adjacency tables, filled here the
    // way the device build fills them (bucket of the neighbour's hash, or the
    // next one with a free slot)
    std::vector<uint32_t> nh;
    if (mode == 2) {
        nh.assign((size_t)acc::kNhWords * (size_t)nnz + 8, 0u);
        for (long long v = 0; v < NV; v++) {
            const uint32_t lg = acc::nh_lg(deg[v]), mask = (1u << lg) - 1u;
            uint32_t *tab = nh.data() + (size_t)acc::kNhWords * (size_t)nptr[v];
            for (long long p = nptr[v]; p < nptr[v + 1]; p++) {
                uint32_t b = acc::nh_bucket(nbr[p] >> 2, lg);
                for (bool done = false; !done; b = (b + 1u) & mask)
                    for (int j = 0; j < 4 && !done; j++)
                        if (tab[4 * b + j] == 0u) {
                            tab[4 * b + j] = nbr[p];
                            done = true;
                        }
            }
        }
    }

    // count mode: the reverse position of each entry (the part of the
    // neighbour's sorted list above the row's vertex: first position,
    // length), as the library's build computes it
    std::vector<uint2> rev(nnz + 1);
    for (long long v = 0; v < NV; v++) {
        const int voff = meta[gid[v]].voff;
        const uint32_t key = (uint32_t)(v - voff) << 2;
        for (long long p = nptr[v]; p < nptr[v + 1]; p++) {
            const long long x = voff + (nbr[p] >> 2);
            const long long i =
                std::lower_bound(nbr.begin() + nptr[x], nbr.begin() + nptr[x] + deg[x], key) - (nbr.begin() + nptr[x]);
            rev[p] = make_uint2((uint32_t)(nptr[x] + i + 1), (uint32_t)(deg[x] - i - 1));
        }
    }

    EnumArgs a{};
    a.src = src.data();
    a.rev = mode != 1 ? rev.data() : nullptr;
    a.nh = mode == 2 ? reinterpret_cast<const uint4 *>(nh.data()) : nullptr;
    a.state = st.data();
    a.deg = deg.data();
    a.lo = lo.data();
    a.nptr = nptr.data();
    a.nbr = nbr.data();
    a.lut = lut_sv.data();
    a.gs.B = (int)B;
    a.gs.NV = NV;
    a.gs.M = nnz / 2;
    if (B == 1) a.gs.one = meta[0];
    a.gs.many = meta.data();
    a.gs.gid = gid.data();
    a.max_n = (int)max_n;
    a.info = &info;
    a.queue = queue.data();
    a.queue_cap = (unsigned long long)h[6];
    a.scratch = scratch.data();
    a.scratch_per_warp = spw;
    a.mode = mode == 2 ? 0 : (int)mode;
    a.light = h[3];
    a.target = h[4];
    a.counts = counts.data();
    a.status = &status;
    const bool count = mode != 1;
    if (NV > 0) {
        if (k == 3) count ? run<3, true>(a, blocks) : run<3, false>(a, blocks);
        else if (k == 4) count ? run<4, true>(a, blocks) : run<4, false>(a, blocks);
        else count ? run<5, true>(a, blocks) : run<5, false>(a, blocks);
    }
    printf("%d %llu %llu", status, info.queue_tail, info.scanned);
    for (size_t i = 0; i < counts.size(); i++) printf(" %llu", counts[i]);
    printf("\n");
    return 0;
}
