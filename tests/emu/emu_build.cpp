// Runs the graph builder (csrc/graph.cu, kernels and host launcher, with each
// launch turned into emu_launch; source in graph_kernels.inc) on the host
// over a set of B graphs given as input CSRs: relabel + 2 sparse + 256 k
// num_sms B (int64; sparse: the build without the dense block; k > 0 turns
// on the count-bound check for that k), then
// n m of each graph (int64), then each graph's rowptr[n + 1] (int64) and
// col[m] (int32).  The set is built twice: first over a pair-state buffer
// full of garbage (swept by the build's zeroing), then, after the builder's
// own clear, over the buffer it left clean.  Output per build, as records of
// int64 (length, values): status, launches, nnz, maxdeg and whether the
// counts were zeroed; label[NV]; deg[NV]; lo[NV]; nptr[NV + 1]; nbr[nnz];
// the state words; the occupancy words (both empty for the sparse build);
// after the clear, whether the state buffer is all zero; src[nnz]; the
// reverse positions (launch_rev_build) as first, length pairs[2 nnz].
#include "shim.h"
#include "common.cuh"
thread_local dim threadIdx, blockIdx;
dim blockDim, gridDim;
thread_local WarpCtx *tw;
#include "graph_kernels.inc"

template <class T> static bool rd(FILE *f, T *p, size_t n) { return n == 0 || fread(p, sizeof(T), n, f) == n; }

static FILE *out;

// one record: its length, then the values, int64 each
template <class T> static void put(const T *v, size_t n) {
    const long long len = (long long)n;
    fwrite(&len, 8, 1, out);
    for (size_t i = 0; i < n; i++) {
        const long long x = (long long)v[i];
        fwrite(&x, 8, 1, out);
    }
}

int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    long long h[3];
    if (!rd(f, h, 3)) return 2;
    const bool relabel = (h[0] & 1) != 0;
    const bool sparse = (h[0] & 2) != 0;
    const int guard_k = (int)(h[0] >> 8);
    const int num_sms = (int)h[1];
    const long long B = h[2];
    std::vector<long long> ns(B), ms(B);
    for (long long g = 0; g < B; g++)
        if (!rd(f, &ns[g], 1) || !rd(f, &ms[g], 1)) return 2;
    std::vector<std::vector<long long>> rowptr(B);
    std::vector<std::vector<int>> col(B);
    std::vector<acc::GMeta> meta(B);
    long long NV = 0, M = 0, words = 0;
    int max_n = 0;
    for (long long g = 0; g < B; g++) {
        rowptr[g].resize(ns[g] + 1);
        col[g].resize(ms[g]);  // exact sizes: a read past either is caught
        if (!rd(f, rowptr[g].data(), ns[g] + 1) || !rd(f, col[g].data(), ms[g])) return 2;
        acc::GMeta &mt = meta[g];
        mt = acc::GMeta{};
        mt.rowptr = rowptr[g].data();
        mt.col = col[g].data();
        mt.m = ms[g];
        mt.n = (int)ns[g];
        mt.pitch = acc::state_pitch(mt.n);
        mt.soff = words;
        mt.moff = M;
        mt.voff = (int)NV;
        words += ns[g] * mt.pitch;
        NV += ns[g];
        M += ms[g];
        max_n = std::max(max_n, mt.n);
    }
    fclose(f);
    out = fopen(argv[2], "wb");

    const int occ_w = acc::occ_words(max_n);
    std::vector<uint32_t> state(words + 4, 0xDEADBEEFu);
    std::vector<int> deg(NV + 1), lo(NV + 1), label(NV + 1), deg_in(NV + 1), gid(NV + 1);
    std::vector<long long> nptr(NV + 1), tiles(acc::scan_tiles_needed(NV) + 1);
    std::vector<uint32_t> nbr(2 * M + 1), occ(NV * occ_w + 1);
    std::vector<uint32_t> src(2 * M + 1), raw(2 * M + 1), merged(2 * M + 1);
    std::vector<uint2> rev(2 * M + 1);
    std::vector<long long> roff(NV + 1);
    std::vector<int> big(acc::sparse_big_rows_cap(M));
    acc::GraphInfo info{};
    std::vector<unsigned long long> counts(7, 123);
    int status = -7;

    acc::GSet gs{};
    gs.B = (int)B;
    gs.NV = NV;
    gs.M = M;
    if (B == 1) gs.one = meta[0];
    gs.many = meta.data();
    gs.gid = gid.data();
    if (acc::launch_graph_ids(gs, gid.data(), nullptr) < 0) return 4;

    acc::BuildBufs bb{};
    bb.state = state.data();
    bb.state_words = words;
    bb.state_clean = false;
    bb.deg = deg.data();
    bb.lo = lo.data();
    bb.label = label.data();
    bb.deg_in = deg_in.data();
    bb.nptr = nptr.data();
    bb.tiles = tiles.data();
    bb.nbr = nbr.data();
    bb.occ = occ.data();
    bb.occ_w = occ_w;
    bb.info = &info;
    bb.k = guard_k;
    bb.src = src.data();
    const acc::SparseBufs sb = {raw.data(), merged.data(), roff.data(), big.data()};
    for (int pass = 0; pass < 2; pass++) {
        std::fill(counts.begin(), counts.end(), 123ull);
        const int launches =
            sparse ? acc::launch_build_graph_sparse(gs, bb, sb, max_n, &status, counts.data(),
                                                    (long long)counts.size(), relabel, num_sms, nullptr)
                   : acc::launch_build_graph(gs, bb, max_n, &status, counts.data(), (long long)counts.size(), relabel,
                                             num_sms, nullptr);
        bool zeroed = true;
        for (auto c : counts) zeroed = zeroed && c == 0;
        const long long nnz = status == 0 ? info.nnz : 0;
        const long long head[5] = {status, launches, nnz, status == 0 ? info.maxdeg : 0, zeroed ? 1 : 0};
        put(head, 5);
        put(label.data(), NV);
        put(deg.data(), NV);
        put(lo.data(), NV);
        put(nptr.data(), NV + 1);
        put(nbr.data(), (size_t)nnz);
        put(state.data(), sparse ? 0 : words);
        put(occ.data(), sparse ? 0 : NV * occ_w);
        if (!sparse && acc::launch_clear_graph(gs, state.data(), occ.data(), occ_w, num_sms, nullptr) < 0) return 4;
        long long clean = 1;
        for (long long i = 0; i < words; i++) clean = clean && (sparse || state[i] == 0);
        put(&clean, 1);
        put(src.data(), (size_t)nnz);
        std::vector<uint32_t> rv;
        if (status == 0 && acc::launch_rev_build(gs, nptr.data(), deg.data(), nbr.data(), src.data(), &info, 2 * M,
                                                 rev.data(), num_sms, nullptr) < 0)
            return 4;
        for (long long p = 0; p < nnz; p++) {
            rv.push_back(rev[p].x);
            rv.push_back(rev[p].y);
        }
        put(rv.data(), rv.size());
        bb.state_clean = true;
    }
    fclose(out);
    return 0;
}
