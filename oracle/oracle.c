/*
 * CPU oracle for exact connected induced k-subgraph counting (k = 3, 4, 5).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg use it.  It shares no code with the
 * CUDA path.
 *
 * What it computes (Problems Motifs-3/4/5, Background section of the paper):
 * for a simple directed graph G(V,E),
 *
 *     counts[c] = #{ S subset of V : |S| = k, G*[S] connected, class(G[S]) = c }
 *
 * where G* is the undirected version of G (Notation section: {u,v} in E*
 * iff (u,v) or (v,u) in E), so "connected" means weakly connected, and the
 * class is the isomorphism class of the induced directed subgraph.  There are
 * 13, 199 and 9364 classes for k = 3, 4, 5 (Problems 1-3).
 *
 * Conventions this file fixes (the paper leaves them open; its histogram
 * positions are arbitrary and "hard coded"):
 *  - adjacency code of an ordered tuple (w_0 .. w_{k-1}): bit
 *    i*(k-1) + (j - [j > i]) is set iff the arc w_i -> w_j is in E;
 *  - canonical code: the minimum of the code over all k! relabellings;
 *  - class index: the rank of the canonical code, ascending, among the
 *    canonical codes of weakly connected k-vertex digraphs.
 *
 * Plain and slow on purpose: canonical forms are found by trying every
 * permutation, the tiny-graph counter tries every k-subset, and the
 * enumeration counter is the ESU procedure of Wernicke (2006, the FANMOD
 * paper the paper cites) with an explicit recursion and plain sets.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAXK 5

static int code_bit(int k, int i, int j) { return i * (k - 1) + (j - (j > i ? 1 : 0)); }

int oracle_num_classes(int k)
{
    switch (k) {
    case 3: return 13;
    case 4: return 199;
    case 5: return 9364;
    default: return -1;
    }
}

/* arc i -> j in the digraph a code describes */
static int code_arc(int k, uint32_t code, int i, int j) { return (int)((code >> code_bit(k, i, j)) & 1u); }

/* Weak connectivity of the code's digraph: depth-first search on the skeleton. */
int oracle_code_connected(int k, uint32_t code)
{
    int seen[ORACLE_MAXK] = {0}, stack[ORACLE_MAXK], top = 0, nseen = 1;
    seen[0] = 1;
    stack[top++] = 0;
    while (top > 0) {
        int a = stack[--top];
        for (int b = 0; b < k; b++) {
            if (seen[b] || b == a) continue;
            if (code_arc(k, code, a, b) || code_arc(k, code, b, a)) {
                seen[b] = 1;
                nseen++;
                stack[top++] = b;
            }
        }
    }
    return nseen == k;
}

/* Code of the digraph relabelled by vertex i -> perm[i]. */
uint32_t oracle_permute_code(int k, uint32_t code, const int *perm)
{
    uint32_t out = 0;
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++)
            if (i != j && code_arc(k, code, i, j)) out |= 1u << code_bit(k, perm[i], perm[j]);
    return out;
}

/* Next permutation in lexicographic order; returns 0 after the last one. */
static int next_perm(int *p, int k)
{
    int i = k - 2;
    while (i >= 0 && p[i] > p[i + 1]) i--;
    if (i < 0) return 0;
    int j = k - 1;
    while (p[j] < p[i]) j--;
    int t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = k - 1; a < b; a++, b--) { t = p[a]; p[a] = p[b]; p[b] = t; }
    return 1;
}

/* Canonical code: the minimum over all k! relabellings. */
uint32_t oracle_canonical_code(int k, uint32_t code)
{
    int p[ORACLE_MAXK];
    for (int i = 0; i < k; i++) p[i] = i;
    uint32_t best = 0xFFFFFFFFu;
    do {
        uint32_t c = oracle_permute_code(k, code, p);
        if (c < best) best = c;
    } while (next_perm(p, k));
    return best;
}

/* Number of relabellings that map the code to itself (automorphisms). */
int oracle_automorphisms(int k, uint32_t code)
{
    int p[ORACLE_MAXK], n = 0;
    for (int i = 0; i < k; i++) p[i] = i;
    do {
        if (oracle_permute_code(k, code, p) == code) n++;
    } while (next_perm(p, k));
    return n;
}

/*
 * Code -> class table for all 2^(k(k-1)) codes (-1 for disconnected codes)
 * and the class -> canonical code list (ascending).  Returns the number of
 * classes, or -1 on a bad k or a too small class_code buffer.
 */
int oracle_build_table(int k, int32_t *class_of_code, uint32_t *class_code, int class_cap)
{
    if (k < 3 || k > ORACLE_MAXK) return -1;
    uint32_t ncodes = 1u << (k * (k - 1));
    uint32_t *canon = (uint32_t *)malloc(sizeof(uint32_t) * ncodes);
    if (!canon) return -1;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t c = 0; c < (int64_t)ncodes; c++)
        canon[c] = oracle_code_connected(k, (uint32_t)c) ? oracle_canonical_code(k, (uint32_t)c) : 0xFFFFFFFFu;
    /* class id of canonical code c = number of canonical codes below c */
    int nclass = 0;
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * ncodes);
    if (!rank) { free(canon); return -1; }
    for (uint32_t c = 0; c < ncodes; c++) {
        if (canon[c] == c) {
            if (nclass >= class_cap) { free(canon); free(rank); return -1; }
            class_code[nclass] = c;
            rank[c] = nclass++;
        } else {
            rank[c] = -1;
        }
    }
    for (uint32_t c = 0; c < ncodes; c++) class_of_code[c] = canon[c] == 0xFFFFFFFFu ? -1 : rank[canon[c]];
    free(canon);
    free(rank);
    return nclass;
}

/* ------------------------------------------------------------------ */
/* Graph: dense out-arc bit matrix plus sorted undirected neighbour lists */
/* ------------------------------------------------------------------ */

/* Graphs of at most this many vertices keep the arc test in a dense bit
   matrix (n^2 / 8 bytes); larger ones in sorted out-neighbour lists. */
static int32_t dense_max = 65536;

void oracle_set_dense_max(int32_t n) { dense_max = n; }

typedef struct {
    int32_t n;
    uint64_t words; /* 64-bit words per bit-matrix row */
    uint64_t *out;  /* bit (a, b) set iff arc a -> b; NULL above dense_max */
    int64_t *optr;  /* out-neighbours of a: oadj[optr[a] .. optr[a+1]), sorted, no repeats */
    int32_t *oadj;
    int64_t *nptr;  /* neighbour lists of G*, sorted ascending */
    int32_t *nbr;
    int64_t maxdeg;
} ograph;

static int arc(const ograph *g, int32_t a, int32_t b)
{
    if (g->out) return (int)((g->out[(uint64_t)a * g->words + ((uint32_t)b >> 6)] >> (b & 63)) & 1u);
    int64_t lo = g->optr[a], hi = g->optr[a + 1] - 1;  /* binary search for b */
    while (lo <= hi) {
        const int64_t mid = (lo + hi) / 2;
        if (g->oadj[mid] == b) return 1;
        if (g->oadj[mid] < b) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

static int adjacent(const ograph *g, int32_t a, int32_t b) { return arc(g, a, b) || arc(g, b, a); }

static int cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* Returns 0, -1 on allocation failure, -2 on a self-loop or a vertex out of range. */
static int ograph_build(ograph *g, int32_t n, int64_t m, const int32_t *src, const int32_t *dst)
{
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->words = ((uint64_t)n + 63) / 64;
    if (n <= dense_max) {
        g->out = (uint64_t *)calloc((size_t)(g->words * (uint64_t)(n > 0 ? n : 1)), sizeof(uint64_t));
        if (!g->out) return -1;
    }
    g->nptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->optr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->nptr || !g->optr) return -1;
    for (int64_t e = 0; e < m; e++) {
        int32_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) return -2;
        if (g->out) g->out[(uint64_t)a * g->words + ((uint32_t)b >> 6)] |= 1ull << (b & 63);
        g->optr[a + 1]++;
    }
    /* out-neighbour lists: sorted, repeats dropped */
    for (int32_t a = 0; a < n; a++) g->optr[a + 1] += g->optr[a];
    g->oadj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t *ofill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->oadj || !ofill) { free(ofill); return -1; }
    for (int64_t e = 0; e < m; e++) g->oadj[g->optr[src[e]] + ofill[src[e]]++] = dst[e];
    free(ofill);
    int64_t ow = 0;
    for (int32_t a = 0; a < n; a++) {
        const int64_t lo = g->optr[a], hi = g->optr[a + 1];
        qsort(g->oadj + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_i32);
        g->optr[a] = ow;
        for (int64_t t = lo; t < hi; t++)
            if (t == lo || g->oadj[t] != g->oadj[t - 1]) g->oadj[ow++] = g->oadj[t];
    }
    g->optr[n] = ow;
    /* neighbour lists of G*: b is listed under a (and a under b) for every
       arc a -> b; each list is then sorted and repeats are dropped */
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!fill) return -1;
    for (int64_t e = 0; e < m; e++) { fill[src[e]]++; fill[dst[e]]++; }
    int64_t total = 0;
    for (int32_t a = 0; a < n; a++) { g->nptr[a] = total; total += fill[a]; fill[a] = 0; }
    g->nptr[n] = total;
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!g->nbr) { free(fill); return -1; }
    for (int64_t e = 0; e < m; e++) {
        int32_t a = src[e], b = dst[e];
        g->nbr[g->nptr[a] + fill[a]++] = b;
        g->nbr[g->nptr[b] + fill[b]++] = a;
    }
    free(fill);
    for (int32_t a = 0; a < n; a++)
        qsort(g->nbr + g->nptr[a], (size_t)(g->nptr[a + 1] - g->nptr[a]), sizeof(int32_t), cmp_i32);
    int64_t w = 0;
    for (int32_t a = 0; a < n; a++) {
        int64_t lo = g->nptr[a], hi = g->nptr[a + 1];
        g->nptr[a] = w;
        for (int64_t t = lo; t < hi; t++)
            if (t == lo || g->nbr[t] != g->nbr[t - 1]) g->nbr[w++] = g->nbr[t];
    }
    g->nptr[n] = w;
    g->maxdeg = 0;
    for (int32_t a = 0; a < n; a++)
        if (g->nptr[a + 1] - g->nptr[a] > g->maxdeg) g->maxdeg = g->nptr[a + 1] - g->nptr[a];
    return 0;
}

static void ograph_free(ograph *g)
{
    free(g->out);
    free(g->nptr);
    free(g->nbr);
    free(g->optr);
    free(g->oadj);
}

/* Adjacency code of the ordered tuple w[0..k-1] in g. */
static uint32_t tuple_code(const ograph *g, int k, const int32_t *w)
{
    uint32_t code = 0;
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++)
            if (i != j && arc(g, w[i], w[j])) code |= 1u << code_bit(k, i, j);
    return code;
}

/* ------------------------------------------------------------------ */
/* Tier 0: every k-subset, canonicalised directly (no table)            */
/* ------------------------------------------------------------------ */

static int class_by_search(const uint32_t *class_code, int nclass, uint32_t canon)
{
    int lo = 0, hi = nclass - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (class_code[mid] == canon) return mid;
        if (class_code[mid] < canon) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/*
 * Counts over all C(n,k) subsets.  class_code is the ascending canonical
 * code list from oracle_build_table.  Returns 0, or a negative error.
 */
int oracle_count_bruteforce(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k,
                            const uint32_t *class_code, int nclass, int64_t *counts)
{
    if (k < 3 || k > ORACLE_MAXK || n < 0) return -3;
    ograph g;
    int rc = ograph_build(&g, n, m, src, dst);
    if (rc) { ograph_free(&g); return rc; }
    memset(counts, 0, sizeof(int64_t) * (size_t)nclass);
    int32_t w[ORACLE_MAXK];
    if (n >= k) {
        for (int i = 0; i < k; i++) w[i] = i;
        for (;;) {
            uint32_t code = tuple_code(&g, k, w);
            if (oracle_code_connected(k, code)) {
                int c = class_by_search(class_code, nclass, oracle_canonical_code(k, code));
                if (c < 0) { ograph_free(&g); return -4; }
                counts[c]++;
            }
            /* next k-combination of 0..n-1 in lexicographic order */
            int i = k - 1;
            while (i >= 0 && w[i] == n - k + i) i--;
            if (i < 0) break;
            w[i]++;
            for (int j = i + 1; j < k; j++) w[j] = w[j - 1] + 1;
        }
    }
    ograph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Tier 1: ESU enumeration (Wernicke 2006)                              */
/* ------------------------------------------------------------------ */

typedef struct {
    const ograph *g;
    int k;
    const int32_t *class_of_code;
    int64_t *counts; /* this worker's histogram */
    int bad;         /* set if a leaf met a disconnected code (cannot happen) */
} esu_ctx;

/* u is in N[Vsub] = Vsub plus every neighbour of Vsub */
static int in_closed_nbhd(const esu_ctx *c, const int32_t *vsub, int nsub, int32_t u)
{
    for (int i = 0; i < nsub; i++)
        if (vsub[i] == u || adjacent(c->g, vsub[i], u)) return 1;
    return 0;
}

/*
 * ExtendSubgraph(Vsub, Vext, v): while Vext is not empty, remove a vertex w
 * from it, form Vext' = Vext plus the exclusive neighbours of w (neighbours
 * of w above the root v that are neither in Vsub nor adjacent to it), and
 * recurse on (Vsub + w, Vext').  Each connected k-set whose smallest vertex
 * is v is reached exactly once.
 */
static void esu_extend(esu_ctx *c, int32_t *vsub, int nsub, const int32_t *vext, int64_t next, int32_t root)
{
    const ograph *g = c->g;
    if (nsub == c->k - 1) {
        /* each remaining choice of w completes a k-set */
        for (int64_t t = 0; t < next; t++) {
            vsub[nsub] = vext[t];
            int cls = c->class_of_code[tuple_code(g, c->k, vsub)];
            if (cls < 0) c->bad = 1; else c->counts[cls]++;
        }
        return;
    }
    int32_t *ext2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(next + g->maxdeg + 1));
    if (!ext2) { c->bad = 2; return; }
    for (int64_t t = 0; t < next; t++) {
        int32_t w = vext[t];
        /* Vext' = the vertices still in Vext after removing w ... */
        int64_t n2 = 0;
        for (int64_t r = t + 1; r < next; r++) ext2[n2++] = vext[r];
        /* ... plus the exclusive neighbours of w with respect to Vsub */
        for (int64_t p = g->nptr[w]; p < g->nptr[w + 1]; p++) {
            int32_t u = g->nbr[p];
            if (u > root && !in_closed_nbhd(c, vsub, nsub, u)) ext2[n2++] = u;
        }
        vsub[nsub] = w;
        esu_extend(c, vsub, nsub + 1, ext2, n2, root);
    }
    free(ext2);
}

/*
 * Counts of the connected k-sets whose smallest vertex lies in
 * [root_lo, root_hi) (the whole graph when root_lo = 0, root_hi = n), using
 * the code -> class table.  nthreads > 1 splits the roots over OpenMP
 * threads, each with its own histogram, summed at the end.  Returns 0, or a
 * negative error.
 */
int oracle_count_esu(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k,
                     const int32_t *class_of_code, int nclass, int32_t root_lo, int32_t root_hi,
                     int nthreads, int64_t *counts)
{
    if (k < 3 || k > ORACLE_MAXK || n < 0) return -3;
    if (root_lo < 0) root_lo = 0;
    if (root_hi > n) root_hi = n;
    ograph g;
    int rc = ograph_build(&g, n, m, src, dst);
    if (rc) { ograph_free(&g); return rc; }
    memset(counts, 0, sizeof(int64_t) * (size_t)nclass);
    if (nthreads < 1) nthreads = 1;
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int64_t *local = (int64_t *)calloc((size_t)nclass, sizeof(int64_t));
        int32_t *ext = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.nptr[n] > 0 ? g.nptr[n] : 1));
        esu_ctx c = {&g, k, class_of_code, local, (local && ext) ? 0 : 2};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int32_t v = root_lo; v < root_hi; v++) {
            if (c.bad) continue;
            int32_t vsub[ORACLE_MAXK];
            vsub[0] = v;
            /* Vext = neighbours of v above v */
            int64_t next = 0;
            for (int64_t p = g.nptr[v]; p < g.nptr[v + 1]; p++)
                if (g.nbr[p] > v) ext[next++] = g.nbr[p];
            esu_extend(&c, vsub, 1, ext, next, v);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (c.bad) bad = c.bad;
            if (local)
                for (int i = 0; i < nclass; i++) counts[i] += local[i];
        }
        free(local);
        free(ext);
    }
    ograph_free(&g);
    return bad ? -4 - bad : 0;
}

/* Number of worker threads OpenMP would use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Significance: Z-scores of a real graph against its randomisations    */
/* ------------------------------------------------------------------ */

/*
 * Z_c = (N_c(real) - mu_c) / sigma_c over R randomisations (step iii of the
 * motif pipeline in the Implementation section; the paper names the step
 * but gives no formula).  mu_c = S1 / R with S1 the exact int64 sum; sigma_c
 * is the population deviation sqrt(sum_i (N_ic - mu_c)^2 / R), the sum taken
 * in increasing i.  Z is NaN when sigma_c = 0.  rand is row-major [R][K].
 */
void oracle_zscores(int K, int R, const int64_t *real, const int64_t *rand, double *z)
{
    for (int c = 0; c < K; c++) {
        int64_t s1 = 0;
        for (int i = 0; i < R; i++) s1 += rand[(int64_t)i * K + c];
        double mu = (double)s1 / (double)R;
        double m2 = 0.0;
        for (int i = 0; i < R; i++) {
            double d = (double)rand[(int64_t)i * K + c] - mu;
            m2 = m2 + d * d; /* built with -ffp-contract=off: no fused multiply-add */
        }
        double var = m2 / (double)R;
        double sd = __builtin_sqrt(var);
        double num = (double)real[c] - mu;
        z[c] = sd == 0.0 ? __builtin_nan("") : num / sd;
    }
}

/* ------------------------------------------------------------------ */
/* Significance: degree-preserving randomised copies                    */
/* ------------------------------------------------------------------ */

/*
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): add the golden-ratio increment to the state,
 * then two xor-shift-multiply rounds and a final xor-shift of the sum.
 */
static uint64_t orand_next(uint64_t *state)
{
    uint64_t z;
    *state = *state + 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* A uniform integer below `bound` by the multiply-shift map (Lemire, "Fast
 * random integer generation in an interval", 2019): the high 64 bits of
 * the 128-bit product of a draw and the bound. */
static uint64_t orand_below(uint64_t *state, uint64_t bound)
{
    unsigned __int128 prod = (unsigned __int128)orand_next(state) * (unsigned __int128)bound;
    return (uint64_t)(prod >> 64);
}

/* Position of target t in row v of the copy, or -1. */
static int64_t orand_find(const int64_t *rowptr, const int32_t *cur, int32_t v, int32_t t)
{
    for (int64_t p = rowptr[v]; p < rowptr[v + 1]; p++)
        if (cur[p] == t) return p;
    return -1;
}

/*
 * Randomised copy of a simple digraph for the random ensemble of the
 * significance step (Implementation section, steps i and iii: the paper
 * counts the real graph and a set of random graphs but fixes no generator).
 *
 * The graph is an out-CSR: arc e runs from the row that holds position e to
 * col[e].  The copy starts as col and keeps rowptr: an accepted swap changes
 * targets only, so every out-degree stays, and it moves targets between
 * arcs, so every in-degree stays.  `attempts` attempts, each drawing e1 then
 * e2 uniformly below m from the stream seeded with `seed`; with
 * a -> b = arc e1 and c -> d = arc e2 of the copy:
 *
 *   mode 0 (double-edge swap): rejected if e1 == e2, a == d, c == b, or
 *     a -> d or c -> b is already an arc; otherwise the arcs become a -> d
 *     and c -> b.
 *   mode 1 (mutual arcs kept): an arc is mutual when its reverse is an arc
 *     too.  Rejected if e1 == e2, a == d, c == b, one arc is mutual and the
 *     other is not, or a, d or c, b are adjacent (an arc either way).  Two
 *     single arcs become a -> d and c -> b; two mutual pairs a <-> b and
 *     c <-> d become a <-> d and c <-> b (the reverse arcs b -> a and d -> c
 *     are retargeted to c and a).  Every vertex keeps its numbers of single
 *     out-arcs, single in-arcs and mutual neighbours.
 *
 * out (int32[m]) receives the copy's targets in the positions of col.
 * Returns the number of accepted swaps, or -1 for an invalid argument.
 */
int64_t oracle_swap_randomise(int32_t n, int64_t m, const int64_t *rowptr, const int32_t *col, int64_t attempts,
                              uint64_t seed, int mode, int32_t *out)
{
    if (n < 0 || m < 0 || attempts < 0 || (mode != 0 && mode != 1)) return -1;
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!row) return -1;
    for (int32_t v = 0; v < n; v++)
        for (int64_t p = rowptr[v]; p < rowptr[v + 1]; p++) row[p] = v;
    for (int64_t e = 0; e < m; e++) out[e] = col[e];
    uint64_t state = seed;
    int64_t accepted = 0;
    for (int64_t t = 0; m >= 2 && t < attempts; t++) {
        int64_t e1 = (int64_t)orand_below(&state, (uint64_t)m);
        int64_t e2 = (int64_t)orand_below(&state, (uint64_t)m);
        if (e1 == e2) continue;
        int32_t a = row[e1], b = out[e1], c = row[e2], d = out[e2];
        if (a == d || c == b) continue;
        if (mode == 0) {
            if (orand_find(rowptr, out, a, d) >= 0 || orand_find(rowptr, out, c, b) >= 0) continue;
            out[e1] = d;
            out[e2] = b;
            accepted++;
            continue;
        }
        int64_t r1 = orand_find(rowptr, out, b, a); /* b -> a, if a -> b is mutual */
        int64_t r2 = orand_find(rowptr, out, d, c);
        if ((r1 >= 0) != (r2 >= 0)) continue;
        if (orand_find(rowptr, out, a, d) >= 0 || orand_find(rowptr, out, d, a) >= 0) continue;
        if (orand_find(rowptr, out, c, b) >= 0 || orand_find(rowptr, out, b, c) >= 0) continue;
        out[e1] = d;
        out[e2] = b;
        if (r1 >= 0) {
            out[r1] = c;
            out[r2] = a;
        }
        accepted++;
    }
    free(row);
    return accepted;
}
