/*
 * Seeded synthetic directed-graph generators.
 *
 * This file holds input preparation only: it draws arc lists whose shapes
 * follow the workloads the motif counter is measured on (Erdos-Renyi,
 * directed Chung-Lu with Pareto weights, hub-and-target "regulatory"
 * graphs, and degree-preserving double-edge-swap randomisations).  It holds
 * none of the counting arithmetic; the CPU oracle and the GPU path both take
 * its output as plain arrays.
 *
 * Determinism across machines: every random number comes from SplitMix64
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014), and the only floating-point operations are IEEE basic
 * operations (+ - * /, comparisons, exact scaling by powers of two and
 * float<->int conversion).  log and exp are written out below as plain
 * series, so no libm routine (whose last bit may differ between x86-64 and
 * aarch64) touches a value.  Build with -ffp-contract=off so the compiler
 * does not fuse multiply-adds.
 *
 * Every generated graph is simple: no self-loops, no repeated arc.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* SplitMix64                                                           */
/* ------------------------------------------------------------------ */

static uint64_t sm_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform integer in [0, bound) by the 128-bit multiply-shift map. */
static uint64_t sm_below(uint64_t *state, uint64_t bound)
{
    unsigned __int128 p = (unsigned __int128)sm_next(state) * bound;
    return (uint64_t)(p >> 64);
}

/* Uniform double in [0, 1) with 53 random bits. */
static double sm_unit(uint64_t *state)
{
    return (double)(sm_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t synth_splitmix_next(uint64_t *state) { return sm_next(state); }
double synth_splitmix_unit(uint64_t *state) { return sm_unit(state); }
uint64_t synth_splitmix_below(uint64_t *state, uint64_t bound) { return sm_below(state, bound); }

/* ------------------------------------------------------------------ */
/* Deterministic log / exp from basic operations                        */
/* ------------------------------------------------------------------ */

static const double LN2_HI = 6.93147180369123816490e-01; /* high bits of ln 2 */
static const double LN2_LO = 1.90821492927058770002e-10; /* ln 2 - LN2_HI     */
static const double SQRT_HALF = 0.70710678118654752440;

/* Split x > 0 into f * 2^e with f in [0.5, 1) by exact scaling. */
static double split_pow2(double x, int *e)
{
    int ee = 0;
    while (x >= 1.0) { x *= 0.5; ee++; }
    while (x < 0.5) { x *= 2.0; ee--; }
    *e = ee;
    return x;
}

static double scale_pow2(double x, int e)
{
    while (e > 0) { x *= 2.0; e--; }
    while (e < 0) { x *= 0.5; e++; }
    return x;
}

/* ln x for x > 0: ln x = e ln 2 + 2 atanh(s), s = (f-1)/(f+1), f near 1. */
double synth_log(double x)
{
    int e;
    double f = split_pow2(x, &e);
    if (f < SQRT_HALF) { f *= 2.0; e -= 1; }
    double s = (f - 1.0) / (f + 1.0);
    double s2 = s * s;
    /* odd series 2 (s + s^3/3 + ... + s^23/23), |s| <= 0.1716 */
    double acc = 0.0;
    for (int j = 23; j >= 3; j -= 2) acc = (acc + 1.0 / (double)j) * s2;
    double lnf = 2.0 * s * (1.0 + acc);
    return (double)e * LN2_HI + ((double)e * LN2_LO + lnf);
}

/* e^y: y = n ln 2 + r with |r| <= ln2/2, Taylor series for e^r. */
double synth_exp(double y)
{
    if (y > 700.0) y = 700.0;
    if (y < -700.0) y = -700.0;
    double t = y / (LN2_HI + LN2_LO) + 0.5;
    long long nn = (long long)t;
    if ((double)nn > t) nn -= 1; /* floor */
    double r = (y - (double)nn * LN2_HI) - (double)nn * LN2_LO;
    double acc = 1.0;
    for (int j = 22; j >= 1; j--) acc = 1.0 + acc * r / (double)j;
    return scale_pow2(acc, (int)nn);
}

/* Pareto sample with x_min = 1 and tail shape alpha: (1-u)^(-1/alpha). */
static double pareto(uint64_t *st, double alpha)
{
    double u = sm_unit(st);
    return synth_exp(-synth_log(1.0 - u) / alpha);
}

/* ------------------------------------------------------------------ */
/* Arc hash set (linear probing, backward-shift deletion)               */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t *keys; /* key = (src << 32 | dst) + 1, 0 = empty */
    uint64_t mask;
} arcset;

static int arcset_init(arcset *h, int64_t expected)
{
    uint64_t cap = 16;
    while (cap < (uint64_t)expected * 3) cap <<= 1;
    h->keys = (uint64_t *)calloc(cap, sizeof(uint64_t));
    h->mask = cap - 1;
    return h->keys ? 0 : -1;
}

static void arcset_free(arcset *h) { free(h->keys); h->keys = NULL; }

static uint64_t arc_key(int32_t s, int32_t t)
{
    return (((uint64_t)(uint32_t)s << 32) | (uint32_t)t) + 1;
}

static uint64_t arc_slot(const arcset *h, uint64_t key)
{
    uint64_t z = key * 0x9E3779B97F4A7C15ULL;
    return (z ^ (z >> 29)) & h->mask;
}

static int arcset_has(const arcset *h, int32_t s, int32_t t)
{
    uint64_t key = arc_key(s, t);
    for (uint64_t i = arc_slot(h, key);; i = (i + 1) & h->mask) {
        if (h->keys[i] == key) return 1;
        if (h->keys[i] == 0) return 0;
    }
}

static void arcset_add(arcset *h, int32_t s, int32_t t)
{
    uint64_t key = arc_key(s, t);
    uint64_t i = arc_slot(h, key);
    while (h->keys[i] != 0 && h->keys[i] != key) i = (i + 1) & h->mask;
    h->keys[i] = key;
}

static void arcset_del(arcset *h, int32_t s, int32_t t)
{
    uint64_t key = arc_key(s, t);
    uint64_t i = arc_slot(h, key);
    while (h->keys[i] != key) {
        if (h->keys[i] == 0) return;
        i = (i + 1) & h->mask;
    }
    /* backward-shift the cluster that follows slot i */
    uint64_t j = i;
    for (;;) {
        j = (j + 1) & h->mask;
        if (h->keys[j] == 0) break;
        uint64_t home = arc_slot(h, h->keys[j]);
        /* keys[j] may move to i if its home is not cyclically in (i, j] */
        int in_range = (i <= j) ? (home > i && home <= j) : (home > i || home <= j);
        if (!in_range) {
            h->keys[i] = h->keys[j];
            i = j;
        }
    }
    h->keys[i] = 0;
}

/* ------------------------------------------------------------------ */
/* Weighted sampling by cumulative integer weights                      */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t *cum; /* cum[i] = sum_{j<=i} W_j */
    int32_t n;
} sampler;

static int sampler_init(sampler *s, const double *w, int32_t n)
{
    s->cum = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    s->n = n;
    if (!s->cum) return -1;
    uint64_t acc = 0;
    for (int32_t i = 0; i < n; i++) {
        acc += (uint64_t)(w[i] * 4294967296.0);
        s->cum[i] = acc;
    }
    return acc > 0 ? 0 : -1;
}

static int32_t sampler_draw(const sampler *s, uint64_t *st)
{
    uint64_t x = sm_below(st, s->cum[s->n - 1]);
    int32_t lo = 0, hi = s->n - 1; /* first i with cum[i] > x */
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (s->cum[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Scale factor c with sum_i min(c * x_i, cap) = target, by bisection. */
static double capped_scale(const double *x, int32_t n, double cap, double target)
{
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; it++) {
        double sum = 0.0;
        for (int32_t i = 0; i < n; i++) { double v = hi * x[i]; sum += v < cap ? v : cap; }
        if (sum >= target) break;
        hi *= 2.0;
    }
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        double sum = 0.0;
        for (int32_t i = 0; i < n; i++) { double v = mid * x[i]; sum += v < cap ? v : cap; }
        if (sum < target) lo = mid; else hi = mid;
    }
    return hi;
}

/* Number of reciprocated pairs for a reciprocity of pct percent of m arcs. */
static int64_t recip_pairs(int64_t m, int32_t pct)
{
    return ((int64_t)pct * m + 100) / 200;
}

/*
 * Reciprocate q of the arcs in (src, dst)[0, m1): walk a seeded random
 * permutation and take the first q arcs whose reverse keeps both degree caps.
 * The reverses are appended at [m1, m1 + q).  Returns the number appended.
 */
static int64_t reciprocate(int32_t *src, int32_t *dst, int64_t m1, int64_t q,
                           int32_t *outdeg, int32_t *indeg, int32_t cap_out, int32_t cap_in,
                           arcset *h, uint64_t *st)
{
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m1 > 0 ? m1 : 1));
    if (!perm) return -1;
    for (int64_t i = 0; i < m1; i++) perm[i] = i;
    int64_t added = 0;
    for (int64_t i = 0; i < m1 && added < q; i++) {
        int64_t j = i + (int64_t)sm_below(st, (uint64_t)(m1 - i));
        int64_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
        int32_t s = src[perm[i]], t = dst[perm[i]];
        if (outdeg[t] >= cap_out || indeg[s] >= cap_in) continue;
        src[m1 + added] = t;
        dst[m1 + added] = s;
        outdeg[t]++; indeg[s]++;
        arcset_add(h, t, s);
        added++;
    }
    free(perm);
    return added;
}

/*
 * Draw m - q single arcs by (source ~ w_out, target ~ w_in), rejecting
 * self-loops, repeats, reverses of drawn arcs and arcs past the degree caps,
 * then reciprocate q of them.  Returns 0, or -1 if the rejection loop stalls.
 */
static int weighted_digraph(int32_t n, int64_t m, const double *w_out, const double *w_in,
                            int32_t cap_out, int32_t cap_in, int32_t recip_pct, uint64_t seed,
                            int32_t *src, int32_t *dst)
{
    uint64_t st = seed;
    int64_t q = recip_pairs(m, recip_pct);
    int64_t m1 = m - q;
    sampler so, si;
    arcset h;
    int32_t *outdeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *indeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int rc = -1;
    if (!outdeg || !indeg) goto done0;
    if (sampler_init(&so, w_out, n)) goto done0;
    if (sampler_init(&si, w_in, n)) { free(so.cum); goto done0; }
    if (arcset_init(&h, m)) goto done1;
    {
        int64_t got = 0, tries = 0, max_tries = 2000 * m + 100000;
        while (got < m1) {
            if (++tries > max_tries) goto done2;
            int32_t s = sampler_draw(&so, &st);
            int32_t t = sampler_draw(&si, &st);
            if (s == t) continue;
            if (outdeg[s] >= cap_out || indeg[t] >= cap_in) continue;
            if (arcset_has(&h, s, t) || arcset_has(&h, t, s)) continue;
            arcset_add(&h, s, t);
            src[got] = s; dst[got] = t;
            outdeg[s]++; indeg[t]++;
            got++;
        }
        if (reciprocate(src, dst, m1, q, outdeg, indeg, cap_out, cap_in, &h, &st) != q) goto done2;
        rc = 0;
    }
done2:
    arcset_free(&h);
done1:
    free(so.cum); free(si.cum);
done0:
    free(outdeg); free(indeg);
    return rc;
}

/* Directed Erdos-Renyi: uniform ordered pairs, pct percent of arcs reciprocal. */
int synth_er(int32_t n, int64_t m, int32_t recip_pct, uint64_t seed, int32_t *src, int32_t *dst)
{
    if (n < 2 || m < 0 || (double)m > (double)n * (double)(n - 1) * 0.5) return -2;
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    if (!w) return -1;
    for (int32_t i = 0; i < n; i++) w[i] = 1.0;
    int rc = weighted_digraph(n, m, w, w, n, n, recip_pct, seed, src, dst);
    free(w);
    return rc;
}

/*
 * Directed Chung-Lu: out- and in-weights drawn independently from a Pareto
 * law with density exponent `exponent` (tail shape exponent - 1, x_min 1),
 * each set scaled so min(c x_i, cap) sums to m; realised out- and in-degrees
 * are capped at `cap`.
 */
int synth_chung_lu(int32_t n, int64_t m, double exponent, int32_t cap, int32_t recip_pct,
                   uint64_t seed, int32_t *src, int32_t *dst)
{
    if (n < 2 || m < 0 || exponent <= 1.0 || cap < 1) return -2;
    if ((double)m > (double)n * (double)cap * 0.9) return -2;
    uint64_t st = seed;
    double alpha = exponent - 1.0;
    double *xo = (double *)malloc(sizeof(double) * (size_t)n);
    double *xi = (double *)malloc(sizeof(double) * (size_t)n);
    if (!xo || !xi) { free(xo); free(xi); return -1; }
    for (int32_t i = 0; i < n; i++) xo[i] = pareto(&st, alpha);
    for (int32_t i = 0; i < n; i++) xi[i] = pareto(&st, alpha);
    double co = capped_scale(xo, n, (double)cap, (double)m);
    double ci = capped_scale(xi, n, (double)cap, (double)m);
    for (int32_t i = 0; i < n; i++) {
        double a = co * xo[i], b = ci * xi[i];
        xo[i] = a < cap ? a : cap;
        xi[i] = b < cap ? b : cap;
    }
    int rc = weighted_digraph(n, m, xo, xi, cap, cap, recip_pct, sm_next(&st), src, dst);
    free(xo); free(xi);
    return rc;
}

/*
 * Regulatory-network shape: n_hubs distinct hub vertices draw out-degrees
 * from a Pareto law (density exponent `exponent`), scaled and capped at `cap`
 * and rounded by largest remainder to sum m - q; each hub's targets are
 * uniform over the other vertices; then q arcs are reciprocated.
 */
int synth_regulatory(int32_t n, int64_t m, int32_t n_hubs, double exponent, int32_t cap,
                     int32_t recip_pct, uint64_t seed, int32_t *src, int32_t *dst)
{
    if (n < 2 || n_hubs < 1 || n_hubs > n || exponent <= 1.0 || cap < 1 || cap > n - 1) return -2;
    int64_t q = recip_pairs(m, recip_pct);
    int64_t m1 = m - q;
    if (m1 > (int64_t)n_hubs * cap) return -2;
    uint64_t st = seed;
    int rc = -1;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n_hubs);
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_hubs);
    double *frac = (double *)malloc(sizeof(double) * (size_t)n_hubs);
    int32_t *outdeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *indeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    arcset h;
    h.keys = NULL;
    if (!ids || !x || !deg || !frac || !outdeg || !indeg) goto done;
    for (int32_t i = 0; i < n; i++) ids[i] = i;
    for (int32_t i = 0; i < n_hubs; i++) { /* partial Fisher-Yates */
        int32_t j = i + (int32_t)sm_below(&st, (uint64_t)(n - i));
        int32_t t = ids[i]; ids[i] = ids[j]; ids[j] = t;
    }
    for (int32_t i = 0; i < n_hubs; i++) x[i] = pareto(&st, exponent - 1.0);
    {
        double c = capped_scale(x, n_hubs, (double)cap, (double)m1);
        int64_t sum = 0;
        for (int32_t i = 0; i < n_hubs; i++) {
            double v = c * x[i];
            if (v > cap) v = cap;
            deg[i] = (int64_t)v;
            frac[i] = v - (double)deg[i];
            sum += deg[i];
        }
        /* largest remainder: repeatedly give one to the largest fraction */
        while (sum < m1) {
            int32_t best = -1;
            for (int32_t i = 0; i < n_hubs; i++)
                if (deg[i] < cap && (best < 0 || frac[i] > frac[best])) best = i;
            if (best < 0) goto done;
            deg[best]++; frac[best] = -1.0; sum++;
        }
        while (sum > m1) {
            int32_t best = -1;
            for (int32_t i = 0; i < n_hubs; i++)
                if (deg[i] > 0 && (best < 0 || frac[i] < frac[best])) best = i;
            if (best < 0) goto done;
            deg[best]--; frac[best] = 2.0; sum--;
        }
    }
    if (arcset_init(&h, m)) goto done;
    {
        int64_t got = 0;
        for (int32_t i = 0; i < n_hubs; i++) {
            int32_t hub = ids[i];
            int64_t tries = 0;
            for (int64_t d = 0; d < deg[i];) {
                if (++tries > 1000 * (int64_t)n + 1000) goto done;
                int32_t t = (int32_t)sm_below(&st, (uint64_t)(n - 1));
                if (t >= hub) t++;
                if (arcset_has(&h, hub, t) || arcset_has(&h, t, hub)) continue;
                arcset_add(&h, hub, t);
                src[got] = hub; dst[got] = t;
                outdeg[hub]++; indeg[t]++;
                got++; d++;
            }
        }
        if (reciprocate(src, dst, m1, q, outdeg, indeg, n, n, &h, &st) != q) goto done;
    }
    rc = 0;
done:
    arcset_free(&h);
    free(ids); free(x); free(deg); free(frac); free(outdeg); free(indeg);
    return rc;
}

/*
 * Degree-preserving randomisation: `attempts` double-edge swaps
 * (a->b, c->d) -> (a->d, c->b) on a copy of the arc list, each rejected if it
 * would create a self-loop or a repeated arc.  Every in- and out-degree is
 * kept.  Returns the number of accepted swaps, or -1 on allocation failure.
 */
int64_t synth_swap_randomise(int32_t n, int64_t m, const int32_t *src_in, const int32_t *dst_in,
                             int64_t attempts, uint64_t seed, int32_t *src, int32_t *dst)
{
    (void)n;
    uint64_t st = seed;
    arcset h;
    if (arcset_init(&h, m)) return -1;
    for (int64_t i = 0; i < m; i++) {
        src[i] = src_in[i];
        dst[i] = dst_in[i];
        arcset_add(&h, src[i], dst[i]);
    }
    int64_t accepted = 0;
    if (m >= 2) {
        for (int64_t it = 0; it < attempts; it++) {
            int64_t e1 = (int64_t)sm_below(&st, (uint64_t)m);
            int64_t e2 = (int64_t)sm_below(&st, (uint64_t)m);
            if (e1 == e2) continue;
            int32_t a = src[e1], b = dst[e1], c = src[e2], d = dst[e2];
            if (a == d || c == b) continue;
            if (arcset_has(&h, a, d) || arcset_has(&h, c, b)) continue;
            arcset_del(&h, a, b);
            arcset_del(&h, c, d);
            arcset_add(&h, a, d);
            arcset_add(&h, c, b);
            dst[e1] = d;
            dst[e2] = b;
            accepted++;
        }
    }
    arcset_free(&h);
    return accepted;
}
