/*
 * graphgen.c -- seeded synthetic graph generators and CSR canonicalisation.
 *
 * This module only produces inputs. It contains none of the orbit-counting
 * arithmetic; both the CPU oracle and the CUDA path consume its output.
 *
 * Random numbers: splitmix64 expands (seed, stream id) into the state of a
 * xoshiro256** generator (Blackman & Vigna, "Scrambled linear pseudorandom
 * number generators", 2018/2021). Work is cut into fixed chunks, each with
 * its own stream, so the output does not depend on the thread count.
 *
 * Generators:
 *   - Erdos-Renyi G(n, p): every pair {i, j} independently with probability
 *     p, sampled by geometric skipping (Batagelj & Brandes, "Efficient
 *     generation of large random networks", Phys. Rev. E 71, 2005). The
 *     paper's ER experiments use G(n, p) graphs (Sec. 7).
 *   - R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004): 2^scale vertices,
 *     edge_factor * 2^scale directed samples, quadrant probabilities
 *     (a, b, c, 1-a-b-c), no noise.
 *   - Chung-Lu with power-law weights w_i ~ (i+1)^(-1/(gamma-1)), scaled to a
 *     target mean degree and capped at sqrt(sum w); endpoints drawn in
 *     proportion to w, Poisson(sum w / 2) pairs ("erased" variant).
 * All generators then drop self-loops, symmetrise and remove duplicates, so
 * the result is a simple undirected graph in CSR form with every row sorted
 * ascending (the input contract of the library).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG */

static inline uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo256;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo256 *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* stream = f(seed, generator kind, chunk index) */
static xo256 xo_stream(uint64_t seed, uint64_t kind, uint64_t chunk) {
    uint64_t sm = seed ^ (kind * 0xD1B54A32D192ED03ULL) ^ (chunk * 0x8CB92BA72F3D8DD7ULL);
    xo256 r;
    for (int i = 0; i < 4; ++i) r.s[i] = splitmix64(&sm);
    return r;
}

/* uniform double in (0, 1] with 53 random bits */
static inline double xo_unit_open0(xo256 *r) {
    return (double)((xo_next(r) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

/* ----------------------------------------------------- growable pair list */

typedef struct { uint64_t *a; size_t len, cap; } u64vec;

static int vpush(u64vec *v, uint64_t x) {
    if (v->len == v->cap) {
        size_t nc = v->cap ? v->cap * 2 : 1024;
        uint64_t *na = (uint64_t *)realloc(v->a, nc * sizeof(uint64_t));
        if (!na) return -1;
        v->a = na;
        v->cap = nc;
    }
    v->a[v->len++] = x;
    return 0;
}

/* ------------------------------------------------------------- radix sort */

/* LSD radix sort of keys < 2^bits, 11-bit digits, OpenMP-parallel. */
static int radix_sort_u64(uint64_t *keys, size_t len, int bits) {
    if (len < 2) return 0;
    uint64_t *tmp = (uint64_t *)malloc(len * sizeof(uint64_t));
    if (!tmp) return -1;
    const int D = 11, B = 1 << D;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    size_t *hist = (size_t *)malloc((size_t)nthreads * B * sizeof(size_t));
    if (!hist) { free(tmp); return -1; }
    uint64_t *src = keys, *dst = tmp;
    for (int shift = 0; shift < bits; shift += D) {
        memset(hist, 0, (size_t)nthreads * B * sizeof(size_t));
#pragma omp parallel num_threads(nthreads)
        {
            int tid = 0, nt = 1;
#ifdef _OPENMP
            tid = omp_get_thread_num();
            nt = omp_get_num_threads();
#endif
            size_t lo = len * (size_t)tid / nt, hi = len * (size_t)(tid + 1) / nt;
            size_t *h = hist + (size_t)tid * B;
            for (size_t i = lo; i < hi; ++i) h[(src[i] >> shift) & (B - 1)]++;
#pragma omp barrier
#pragma omp single
            {
                size_t run = 0;
                for (int d = 0; d < B; ++d)
                    for (int t = 0; t < nt; ++t) {
                        size_t c = hist[(size_t)t * B + d];
                        hist[(size_t)t * B + d] = run;
                        run += c;
                    }
            }
            for (size_t i = lo; i < hi; ++i) {
                uint64_t k = src[i];
                dst[h[(k >> shift) & (B - 1)]++] = k;
            }
        }
        uint64_t *sw = src; src = dst; dst = sw;
    }
    if (src != keys) memcpy(keys, src, len * sizeof(uint64_t));
    free(hist);
    free(tmp);
    return 0;
}

/* ------------------------------------------------------- CSR result handle */

typedef struct {
    int32_t n;
    int64_t m;          /* number of CSR entries = 2|E| */
    int32_t *rowptr;    /* n + 1 */
    int32_t *colidx;    /* m */
} gg_graph;

void gg_free(gg_graph *g) {
    if (!g) return;
    free(g->rowptr);
    free(g->colidx);
    free(g);
}

int32_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_m(const gg_graph *g) { return g->m; }

void gg_copy_out(const gg_graph *g, int32_t *rowptr, int32_t *colidx) {
    memcpy(rowptr, g->rowptr, sizeof(int32_t) * ((size_t)g->n + 1));
    if (g->m) memcpy(colidx, g->colidx, sizeof(int32_t) * (size_t)g->m);
}

static int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b ? b : 1;
}

/*
 * Canonicalise undirected pairs (u, v), 0 <= u, v < n, into CSR: self-loops
 * dropped, both directions added, duplicates removed, rows sorted. Takes
 * ownership of nothing; `pairs` holds u * n + v keys of one direction each.
 */
static gg_graph *csr_from_pairs(int32_t n, const uint64_t *pairs, size_t npairs) {
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) return NULL;
    g->n = n;
    g->rowptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!g->rowptr) { gg_free(g); return NULL; }
    uint64_t *keys = (uint64_t *)malloc((2 * npairs + 1) * sizeof(uint64_t));
    if (!keys) { gg_free(g); return NULL; }
    size_t k = 0;
    const uint64_t N = (uint64_t)n;
    for (size_t i = 0; i < npairs; ++i) {
        uint64_t u = pairs[i] / N, v = pairs[i] % N;
        if (u == v) continue;
        keys[k++] = u * N + v;
        keys[k++] = v * N + u;
    }
    if (n > 0 && radix_sort_u64(keys, k, bits_for(N * N - 1)) != 0) { free(keys); gg_free(g); return NULL; }
    size_t w = 0;
    for (size_t i = 0; i < k; ++i)
        if (i == 0 || keys[i] != keys[i - 1]) keys[w++] = keys[i];
    g->m = (int64_t)w;
    g->colidx = (int32_t *)malloc((w ? w : 1) * sizeof(int32_t));
    if (!g->colidx) { free(keys); gg_free(g); return NULL; }
    for (size_t i = 0; i < w; ++i) {
        uint64_t u = keys[i] / N, v = keys[i] % N;
        g->rowptr[u + 1]++;
        g->colidx[i] = (int32_t)v;
    }
    for (int32_t i = 0; i < n; ++i) g->rowptr[i + 1] += g->rowptr[i];
    free(keys);
    return g;
}

/* Build a CSR from an explicit undirected edge list (used for small named graphs). */
gg_graph *gg_from_edges(int32_t n, int64_t nedges, const int32_t *eu, const int32_t *ev) {
    if (n < 0 || nedges < 0) return NULL;
    uint64_t *p = (uint64_t *)malloc(((size_t)nedges + 1) * sizeof(uint64_t));
    if (!p) return NULL;
    size_t k = 0;
    for (int64_t i = 0; i < nedges; ++i) {
        if (eu[i] < 0 || eu[i] >= n || ev[i] < 0 || ev[i] >= n) { free(p); return NULL; }
        p[k++] = (uint64_t)eu[i] * (uint64_t)n + (uint64_t)ev[i];
    }
    gg_graph *g = csr_from_pairs(n, p, k);
    free(p);
    return g;
}

/* ------------------------------------------------------------- generators */

enum { KIND_ER = 1, KIND_RMAT = 2, KIND_CL = 3 };

/* Erdos-Renyi G(n, p) by geometric skipping; rows are cut into fixed chunks. */
gg_graph *gg_er(int32_t n, double p, uint64_t seed) {
    if (n < 0 || !(p >= 0.0)) return NULL;
    const int32_t ROWS = 4096;
    int32_t nchunks = n > 0 ? (n + ROWS - 1) / ROWS : 0;
    u64vec *parts = (u64vec *)calloc((size_t)nchunks + 1, sizeof(u64vec));
    if (!parts) return NULL;
    int fail = 0;
    const double lq = (p < 1.0) ? log1p(-p) : 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int32_t c = 0; c < nchunks; ++c) {
        xo256 r = xo_stream(seed, KIND_ER, (uint64_t)c);
        int64_t lo = (int64_t)c * ROWS, hi = lo + ROWS;
        if (hi > n) hi = n;
        if (p <= 0.0) continue;
        if (p >= 1.0) {
            for (int64_t i = lo; i < hi; ++i)
                for (int64_t j = 0; j < i; ++j)
                    fail |= vpush(&parts[c], (uint64_t)i * (uint64_t)n + (uint64_t)j) != 0;
            continue;
        }
        /* pairs (i, j) with j < i, walked row by row; the next present pair is
           1 + Geometric(p) positions further on. */
        int64_t i = lo < 1 ? 1 : lo, j = -1;
        while (i < hi) {
            double u = xo_unit_open0(&r);
            double skip = floor(log(u) / lq);
            if (skip > 9.0e15) break;
            j += 1 + (int64_t)skip;
            while (j >= i && i < hi) { j -= i; ++i; }
            if (i < hi) fail |= vpush(&parts[c], (uint64_t)i * (uint64_t)n + (uint64_t)j) != 0;
        }
    }
    size_t total = 0;
    for (int32_t c = 0; c < nchunks; ++c) total += parts[c].len;
    uint64_t *all = (uint64_t *)malloc((total + 1) * sizeof(uint64_t));
    gg_graph *g = NULL;
    if (all && !fail) {
        size_t off = 0;
        for (int32_t c = 0; c < nchunks; ++c) {
            if (parts[c].len) memcpy(all + off, parts[c].a, parts[c].len * sizeof(uint64_t));
            off += parts[c].len;
        }
        g = csr_from_pairs(n, all, total);
    }
    for (int32_t c = 0; c < nchunks; ++c) free(parts[c].a);
    free(parts);
    free(all);
    return g;
}

/* R-MAT: edge_factor * 2^scale samples, quadrants a | b / c | d, MSB first. */
gg_graph *gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed) {
    if (scale < 1 || scale > 30 || edge_factor < 0) return NULL;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return NULL;
    const int32_t n = (int32_t)1 << scale;
    const size_t M = (size_t)edge_factor << scale;
    uint64_t *pairs = (uint64_t *)malloc((M + 1) * sizeof(uint64_t));
    if (!pairs) return NULL;
    const double two64 = 18446744073709551616.0;
    const uint64_t ta = (uint64_t)(a * two64 * (1.0 - 1e-16));
    const uint64_t tab = (uint64_t)((a + b) * two64 * (1.0 - 1e-16));
    const uint64_t tabc = (uint64_t)((a + b + c) * two64 * (1.0 - 1e-16));
    const size_t CH = (size_t)1 << 18;
    const size_t nch = (M + CH - 1) / CH;
#pragma omp parallel for schedule(dynamic, 4)
    for (size_t ch = 0; ch < nch; ++ch) {
        xo256 r = xo_stream(seed, KIND_RMAT, (uint64_t)ch);
        size_t lo = ch * CH, hi = lo + CH < M ? lo + CH : M;
        for (size_t e = lo; e < hi; ++e) {
            uint64_t u = 0, v = 0;
            for (int l = scale - 1; l >= 0; --l) {
                uint64_t x = xo_next(&r);
                uint64_t ub = x >= tab;                       /* quadrants c, d */
                uint64_t vb = (x >= ta && x < tab) || x >= tabc; /* quadrants b, d */
                u |= ub << l;
                v |= vb << l;
            }
            pairs[e] = u * (uint64_t)n + v;
        }
    }
    gg_graph *g = csr_from_pairs(n, pairs, M);
    free(pairs);
    return g;
}

/* Poisson sample: inversion for small means, rounded normal otherwise. */
static uint64_t poisson(xo256 *r, double lam) {
    if (lam <= 0) return 0;
    if (lam < 30.0) {
        double L = exp(-lam), p = 1.0;
        uint64_t k = 0;
        do { ++k; p *= xo_unit_open0(r); } while (p > L);
        return k - 1;
    }
    double u1 = xo_unit_open0(r), u2 = xo_unit_open0(r);
    double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    double x = floor(lam + sqrt(lam) * z + 0.5);
    return x < 0 ? 0 : (uint64_t)x;
}

/* Chung-Lu power-law graph with exponent gamma and target mean degree dmean. */
gg_graph *gg_chunglu(int32_t n, double gamma, double dmean, uint64_t seed) {
    if (n < 0 || !(gamma > 1.0) || !(dmean >= 0.0)) return NULL;
    if (n < 2) return csr_from_pairs(n, NULL, 0);
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *cdf = (double *)malloc(((size_t)n + 1) * sizeof(double));
    if (!w || !cdf) { free(w); free(cdf); return NULL; }
    double s = 0;
    const double ex = -1.0 / (gamma - 1.0);
    for (int32_t i = 0; i < n; ++i) { w[i] = pow((double)i + 1.0, ex); s += w[i]; }
    const double scale = dmean * (double)n / s;
    const double cap = sqrt(dmean * (double)n);
    cdf[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        double wi = w[i] * scale;
        if (wi > cap) wi = cap;
        cdf[i + 1] = cdf[i] + wi;
    }
    const double S = cdf[n];
    xo256 r = xo_stream(seed, KIND_CL, 0);
    uint64_t M = poisson(&r, S / 2.0);
    uint64_t *pairs = (uint64_t *)malloc((M + 1) * sizeof(uint64_t));
    if (!pairs) { free(w); free(cdf); return NULL; }
    for (uint64_t e = 0; e < M; ++e) {
        uint64_t ends[2];
        for (int k = 0; k < 2; ++k) {
            double x = (double)(xo_next(&r) >> 11) * (1.0 / 9007199254740992.0) * S;
            int32_t lo = 0, hi = n - 1; /* largest i with cdf[i] <= x */
            while (lo < hi) {
                int32_t mid = lo + (hi - lo + 1) / 2;
                if (cdf[mid] <= x) lo = mid; else hi = mid - 1;
            }
            ends[k] = (uint64_t)lo;
        }
        pairs[e] = ends[0] * (uint64_t)n + ends[1];
    }
    gg_graph *g = csr_from_pairs(n, pairs, (size_t)M);
    free(pairs);
    free(w);
    free(cdf);
    return g;
}

/* Seeded uniform doubles in [0,1) for host-side recipes (sizes, arrivals). */
void gg_uniform(uint64_t seed, uint64_t stream, int64_t count, double *out) {
    xo256 r = xo_stream(seed, 0x5151, stream);
    for (int64_t i = 0; i < count; ++i) out[i] = (double)(xo_next(&r) >> 11) * (1.0 / 9007199254740992.0);
}
