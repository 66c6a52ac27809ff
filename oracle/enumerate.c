/*
 * enumerate.c -- ORACLE (test infrastructure, not the product).
 *
 * Non-induced orbit counts straight from the definitions (Defs. 1-5, Sec. 3):
 * psi_k(x) is the number of subgraphs (V', E') of G with |V'| <= 4,
 * E' a subset of the edges of G inside V', (V', E') connected, in which x
 * sits in orbit k. Every connected vertex set V' of size 2..4 is listed once
 * with the ESU algorithm (Wernicke, "Efficient detection of network motifs",
 * IEEE/ACM TCBB 2006); for each, every subset E' of its induced edges that
 * connects all of V' is classified, and each vertex is credited with its
 * orbit.
 *
 * Orbit numbering (the paper's Fig. 2 is missing from the text; this is the
 * numbering under which every printed equation holds, checked by the tests):
 *   0 edge; 1 path-P3 end, 2 P3 middle; 3 triangle; 4 P4 end, 5 P4 interior;
 *   6 3-star leaf, 7 3-star centre; 8 4-cycle; 9 paw degree-1 vertex,
 *   10 paw degree-2 vertex, 11 paw degree-3 vertex; 12 diamond degree-2
 *   vertex, 13 diamond degree-3 vertex; 14 K4.
 * Within each graphlet the orbit is fixed by the vertex's degree in E'.
 *
 * Only tests/ may load this code. It shares no code with the CUDA path or
 * with the three-stage oracle.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    const int32_t *rp;
    const int32_t *ci;
} dgraph;

static int adjacent(const dgraph *g, int32_t a, int32_t b) {
    int64_t lo = g->rp[a], hi = (int64_t)g->rp[a + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t v = g->ci[mid];
        if (v == b) return 1;
        if (v < b) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

/* orbit of a vertex of subgraph degree `dv` in a connected graphlet with k
   vertices, `ne` edges and maximum degree `dmax` and all-degree-2 flag */
static int orbit_of(int k, int ne, int dv, int dmax, int regular2) {
    if (k == 2) return 0;
    if (k == 3) return ne == 3 ? 3 : (dv == 1 ? 1 : 2);
    switch (ne) {
    case 3: return dmax == 3 ? (dv == 3 ? 7 : 6) : (dv == 1 ? 4 : 5);
    case 4: return regular2 ? 8 : (dv == 1 ? 9 : (dv == 2 ? 10 : 11));
    case 5: return dv == 2 ? 12 : 13;
    default: return 14;
    }
}

static int uf_find(int *p, int a) {
    while (p[a] != a) a = p[a] = p[p[a]];
    return a;
}

/*
 * Credit every connected spanning edge subset of the vertex set s[0..k-1].
 * If `only` >= 0, only that vertex is credited and `out` is its 15-entry row;
 * otherwise `out` is the n x 15 table.
 */
static int g_induced = 0;  /* 1: only E' = every edge inside V' (Def. 2) */

static void credit_set(const dgraph *g, const int32_t *s, int k, int64_t *out, int32_t only) {
    int ea[6], eb[6], ne = 0;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j)
            if (adjacent(g, s[i], s[j])) { ea[ne] = i; eb[ne] = j; ++ne; }
    for (int mask = g_induced ? (1 << ne) - 1 : 1; mask < (1 << ne); ++mask) {
        int dv[4] = {0, 0, 0, 0}, par[4] = {0, 1, 2, 3}, cnt = 0, comps = k;
        for (int e = 0; e < ne; ++e) {
            if (!((mask >> e) & 1)) continue;
            ++cnt;
            dv[ea[e]]++;
            dv[eb[e]]++;
            int ra = uf_find(par, ea[e]), rb = uf_find(par, eb[e]);
            if (ra != rb) { par[ra] = rb; --comps; }
        }
        if (comps != 1) continue;
        int dmax = 0, reg2 = 1;
        for (int i = 0; i < k; ++i) {
            if (dv[i] > dmax) dmax = dv[i];
            if (dv[i] != 2) reg2 = 0;
        }
        for (int i = 0; i < k; ++i) {
            if (only >= 0 && s[i] != only) continue;
            int o = orbit_of(k, cnt, dv[i], dmax, reg2);
            if (only >= 0) { out[o]++; continue; }
#pragma omp atomic
            out[(size_t)s[i] * 15 + o]++;
        }
    }
}

/* ESU extension: sub has k vertices, ext lists candidates; `root` is the
   first vertex; in whole-graph mode only vertices above it may join. */
static void esu_extend(const dgraph *g, int32_t *sub, int k, const int32_t *ext, int next, int32_t root,
                       int whole, int64_t *out, int32_t only) {
    if (k >= 2) credit_set(g, sub, k, out, only);
    if (k == 4) return;
    int32_t *work = (int32_t *)malloc(((size_t)next + 1) * sizeof(int32_t));
    if (!work) return;
    memcpy(work, ext, (size_t)next * sizeof(int32_t));
    int left = next;
    while (left > 0) {
        int32_t w = work[--left];
        /* new extension = remaining candidates + exclusive neighbours of w */
        size_t cap = (size_t)left + (size_t)(g->rp[w + 1] - g->rp[w]) + 1;
        int32_t *next_ext = (int32_t *)malloc(cap * sizeof(int32_t));
        if (!next_ext) break;
        memcpy(next_ext, work, (size_t)left * sizeof(int32_t));
        int nn = left;
        for (int64_t p = g->rp[w]; p < g->rp[w + 1]; ++p) {
            int32_t u = g->ci[p];
            if (whole && u <= root) continue;
            int excl = 1;
            for (int i = 0; i < k && excl; ++i)
                if (u == sub[i] || adjacent(g, u, sub[i])) excl = 0;
            if (excl) next_ext[nn++] = u;
        }
        sub[k] = w;
        esu_extend(g, sub, k + 1, next_ext, nn, root, whole, out, only);
        free(next_ext);
    }
    free(work);
}

static void esu_root(const dgraph *g, int32_t v, int whole, int64_t *out, int32_t only) {
    int32_t sub[4];
    sub[0] = v;
    int64_t d = g->rp[v + 1] - g->rp[v];
    int32_t *ext = (int32_t *)malloc(((size_t)d + 1) * sizeof(int32_t));
    if (!ext) return;
    int nn = 0;
    for (int64_t p = g->rp[v]; p < g->rp[v + 1]; ++p)
        if (!whole || g->ci[p] > v) ext[nn++] = g->ci[p];
    esu_extend(g, sub, 1, ext, nn, v, whole, out, only);
    free(ext);
}

/* All vertices: out is n x 15 int64, zeroed here. */
void def_count(int32_t n, const int32_t *rowptr, const int32_t *colidx, int64_t *out) {
    dgraph g = {n, rowptr, colidx};
    g_induced = 0;
    memset(out, 0, sizeof(int64_t) * 15 * (size_t)n);
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t v = 0; v < n; ++v) esu_root(&g, v, 1, out, -1);
}

/*
 * Selected vertices: every connected set that contains x is listed from x
 * (ESU rooted at x without the ordering filter) and only x is credited.
 * out is nq x 15 int64.
 */
void def_count_vertices(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t nq, const int32_t *verts,
                        int64_t *out) {
    dgraph g = {n, rowptr, colidx};
    g_induced = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < nq; ++i) {
        int64_t *row = out + (size_t)i * 15;
        memset(row, 0, 15 * sizeof(int64_t));
        int32_t x = verts[i];
        if (x < 0 || x >= n) continue;
        esu_root(&g, x, 0, row, x);
    }
}

/*
 * Induced orbit counts by definition (Def. 2: E' is every edge of G inside
 * V'): the same enumeration with only the full induced edge set kept.
 */
void def_count_induced(int32_t n, const int32_t *rowptr, const int32_t *colidx, int64_t *out) {
    dgraph g = {n, rowptr, colidx};
    memset(out, 0, sizeof(int64_t) * 15 * (size_t)n);
    g_induced = 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t v = 0; v < n; ++v) esu_root(&g, v, 1, out, -1);
    g_induced = 0;
}
