/*
 * niorca_oracle.c -- ORACLE (test infrastructure, not the product).
 *
 * A plain, slow CPU implementation of NI-ORCA as the paper states it:
 *   Stage I   per-edge triangle counts            (Algorithm 1, Stage I; Sec. 6)
 *   Stage II  CountK4(x) for every x              (Algorithm 2; Sec. 6, Table 2 "ARR")
 *   Stage III the nine f* variables of Table 1 over the substructures of
 *             Fig. 3 (a)-(d), with the per-thread dense `common` array
 *             (Sec. 6, Table 3 "ARR (T)"), then the orbit equations of
 *             Sec. 5 (Eqs. o13, o12, o11, o10) and the Appendix (o9 .. o4).
 *
 * Only tests/, the smoke entry point and the CPU-baseline leg of the bench
 * may load or run this code. It shares no code with the CUDA path.
 *
 * Readings taken where the paper is ambiguous (each is pinned by the
 * brute-force definition in the tests; ORC_READ_* flags switch to the
 * rejected literal reading so that tests can show it fails):
 *   - Alg. 2: `neigh` is emptied for every y (it is declared once per x),
 *     the inner index runs j > i, and id comparisons are strict.
 *   - Fig. 3a/3b: every unordered triangle {x, y, z} is visited once.
 *   - Fig. 3d: the path x-y-z visits every y in N(x) and every z in N(y)
 *     with z != x and z not adjacent to x; `common[z]` counts such paths.
 *   - Table 1, f_6^9: neighbours of y other than x and z that do not close
 *     a triangle with the edge x-y, i.e. d_y - 2 - t_xy per path.
 *   - psi_1, psi_2, psi_3 are counted while probing (Sec. 5): paths x-y-z,
 *     pairs of neighbours, and adjacent pairs of neighbours.
 * All counts are int64; every halving in the equations is checked to be
 * exact and a failed check is reported as an error.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
    ORC_OK = 0,
    ORC_EODD = 1,     /* a halving in the equations had an odd numerator */
    ORC_ENOMEM = 2,
    ORC_EINVAL = 3,
};

/* Reading switches (tests only): each selects a rejected literal reading. */
enum {
    ORC_READ_F69_EYZ = 1,       /* f_6^9 with t_yz instead of t_xy            */
    ORC_READ_NEIGH_NO_RESET = 2,/* Alg. 2 neigh kept across y                 */
    ORC_READ_FIG3B_ORDERED = 4, /* Fig. 3b visited as ordered pairs           */
};

typedef struct {
    int32_t n;
    const int32_t *rp; /* rowptr, n + 1 */
    const int32_t *ci; /* colidx, rows sorted ascending */
} graph_t;

static inline int32_t deg(const graph_t *g, int32_t x) { return g->rp[x + 1] - g->rp[x]; }

/* position of b in the sorted row of a, or -1 */
static int64_t pos_in_row(const graph_t *g, int32_t a, int32_t b) {
    int64_t lo = g->rp[a], hi = (int64_t)g->rp[a + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t v = g->ci[mid];
        if (v == b) return mid;
        if (v < b) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static inline int is_edge(const graph_t *g, int32_t a, int32_t b) { return pos_in_row(g, a, b) >= 0; }

static int32_t max_degree(const graph_t *g) {
    int32_t m = 0;
    for (int32_t x = 0; x < g->n; ++x) if (deg(g, x) > m) m = deg(g, x);
    return m;
}

/* |N(x) ∩ N(y)| by merging the two sorted rows (the `common_neighbours` of Alg. 1). */
static int32_t common_neighbours(const graph_t *g, int32_t x, int32_t y) {
    int64_t i = g->rp[x], ie = g->rp[x + 1], j = g->rp[y], je = g->rp[y + 1];
    int32_t c = 0;
    /* skip-ahead by binary search when one row is much longer */
    int64_t lx = ie - i, ly = je - j;
    if (lx * 16 < ly || ly * 16 < lx) {
        int32_t s = lx <= ly ? x : y, t = lx <= ly ? y : x;
        for (int64_t p = g->rp[s]; p < g->rp[s + 1]; ++p) c += is_edge(g, t, g->ci[p]);
        return c;
    }
    while (i < ie && j < je) {
        int32_t a = g->ci[i], b = g->ci[j];
        if (a == b) { ++c; ++i; ++j; }
        else if (a < b) ++i;
        else ++j;
    }
    return c;
}

/* ------------------------------------------------------------- Stage I */

/*
 * Stage I (Algorithm 1): for every edge (x, y), tri = |common_neighbours(x, y)|.
 * Each undirected edge is intersected once (x < y) and the count is stored at
 * both CSR positions, so tri[p] is the triangle count of the edge at CSR
 * position p.
 */
void orc_stage1(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *tri) {
    graph_t g = {n, rowptr, colidx};
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t x = 0; x < n; ++x) {
        for (int64_t p = rowptr[x]; p < rowptr[x + 1]; ++p) {
            int32_t y = colidx[p];
            if (y <= x) continue;
            int32_t c = common_neighbours(&g, x, y);
            tri[p] = c;
            tri[pos_in_row(&g, y, x)] = c;
        }
    }
}

/* ------------------------------------------------------------ Stage II */

/*
 * Algorithm 2, CountK4(x): for y in N(x), y > x, collect in `neigh` every
 * z in N(y) with z > y and (x, z) in E; every adjacent pair of `neigh`
 * closes a K4 {x, y, z, z'} and all four counts are incremented. K4 is
 * shared between threads, so increments are atomic (Table 2, "ARR").
 */
static void count_k4(const graph_t *g, int32_t x, int64_t *K4, int32_t *neigh, int flags) {
    int32_t len = 0;
    for (int64_t p = g->rp[x]; p < g->rp[x + 1]; ++p) {
        int32_t y = g->ci[p];
        if (y <= x) continue;
        if (!(flags & ORC_READ_NEIGH_NO_RESET)) len = 0; /* neigh emptied for every y */
        for (int64_t q = g->rp[y]; q < g->rp[y + 1]; ++q) {
            int32_t z = g->ci[q];
            if (z <= y) continue;
            if (is_edge(g, x, z)) neigh[len++] = z;
        }
        for (int32_t i = 0; i < len; ++i) {
            int32_t z = neigh[i];
            for (int32_t j = i + 1; j < len; ++j) {
                int32_t zz = neigh[j];
                if (is_edge(g, z, zz)) {
#pragma omp atomic
                    K4[x]++;
#pragma omp atomic
                    K4[y]++;
#pragma omp atomic
                    K4[z]++;
#pragma omp atomic
                    K4[zz]++;
                }
            }
        }
    }
}

int orc_stage2(int32_t n, const int32_t *rowptr, const int32_t *colidx, int64_t *K4, int flags) {
    graph_t g = {n, rowptr, colidx};
    const int32_t maxdeg = max_degree(&g);
    memset(K4, 0, sizeof(int64_t) * (size_t)n);
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        /* per-thread neigh buffer; the rejected reading can overflow maxdeg,
           so it is sized for the sum of all out-degrees of one x */
        size_t cap = (flags & ORC_READ_NEIGH_NO_RESET) ? (size_t)maxdeg * (size_t)maxdeg + 1
                                                      : (size_t)maxdeg + 1;
        int32_t *neigh = (int32_t *)malloc(cap * sizeof(int32_t));
        if (!neigh) err |= 1;
        else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t x = 0; x < n; ++x) count_k4(&g, x, K4, neigh, flags);
        }
        free(neigh);
    }
    return err ? ORC_ENOMEM : ORC_OK;
}

/* ----------------------------------------------------------- Stage III */

typedef struct {
    int64_t f12_14, f10_13, f13_14, f11_13, f5_8, f6_9, f9_12, f4_8, f8_12;
    int64_t p1, p2, p3; /* psi_1..psi_3, counted while probing (Sec. 5) */
} fvars;

/* triangle count of the edge (a, b); `tri` is per CSR position, or NULL to
   intersect on demand */
static inline int64_t tri_ab(const graph_t *g, const int32_t *tri, int32_t a, int64_t pab, int32_t b) {
    if (tri) return tri[pab];
    return common_neighbours(g, a, b);
}

/*
 * Table 1 over the substructures of Fig. 3 for one vertex x.
 * `mark` and `common` are per-thread dense arrays of n entries that are zero
 * on entry and zero again on return (ARR (T) of Table 3).
 */
static void count_f_vars(const graph_t *g, const int32_t *tri, int32_t x, int32_t *mark, int32_t *common,
                         int32_t *ymark, int64_t *tx, fvars *f, int flags) {
    memset(f, 0, sizeof(*f));
    const int64_t dx = deg(g, x);
    const int64_t b = g->rp[x], e = g->rp[x + 1];
    for (int64_t p = b; p < e; ++p) {
        mark[g->ci[p]] = 1;
        tx[p - b] = tri_ab(g, tri, x, p, g->ci[p]); /* t_xy for every y in N(x) */
    }

    /* Fig. 3a, 3b (triangle x-y-z, each unordered pair once) and 3c (two-star) */
    for (int64_t i = b; i < e; ++i) {
        const int32_t y = g->ci[i];
        const int64_t dy = deg(g, y), txy = tx[i - b];
        for (int64_t j = i + 1; j < e; ++j) {
            const int32_t z = g->ci[j];
            const int64_t dz = deg(g, z), txz = tx[j - b];
            f->p2 += 1;
            const int64_t pyz = pos_in_row(g, y, z);
            if (pyz >= 0) {
                const int64_t tyz = tri_ab(g, tri, y, pyz, z);
                f->p3 += 1;
                f->f12_14 += tyz - 1;                                   /* Fig. 3a */
                f->f10_13 += (dy - 1 - tyz) + (dz - 1 - tyz);           /* Fig. 3a */
                int64_t k13 = (txy - 1) + (txz - 1);                    /* Fig. 3b */
                int64_t k11 = (dx - 1 - txy) + (dx - 1 - txz);          /* Fig. 3b */
                int mult = (flags & ORC_READ_FIG3B_ORDERED) ? 2 : 1;
                f->f13_14 += mult * k13;
                f->f11_13 += mult * k11;
            } else {
                f->f5_8 += (dy - 1 - txy) + (dz - 1 - txz);             /* Fig. 3c */
            }
        }
    }
    /* common[z]: induced 2-paths x-y-z with z outside N(x) ∪ {x} */
    for (int64_t i = b; i < e; ++i) {
        const int32_t y = g->ci[i];
        for (int64_t q = g->rp[y]; q < g->rp[y + 1]; ++q) {
            const int32_t z = g->ci[q];
            if (z != x && !mark[z]) common[z]++;
        }
    }
    /* Fig. 3d: the path x-y-z; psi_1 counts every path x-y-z with z != x */
    for (int64_t i = b; i < e; ++i) {
        const int32_t y = g->ci[i];
        const int64_t dy = deg(g, y), txy = tx[i - b];
        /* without a Stage I table, |N(y) ∩ N(z)| is counted against a marker
           array of N(y) when N(z) is the shorter row */
        const int use_ymark = (tri == NULL) && dy >= 64;
        if (use_ymark)
            for (int64_t q = g->rp[y]; q < g->rp[y + 1]; ++q) ymark[g->ci[q]] = 1;
        for (int64_t q = g->rp[y]; q < g->rp[y + 1]; ++q) {
            const int32_t z = g->ci[q];
            if (z == x) continue;
            f->p1 += 1;
            if (mark[z]) continue;
            const int64_t dz = deg(g, z);
            int64_t tyz;
            if (use_ymark && dz < dy) {
                tyz = 0;
                for (int64_t r = g->rp[z]; r < g->rp[z + 1]; ++r) tyz += ymark[g->ci[r]];
            } else {
                tyz = tri_ab(g, tri, y, q, z);
            }
            if (flags & ORC_READ_F69_EYZ) f->f6_9 += dy - 2 - tyz;
            else f->f6_9 += dy - 2 - txy;
            f->f9_12 += tyz;
            f->f4_8 += dz - 1 - tyz;
            f->f8_12 += common[z] - 1;
        }
        if (use_ymark)
            for (int64_t q = g->rp[y]; q < g->rp[y + 1]; ++q) ymark[g->ci[q]] = 0;
    }
    for (int64_t i = b; i < e; ++i) {
        const int32_t y = g->ci[i];
        for (int64_t q = g->rp[y]; q < g->rp[y + 1]; ++q) common[g->ci[q]] = 0;
    }
    for (int64_t p = b; p < e; ++p) mark[g->ci[p]] = 0;
}

static inline int64_t choose2(int64_t a) { return a < 2 ? 0 : a * (a - 1) / 2; }
static inline int64_t choose3(int64_t a) { return a < 3 ? 0 : a * (a - 1) / 2 * (a - 2) / 3; }

/*
 * Sec. 5 and the Appendix: the orbit counts of x from the f* variables.
 * `mutation` (tests only, 0 = none) perturbs one term so that tests can show
 * that the pins detect it.
 */
static int solve_equations(const fvars *f, int64_t dx, int64_t k4, int64_t *psi, int mutation) {
    const int64_t f12 = f->f12_14, f10 = f->f10_13, f13 = f->f13_14, f11 = f->f11_13;
    const int64_t f5 = f->f5_8, f6 = f->f6_9, f9 = f->f9_12, f4 = f->f4_8, f8 = f->f8_12;
    int err = 0;
    if ((f13 & 1) || ((f11 + f13) & 1) || (f9 & 1) || ((f13 + f8) & 1) || ((f6 - f13) & 1)) err = ORC_EODD;
    psi[0] = dx;                                   /* deg[x] */
    psi[1] = f->p1;
    psi[2] = f->p2;
    psi[3] = f->p3;
    psi[14] = k4;                                  /* K4[x] from Stage II */
    psi[13] = f13 / 2;                             /* Eq. o13 */
    psi[12] = f12;                                 /* Eq. o12 */
    psi[11] = (f11 + f13) / 2;                     /* Eq. o11 */
    psi[10] = f10 + 2 * f12;                       /* Eq. o10 */
    psi[9] = f12 + f9 / 2;                         /* Appendix, o9 */
    psi[8] = (f13 + f8) / 2;                       /* Appendix, o8 */
    psi[7] = choose3(dx);                          /* Appendix, o7 = C(psi_0, 3) */
    psi[6] = (f6 - f13) / 2 + f10 + 2 * f12;       /* Appendix, o6 */
    psi[5] = 2 * f12 + f5 + f10 + f11;             /* Appendix, o5 */
    psi[4] = 2 * f12 + f4 + f10 + f9;              /* Appendix, o4 */
    switch (mutation) {                            /* planted mistakes for pin tests */
    case 1: psi[4] = 2 * f12 + f4 + f9; break;             /* dropped f10 in o4 */
    case 2: psi[5] = 2 * f12 + f5 + f10 - f11; break;      /* sign of f11 in o5 */
    case 3: psi[6] = (f6 + f13) / 2 + f10 + 2 * f12; break;/* sign of f13 in o6 */
    case 4: psi[8] = (f13 + f8); break;                    /* missing halving */
    case 5: psi[9] = f12 + f9; break;                      /* missing halving */
    case 6: psi[10] = f10 + f12; break;                    /* factor 2 dropped */
    case 7: psi[11] = (f11 - f13) / 2; break;              /* sign */
    case 8: psi[12] = f10; break;                          /* transposed operand */
    case 9: psi[13] = f11 / 2; break;                      /* transposed operand */
    case 10: psi[7] = choose2(dx); break;                  /* wrong binomial */
    case 11: psi[1] = f->p2; break;                        /* transposed */
    case 12: psi[3] = f->p3 * 2; break;                    /* double count */
    default: break;
    }
    return err;
}

/* Stage III for all vertices (Algorithm 1, Stage III), using tri and K4. */
int orc_stage3(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *tri, const int64_t *K4,
               int64_t *out, int flags, int mutation) {
    graph_t g = {n, rowptr, colidx};
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        int32_t *mark = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int32_t *common = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int32_t *ymark = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int64_t *tx = (int64_t *)malloc(((size_t)max_degree(&g) + 1) * sizeof(int64_t));
        if (!mark || !common || !ymark || !tx) err |= ORC_ENOMEM;
        else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t x = 0; x < n; ++x) {
                fvars f;
                count_f_vars(&g, tri, x, mark, common, ymark, tx, &f, flags);
                err |= solve_equations(&f, deg(&g, x), K4[x], out + (size_t)x * 15, mutation);
            }
        }
        free(mark);
        free(common);
        free(ymark);
        free(tx);
    }
    return err;
}

/* Set the OpenMP thread count for subsequent calls (0 = leave unchanged). */
void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* All three stages (Algorithm 1). out: n x 15 int64, row-major. */
int orc_count(int32_t n, const int32_t *rowptr, const int32_t *colidx, int64_t *out, int flags, int mutation) {
    if (n < 0) return ORC_EINVAL;
    const int64_t m = rowptr[n];
    int32_t *tri = (int32_t *)malloc(((size_t)m + 1) * sizeof(int32_t));
    int64_t *K4 = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int err = ORC_OK;
    if (!tri || !K4) err = ORC_ENOMEM;
    if (!err) orc_stage1(n, rowptr, colidx, tri);
    if (!err) err = orc_stage2(n, rowptr, colidx, K4, flags);
    if (!err) err = orc_stage3(n, rowptr, colidx, tri, K4, out, flags, mutation);
    free(tri);
    free(K4);
    return err;
}

/*
 * K4 containing x, by definition: triples y < z < w of N(x) that are
 * pairwise adjacent (used where Stage II is not run for the whole graph).
 */
static int64_t k4_of_vertex(const graph_t *g, int32_t x) {
    int64_t c = 0;
    const int64_t b = g->rp[x], e = g->rp[x + 1];
    for (int64_t i = b; i < e; ++i)
        for (int64_t j = i + 1; j < e; ++j) {
            int32_t y = g->ci[i], z = g->ci[j];
            if (!is_edge(g, y, z)) continue;
            for (int64_t k = j + 1; k < e; ++k) {
                int32_t w = g->ci[k];
                if (is_edge(g, y, w) && is_edge(g, z, w)) ++c;
            }
        }
    return c;
}

/*
 * Orbit counts of selected vertices only (for graphs too large for the full
 * oracle): Stage III's f* for each listed x with triangle counts intersected
 * on demand, and psi_14 from the K4s that contain x.
 */
int orc_count_vertices(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t nq, const int32_t *verts,
                       int64_t *out, int flags, int mutation) {
    graph_t g = {n, rowptr, colidx};
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        int32_t *mark = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int32_t *common = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int32_t *ymark = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int64_t *tx = (int64_t *)malloc(((size_t)max_degree(&g) + 1) * sizeof(int64_t));
        if (!mark || !common || !ymark || !tx) err |= ORC_ENOMEM;
        else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t i = 0; i < nq; ++i) {
                const int32_t x = verts[i];
                if (x < 0 || x >= n) { err |= ORC_EINVAL; continue; }
                fvars f;
                count_f_vars(&g, NULL, x, mark, common, ymark, tx, &f, flags);
                err |= solve_equations(&f, deg(&g, x), k4_of_vertex(&g, x), out + (size_t)i * 15, mutation);
            }
        }
        free(mark);
        free(common);
        free(ymark);
        free(tx);
    }
    return err;
}
