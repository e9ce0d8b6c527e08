/*
 * CPU oracle for the join-aggregate hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C (fp64 / uint64) that computes the result
 * each query is DEFINED to have (AJAR semantics, Section 2.3: join tuples
 * multiply annotations, the aggregation sums them), not the method's way of
 * reaching it.  Only tests/, __graft_entry__.smoke() and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or
 * constant with the CUDA path.
 *
 * Conventions: a graph relation E is a SET of oriented pairs (a, b) with
 * a < b (inputs are deduplicated here); sums use Neumaier compensation in
 * fp64; OpenMP only splits independent outer loops.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---------------------------------------------------------------- sums */
typedef struct { double s, c; } neu_t;   /* Neumaier running sum */

static inline void neu_add(neu_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double neu_val(const neu_t *a) { return a->s + a->c; }

/* ------------------------------------------------------- sorted edge set */
static int cmp_u64(const void *x, const void *y) {
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

/* Edge set as sorted unique packed keys (a<<32|b) plus a CSR adjacency of
 * out-neighbours (b > a), sorted. */
typedef struct {
    uint64_t m;         /* distinct edges */
    uint32_t n;         /* 1 + max vertex id */
    uint64_t *key;      /* sorted packed keys */
    uint64_t *off;      /* n+1 */
    uint32_t *adj;      /* m */
} eset_t;

static void eset_build(eset_t *E, uint64_t m, const uint32_t *src, const uint32_t *dst) {
    uint64_t *k = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t w = 0;
    uint32_t n = 0;
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = src[i], b = dst[i];
        if (a == b) continue;
        if (a > b) { uint32_t t = a; a = b; b = t; }
        k[w++] = ((uint64_t)a << 32) | b;
        if (b + 1 > n) n = b + 1;
    }
    qsort(k, w, sizeof(uint64_t), cmp_u64);
    uint64_t u = 0;
    for (uint64_t i = 0; i < w; ++i)
        if (i == 0 || k[i] != k[i - 1]) k[u++] = k[i];
    E->m = u; E->n = n; E->key = k;
    E->off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    E->adj = (uint32_t *)malloc((u ? u : 1) * sizeof(uint32_t));
    for (uint64_t i = 0; i < u; ++i) E->off[(k[i] >> 32) + 1]++;
    for (uint32_t v = 0; v < n; ++v) E->off[v + 1] += E->off[v];
    for (uint64_t i = 0; i < u; ++i) E->adj[i] = (uint32_t)k[i];  /* keys sorted => CSR order */
}

static void eset_free(eset_t *E) { free(E->key); free(E->off); free(E->adj); }

static int eset_has(const eset_t *E, uint32_t a, uint32_t b) {
    if (a >= E->n) return 0;
    uint64_t lo = E->off[a], hi = E->off[a + 1];
    while (lo < hi) {                       /* binary search in adj+(a) */
        uint64_t mid = (lo + hi) / 2;
        if (E->adj[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < E->off[a + 1] && E->adj[lo] == b;
}

/* --------------------------------------------------------- graph counts */

/* Triangle join R(a,b) S(b,c) T(a,c) over three (possibly different) edge
 * sets: for each (a,b) in R and each c with (b,c) in S, test (a,c) in T. */
uint64_t orc_join_rst_count(uint64_t mR, const uint32_t *Ra, const uint32_t *Rb,
                            uint64_t mS, const uint32_t *Sb, const uint32_t *Sc,
                            uint64_t mT, const uint32_t *Ta, const uint32_t *Tc) {
    eset_t R, S, T;
    eset_build(&R, mR, Ra, Rb); eset_build(&S, mS, Sb, Sc); eset_build(&T, mT, Ta, Tc);
    uint64_t cnt = 0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+:cnt)
    for (int64_t e = 0; e < (int64_t)R.m; ++e) {
        uint32_t a = (uint32_t)(R.key[e] >> 32), b = (uint32_t)R.key[e];
        if (b >= S.n) continue;
        for (uint64_t j = S.off[b]; j < S.off[b + 1]; ++j)
            cnt += (uint64_t)eset_has(&T, a, S.adj[j]);
    }
    eset_free(&R); eset_free(&S); eset_free(&T);
    return cnt;
}

uint64_t orc_triangle_count(uint64_t m, const uint32_t *src, const uint32_t *dst) {
    return orc_join_rst_count(m, src, dst, m, src, dst, m, src, dst);
}

/* Triangle count of the undirected graph (each triangle once) by a
 * different route than the join above: every edge is oriented from its
 * endpoint of lower (degree, id) to the higher one, so each triangle has
 * exactly one vertex u whose two out-neighbours v, w close it; per u the
 * out-set N+(u) is marked and every 2-path u -> v -> w with w marked counts.
 * The join R(a,b) S(b,c) T(a,c) over the id-oriented edge set has one
 * result per triangle as well (Section 2.4: the count is the same whatever
 * orientation the relations use). */
uint64_t orc_triangle_count_degree(uint64_t m, const uint32_t *src, const uint32_t *dst) {
    eset_t E; eset_build(&E, m, src, dst);
    const uint32_t n = E.n;
    uint64_t *deg = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < E.m; ++i) { deg[E.key[i] >> 32]++; deg[(uint32_t)E.key[i]]++; }
    /* out-degree under the degree order, then the oriented CSR */
    uint64_t *off = (uint64_t *)calloc((size_t)n + 2, sizeof(uint64_t));
    #define ORC_BEFORE(x, y) (deg[x] < deg[y] || (deg[x] == deg[y] && (x) < (y)))
    for (uint64_t i = 0; i < E.m; ++i) {
        uint32_t a = (uint32_t)(E.key[i] >> 32), b = (uint32_t)E.key[i];
        off[(ORC_BEFORE(a, b) ? a : b) + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) off[v + 1] += off[v];
    uint32_t *adj = (uint32_t *)malloc((E.m ? E.m : 1) * sizeof(uint32_t));
    uint64_t *fill = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    memcpy(fill, off, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < E.m; ++i) {
        uint32_t a = (uint32_t)(E.key[i] >> 32), b = (uint32_t)E.key[i];
        if (ORC_BEFORE(a, b)) adj[fill[a]++] = b; else adj[fill[b]++] = a;
    }
    #undef ORC_BEFORE
    free(fill);
    uint64_t cnt = 0;
    #pragma omp parallel reduction(+:cnt)
    {
        uint8_t *mark = (uint8_t *)calloc((size_t)n + 1, 1);
        #pragma omp for schedule(dynamic, 64)
        for (int64_t u = 0; u < (int64_t)n; ++u) {
            for (uint64_t i = off[u]; i < off[u + 1]; ++i) mark[adj[i]] = 1;
            for (uint64_t i = off[u]; i < off[u + 1]; ++i) {
                uint32_t v = adj[i];
                for (uint64_t j = off[v]; j < off[v + 1]; ++j) cnt += mark[adj[j]];
            }
            for (uint64_t i = off[u]; i < off[u + 1]; ++i) mark[adj[i]] = 0;
        }
        free(mark);
    }
    free(adj); free(off); free(deg);
    eset_free(&E);
    return cnt;
}

/* 4-clique join E(a,b)E(a,c)E(a,d)E(b,c)E(b,d)E(c,d). */
uint64_t orc_clique4_count(uint64_t m, const uint32_t *src, const uint32_t *dst) {
    eset_t E; eset_build(&E, m, src, dst);
    uint64_t cnt = 0;
    #pragma omp parallel for schedule(dynamic, 64) reduction(+:cnt)
    for (int64_t e = 0; e < (int64_t)E.m; ++e) {
        uint32_t a = (uint32_t)(E.key[e] >> 32), b = (uint32_t)E.key[e];
        for (uint64_t i = E.off[a]; i < E.off[a + 1]; ++i) {
            uint32_t c = E.adj[i];
            if (!eset_has(&E, b, c)) continue;               /* c in adj+(a) and adj+(b) */
            for (uint64_t j = E.off[a]; j < E.off[a + 1]; ++j) {
                uint32_t d = E.adj[j];
                if (eset_has(&E, b, d) && eset_has(&E, c, d)) cnt++;
            }
        }
    }
    eset_free(&E);
    return cnt;
}

/* 4-cycle join E(a,b)E(b,c)E(c,d)E(a,d).  Per a: P[c] = number of b with
 * (a,b),(b,c) in E; then add P[c] * |{d : (c,d) in E and (a,d) in E}|. */
uint64_t orc_cycle4_count(uint64_t m, const uint32_t *src, const uint32_t *dst) {
    eset_t E; eset_build(&E, m, src, dst);
    uint64_t cnt = 0;
    #pragma omp parallel reduction(+:cnt)
    {
        uint64_t *P = (uint64_t *)calloc((size_t)E.n + 1, sizeof(uint64_t));
        uint8_t *inA = (uint8_t *)calloc((size_t)E.n + 1, 1);
        uint32_t *touched = (uint32_t *)malloc(((size_t)E.n + 1) * sizeof(uint32_t));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < (int64_t)E.n; ++a) {
            uint64_t nt = 0;
            for (uint64_t i = E.off[a]; i < E.off[a + 1]; ++i) inA[E.adj[i]] = 1;
            for (uint64_t i = E.off[a]; i < E.off[a + 1]; ++i) {
                uint32_t b = E.adj[i];
                for (uint64_t j = E.off[b]; j < E.off[b + 1]; ++j) {
                    uint32_t c = E.adj[j];
                    if (P[c]++ == 0) touched[nt++] = c;
                }
            }
            for (uint64_t t = 0; t < nt; ++t) {
                uint32_t c = touched[t];
                uint64_t q = 0;
                for (uint64_t j = E.off[c]; j < E.off[c + 1]; ++j) q += inA[E.adj[j]];
                cnt += P[c] * q;
                P[c] = 0;
            }
            for (uint64_t i = E.off[a]; i < E.off[a + 1]; ++i) inA[E.adj[i]] = 0;
        }
        free(P); free(inA); free(touched);
    }
    eset_free(&E);
    return cnt;
}

/* Lollipop join E(a,b)E(b,c)E(a,c)E(c,d): sum over triangles (a,b,c) of the
 * out-degree of c. */
uint64_t orc_lollipop_count(uint64_t m, const uint32_t *src, const uint32_t *dst) {
    eset_t E; eset_build(&E, m, src, dst);
    uint64_t cnt = 0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+:cnt)
    for (int64_t e = 0; e < (int64_t)E.m; ++e) {
        uint32_t a = (uint32_t)(E.key[e] >> 32), b = (uint32_t)E.key[e];
        if (b >= E.n) continue;
        for (uint64_t j = E.off[b]; j < E.off[b + 1]; ++j) {
            uint32_t c = E.adj[j];
            if (eset_has(&E, a, c)) cnt += (c < E.n) ? (E.off[c + 1] - E.off[c]) : 0;
        }
    }
    eset_free(&E);
    return cnt;
}

/* |A cap B| of two sorted duplicate-free uint32 arrays by a plain merge. */
uint64_t orc_intersect_count(uint64_t na, const uint32_t *A, uint64_t nb, const uint32_t *B) {
    uint64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (A[i] < B[j]) ++i;
        else if (A[i] > B[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* ------------------------------------------------------------ sparse LA */

/* y(i) = sum_j A(i,j) x(j) over COO triples; also absy(i) = sum_j |A(i,j) x(j)|
 * for componentwise error bounds. */
void orc_spmv(uint64_t nnz, const uint32_t *row, const uint32_t *col, const float *val,
              uint32_t nrows, const float *x, double *y, double *absy) {
    neu_t *acc = (neu_t *)calloc(nrows, sizeof(neu_t));
    for (uint32_t i = 0; i < nrows; ++i) absy[i] = 0.0;
    for (uint64_t e = 0; e < nnz; ++e) {
        double t = (double)val[e] * (double)x[col[e]];
        neu_add(&acc[row[e]], t);
        absy[row[e]] += fabs(t);
    }
    for (uint32_t i = 0; i < nrows; ++i) y[i] = neu_val(&acc[i]);
    free(acc);
}

/* CSR view built from COO by counting sort on the row (stable). */
typedef struct { uint32_t n; uint64_t *off; uint32_t *col; float *val; } csr_t;

static void csr_from_coo(csr_t *M, uint32_t nrows, uint64_t nnz, const uint32_t *row,
                         const uint32_t *col, const float *val) {
    M->n = nrows;
    M->off = (uint64_t *)calloc((size_t)nrows + 1, sizeof(uint64_t));
    M->col = (uint32_t *)malloc((nnz ? nnz : 1) * sizeof(uint32_t));
    M->val = (float *)malloc((nnz ? nnz : 1) * sizeof(float));
    for (uint64_t e = 0; e < nnz; ++e) M->off[row[e] + 1]++;
    for (uint32_t i = 0; i < nrows; ++i) M->off[i + 1] += M->off[i];
    uint64_t *fill = (uint64_t *)malloc(((size_t)nrows + 1) * sizeof(uint64_t));
    memcpy(fill, M->off, ((size_t)nrows + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < nnz; ++e) {
        uint64_t p = fill[row[e]]++;
        M->col[p] = col[e]; M->val[p] = val[e];
    }
    free(fill);
}
static void csr_free(csr_t *M) { free(M->off); free(M->col); free(M->val); }

/* C(i,k) = sum_j A(i,j) B(j,k) for the selected rows i (Gustavson's row-wise
 * product with a dense accumulator).  Output per selected row: its distinct k
 * in ascending order, the fp64 value and sum_j |A(i,j) B(j,k)|.  Pass 1
 * (out==NULL) returns per-row counts in cnt[]; pass 2 fills at offsets
 * ooff[] (size nsel+1). */
void orc_spgemm_rows(uint32_t nrowsA, uint64_t nnzA, const uint32_t *Ar, const uint32_t *Ac,
                     const float *Av, uint32_t nrowsB, uint64_t nnzB, const uint32_t *Br,
                     const uint32_t *Bc, const float *Bv, uint32_t ncolsB,
                     uint64_t nsel, const uint32_t *sel, uint64_t *cnt,
                     const uint64_t *ooff, uint32_t *ocol, double *oval, double *oabs) {
    csr_t A, B;
    csr_from_coo(&A, nrowsA, nnzA, Ar, Ac, Av);
    csr_from_coo(&B, nrowsB, nnzB, Br, Bc, Bv);
    #pragma omp parallel
    {
        neu_t *acc = (neu_t *)calloc(ncolsB, sizeof(neu_t));
        double *aab = (double *)calloc(ncolsB, sizeof(double));
        uint8_t *flag = (uint8_t *)calloc(ncolsB, 1);
        uint32_t *list = (uint32_t *)malloc((size_t)ncolsB * sizeof(uint32_t));
        #pragma omp for schedule(dynamic, 64)
        for (int64_t s = 0; s < (int64_t)nsel; ++s) {
            uint32_t i = sel[s];
            uint64_t nl = 0;
            for (uint64_t p = A.off[i]; p < A.off[i + 1]; ++p) {
                uint32_t j = A.col[p];
                if (j >= B.n) continue;
                for (uint64_t q = B.off[j]; q < B.off[j + 1]; ++q) {
                    uint32_t k = B.col[q];
                    double t = (double)A.val[p] * (double)B.val[q];
                    if (!flag[k]) { flag[k] = 1; list[nl++] = k; }
                    neu_add(&acc[k], t);
                    aab[k] += fabs(t);
                }
            }
            /* ascending k: insertion into a sorted list is plain and fine for
             * the few hundred entries of a row */
            for (uint64_t x = 1; x < nl; ++x) {
                uint32_t v = list[x]; uint64_t y = x;
                while (y > 0 && list[y - 1] > v) { list[y] = list[y - 1]; --y; }
                list[y] = v;
            }
            if (!ocol) cnt[s] = nl;
            for (uint64_t x = 0; x < nl; ++x) {
                uint32_t k = list[x];
                if (ocol) {
                    ocol[ooff[s] + x] = k;
                    oval[ooff[s] + x] = neu_val(&acc[k]);
                    oabs[ooff[s] + x] = aab[k];
                }
                acc[k].s = 0; acc[k].c = 0; aab[k] = 0; flag[k] = 0;
            }
        }
        free(acc); free(aab); free(flag); free(list);
    }
    csr_free(&A); csr_free(&B);
}

/* ----------------------------------------------------------- star schema */

/* SUM(price * (1 - disc/100)) over fact rows that pass
 *   f1lo <= d1_date[k1] <= f1hi  and  f2lo <= d2_cat[k2] <= f2hi,
 * GROUP BY (d3_grp[k3], d4_region[k4]) -> group g = g1 * n_g2 + g2.
 * A pairwise hash join: each dimension is addressed by its key (the keys are
 * dense 0..|D|-1, so the "hash" is the key itself). */
void orc_star_sum(uint64_t nfact, const uint32_t *k1, const uint32_t *k2, const uint32_t *k3,
                  const uint32_t *k4, const double *price, const int8_t *disc,
                  const int32_t *d1_date, int32_t f1lo, int32_t f1hi,
                  const int32_t *d2_cat, int32_t f2lo, int32_t f2hi,
                  const int32_t *d3_grp, const int32_t *d4_region, uint32_t n_g2,
                  uint32_t ngroups, double *gsum, uint64_t *gcnt) {
    int nt = orc_num_threads();
    neu_t *part = (neu_t *)calloc((size_t)nt * ngroups, sizeof(neu_t));
    uint64_t *pc = (uint64_t *)calloc((size_t)nt * ngroups, sizeof(uint64_t));
    #pragma omp parallel
    {
#ifdef _OPENMP
        int t = omp_get_thread_num();
#else
        int t = 0;
#endif
        neu_t *my = part + (size_t)t * ngroups;
        uint64_t *mc = pc + (size_t)t * ngroups;
        #pragma omp for schedule(static)
        for (int64_t r = 0; r < (int64_t)nfact; ++r) {
            int32_t dd = d1_date[k1[r]], cc = d2_cat[k2[r]];
            if (dd < f1lo || dd > f1hi || cc < f2lo || cc > f2hi) continue;
            uint32_t g = (uint32_t)d3_grp[k3[r]] * n_g2 + (uint32_t)d4_region[k4[r]];
            neu_add(&my[g], price[r] * (1.0 - (double)disc[r] / 100.0));
            mc[g]++;
        }
    }
    for (uint32_t g = 0; g < ngroups; ++g) {
        neu_t a = {0, 0};
        uint64_t c = 0;
        for (int t = 0; t < nt; ++t) {
            neu_add(&a, part[(size_t)t * ngroups + g].s);
            neu_add(&a, part[(size_t)t * ngroups + g].c);
            c += pc[(size_t)t * ngroups + g];
        }
        gsum[g] = neu_val(&a);
        gcnt[g] = c;
    }
    free(part); free(pc);
}

/* Fact rows passing f1lo <= d1_date[k1] <= f1hi and f2lo <= d2_cat[k2] <=
 * f2hi (pass[r] = 1) and every row's price * (1 - disc/100) in fp64: the
 * selections and the aggregated expression of the star join, with no
 * grouping (the caller forms key tuples). */
void orc_star_pass(uint64_t nfact, const uint32_t *k1, const uint32_t *k2, const double *price,
                   const int8_t *disc, const int32_t *d1_date, int32_t f1lo, int32_t f1hi,
                   const int32_t *d2_cat, int32_t f2lo, int32_t f2hi, uint8_t *pass, double *val) {
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < (int64_t)nfact; ++r) {
        int32_t dd = d1_date[k1[r]], cc = d2_cat[k2[r]];
        pass[r] = (dd >= f1lo && dd <= f1hi && cc >= f2lo && cc <= f2hi) ? 1 : 0;
        val[r] = price[r] * (1.0 - (double)disc[r] / 100.0);
    }
}

/* Per-group Neumaier sums and counts of values v[i] in group gid[i]. */
void orc_group_sum(uint64_t n, const uint64_t *gid, const double *v, uint64_t ngroups, double *sum,
                   uint64_t *cnt) {
    neu_t *acc = (neu_t *)calloc(ngroups ? ngroups : 1, sizeof(neu_t));
    for (uint64_t g = 0; g < ngroups; ++g) cnt[g] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        neu_add(&acc[gid[i]], v[i]);
        cnt[gid[i]]++;
    }
    for (uint64_t g = 0; g < ngroups; ++g) sum[g] = neu_val(&acc[g]);
    free(acc);
}

/* The six-relation BI query of the two-node GHD example (Section 3.1):
 * SUM(price * (1 - disc/100)) over fact rows f joined with orders o
 * (f.order = o), customer c (o.cust = c), supplier s (f.supp = s) where
 * c.nation = s.nation = n, nation n's region r has name region_pick, and o's
 * date lies in [dlo, dhi]; GROUP BY the nation's name.  A plain pairwise
 * hash join: keys are row ids, so each lookup is an index.  gsum / gcnt are
 * indexed by nation name (n_names entries). */
void orc_bi_q5(uint64_t nfact, const uint32_t *f_order, const uint32_t *f_supp, const double *price,
               const int8_t *disc, const uint32_t *o_cust, const int32_t *o_date, const uint32_t *c_nation,
               const uint32_t *s_nation, const uint32_t *n_region, const int32_t *n_name,
               const int32_t *r_name, int32_t region_pick, int32_t dlo, int32_t dhi, uint32_t n_names,
               double *gsum, uint64_t *gcnt) {
    int nt = orc_num_threads();
    neu_t *part = (neu_t *)calloc((size_t)nt * n_names, sizeof(neu_t));
    uint64_t *pc = (uint64_t *)calloc((size_t)nt * n_names, sizeof(uint64_t));
    #pragma omp parallel
    {
#ifdef _OPENMP
        int t = omp_get_thread_num();
#else
        int t = 0;
#endif
        #pragma omp for schedule(static)
        for (int64_t r = 0; r < (int64_t)nfact; ++r) {
            uint32_t o = f_order[r];
            int32_t d = o_date[o];
            if (d < dlo || d > dhi) continue;
            uint32_t n = c_nation[o_cust[o]];
            if (n != s_nation[f_supp[r]]) continue;
            if (r_name[n_region[n]] != region_pick) continue;
            uint32_t g = (uint32_t)n_name[n];
            neu_add(&part[(size_t)t * n_names + g], price[r] * (1.0 - (double)disc[r] / 100.0));
            pc[(size_t)t * n_names + g]++;
        }
    }
    for (uint32_t g = 0; g < n_names; ++g) {
        neu_t a = {0, 0};
        uint64_t c = 0;
        for (int t = 0; t < nt; ++t) {
            neu_add(&a, part[(size_t)t * n_names + g].s);
            neu_add(&a, part[(size_t)t * n_names + g].c);
            c += pc[(size_t)t * n_names + g];
        }
        gsum[g] = neu_val(&a);
        gcnt[g] = c;
    }
    free(part); free(pc);
}
