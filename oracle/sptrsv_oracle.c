/*
 * CPU oracle for the SpTRSV hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, sequential, FP64 C written from the definitions in the paper
 * ("Reinforcement Learning-Guided Graph Transformations for SpTRSV
 * Optimization"):
 *   - Section 2.1: L x = b, rows are DAG nodes, every off-diagonal L[i][j]
 *     is an edge j -> i, a row can be computed only after its predecessors;
 *     the level-set method partitions the DAG into levels of independent rows.
 *   - Section 2.2: equation rewriting replaces a row's dependencies by their
 *     predecessors so that the row moves to an earlier level; it is a
 *     preprocessing step and the result is again a CSR lower-triangular system.
 *   - Section 4.1 / Tables 4-5: level cost, ALC, ARL, AIR; Section 4.1 and
 *     Table 1: coefficient of variation of level costs and node counts, and
 *     the thin-level threshold ALC * (1 + alpha * max(0, 1 - CV)).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * use this file; the CUDA library never links it and shares no code with it.
 * Build with -ffp-contract=off so that every a - m*b is a separate multiply
 * and subtract.
 *
 * Conventions: CSR with int32 row_ptr[n+1], col_idx[nnz]; every row lists its
 * off-diagonal columns in strictly increasing order followed by the diagonal.
 * Dense right-hand sides are [n x k] row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOTLOWER 2
#define ORC_EDIAG 3
#define ORC_EUNSORTED 4
#define ORC_ETARGET 5
#define ORC_ENOMEM 6

/* ---------------------------------------------------------------------- */
/* Validation: the CSR describes a lower-triangular system with the diagonal
 * stored last in every row (Section 2.1).  Returns the status of the first
 * offending row (in row order) and writes that row to *bad_row.           */
int orc_validate(int32_t n, const int32_t *rp, const int32_t *ci,
                 const double *v, int32_t *bad_row)
{
    *bad_row = -1;
    if (n < 0) return ORC_EINVAL;
    if (n > 0 && rp[0] != 0) { *bad_row = 0; return ORC_EINVAL; }
    for (int32_t i = 0; i < n; ++i) {
        int32_t a = rp[i], e = rp[i + 1];
        if (e <= a) { *bad_row = i; return (e < a) ? ORC_EINVAL : ORC_EDIAG; }
        for (int32_t p = a; p < e; ++p) {
            if (ci[p] < 0 || ci[p] > i) { *bad_row = i; return ORC_ENOTLOWER; }
            if (p > a && ci[p] <= ci[p - 1]) { *bad_row = i; return ORC_EUNSORTED; }
        }
        if (ci[e - 1] != i || v[e - 1] == 0.0) { *bad_row = i; return ORC_EDIAG; }
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Forward substitution in row order (Section 2.1):
 *   x_i = (b_i - sum_{p < diag} L[p] * x[col[p]]) / L_ii,
 * the sum taken in stored column order.                                  */
void orc_solve(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
               int32_t k, const double *b, double *x)
{
    for (int32_t i = 0; i < n; ++i) {
        int32_t a = rp[i], d = rp[i + 1] - 1;
        for (int32_t r = 0; r < k; ++r) {
            double s = b[(int64_t)i * k + r];
            for (int32_t p = a; p < d; ++p)
                s = s - v[p] * x[(int64_t)ci[p] * k + r];
            x[(int64_t)i * k + r] = s / v[d];
        }
    }
}

/* Backward substitution for L^T g_b = g_x (the adjoint of the solve), column
 * sweep over rows of L from the last to the first:
 *   g_b_i = r_i / L_ii, then r_j -= L_ij * g_b_i for every off-diagonal j. */
void orc_solve_transpose(int32_t n, const int32_t *rp, const int32_t *ci,
                         const double *v, int32_t k, const double *gx, double *gb)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(k > 0 ? k : 1));
    memcpy(r, gx, sizeof(double) * (size_t)n * (size_t)k);
    for (int32_t i = n - 1; i >= 0; --i) {
        int32_t a = rp[i], d = rp[i + 1] - 1;
        for (int32_t q = 0; q < k; ++q) {
            double g = r[(int64_t)i * k + q] / v[d];
            gb[(int64_t)i * k + q] = g;
            for (int32_t p = a; p < d; ++p)
                r[(int64_t)ci[p] * k + q] = r[(int64_t)ci[p] * k + q] - v[p] * g;
        }
    }
    free(r);
}

/* Gradient of a loss with respect to the stored values of L, given
 * g_b = L^{-T} g_x and x = L^{-1} b:  dL/dL_ij = -sum_r g_b[i,r] * x[j,r],
 * on L's pattern, diagonal included.                                      */
void orc_grad_vals(int32_t n, const int32_t *rp, const int32_t *ci, int32_t k,
                   const double *gb, const double *x, double *gv)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
            double s = 0.0;
            for (int32_t q = 0; q < k; ++q)
                s = s + gb[(int64_t)i * k + q] * x[(int64_t)ci[p] * k + q];
            gv[p] = -s;
        }
}

/* ---------------------------------------------------------------------- */
/* Level-set analysis, Kahn style (Section 2.1 / related work on the
 * level-set method): indegree = number of off-diagonals; round r takes every
 * row whose predecessors are all done and gives it level r.  Returns the
 * number of rounds (levels).                                              */
int32_t orc_levels(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *lev)
{
    if (n <= 0) return 0;
    int32_t *indeg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int64_t noff = 0;
    for (int32_t i = 0; i < n; ++i) {
        indeg[i] = rp[i + 1] - rp[i] - 1;
        noff += indeg[i];
        for (int32_t p = rp[i]; p < rp[i + 1] - 1; ++p) sp[ci[p] + 1]++;
    }
    for (int32_t j = 0; j < n; ++j) sp[j + 1] += sp[j];
    int32_t *succ = (int32_t *)malloc(sizeof(int32_t) * (size_t)(noff > 0 ? noff : 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    memcpy(fill, sp, sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = rp[i]; p < rp[i + 1] - 1; ++p) succ[fill[ci[p]]++] = i;
    int32_t *front = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t nf = 0;
    for (int32_t i = 0; i < n; ++i) if (indeg[i] == 0) front[nf++] = i;
    int32_t round = 0;
    while (nf > 0) {
        int32_t nn = 0;
        for (int32_t f = 0; f < nf; ++f) lev[front[f]] = round;
        for (int32_t f = 0; f < nf; ++f) {
            int32_t j = front[f];
            for (int32_t q = sp[j]; q < sp[j + 1]; ++q)
                if (--indeg[succ[q]] == 0) next[nn++] = succ[q];
        }
        int32_t *t = front; front = next; next = t;
        nf = nn;
        ++round;
    }
    free(indeg); free(sp); free(succ); free(fill); free(front); free(next);
    return round;
}

/* Level table (Section 4.1: rows on each level and level costs):
 * perm lists the rows of level 0 in ascending order, then level 1, ...;
 * level_ptr[l] is where level l starts in perm; the cost of a level is
 * sum over its rows of (2 * offdiag(i) + 1): one multiply and one add per
 * off-diagonal plus the division by the diagonal.                        */
void orc_partition(int32_t n, const int32_t *rp, const int32_t *lev, int32_t nlevels,
                   int32_t *perm, int32_t *level_ptr, int64_t *cost)
{
    memset(level_ptr, 0, sizeof(int32_t) * ((size_t)nlevels + 1));
    memset(cost, 0, sizeof(int64_t) * (size_t)nlevels);
    for (int32_t i = 0; i < n; ++i) {
        level_ptr[lev[i] + 1]++;
        cost[lev[i]] += 2 * (int64_t)(rp[i + 1] - rp[i] - 1) + 1;
    }
    for (int32_t l = 0; l < nlevels; ++l) level_ptr[l + 1] += level_ptr[l];
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nlevels + 1));
    memcpy(pos, level_ptr, sizeof(int32_t) * ((size_t)nlevels + 1));
    for (int32_t i = 0; i < n; ++i) perm[pos[lev[i]]++] = i;
    free(pos);
}

/* Population coefficient of variation of m non-negative integers whose sum
 * is S1 and whose sum of squares is S2:
 *   CV = sqrt(m*S2 - S1^2) / S1,
 * the difference taken exactly in 128-bit integers and rounded to double
 * once; sqrt and the division are IEEE correctly rounded.                 */
static double cov_exact(int64_t m, int64_t S1, unsigned __int128 S2)
{
    if (m <= 0 || S1 <= 0) return 0.0;
    unsigned __int128 a = (unsigned __int128)(uint64_t)m * S2;
    unsigned __int128 s1 = (unsigned __int128)(uint64_t)S1;
    unsigned __int128 b = s1 * s1;
    unsigned __int128 d = (a > b) ? (a - b) : 0;
    return sqrt((double)d) / (double)S1;
}

/* Thin-level threshold of Section 4.1: ALC * (1 + alpha * max(0, 1 - CV)). */
double orc_thin_threshold(double alc, double cv, double alpha)
{
    double relax = 1.0 - cv;
    if (relax < 0.0) relax = 0.0;
    return alc * (1.0 + alpha * relax);
}

/* Level summary that the paper's environment observes after every rewrite
 * (Section 4.1 and Section 4.3, Tables 4-5):
 *   thin[l]  = 1 when cost[l] < threshold (a thin level: its cost is below
 *              the thin-level threshold), else 0;
 *   pick[l]  = the row of level l with the smallest number of dependencies
 *              (off-diagonals), the smallest row index among equals -- the
 *              node a rewrite of level l moves (Section 4.3);
 *   out[0] number of thin levels, out[1] largest row count of a thin level,
 *   out[2] largest cost of a thin level (0 when there is none).
 * The cost comparison is in double, as the threshold.                    */
void orc_level_summary(int32_t n, const int32_t *rp, int32_t nlevels, const int32_t *level_ptr,
                       const int32_t *perm, const int64_t *cost, double threshold,
                       uint8_t *thin, int32_t *pick, int64_t *out)
{
    (void)n;
    out[0] = out[1] = out[2] = 0;
    for (int32_t l = 0; l < nlevels; ++l) {
        int32_t best = -1, best_deps = 0;
        for (int32_t q = level_ptr[l]; q < level_ptr[l + 1]; ++q) {
            const int32_t i = perm[q];
            const int32_t deps = rp[i + 1] - rp[i] - 1;
            if (best < 0 || deps < best_deps || (deps == best_deps && i < best)) {
                best = i;
                best_deps = deps;
            }
        }
        pick[l] = best;
        thin[l] = (double)cost[l] < threshold ? 1 : 0;
        if (thin[l]) {
            const int64_t rows = level_ptr[l + 1] - level_ptr[l];
            out[0] += 1;
            if (rows > out[1]) out[1] = rows;
            if (cost[l] > out[2]) out[2] = cost[l];
        }
    }
}

/* Scalar statistics of a level table (Tables 4-5, Section 4.1):
 * out[0] ALC  = sum(cost) / L        (average level cost)
 * out[1] ARL  = n / L                (average rows per level)
 * out[2] AIR  = (nnz - n) / n        (average incoming dependencies per row)
 * out[3] CV of level costs, out[4] CV of rows per level,
 * out[5] thin-level threshold ALC * (1 + alpha * max(0, 1 - CV)), alpha = 1.
 */
void orc_stats(int32_t n, int64_t nnz, int32_t nlevels, const int32_t *level_ptr,
               const int64_t *cost, double *out)
{
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    if (n <= 0 || nlevels <= 0) return;
    int64_t S1 = 0, R1 = 0;
    unsigned __int128 S2 = 0, R2 = 0;
    for (int32_t l = 0; l < nlevels; ++l) {
        int64_t c = cost[l];
        int64_t r = level_ptr[l + 1] - level_ptr[l];
        S1 += c;
        S2 += (unsigned __int128)(uint64_t)c * (uint64_t)c;
        R1 += r;
        R2 += (unsigned __int128)(uint64_t)r * (uint64_t)r;
    }
    double L = (double)nlevels;
    out[0] = (double)S1 / L;
    out[1] = (double)n / L;
    out[2] = (double)(nnz - (int64_t)n) / (double)n;
    out[3] = cov_exact(nlevels, S1, S2);
    out[4] = cov_exact(nlevels, R1, R2);
    out[5] = orc_thin_threshold(out[0], out[3], 1.0);
}

/* ---------------------------------------------------------------------- */
/* Equation rewriting (Section 2.2; rewriting list of Section 4.3): textbook
 * row substitution.  For a listed row i with target level t < lev(i):
 *
 *   acc <- row i (off-diagonals, column -> value);  tb <- {}
 *   repeat: take the LARGEST column j in acc with lev(j) >= t (original
 *           levels);  m = acc[j] / L_jj;  drop j from acc;
 *           for every off-diagonal (k, L_jk) of the ORIGINAL row j:
 *               acc[k] = acc[k] - m * L_jk   (k inserted with 0 if absent)
 *           tb[j] = tb[j] - m                 (j inserted with 0 if absent)
 *   until no such column is left.
 *
 * Row i of L' is acc sorted by column followed by the unchanged diagonal;
 * row i of T is tb sorted by column, so that L' x = b + T b.  Rows not
 * listed are copied.  Every fill column is smaller than the column that
 * produced it, so each j is eliminated at most once and the loop ends.
 * Exact zeros produced by cancellation stay as explicit entries.
 * A row listed twice keeps its smallest target.                          */

typedef struct {
    int32_t *a;
    int32_t n, cap;
} orc_heap;

static int heap_push(orc_heap *h, int32_t v)
{
    if (h->n == h->cap) {
        int32_t nc = h->cap ? 2 * h->cap : 64;
        int32_t *na = (int32_t *)realloc(h->a, sizeof(int32_t) * (size_t)nc);
        if (!na) return -1;
        h->a = na; h->cap = nc;
    }
    int32_t c = h->n++;
    h->a[c] = v;
    while (c > 0) {
        int32_t p = (c - 1) / 2;
        if (h->a[p] >= h->a[c]) break;
        int32_t t = h->a[p]; h->a[p] = h->a[c]; h->a[c] = t;
        c = p;
    }
    return 0;
}

static int32_t heap_pop(orc_heap *h)
{
    int32_t top = h->a[0];
    h->a[0] = h->a[--h->n];
    int32_t c = 0;
    for (;;) {
        int32_t l = 2 * c + 1, r = l + 1, m = c;
        if (l < h->n && h->a[l] > h->a[m]) m = l;
        if (r < h->n && h->a[r] > h->a[m]) m = r;
        if (m == c) break;
        int32_t t = h->a[m]; h->a[m] = h->a[c]; h->a[c] = t;
        c = m;
    }
    return top;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct {
    double *acc;
    int32_t *in_acc;    /* == stamp when the column is in acc            */
    int32_t *gone;      /* == stamp when the column has been eliminated   */
    int32_t *cols;      /* every column ever inserted for the current row */
    int32_t ncols, capcols;
    int32_t *elim;      /* eliminated columns, in elimination order       */
    double *elim_v;     /* their T coefficients                           */
    int32_t nelim, capelim;
    orc_heap h;
    int32_t stamp;
} orc_ws;

static int ws_grow_cols(orc_ws *w)
{
    int32_t nc = w->capcols ? 2 * w->capcols : 256;
    int32_t *na = (int32_t *)realloc(w->cols, sizeof(int32_t) * (size_t)nc);
    if (!na) return -1;
    w->cols = na; w->capcols = nc;
    return 0;
}

static int ws_grow_elim(orc_ws *w)
{
    int32_t nc = w->capelim ? 2 * w->capelim : 256;
    int32_t *na = (int32_t *)realloc(w->elim, sizeof(int32_t) * (size_t)nc);
    double *nv = (double *)realloc(w->elim_v, sizeof(double) * (size_t)nc);
    if (!na || !nv) return -1;
    w->elim = na; w->elim_v = nv; w->capelim = nc;
    return 0;
}

/* Runs the substitution for row i; afterwards the surviving columns are in
 * w->cols (filtered by in_acc/gone) and the eliminated ones in w->elim.   */
static int rewrite_row(orc_ws *w, const int32_t *rp, const int32_t *ci, const double *v,
                       const int32_t *lev, int32_t i, int32_t t)
{
    w->stamp++;
    w->ncols = 0; w->nelim = 0; w->h.n = 0;
    for (int32_t p = rp[i]; p < rp[i + 1] - 1; ++p) {
        int32_t j = ci[p];
        w->acc[j] = v[p];
        w->in_acc[j] = w->stamp;
        if (w->ncols == w->capcols && ws_grow_cols(w)) return ORC_ENOMEM;
        w->cols[w->ncols++] = j;
        if (lev[j] >= t && heap_push(&w->h, j)) return ORC_ENOMEM;
    }
    while (w->h.n > 0) {
        int32_t j = heap_pop(&w->h);
        int32_t dj = rp[j + 1] - 1;
        double m = w->acc[j] / v[dj];
        w->gone[j] = w->stamp;
        for (int32_t p = rp[j]; p < dj; ++p) {
            int32_t k = ci[p];
            if (w->in_acc[k] != w->stamp) {
                w->acc[k] = 0.0;
                w->in_acc[k] = w->stamp;
                if (w->ncols == w->capcols && ws_grow_cols(w)) return ORC_ENOMEM;
                w->cols[w->ncols++] = k;
                if (lev[k] >= t && heap_push(&w->h, k)) return ORC_ENOMEM;
            }
            w->acc[k] = w->acc[k] - m * v[p];
        }
        if (w->nelim == w->capelim && ws_grow_elim(w)) return ORC_ENOMEM;
        w->elim[w->nelim] = j;
        w->elim_v[w->nelim] = 0.0 - m;
        w->nelim++;
    }
    return ORC_OK;
}

/* Sizing pass when lp_ci == NULL (fills lp_rp[n+1], t_rp[n+1] only);
 * otherwise also fills lp_ci/lp_v and t_ci/t_v.  Returns a status; on
 * ORC_ETARGET/ORC_EINVAL *bad is the offending list position.            */
int orc_rewrite(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                const int32_t *lev, int32_t nrows, const int32_t *rows,
                const int32_t *targets, int32_t *lp_rp, int32_t *lp_ci, double *lp_v,
                int32_t *t_rp, int32_t *t_ci, double *t_v, int32_t *bad)
{
    *bad = -1;
    int32_t *tgt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!tgt) return ORC_ENOMEM;
    for (int32_t i = 0; i < n; ++i) tgt[i] = -1;
    for (int32_t q = 0; q < nrows; ++q) {
        int32_t i = rows[q];
        if (i < 0 || i >= n) { *bad = q; free(tgt); return ORC_EINVAL; }
        int32_t t = targets ? targets[q] : lev[i] - 1;
        if (lev[i] == 0 || t < 0 || t >= lev[i]) { *bad = q; free(tgt); return ORC_ETARGET; }
        if (tgt[i] < 0 || t < tgt[i]) tgt[i] = t;
    }
    orc_ws w;
    memset(&w, 0, sizeof(w));
    w.acc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    w.in_acc = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    w.gone = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    int status = ORC_OK;
    if (!w.acc || !w.in_acc || !w.gone) { status = ORC_ENOMEM; goto done; }
    lp_rp[0] = 0;
    t_rp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t len = rp[i + 1] - rp[i];
        if (tgt[i] < 0) {
            if (lp_ci) {
                memcpy(lp_ci + lp_rp[i], ci + rp[i], sizeof(int32_t) * (size_t)len);
                memcpy(lp_v + lp_rp[i], v + rp[i], sizeof(double) * (size_t)len);
            }
            lp_rp[i + 1] = lp_rp[i] + len;
            t_rp[i + 1] = t_rp[i];
            continue;
        }
        status = rewrite_row(&w, rp, ci, v, lev, i, tgt[i]);
        if (status != ORC_OK) goto done;
        int32_t keep = 0;
        for (int32_t c = 0; c < w.ncols; ++c) {
            int32_t j = w.cols[c];
            if (w.gone[j] != w.stamp) w.cols[keep++] = j;
        }
        qsort(w.cols, (size_t)keep, sizeof(int32_t), cmp_i32);
        if (lp_ci) {
            int32_t o = lp_rp[i];
            for (int32_t c = 0; c < keep; ++c) {
                lp_ci[o + c] = w.cols[c];
                lp_v[o + c] = w.acc[w.cols[c]];
            }
            lp_ci[o + keep] = i;
            lp_v[o + keep] = v[rp[i + 1] - 1];
            int32_t to = t_rp[i];
            for (int32_t e = 0; e < w.nelim; ++e) {   /* elimination order is descending */
                t_ci[to + e] = w.elim[w.nelim - 1 - e];
                t_v[to + e] = w.elim_v[w.nelim - 1 - e];
            }
        }
        lp_rp[i + 1] = lp_rp[i] + keep + 1;
        t_rp[i + 1] = t_rp[i] + w.nelim;
    }
done:
    free(tgt); free(w.acc); free(w.in_acc); free(w.gone); free(w.cols);
    free(w.elim); free(w.elim_v); free(w.h.a);
    return status;
}

/* Solve of the rewritten system L' x = b + T b (T has no diagonal): the
 * right-hand side b_i + sum_j T_ij b_j is formed first, then forward
 * substitution with L'.                                                   */
void orc_solve_rewritten(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                         const int32_t *trp, const int32_t *tci, const double *tv,
                         int32_t k, const double *b, double *x)
{
    double *bt = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(k > 0 ? k : 1));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t r = 0; r < k; ++r) {
            double s = b[(int64_t)i * k + r];
            for (int32_t p = trp[i]; p < trp[i + 1]; ++p)
                s = s + tv[p] * b[(int64_t)tci[p] * k + r];
            bt[(int64_t)i * k + r] = s;
        }
    orc_solve(n, rp, ci, v, k, bt, x);
    free(bt);
}

/* Adjoint of b -> b + T b:  g_b = g_b' + T^T g_b'.                        */
void orc_tt_apply(int32_t n, const int32_t *trp, const int32_t *tci, const double *tv,
                  int32_t k, const double *gbp, double *gb)
{
    memcpy(gb, gbp, sizeof(double) * (size_t)n * (size_t)k);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = trp[i]; p < trp[i + 1]; ++p)
            for (int32_t r = 0; r < k; ++r)
                gb[(int64_t)tci[p] * k + r] = gb[(int64_t)tci[p] * k + r] + tv[p] * gbp[(int64_t)i * k + r];
}
