/*
 * FP64 CPU oracle for the context-enhanced tensor join.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * What it computes is the plain definition of the operator, written out:
 *
 *   sim(r, s) = (sum_k r_k s_k) / (||r|| ||s||)          -- Sec. III-A, Eq. (Cosine Similarity)
 *   R join_{E,mu,theta} S = sigma_theta(E(R) x E(S))      -- Sec. III-C, Eq. (E-theta-Join),
 *                                                            Eq. (theta-Join Generalization)
 *   theta(r, s) = selR(r) and selS(s) and sim(r, s) >= eps -- Sec. III-B (threshold predicate),
 *                                                            Sec. III-C (Selection), Sec. VI-E
 *                                                            (relational pre-filter)
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * design notes): the threshold test is ">=" (the paper says "larger than"; the
 * two differ only on the measure-zero set sim == eps); a zero-norm row has
 * similarity 0 with every row; a similarity that rounds outside [-1, 1] is
 * clamped; pair ids are 0-based row numbers of the ORIGINAL (pre-selection)
 * relations (Sec. IV-C: pairs are mapped back to tuples through partition
 * offsets); a self-join yields every ordered pair, the diagonal included.
 *
 * Arithmetic: every float input is widened exactly to double; norms and dot
 * products are summed in index order (k = 0 .. d-1) with no fused multiply-add
 * (the library is compiled with -ffp-contract=off), so that the result is the
 * same on every host and sim(i, j) and sim(j, i) are bitwise equal.
 *
 * Output order: sorted by (i, j).  Rows of R are processed in ascending order
 * (the sample list, when given, must be ascending), S rows ascending inside.
 *
 * Parity pins for this file live in tests/test_oracle_pins.py (exact rational
 * arithmetic, closed forms, invariants, planted pairs, mutation checks).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Build-time mutants (tests only): ORACLE_MUTANT selects one deliberate
 * mistake so that the pin suite can show it is caught.  0 = the oracle. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

enum { OP_LT = 0, OP_LE = 1, OP_GT = 2, OP_GE = 3, OP_EQ = 4, OP_NE = 5 };

/* sigma_theta(R) = { t in R : theta(t) }  (Sec. III-C, Eq. Selection), with
 * theta an attribute comparison "attr op c" (Sec. VI-E pre-filter). */
static int keep_row(const int32_t *attr, int32_t op, int32_t c, int64_t row)
{
    if (attr == NULL) return 1;
    int32_t a = attr[row];
    switch (op) {
    case OP_LT: return a < c;
    case OP_LE: return a <= c;
    case OP_GT: return a > c;
    case OP_GE: return a >= c;
    case OP_EQ: return a == c;
    case OP_NE: return a != c;
    default: return 0;
    }
}

/* ||x|| = sqrt(sum_k x_k^2), the denominator factor of Eq. (Cosine Similarity). */
double oracle_norm(const float *x, int32_t d)
{
    double acc = 0.0;
#if ORACLE_MUTANT == 1
    /* mutant 1: dropped last term */
    for (int32_t k = 0; k + 1 < d; ++k) { double v = (double)x[k]; acc += v * v; }
#else
    for (int32_t k = 0; k < d; ++k) { double v = (double)x[k]; acc += v * v; }
#endif
#if ORACLE_MUTANT == 2
    /* mutant 2: squared norm instead of norm */
    return acc;
#else
    return sqrt(acc);
#endif
}

/* A . B = sum_k A_k B_k, the numerator of Eq. (Cosine Similarity). */
double oracle_dot(const float *a, const float *b, int32_t d)
{
    double acc = 0.0;
    for (int32_t k = 0; k < d; ++k) {
#if ORACLE_MUTANT == 3
        /* mutant 3: wrong index into the second operand */
        acc += (double)a[k] * (double)b[(k + 1) % d];
#else
        acc += (double)a[k] * (double)b[k];
#endif
    }
    return acc;
}

/* cos(theta) = (A . B) / (||A|| ||B||), clamped to [-1, 1]; 0 for a zero row. */
static double cosine_from(double dot, double nr, double ns)
{
    if (nr == 0.0 || ns == 0.0) return 0.0;
    double s = dot / (nr * ns);
#if ORACLE_MUTANT == 4
    s = -s; /* mutant 4: wrong sign */
#endif
#if ORACLE_MUTANT != 5
    /* mutant 5 drops the clamp */
    if (s > 1.0) s = 1.0;
    if (s < -1.0) s = -1.0;
#endif
    return s;
}

double oracle_sim(const float *r, const float *s, int32_t d)
{
    return cosine_from(oracle_dot(r, s, d), oracle_norm(r, d), oracle_norm(s, d));
}

static int matches(double sim, double eps)
{
#if ORACLE_MUTANT == 6
    return sim > eps; /* mutant 6: strict comparison */
#else
    return sim >= eps;
#endif
}

typedef struct {
    uint32_t *i, *j;
    double *sim;
    int64_t n, cap;
} pair_buf;

static int buf_push(pair_buf *b, uint32_t i, uint32_t j, double sim)
{
    if (b->n == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 1024;
        uint32_t *ni = (uint32_t *)realloc(b->i, (size_t)nc * sizeof(uint32_t));
        if (!ni) return -1;
        b->i = ni;
        uint32_t *nj = (uint32_t *)realloc(b->j, (size_t)nc * sizeof(uint32_t));
        if (!nj) return -1;
        b->j = nj;
        double *ns = (double *)realloc(b->sim, (size_t)nc * sizeof(double));
        if (!ns) return -1;
        b->sim = ns;
        b->cap = nc;
    }
    b->i[b->n] = i;
    b->j[b->n] = j;
    b->sim[b->n] = sim;
    b->n++;
    return 0;
}

/*
 * The E-theta-join of Sec. III-C evaluated pair by pair.
 *
 *   R, S         row-major FP32 relations, nR x d (row stride ldR) and nS x d (ldS)
 *   attrR/opR/cR optional selection on R (attrR == NULL: keep every row); same for S
 *   eps          similarity threshold, compared as (double)eps
 *   rows/n_rows  optional ascending list of R rows to evaluate (NULL: all rows);
 *                this is how large workloads are sampled
 *   out_*        output arrays with room for cap pairs (may be NULL when cap == 0)
 *   n_threads    OpenMP threads (<= 0: the runtime default)
 *
 * Returns the total number of matching pairs (which may exceed cap; only the
 * first cap are written), or -1 on allocation failure.
 */
int64_t oracle_join(const float *R, int64_t nR, int64_t ldR,
                    const float *S, int64_t nS, int64_t ldS, int32_t d,
                    const int32_t *attrR, int32_t opR, int32_t cR,
                    const int32_t *attrS, int32_t opS, int32_t cS,
                    float eps, const int64_t *rows, int64_t n_rows,
                    uint32_t *out_i, uint32_t *out_j, double *out_sim, int64_t cap,
                    int32_t n_threads)
{
    const double e = (double)eps;
    const int64_t n_eval = rows ? n_rows : nR;
    if (n_eval <= 0 || nS <= 0) return 0;

    /* Norms of S are needed by every R row: compute each once (the
     * "prefetch" formulation of Sec. IV-A, Eq. nlj-prefetch). */
    double *ns = (double *)malloc((size_t)nS * sizeof(double));
    if (!ns) return -1;
    for (int64_t j = 0; j < nS; ++j) ns[j] = oracle_norm(S + j * ldS, d);

    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#endif
    pair_buf *bufs = (pair_buf *)calloc((size_t)nt, sizeof(pair_buf));
    int failed = 0;
    if (!bufs) { free(ns); return -1; }

#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        /* contiguous, ascending block of the R rows per thread: concatenating
         * the per-thread buffers in thread order keeps the (i, j) order */
        int64_t chunk = (n_eval + nt - 1) / nt;
        int64_t lo = (int64_t)t * chunk, hi = lo + chunk;
        if (hi > n_eval) hi = n_eval;
        for (int64_t q = lo; q < hi; ++q) {
            int64_t i = rows ? rows[q] : q;
            if (!keep_row(attrR, opR, cR, i)) continue;
            const float *r = R + i * ldR;
            double nr = oracle_norm(r, d);
            for (int64_t j = 0; j < nS; ++j) {
                if (!keep_row(attrS, opS, cS, j)) continue;
                double sim = cosine_from(oracle_dot(r, S + j * ldS, d), nr, ns[j]);
                if (matches(sim, e)) {
                    if (buf_push(&bufs[t], (uint32_t)i, (uint32_t)j, sim)) failed = 1;
                }
            }
        }
    }

    int64_t total = 0;
    for (int t = 0; t < nt; ++t) {
        for (int64_t k = 0; k < bufs[t].n; ++k) {
            if (total < cap) {
                out_i[total] = bufs[t].i[k];
                out_j[total] = bufs[t].j[k];
                out_sim[total] = bufs[t].sim[k];
            }
            ++total;
        }
        free(bufs[t].i);
        free(bufs[t].j);
        free(bufs[t].sim);
    }
    free(bufs);
    free(ns);
    return failed ? -1 : total;
}

/* FP64 similarity of given (i, j) pairs, one by one: used to check sampled
 * outputs of workloads too large for a full join.  Same arithmetic as above. */
void oracle_sim_pairs(const float *R, int64_t ldR, const float *S, int64_t ldS, int32_t d,
                      const uint32_t *pi, const uint32_t *pj, int64_t n_pairs, double *out_sim,
                      int32_t n_threads)
{
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
    for (int64_t q = 0; q < n_pairs; ++q) {
        const float *r = R + (int64_t)pi[q] * ldR;
        const float *s = S + (int64_t)pj[q] * ldS;
        out_sim[q] = cosine_from(oracle_dot(r, s, d), oracle_norm(r, d), oracle_norm(s, d));
    }
    (void)nt;
}

/* Number of rows kept by the selection (Sec. III-C, Eq. Selection). */
int64_t oracle_count_selected(const int32_t *attr, int32_t op, int32_t c, int64_t n)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) k += keep_row(attr, op, c, i);
    return k;
}

/*
 * The top-1 join condition (Sec. VI-E, "top-k" join predicate with k = 1):
 * for every kept row i of R, the kept row j of S with the largest similarity,
 * ties broken towards the smaller j.  Same arithmetic as oracle_join.
 *
 *   rows/n_rows  optional ascending list of R rows to evaluate (NULL: all rows)
 *   out_*        room for one record per evaluated row
 *
 * Writes one record (i, j, sim) per kept R row, in ascending i, when S has at
 * least one kept row; returns the number written, or -1 on allocation failure.
 */
int64_t oracle_top1(const float *R, int64_t nR, int64_t ldR,
                    const float *S, int64_t nS, int64_t ldS, int32_t d,
                    const int32_t *attrR, int32_t opR, int32_t cR,
                    const int32_t *attrS, int32_t opS, int32_t cS,
                    const int64_t *rows, int64_t n_rows,
                    uint32_t *out_i, uint32_t *out_j, double *out_sim, int32_t n_threads)
{
    const int64_t n_eval = rows ? n_rows : nR;
    if (n_eval <= 0 || nS <= 0) return 0;
    double *ns = (double *)malloc((size_t)nS * sizeof(double));
    int64_t *best_j = (int64_t *)malloc((size_t)n_eval * sizeof(int64_t));
    double *best_s = (double *)malloc((size_t)n_eval * sizeof(double));
    if (!ns || !best_j || !best_s) {
        free(ns);
        free(best_j);
        free(best_s);
        return -1;
    }
    for (int64_t j = 0; j < nS; ++j) ns[j] = oracle_norm(S + j * ldS, d);
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
#endif
    for (int64_t q = 0; q < n_eval; ++q) {
        const int64_t i = rows ? rows[q] : q;
        best_j[q] = -1;
        best_s[q] = 0.0;
        if (!keep_row(attrR, opR, cR, i)) continue;
        const float *r = R + i * ldR;
        const double nr = oracle_norm(r, d);
        for (int64_t j = 0; j < nS; ++j) {
            if (!keep_row(attrS, opS, cS, j)) continue;
            const double sim = cosine_from(oracle_dot(r, S + j * ldS, d), nr, ns[j]);
#if ORACLE_MUTANT == 7
            if (best_j[q] < 0 || sim >= best_s[q]) { /* mutant 7: a tie goes to the larger j */
#else
            if (best_j[q] < 0 || sim > best_s[q]) { /* strict: the smaller j keeps a tie */
#endif
                best_j[q] = j;
                best_s[q] = sim;
            }
        }
    }
    (void)nt;
    int64_t n_out = 0;
    for (int64_t q = 0; q < n_eval; ++q) {
        if (best_j[q] < 0) continue;
        out_i[n_out] = (uint32_t)(rows ? rows[q] : q);
        out_j[n_out] = (uint32_t)best_j[q];
        out_sim[n_out] = best_s[q];
        ++n_out;
    }
    free(ns);
    free(best_j);
    free(best_s);
    return n_out;
}

/*
 * The top-k join condition (Sec. VI-E, "top-k" join predicate; the paper's
 * figures use k = 1 and k = 32): for every kept row i of R, the min(k, kept S
 * rows) kept rows j of S of largest similarity, in descending similarity, ties
 * broken towards the smaller j.  Same arithmetic as oracle_join.
 *
 *   rows/n_rows  optional ascending list of R rows to evaluate (NULL: all rows)
 *   out_*        room for k records per evaluated row
 *
 * Writes the records of each kept R row consecutively, rows in ascending i;
 * returns the number written, or -1 on allocation failure.  Each row keeps its
 * list sorted by (sim descending, j ascending): S rows are visited in
 * ascending j and a new row enters only if its similarity is strictly larger
 * than that of the list entry it passes, so an earlier j stays ahead on ties.
 */
int64_t oracle_topk(const float *R, int64_t nR, int64_t ldR,
                    const float *S, int64_t nS, int64_t ldS, int32_t d, int32_t k,
                    const int32_t *attrR, int32_t opR, int32_t cR,
                    const int32_t *attrS, int32_t opS, int32_t cS,
                    const int64_t *rows, int64_t n_rows,
                    uint32_t *out_i, uint32_t *out_j, double *out_sim, int32_t n_threads)
{
    const int64_t n_eval = rows ? n_rows : nR;
    if (n_eval <= 0 || nS <= 0 || k <= 0) return 0;
    double *ns = (double *)malloc((size_t)nS * sizeof(double));
    int64_t *list_j = (int64_t *)malloc((size_t)n_eval * k * sizeof(int64_t));
    double *list_s = (double *)malloc((size_t)n_eval * k * sizeof(double));
    int64_t *list_n = (int64_t *)malloc((size_t)n_eval * sizeof(int64_t));
    if (!ns || !list_j || !list_s || !list_n) {
        free(ns);
        free(list_j);
        free(list_s);
        free(list_n);
        return -1;
    }
    for (int64_t j = 0; j < nS; ++j) ns[j] = oracle_norm(S + j * ldS, d);
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
#endif
    for (int64_t q = 0; q < n_eval; ++q) {
        const int64_t i = rows ? rows[q] : q;
        int64_t *lj = list_j + q * k;
        double *ls = list_s + q * k;
        int64_t n = 0;
        list_n[q] = 0;
        if (!keep_row(attrR, opR, cR, i)) continue;
        const float *r = R + i * ldR;
        const double nr = oracle_norm(r, d);
        for (int64_t j = 0; j < nS; ++j) {
            if (!keep_row(attrS, opS, cS, j)) continue;
            const double sim = cosine_from(oracle_dot(r, S + j * ldS, d), nr, ns[j]);
            /* position p: the first entry that sim beats */
            int64_t p = n;
#if ORACLE_MUTANT == 8
            while (p > 0 && sim >= ls[p - 1]) --p; /* mutant 8: a tie goes to the larger j */
#else
            while (p > 0 && sim > ls[p - 1]) --p;
#endif
            if (p >= k) continue;
            const int64_t last = n < k ? n : k - 1; /* entries p .. last-1 move down by one */
            for (int64_t t = last; t > p; --t) {
                lj[t] = lj[t - 1];
                ls[t] = ls[t - 1];
            }
            lj[p] = j;
            ls[p] = sim;
            if (n < k) ++n;
        }
        list_n[q] = n;
    }
    (void)nt;
    int64_t n_out = 0;
    for (int64_t q = 0; q < n_eval; ++q) {
        for (int64_t t = 0; t < list_n[q]; ++t) {
            out_i[n_out] = (uint32_t)(rows ? rows[q] : q);
            out_j[n_out] = (uint32_t)list_j[q * k + t];
            out_sim[n_out] = list_s[q * k + t];
            ++n_out;
        }
    }
    free(ns);
    free(list_j);
    free(list_s);
    free(list_n);
    return n_out;
}
