/*
 * pagerank_oracle.c — plain, slow, FP64 CPU oracle for pull-based PageRank.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only the test-suite, the package's smoke check and the
 * benchmark's CPU-baseline leg do. It shares no code with the CUDA path.
 *
 * What it computes (Adjusting PageRank parameters and Comparing results,
 * Section 2 for the iteration and the teleport term, Section 3 for the norms,
 * Section 2 for the 500-iteration cap and Section 4 for halting at the cap):
 *
 *   r^0          = 1/N for every vertex, or the caller's start vector
 *   for i = 1 .. max_iter:
 *     D          = sum of r^{i-1}[u] over vertices u with out-degree 0
 *     c0         = (1 - alpha)/N + alpha * D / N          (common teleport)
 *     r^i[v]     = c0 + alpha * sum over in-edges u->v of r^{i-1}[u] / d_u
 *     err        = ||r^i - r^{i-1}|| in the chosen norm
 *                  L1  : sum |x|
 *                  L2  : sqrt(sum |x|^2)
 *                  Linf: max |x|
 *     stop, converged, when err < tau
 *   otherwise stop, not converged, after max_iter updates.
 *
 * The iteration is Jacobi-style: every term uses the previous iterate. Every
 * sum (a vertex's in-edge sum in CSR order, the dangling sum and the norms in
 * vertex order) is a sequential FP64 sum with Neumaier's compensation
 * (Neumaier 1974): the same sum as written, with its rounding error carried
 * in a second accumulator, so that long sums over hub rows keep the total
 * mass at 1 to rounding. Optional threads split only the vertex loop, whose
 * entries are independent, so the result is bit-identical for every thread
 * count.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused and x86-64
 * and aarch64 hosts produce identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_L1 = 1, OR_L2 = 2, OR_LINF = 3 };

/* Compensated running sum (Neumaier's variant of Kahan summation). */
typedef struct { double s, c; } csum;
static inline void csum_add(csum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double csum_get(const csum *a) { return a->s + a->c; }

/* The three norms of a - b (Section 3). out[0] = L1, out[1] = L2, out[2] = Linf. */
void oracle_norms(int32_t n, const double *a, const double *b, double *out) {
    csum l1 = {0.0, 0.0}, sq = {0.0, 0.0};
    double mx = 0.0;
    for (int32_t v = 0; v < n; v++) {
        double x = fabs(a[v] - b[v]);
        csum_add(&l1, x);
        csum_add(&sq, x * x);
        if (x > mx) mx = x;
    }
    out[0] = csum_get(&l1);
    out[1] = sqrt(csum_get(&sq));
    out[2] = mx;
}

/* One PageRank update r_new = c0 + alpha * A^T (r / d) (Section 2).
 * Returns the dangling sum D that entered c0 through *dangling_out. */
void oracle_step(int32_t n, const int32_t *offsets, const int32_t *sources, const int32_t *outdeg,
                 double alpha, const double *r, double *r_new, double *dangling_out, int nthreads) {
    csum Dc = {0.0, 0.0};
    for (int32_t u = 0; u < n; u++)
        if (outdeg[u] == 0) csum_add(&Dc, r[u]);
    double D = csum_get(&Dc);
    double N = (double)n;
    double c0 = (1.0 - alpha) / N + alpha * D / N;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int32_t v = 0; v < n; v++) {
        csum s = {0.0, 0.0};
        for (int32_t e = offsets[v]; e < offsets[v + 1]; e++) {
            int32_t u = sources[e];
            csum_add(&s, r[u] / (double)outdeg[u]);
        }
        r_new[v] = c0 + alpha * csum_get(&s);
    }
    if (dangling_out) *dangling_out = D;
}

/*
 * Full solve. Returns 0 on success, 1 on bad arguments, 2 on allocation failure.
 *   init          : n doubles or NULL for the uniform start 1/N
 *   ranks_out     : n doubles (the iterate at the stopping iteration)
 *   iters_out     : number of updates performed (max_iter when not converged)
 *   err_out       : the chosen norm at the stopping iteration
 *   converged_out : 1 when err < tau was reached
 *   err_hist      : NULL or 3*max_iter doubles; row i-1 holds (L1, L2, Linf)
 *                   of r^i - r^{i-1}
 */
int oracle_pagerank(int32_t n, const int32_t *offsets, const int32_t *sources, const int32_t *outdeg,
                    double alpha, double tau, int32_t norm, int32_t max_iter, const double *init,
                    double *ranks_out, int32_t *iters_out, double *err_out, int32_t *converged_out,
                    double *err_hist, int nthreads) {
    if (n < 1 || !offsets || !outdeg || !ranks_out || max_iter < 1) return 1;
    if (norm < OR_L1 || norm > OR_LINF) return 1;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !s) { free(r); free(s); return 2; }
    for (int32_t v = 0; v < n; v++) r[v] = init ? init[v] : 1.0 / (double)n;
    int32_t it = 0, conv = 0;
    double err = 0.0;
    while (it < max_iter) {
        oracle_step(n, offsets, sources, outdeg, alpha, r, s, NULL, nthreads);
        double nv[3];
        oracle_norms(n, s, r, nv);
        it++;
        if (err_hist) { err_hist[3 * (it - 1)] = nv[0]; err_hist[3 * (it - 1) + 1] = nv[1]; err_hist[3 * (it - 1) + 2] = nv[2]; }
        err = nv[norm - 1];
        double *t = r; r = s; s = t;
        if (err < tau) { conv = 1; break; }
    }
    memcpy(ranks_out, r, sizeof(double) * (size_t)n);
    if (iters_out) *iters_out = it;
    if (err_out) *err_out = err;
    if (converged_out) *converged_out = conv;
    free(r);
    free(s);
    return 0;
}

/*
 * Per-vertex features for the learned warm start (spec workload; no
 * counterpart in the paper): for every vertex v
 *   f0 = log(1 + in-degree(v))
 *   f1 = log(1 + out-degree(v))
 *   f2 = mean over in-neighbours u of log(1 + out-degree(u))   (0 if none)
 *   f3 = max  over in-neighbours u of log(1 + out-degree(u))   (0 if none)
 *   f4 = alpha
 * written row-major into feat[5*v + k].
 */
void oracle_features(int32_t n, const int32_t *offsets, const int32_t *sources, const int32_t *outdeg,
                     double alpha, double *feat) {
    for (int32_t v = 0; v < n; v++) {
        int32_t deg = offsets[v + 1] - offsets[v];
        csum sc = {0.0, 0.0};
        double mx = 0.0;
        for (int32_t e = offsets[v]; e < offsets[v + 1]; e++) {
            double x = log(1.0 + (double)outdeg[sources[e]]);
            csum_add(&sc, x);
            if (x > mx) mx = x;
        }
        double sum = csum_get(&sc);
        feat[5 * (size_t)v + 0] = log(1.0 + (double)deg);
        feat[5 * (size_t)v + 1] = log(1.0 + (double)outdeg[v]);
        feat[5 * (size_t)v + 2] = deg > 0 ? sum / (double)deg : 0.0;
        feat[5 * (size_t)v + 3] = deg > 0 ? mx : 0.0;
        feat[5 * (size_t)v + 4] = alpha;
    }
}
