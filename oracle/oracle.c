/*
 * FP64 CPU oracle of the alternating NNLS method of Nguyen & Ho,
 * "Accelerated Parallel and Distributed Algorithm using Limited Internal
 * Memory for Nonnegative Matrix Factorization" (arXiv 1506.08938).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is compared against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * library never links it and shares no code, header or constant with it.
 *
 * Notation (row-major everywhere):
 *   V  m x n data, one instance per row            (paper: V is n x m, columns)
 *   W  m x r coefficients  (paper F^T)             E-step of Alg. 1/2
 *   Ht n x r components    (paper G, i.e. H^T)     M-step of Alg. 1/2
 *   Objective  J = 1/2||V - W Ht^T||_F^2 + a_w sum(W) + a_h sum(Ht)
 *                  + b_w/2 ||W||_F^2 + b_h/2 ||Ht||_F^2
 * Each factor row solves the NQP of Eq. 2 (§3.2),
 *   min_x 1/2 x^T Q x + q^T x,  x >= 0,
 * with Q = X^T X + b I and q = -c + a 1 (L2 on the diagonal, L1 on the
 * linear term; the §3.5 text swaps the two coefficients, this follows its
 * objective), c being the row of the cross term.
 *
 * Parity status of each function is stated beside it; all are pinned by
 * tests under tests/ (closed forms, brute force, a textbook solver, the worked
 * example of §3.4 Eqs. 4-5, and invariants of §4.1).
 *
 * No blocking, fusion or reordering: loops follow the definitions.  OpenMP
 * is used only to run independent rows (independent NQP problems, Alg. 2)
 * at the same time; each row's arithmetic is sequential.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------------- */
/* Options of Alg. 3 (§3.4).                                                */
/* ---------------------------------------------------------------------- */
typedef struct {
    int max_inner;      /* K_max: cap on repeat-loop iterations (paper: none)  */
    double eps;         /* accelerated condition  s_k <= eps * s_0             */
    double abs_tol;     /* extra absolute stop    s_k <= abs_tol (0 = off)     */
    int cd_steps;       /* coordinate steps per iteration; -1 means r          */
    int rescale;        /* 1 = anti-lopsided rescaling (paper); 0 = off        */
    int pg;             /* 1 = exact line-search projected-gradient part       */
    int maxstop_mode;   /* 0 off; 1 'prev' (max of the previous half-step);
                           2 sequential per-thread as printed in Alg. 3        */
} oracle_nqp_opts;

/* ---------------------------------------------------------------------- */
/* Plain definitions: Gram, cross term.  Parity: pinned against numpy.       */
/* ---------------------------------------------------------------------- */

/* Q = X^T X + beta I, X rows x r (Alg. 2 "Q = G^T G", §4.2). */
OR_API void oracle_gram(const double *X, int64_t rows, int r, double beta, double *Q)
{
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < rows; ++k)
                s += X[k * r + i] * X[k * r + j];
            Q[i * r + j] = s + (i == j ? beta : 0.0);
        }
}

/* C = A B, A rows x k (row-major, leading dim lda), B k x r (Alg. 2 Y = F V^T). */
OR_API void oracle_cross_dense(const double *A, int64_t rows, int64_t k, int64_t lda,
                               const double *B, int r, double *C)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i)
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int64_t t = 0; t < k; ++t)
                s += A[i * lda + t] * B[t * r + j];
            C[i * r + j] = s;
        }
}

/* C = A B with A in CSR (rows x k), B k x r (Theorem 2: sparse cross term). */
OR_API void oracle_cross_csr(const int64_t *rowptr, const int32_t *colidx, const double *vals,
                             int64_t rows, const double *B, int r, double *C)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < rows; ++i)
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                s += vals[p] * B[(int64_t)colidx[p] * r + j];
            C[i * r + j] = s;
        }
}

/* ---------------------------------------------------------------------- */
/* Anti-lopsided rescaling (§3.4 Eq. 3; first lines of Alg. 3).             */
/*   d_i = sqrt(H_ii),  Qt = H / (d d^T),  diag(Qt) = 1.                    */
/* A coordinate with H_ii <= 0 (an all-zero factor column and no L2 term)   */
/* is "dead": the paper divides by zero there.  Reading: d_i = 1, its row   */
/* and column of Qt are zero and x_i is held at 0 (which is optimal, since  */
/* its linear term is then a >= 0).                                         */
/* Parity: pinned by invariants (unit diagonal, cosines in [0,1] for        */
/* nonnegative factors, sqrt(r) <= ||Qt||_F <= r, f(x) = ft(x.*d)).         */
/* ---------------------------------------------------------------------- */
OR_API void oracle_rescale(const double *H, int r, double *Qt, double *d, uint8_t *dead)
{
    for (int i = 0; i < r; ++i) {
        double hii = H[i * r + i];
        if (hii > 0.0) {
            d[i] = sqrt(hii);
            dead[i] = 0;
        } else {
            d[i] = 1.0;
            dead[i] = 1;
        }
    }
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
            if (dead[i] || dead[j])
                Qt[i * r + j] = 0.0;
            else if (i == j)
                Qt[i * r + j] = 1.0;   /* Q_ii = H_ii / sqrt(H_ii H_ii) = 1 */
            else
                Qt[i * r + j] = H[i * r + j] / (d[i] * d[j]);
        }
}

/* projected gradient of the bound-constrained problem: the passive set is
 * { i : y_i > 0 or g_i < 0 } (§3.4, "passive variables"). */
static double proj_grad_sq(const double *y, const double *g, const uint8_t *dead, int r)
{
    double s = 0.0;
    for (int i = 0; i < r; ++i)
        if (!dead[i] && (y[i] > 0.0 || g[i] < 0.0))
            s += g[i] * g[i];
    return s;
}

/* ---------------------------------------------------------------------- */
/* Alg. 3: fast combinational algorithm for one NQP.                        */
/*   H (r x r), h (r); x in: x0 (warm start), out: solution.                */
/*   *maxstop: the per-thread fast-break threshold (read when mode != 0,    */
/*   raised after the solve in mode 2).                                     */
/*   Returns the number of repeat-loop iterations performed.               */
/*   *s_final receives ||P(y_k, g_k)||^2 in the rescaled space.             */
/* Parity: the converged answer is pinned exactly (brute-force support      */
/* enumeration, Lawson-Hanson, KKT, closed forms); the iteration itself is  */
/* pinned by the §3.4 worked example (59 plain line-search steps).          */
/* ---------------------------------------------------------------------- */
/* min_gap (optional, instrumentation only): over all coordinate steps taken,
 * the smallest margin between the two largest gains, best - second, in units
 * of what an FP32 rendering of the same step cannot resolve: a gain D_i moves
 * by about |dx_i| dg when the gradient entry g_i is off by dg, and an FP32
 * gradient carries rounding of order dg = 2^-24 G with
 * G = max_i (|q_i| + sum_j |Q_ij| |y_j|), the size of the terms it is built
 * from.  min_gap[0] = min (best - second) / ((|dx_p| + |dx_s|) 2^-24 G);
 * min_gap[1] = min (best - second) / best, the plain relative margin;
 * min_gap[2] = the largest |dx_p| + |dx_s| over the steps whose margin is
 * below min_gap[3] such units (the size of a move that an unresolved choice
 * could have swapped). */
static int nqp_core(const double *H, const double *h, int r, double *x,
                    const oracle_nqp_opts *o, double *maxstop, double *s_final,
                    double *min_gap)
{
    double *Q = (double *)malloc(sizeof(double) * (size_t)r * r);
    double *buf = (double *)malloc(sizeof(double) * (size_t)r * 7);
    uint8_t *dead = (uint8_t *)malloc((size_t)r);
    double *d = buf, *q = buf + r, *y = buf + 2 * r, *g = buf + 3 * r;
    double *gb = buf + 4 * r, *u = buf + 5 * r, *yn = buf + 6 * r;
    int T = o->cd_steps < 0 ? r : o->cd_steps;

    /* re-scaling variables */
    if (o->rescale) {
        oracle_rescale(H, r, Q, d, dead);
    } else {
        for (int i = 0; i < r; ++i) {
            d[i] = 1.0;
            dead[i] = H[i * r + i] > 0.0 ? 0 : 1;
        }
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < r; ++j)
                Q[i * r + j] = (dead[i] || dead[j]) ? 0.0 : H[i * r + j];
    }
    for (int i = 0; i < r; ++i) {
        q[i] = dead[i] ? 0.0 : h[i] / d[i];
        y[i] = dead[i] ? 0.0 : x[i] * d[i];
    }
    /* gradient f = Q y + q */
    for (int i = 0; i < r; ++i) {
        double s = q[i];
        for (int j = 0; j < r; ++j)
            s += Q[i * r + j] * y[j];
        g[i] = dead[i] ? 0.0 : s;
    }
    double s0 = proj_grad_sq(y, g, dead, r);
    double sk = s0;
    int k = 0;
    if (s0 > 0.0) {
        for (k = 1; k <= o->max_inner; ++k) {
            /* exact line search on the masked gradient */
            if (o->pg) {
                double s = 0.0;
                for (int i = 0; i < r; ++i) {
                    gb[i] = (!dead[i] && (y[i] > 0.0 || g[i] < 0.0)) ? g[i] : 0.0;
                    s += gb[i] * gb[i];
                }
                if (s > 0.0) {
                    double den = 0.0;
                    for (int i = 0; i < r; ++i) {
                        double t = 0.0;
                        for (int j = 0; j < r; ++j)
                            t += Q[i * r + j] * gb[j];
                        u[i] = t;
                        den += gb[i] * t;
                    }
                    if (den > 0.0) {
                        double alpha = s / den;
                        for (int i = 0; i < r; ++i) {
                            double v = y[i] - alpha * gb[i];
                            yn[i] = v > 0.0 ? v : 0.0;
                        }
                        /* f_k = f_{k-1} + Q (x_k - x_{k-1}) */
                        for (int i = 0; i < r; ++i)
                            u[i] = yn[i] - y[i];
                        for (int i = 0; i < r; ++i) {
                            double t = 0.0;
                            for (int j = 0; j < r; ++j)
                                t += Q[i * r + j] * u[j];
                            g[i] += t;
                        }
                        for (int i = 0; i < r; ++i)
                            y[i] = yn[i];
                    }
                }
            }
            /* greedy block coordinate descent */
            for (int t = 0; t < T; ++t) {
                int p = -1;
                double best = 0.0, dp = 0.0, second = 0.0, ds = 0.0;
                for (int i = 0; i < r; ++i) {
                    if (dead[i])
                        continue;
                    double qii = Q[i * r + i];
                    double v = y[i] - g[i] / qii;
                    double di = (v > 0.0 ? v : 0.0) - y[i];
                    double gain = -(g[i] * di + 0.5 * qii * di * di);
                    if (gain > best) {    /* strict: lowest index wins ties */
                        second = best;
                        ds = dp;
                        best = gain;
                        p = i;
                        dp = di;
                    } else if (gain > second) {
                        second = gain;
                        ds = di;
                    }
                }
                if (p < 0)
                    break;
                if (min_gap) {
                    double G = 0.0;
                    for (int i = 0; i < r; ++i) {
                        double s = fabs(q[i]);
                        for (int j = 0; j < r; ++j)
                            s += fabs(Q[i * r + j]) * fabs(y[j]);
                        if (s > G)
                            G = s;
                    }
                    double unit = (fabs(dp) + fabs(ds)) * ldexp(G, -24);
                    double m0 = unit > 0.0 ? (best - second) / unit : 1e300;
                    if (m0 < min_gap[0])
                        min_gap[0] = m0;
                    if (m0 < min_gap[3] && fabs(dp) + fabs(ds) > min_gap[2])
                        min_gap[2] = fabs(dp) + fabs(ds);
                    if ((best - second) / best < min_gap[1])
                        min_gap[1] = (best - second) / best;
                }
                for (int i = 0; i < r; ++i)
                    g[i] += Q[i * r + p] * dp;   /* Q symmetric: column p */
                y[p] += dp;
            }
            sk = proj_grad_sq(y, g, dead, r);
            if (sk <= o->eps * s0)
                break;
            if (o->abs_tol > 0.0 && sk <= o->abs_tol)
                break;
            if (o->maxstop_mode != 0 && maxstop && sk <= *maxstop)
                break;
        }
        if (k > o->max_inner)
            k = o->max_inner;
    }
    if (o->maxstop_mode == 2 && maxstop && sk > *maxstop)
        *maxstop = sk;
    if (s_final)
        *s_final = sk;
    for (int i = 0; i < r; ++i)
        x[i] = dead[i] ? 0.0 : y[i] / d[i];
    free(Q);
    free(buf);
    free(dead);
    return k;
}

OR_API int oracle_nqp(const double *H, const double *h, int r, double *x,
                      const oracle_nqp_opts *o, double *maxstop, double *s_final)
{
    return nqp_core(H, h, r, x, o, maxstop, s_final, NULL);
}

/* Alg. 3 as oracle_nqp, also reporting the margins between the two largest
 * gains of its coordinate steps described at nqp_core: out[0..2] as
 * min_gap[0..2] there (1e300, 1 and 0 if it took no step), with the
 * unresolved-step threshold tie_units in FP32 gain-resolution units. */
OR_API int oracle_nqp_min_gap(const double *H, const double *h, int r, double *x,
                              const oracle_nqp_opts *o, double tie_units, double *out)
{
    double mg[4] = {1e300, 1.0, 0.0, tie_units};
    int k = nqp_core(H, h, r, x, o, NULL, NULL, mg);
    out[0] = mg[0];
    out[1] = mg[1];
    out[2] = mg[2];
    return k;
}

/* ---------------------------------------------------------------------- */
/* One half-step: every row of X solves the NQP with the shared Q and      */
/* q_i = -C_i + alpha 1 (Alg. 2 loops; §3.5 for alpha).                     */
/* Mode 1 ('prev'): maxstop_in is the fixed threshold of every row and     */
/*   *maxstop_out receives the max final s over rows.                       */
/* Mode 2 (sequential, as printed): rows run in order on one thread whose   */
/*   running maxStop starts at maxstop_in and is returned in *maxstop_out.  */
/* Returns the total number of inner iterations.                            */
/* ---------------------------------------------------------------------- */
OR_API int64_t oracle_nnls_update(const double *Q, const double *C, int64_t rows, int r,
                                  double alpha, double *X, const oracle_nqp_opts *o,
                                  double maxstop_in, double *maxstop_out, int32_t *iters)
{
    int64_t total = 0;
    double smax = 0.0;
    if (o->maxstop_mode == 2) {
        double ms = maxstop_in;   /* the one thread's running maxStop */
        double *h = (double *)malloc(sizeof(double) * r);
        for (int64_t i = 0; i < rows; ++i) {
            for (int j = 0; j < r; ++j)
                h[j] = -C[i * r + j] + alpha;
            double sf = 0.0;
            int k = oracle_nqp(Q, h, r, X + i * r, o, &ms, &sf);
            if (iters)
                iters[i] = k;
            total += k;
        }
        smax = ms;
        free(h);
    } else {
#pragma omp parallel
        {
            double *h = (double *)malloc(sizeof(double) * r);
            int64_t tot = 0;
            double sm = 0.0;
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < rows; ++i) {
                for (int j = 0; j < r; ++j)
                    h[j] = -C[i * r + j] + alpha;
                double ms = maxstop_in, sf = 0.0;
                int k = oracle_nqp(Q, h, r, X + i * r, o, &ms, &sf);
                if (iters)
                    iters[i] = k;
                tot += k;
                if (sf > sm)
                    sm = sf;
            }
#pragma omp critical
            {
                total += tot;
                if (sm > smax)
                    smax = sm;
            }
            free(h);
        }
    }
    if (maxstop_out)
        *maxstop_out = smax;
    return total;
}

/* ---------------------------------------------------------------------- */
/* Objective (Def. 1, reported as 1/2||.||^2 per Table 4) plus penalties,   */
/* evaluated directly from the residual.  Parity: pinned (tests compute the */
/* residual with numpy and check the trace identity).                       */
/* ---------------------------------------------------------------------- */
OR_API double oracle_objective_dense(const double *V, int64_t m, int64_t n, const double *W,
                                     const double *Ht, int r, double aw, double ah,
                                     double bw, double bh)
{
    double fit = 0.0;
#pragma omp parallel for reduction(+ : fit) schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < r; ++k)
                s += W[i * r + k] * Ht[j * r + k];
            double e = V[i * n + j] - s;
            fit += e * e;
        }
    double l1w = 0, l2w = 0, l1h = 0, l2h = 0;
    for (int64_t i = 0; i < m * r; ++i) {
        l1w += W[i];
        l2w += W[i] * W[i];
    }
    for (int64_t i = 0; i < n * r; ++i) {
        l1h += Ht[i];
        l2h += Ht[i] * Ht[i];
    }
    return 0.5 * fit + aw * l1w + ah * l1h + 0.5 * bw * l2w + 0.5 * bh * l2h;
}

/* Same for CSR V: ||V - W Ht^T||^2 = ||V||^2 - 2<V, W Ht^T> + ||W Ht^T||^2,
 * the last term expanded as sum_{k,l} (W^T W)_{kl} (Ht^T Ht)_{kl}; every term
 * is a plain sum written out. */
OR_API double oracle_objective_csr(const int64_t *rowptr, const int32_t *colidx,
                                   const double *vals, int64_t m, int64_t n, const double *W,
                                   const double *Ht, int r, double aw, double ah, double bw,
                                   double bh)
{
    double vv = 0.0, vwh = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            double s = 0.0;
            for (int k = 0; k < r; ++k)
                s += W[i * r + k] * Ht[(int64_t)colidx[p] * r + k];
            vv += vals[p] * vals[p];
            vwh += vals[p] * s;
        }
    double *GW = (double *)malloc(sizeof(double) * r * r);
    double *GH = (double *)malloc(sizeof(double) * r * r);
    oracle_gram(W, m, r, 0.0, GW);
    oracle_gram(Ht, n, r, 0.0, GH);
    double whwh = 0.0;
    for (int i = 0; i < r * r; ++i)
        whwh += GW[i] * GH[i];
    free(GW);
    free(GH);
    double l1w = 0, l2w = 0, l1h = 0, l2h = 0;
    for (int64_t i = 0; i < m * r; ++i) {
        l1w += W[i];
        l2w += W[i] * W[i];
    }
    for (int64_t i = 0; i < n * r; ++i) {
        l1h += Ht[i];
        l2h += Ht[i] * Ht[i];
    }
    return 0.5 * (vv - 2.0 * vwh + whwh) + aw * l1w + ah * l1h + 0.5 * bw * l2w + 0.5 * bh * l2h;
}

/* KKT residuals of one half-step's NQPs (Eq. 2 optimality: x >= 0,
 * grad >= 0, x.*grad = 0): out[0] = max_i |min(x_i, grad_i)|,
 * out[1] = max_i |x_i grad_i|, with grad = Q x + q, q = -c + alpha. */
OR_API void oracle_kkt(const double *Q, const double *C, int64_t rows, int r, double alpha,
                       const double *X, double *out)
{
    double m1 = 0.0, m2 = 0.0;
    for (int64_t i = 0; i < rows; ++i)
        for (int j = 0; j < r; ++j) {
            double gj = -C[i * r + j] + alpha;
            for (int k = 0; k < r; ++k)
                gj += Q[j * r + k] * X[i * r + k];
            double x = X[i * r + j];
            double a = fabs(x < gj ? x : gj);
            double b = fabs(x * gj);
            if (a > m1)
                m1 = a;
            if (b > m2)
                m2 = b;
        }
    out[0] = m1;
    out[1] = m2;
}

/* ---------------------------------------------------------------------- */
/* Alg. 1/2 outer loop: W-update (E-step) then H-update (M-step).           */
/* V given dense (Vd, m x n) or CSR (rowptr...; and its transpose).         */
/* hist[2t] = J after the W-update of iteration t, hist[2t+1] = J after the */
/* H-update.  iters_total receives the total inner iterations, for          */
/* kbar = iters_total / (T (m + n)) (§5.3).                                 */
/* ---------------------------------------------------------------------- */
typedef struct {
    int outer_iters;
    double alpha_w, alpha_h, beta_w, beta_h;
    oracle_nqp_opts nqp;
} oracle_solve_opts;

static double obj_any(const double *Vd, const int64_t *rp, const int32_t *ci, const double *va,
                      int64_t m, int64_t n, const double *W, const double *Ht, int r,
                      const oracle_solve_opts *o)
{
    if (Vd)
        return oracle_objective_dense(Vd, m, n, W, Ht, r, o->alpha_w, o->alpha_h, o->beta_w,
                                      o->beta_h);
    return oracle_objective_csr(rp, ci, va, m, n, W, Ht, r, o->alpha_w, o->alpha_h, o->beta_w,
                                o->beta_h);
}

OR_API int64_t oracle_nmf_solve(const double *Vd, const int64_t *rp, const int32_t *ci,
                                const double *va, const int64_t *trp, const int32_t *tci,
                                const double *tva, int64_t m, int64_t n, int r, double *W,
                                double *Ht, const oracle_solve_opts *o, double *hist)
{
    double *Q = (double *)malloc(sizeof(double) * r * r);
    double *CW = (double *)malloc(sizeof(double) * (size_t)m * r);
    double *CH = (double *)malloc(sizeof(double) * (size_t)n * r);
    double *VT = NULL;
    if (Vd) {
        VT = (double *)malloc(sizeof(double) * (size_t)m * n);
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < n; ++j)
                VT[j * m + i] = Vd[i * n + j];
    }
    int64_t total = 0;
    double msw = 0.0, msh = 0.0;   /* mode 1: previous half-step max, per factor */
    for (int t = 0; t < o->outer_iters; ++t) {
        double ms_next = 0.0, ms_seq = 0.0;   /* mode 2: Alg. 2 resets maxStop per iteration */
        /* E-step: Q = H H^T + b_w I, C = V H^T */
        oracle_gram(Ht, n, r, o->beta_w, Q);
        if (Vd)
            oracle_cross_dense(Vd, m, n, n, Ht, r, CW);
        else
            oracle_cross_csr(rp, ci, va, m, Ht, r, CW);
        total += oracle_nnls_update(Q, CW, m, r, o->alpha_w, W, &o->nqp,
                                    o->nqp.maxstop_mode == 2 ? ms_seq : msw, &ms_next, NULL);
        if (o->nqp.maxstop_mode == 2)
            ms_seq = ms_next;
        else
            msw = ms_next;
        if (hist)
            hist[2 * t] = obj_any(Vd, rp, ci, va, m, n, W, Ht, r, o);
        /* M-step: Q = W^T W + b_h I, C = V^T W */
        oracle_gram(W, m, r, o->beta_h, Q);
        if (Vd)
            oracle_cross_dense(VT, n, m, m, W, r, CH);
        else
            oracle_cross_csr(trp, tci, tva, n, W, r, CH);
        total += oracle_nnls_update(Q, CH, n, r, o->alpha_h, Ht, &o->nqp,
                                    o->nqp.maxstop_mode == 2 ? ms_seq : msh, &ms_next, NULL);
        if (o->nqp.maxstop_mode != 2)
            msh = ms_next;
        if (hist)
            hist[2 * t + 1] = obj_any(Vd, rp, ci, va, m, n, W, Ht, r, o);
    }
    free(Q);
    free(CW);
    free(CH);
    free(VT);
    return total;
}

OR_API int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
