/*
 * nmf.h - C ABI of the GB300 alternating-NNLS NMF library (libnmf.so).
 *
 * Method: Nguyen & Ho, "Accelerated Parallel and Distributed Algorithm using
 * Limited Internal Memory for Nonnegative Matrix Factorization",
 * arXiv 1506.08938.  Minimise
 *     J(W, H) = 1/2 ||V - W H||_F^2 + a_w sum(W) + a_h sum(H)
 *               + b_w/2 ||W||_F^2 + b_h/2 ||H||_F^2,   W, H >= 0,
 * by alternating updates (Alg. 1 and Alg. 2 of §3).  Each half-step splits into
 * independent r-dimensional nonnegative quadratic programs (Eq. 2, §3.2)
 *     min_x 1/2 x^T Q x + q^T x,  x >= 0,
 * that share one Q, solved by the anti-lopsided + greedy coordinate descent
 * iteration (Alg. 3, §3.4).  L1/L2 penalties fold into q and Q (§3.5).
 *
 * Conventions for every call:
 *  - Layout.  Matrices are row-major.  V is m x n with one instance per row
 *    (the paper stores instances as columns: V_here = V_paper^T).  W is m x r.
 *    H is kept as its transpose Ht (n x r) so that every NQP works on one
 *    contiguous r-vector.  r <= 128 (NMF_E_SHAPE above).
 *  - Memory.  Unless stated otherwise every pointer is DEVICE memory owned by
 *    the caller.  The library owns only its handle's workspace, which it
 *    allocates on first use at a given size and frees in nmf_destroy.
 *  - Execution.  Calls enqueue work on the handle's stream and return without
 *    waiting, except where stated.  Argument errors (NULL pointers, negative
 *    sizes, r out of range, unsupported dtype) are returned before anything
 *    is launched.  Errors found on the device (non-finite input, a wait that
 *    ran out) are latched in a device status word and returned by the next
 *    synchronising call (nmf_sync, nmf_solve).
 *  - Threads.  A handle is used by one host thread at a time.  No exception
 *    crosses this interface.
 */
#ifndef NMF_GB300_H
#define NMF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NMF_OK = 0,
    NMF_E_ARG = 1,        /* NULL pointer, negative size, bad option value     */
    NMF_E_SHAPE = 2,      /* inconsistent shapes, r < 1 or r > 128             */
    NMF_E_DTYPE = 3,      /* dtype not supported by this call                  */
    NMF_E_NOMEM = 4,      /* workspace allocation failed                      */
    NMF_E_CUDA = 5,       /* a CUDA runtime call failed (no device, launch)   */
    NMF_E_NONFINITE = 6,  /* NaN/Inf met in an input row (row left unchanged) */
    NMF_E_TIMEOUT = 7,    /* a bounded device-side wait ran out                */
    NMF_E_BUSY = 8,       /* admission refused (serving: over memory budget)   */
    NMF_E_NOTIMPL = 9     /* combination of options not implemented           */
} nmf_status;

typedef enum { NMF_F32 = 0, NMF_BF16 = 1, NMF_F64 = 2 } nmf_dtype;

/* Arithmetic of the dense cross-term products (the NNLS sweeps are always
 * FP32, the Gram matrices FP32 on CUDA cores).
 *  FP32       FP32-accurate: on tcgen05 tensor cores each operand is split
 *             into a TF32-exact high part and its remainder and
 *             hi*hi + hi*lo + lo*hi is accumulated in FP32 (relative error
 *             ~1e-7, as FP32 summation); falls back to FP32_SIMT when the
 *             data's row pitch is not a multiple of 16 bytes.
 *  TF32       operands truncated to TF32 (10-bit mantissa), FP32 accumulate.
 *  BF16       operands rounded to BF16, FP32 accumulate (the solve keeps a
 *             BF16 copy of V and V^T on the device).
 *  BF16X2     split BF16 (hi + lo).  Cross term (nmf_cross with BF16 V,
 *             nmf_solve): V read once rounded to BF16 (as for BF16), the
 *             factor split as hi = bf16(x), lo = bf16(x - hi), both products
 *             in one MMA, FP32 accumulate: the factor enters with relative
 *             error <= 2^-16 instead of BF16's 2^-8, so the NQP's cross term
 *             stays consistent with its FP32 Gram from one outer iteration to
 *             the next.  nmf_gram: see there.
 *  FP32_SIMT  plain FP32 fused multiply-adds on CUDA cores. */
typedef enum {
    NMF_PREC_FP32 = 0,
    NMF_PREC_TF32 = 1,
    NMF_PREC_BF16 = 2,
    NMF_PREC_BF16X2 = 3,
    NMF_PREC_FP32_SIMT = 4
} nmf_prec;

typedef struct nmf_ctx *nmf_handle;

/* Dense row-major matrix: element (i, j) at data[i * ld + j]. */
typedef struct {
    int64_t rows, cols, ld;
    nmf_dtype dt;
    const void *data;
} nmf_dense;

/* CSR matrix: row i holds colidx/vals[rowptr[i] .. rowptr[i+1]). */
typedef struct {
    int64_t rows, cols, nnz;
    const int64_t *rowptr;   /* rows + 1 entries, rowptr[0] = 0 */
    const int32_t *colidx;   /* nnz entries, each in [0, cols)  */
    const void *vals;        /* nnz entries of type dt          */
    nmf_dtype dt;
} nmf_csr;

typedef struct {
    int is_sparse;           /* 0: d is used, 1: s is used */
    nmf_dense d;
    nmf_csr s;
} nmf_matrix;

/* Options of Alg. 3 (§3.4).  Zero-initialised fields select the defaults
 * noted in brackets via nmf_nnls_opts_default(). */
typedef struct {
    int max_inner;       /* cap on repeat-loop iterations per NQP [50]         */
    double eps;          /* accelerated condition ||f_k||^2 <= eps ||f_0||^2,
                            f = projected gradient in the rescaled space [1e-3] */
    int cd_steps;        /* greedy coordinate steps per iteration, -1 = r [-1] */
    int maxstop_mode;    /* fast-break rule of Alg. 3: 0 off; 1 = a row stops
                            once ||f||^2 <= threshold; in nmf_solve the
                            threshold is the largest final ||f||^2 of the
                            previous update of the same factor (0 before the
                            first), a deterministic reading [0]              */
    float maxstop;       /* threshold for mode 1 in nmf_nnls_update [0]       */
    int lanes;           /* lanes of a warp per row problem: 1, 2, 4, ..., 32
                            with lanes * 16 >= r; 0 = chosen from r [0]       */
    int grad_refresh;    /* > 0: every grad_refresh-th repeat-loop iteration of
                            a row recomputes its gradient Qt y + qt from
                            scratch instead of carrying it by the updates of
                            Alg. 3 (the FP32 rounding those accumulate over
                            hundreds of iterations otherwise shifts the point
                            a long solve converges to); 0 = off [0]           */
} nmf_nnls_opts;

/* Options of the outer loop (Alg. 1 / Alg. 2). */
typedef struct {
    int outer_iters;         /* iterations to run (upper bound if a gap target) */
    double rel_gap_target;   /* stop once (J - f_star)/f_star <= target; 0 off  */
    double f_star;           /* reference optimum for the gap test             */
    float alpha_w, alpha_h;  /* L1 weights                                     */
    float beta_w, beta_h;    /* L2 weights (added to the Gram diagonal)        */
    nmf_prec prec;           /* product arithmetic                            */
    nmf_nnls_opts nnls;
    int check_every;         /* gap test period in iterations (0 = 1); < 0:
                                adaptive - the next test is scheduled from
                                the gap's measured rate of decrease         */
    int use_graph;           /* 1: capture one iteration as a CUDA graph       */
    int objective;           /* how J is evaluated after each iteration:
                                0 = FP64 trace identity (cheap; its FP32 inputs
                                limit it to about 1e-7 ||V||^2 / J relative),
                                1 = FP64 sum of element-wise residuals (dense
                                V only; one extra pass over V)               */
    double *obj_hist;        /* optional HOST array [outer_iters]: J after each
                                full iteration (evaluated as `objective` says) */
} nmf_solve_opts;

typedef struct {
    int iters_done;          /* outer iterations performed                    */
    double objective;        /* J after the last iteration (FP64)             */
    double rel_gap;          /* (J - f_star)/f_star, or 0 without f_star       */
    double kbar;             /* inner iterations / (iters_done (m + n)) (§5.3) */
    double kkt_max;          /* max |min(x, grad)| over both factors (FP64)   */
    double ms_total;         /* device time of the loop (CUDA events)         */
    int64_t inner_total;     /* inner iterations summed over all NQPs         */
} nmf_report;

/* ---- handle -------------------------------------------------------------- */

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Returns NMF_E_CUDA if
 * the device cannot be used. */
nmf_status nmf_create(nmf_handle *out, int device, void *cuda_stream);
/* Free the handle's workspace (waits for its stream first). */
nmf_status nmf_destroy(nmf_handle h);
/* Re-bind the handle to another stream of the same device. */
nmf_status nmf_set_stream(nmf_handle h, void *cuda_stream);
/* Wait for the handle's stream; return and clear the latched device status. */
nmf_status nmf_sync(nmf_handle h);
/* Static description of a status code. */
const char *nmf_status_string(nmf_status s);
/* Fill `o` with the defaults listed in nmf_nnls_opts. */
void nmf_nnls_opts_default(nmf_nnls_opts *o);
/* Number of kernels this process has launched through the library. */
int64_t nmf_launch_count(void);

/* ---- steps of one half-step ------------------------------------------------ */

/* Gram matrix Q = X^T X + beta I (r x r, FP32), X rows x r (F32, ld >= r).
 * Alg. 2 "Q = G^T G" (the printed "G G^T" is r x r only as G^T G; §4.2 gives
 * its O(n r^2) cost); beta is the L2 weight of §3.5.  prec selects the
 * operand arithmetic, always with FP32 accumulation on CUDA cores:
 *   FP32, FP32_SIMT  the stored FP32 values;
 *   TF32             each element rounded to the nearest TF32 (11 significant bits);
 *   BF16             each element rounded to the nearest BF16 (8 significant bits);
 *   BF16X2           each element split as hi = bf16(x), lo = bf16(x - hi) and
 *                    hi hi + hi lo + lo hi accumulated (relative error of
 *                    each product ~2^-16: a Gram from BF16 storage accurate
 *                    to about FP32 level where conditioning needs it).
 * nmf_solve forms its Grams from the FP32 factors in FP32 under every prec. */
nmf_status nmf_gram(nmf_handle h, const nmf_dense *X, float beta, nmf_prec prec, float *Q);

/* Cross term C = V B (V rows x k dense F32/BF16 or CSR with F32/BF16 values;
 * B k x r F32 row-major; C rows x r F32).  Alg. 2 "Y = F V^T" and the linear
 * term of Eq. 2 (h = -A^T b); Theorem 2 for the sparse cost.  Dense V uses
 * prec; CSR V always accumulates in FP32 from its stored values. */
nmf_status nmf_cross(nmf_handle h, const nmf_matrix *V, const float *B, int r, nmf_prec prec,
                     float *C);

/* Anti-lopsided rescaling (§3.4 Eq. 3, first lines of Alg. 3):
 * d_i = sqrt(Q_ii), Qt = Q ./ (d d^T) with unit diagonal.  A coordinate with
 * Q_ii <= 0 is dead: d_i = 1 and its row and column of Qt are zero (its
 * variable is then held at 0).  Q, Qt r x r; d length r. */
nmf_status nmf_rescale(nmf_handle h, const float *Q, int r, float *Qt, float *d);

/* Batched NQP solve (Alg. 3) for `rows` problems sharing Qt:
 * row i minimises 1/2 x^T Q x + (alpha 1 - C_i)^T x, x >= 0, with
 * Q = D Qt D, D = diag(d) (Qt, d from nmf_rescale).  X (rows x r) is the warm
 * start on entry (Alg. 3 input x0) and the solution on return.  inner_iters
 * (optional, rows entries) receives each row's repeat-loop count. */
nmf_status nmf_nnls_update(nmf_handle h, const float *Qt, const float *d, const float *C,
                           int64_t rows, int r, float alpha, float *X,
                           const nmf_nnls_opts *opts, int32_t *inner_iters);

/* ---- objective and optimality ---------------------------------------------- */

/* J by the trace identity in FP64 (Def. 1, Table 4's 1/2 ||.||^2):
 *   J = 1/2 (vv - 2 <Ht, Ch> + <Gw, Gh>) + a_w sum W + a_h sum Ht
 *       + b_w/2 tr Gw + b_h/2 tr Gh
 * vv = ||V||_F^2, Ch = V^T W (n x r), Gw = W^T W, Gh = Ht^T Ht (r x r,
 * without the L2 term).  Writes one double to *J_dev (device). */
nmf_status nmf_objective(nmf_handle h, double vv, const float *W, int64_t m, const float *Ht,
                         int64_t n, int r, const float *Ch, const float *Gw, const float *Gh,
                         float alpha_w, float alpha_h, float beta_w, float beta_h,
                         double *J_dev);

/* J from the element-wise residual, FP64 (Def. 1, Table 4's 1/2 ||.||^2):
 *   J = 1/2 sum_ij (V_ij - W_i . Ht_j)^2 + a_w sum W + a_h sum Ht
 *       + b_w/2 ||W||^2 + b_h/2 ||Ht||^2,
 * each W_i . Ht_j formed in FP32, the squares summed in FP64.  V dense F32
 * m x n; W m x r; Ht n x r.  Writes one double to *J_dev (device). */
nmf_status nmf_objective_direct(nmf_handle h, const nmf_dense *V, const float *W, const float *Ht,
                                int r, float alpha_w, float alpha_h, float beta_w, float beta_h,
                                double *J_dev);

/* KKT residuals of Eq. 2 for one factor: with
 * grad_i = Q X_i - C_i + alpha (Q r x r including the L2 term; symmetric, as
 * every Gram is - it is read by columns),
 * out_dev[0] = max |min(X_ij, grad_ij)|, out_dev[1] = max |X_ij grad_ij|.
 * The sums of Q X_i run in float-float (exact FP32 products, compensated
 * sums, ~44 bits); the residuals and maxima are FP64.  r <= 128. */
nmf_status nmf_kkt(nmf_handle h, const float *Q, const float *C, int64_t rows, int r,
                   float alpha, const float *X, double *out_dev);

/* ---- whole method ---------------------------------------------------------- */

/* Alternating solve (Alg. 1 / Alg. 2): for t = 1..outer_iters
 *   W-update:  Q = Ht^T Ht + b_w I, C = V Ht,  every row of W by Alg. 3;
 *   H-update:  Q = W^T W + b_h I,   C = V^T W, every row of Ht by Alg. 3;
 * then J by the FP64 trace identity.  V is dense (F32, or BF16 when
 * prec = BF16) or CSR; Vt is V^T in the same format (required for CSR;
 * optional for dense, built on the device when NULL).  W (m x r) and Ht
 * (n x r) hold the initial factors and receive the result.  Synchronises
 * before returning and fills *rep (host). */
nmf_status nmf_solve(nmf_handle h, const nmf_matrix *V, const nmf_matrix *Vt, int r, float *W,
                     float *Ht, const nmf_solve_opts *opts, nmf_report *rep);

/* One-pass alternating solve with V streamed in row chunks (Alg. 2 as
 * printed in §3.3: while the coefficients F_i of a chunk are solved, the
 * M-step's inputs Y += F_i V_i^T and H += F_i F_i^T are accumulated, so each
 * outer iteration reads V once).  For chunk b of `chunk_rows` rows of V:
 * C_W = V_b Ht (tensor cores when n % 4 == 0, else CUDA cores), the rows of
 * W_b by Alg. 3, G_W += W_b^T W_b, C_H += V_b^T W_b (CUDA cores, FP32); then
 * Q_H = G_W + b_h I, every row of Ht against C_H, and J by the FP64 trace
 * identity after every iteration that obj_hist, rel_gap_target or the last
 * one asks for.
 *  V        m x n F32, contiguous (ld = n), in DEVICE or HOST memory.  In host
 *           memory (pinned for full speed) it is the limited-internal-memory
 *           mode of §1 / Table 1: the device holds two chunk buffers of V
 *           (2 chunk_rows n floats), W, Ht and O(r (r + n)) of M-step state;
 *           chunks are copied on a second stream while the previous chunk is
 *           computed.  The same chunking gives bitwise the same result
 *           whether V is on the host or the device.
 *  W, Ht    DEVICE memory (m x r, n x r): initial factors in, result out.
 *  opts     outer_iters, rel_gap_target / f_star, penalties and nnls as for
 *           nmf_solve; prec FP32 or FP32_SIMT (NMF_E_NOTIMPL otherwise);
 *           maxstop_mode must be 0; check_every, use_graph and objective are
 *           not used (no CUDA graph: the chunk loop is launched directly).
 * Synchronises before returning and fills *rep (host). */
nmf_status nmf_solve_streamed(nmf_handle h, const nmf_dense *V, int r, float *W, float *Ht,
                              const nmf_solve_opts *opts, int64_t chunk_rows, nmf_report *rep);

/* ---- many independent instances ------------------------------------------ */

/* One NMF instance of a batch (all pointers device memory, row-major F32,
 * contiguous): V m x n and its transpose Vt n x m, W m x r, Ht n x r (initial
 * factors in, result out).  r <= 64. */
typedef struct {
    int64_t m, n;
    int r;
    const float *V, *Vt;
    float *W, *Ht;
} nmf_instance;

/* Advance `count` independent instances by opts->outer_iters outer
 * iterations of Alg. 2 each (shared L1/L2 weights and NNLS options).  The
 * cross term's products follow opts->prec: NMF_PREC_FP32 runs them as 3xTF32
 * tcgen05 MMAs (FP32-accurate, each 32-wide k block added into FP32 with
 * round-to-nearest), NMF_PREC_FP32_SIMT as FFMA on the CUDA cores; any other
 * precision returns NMF_E_NOTIMPL.  Gram, rescale and NNLS are FP32 on the
 * CUDA cores.  With NMF_PREC_FP32 the cross phase reads its tiles 16 bytes at
 * a time: an instance whose V rows (Vt rows) do not start 16 bytes apart -
 * n (m) not a multiple of 4, or the array not 16-byte aligned - is copied
 * once per call into a row-padded workspace array (pad columns zeroed) of m x round4(n)
 * (n x round4(m)) floats.
 *  mode 0: persistent - one cooperative launch per outer iteration runs all
 *          eight phases (Gram, rescale, cross term, NNLS for W, then for H)
 *          for all instances with grid barriers between phases (with FP32
 *          products the two cross phases run in tensor-core launches of
 *          their own between three cooperative launches); captured in a
 *          CUDA graph when opts->use_graph;
 *  mode 1: per-instance loop - the same phase code launched per instance and
 *          phase (the baseline);
 *  mode 2: as mode 0, with the first iterations spent timing candidate
 *          launch shapes (CTAs per SM, NNLS rows per work item) and the
 *          fastest kept for the rest;
 *  mode 3: one ordinary launch per phase over all instances (eight per
 *          outer iteration; no cooperative launch, no grid barrier).
 * reps (host, `count` entries, optional) receive each instance's final J
 * (FP64 element-wise objective), iterations and, in every entry, the batch's
 * device time and mean inner iterations.  Synchronises before returning. */
nmf_status nmf_solve_batched(nmf_handle h, int count, const nmf_instance *inst,
                             const nmf_solve_opts *opts, int mode, nmf_report *reps);

/* ---- diagnostics ------------------------------------------------------------ */

/* FP32 FFMA throughput of the current device in TFLOP/s (*tflops, host),
 * measured with independent fmaf chains on every SM: the ALU roofline of
 * the CUDA-core kernels.  Synchronises the device; allocates a few bytes. */
nmf_status nmf_peak_fp32(double *tflops);

/* Bandwidth of the sparse cross term's access pattern with its dense operand
 * resident in L2, in GB/s of gathered data (*gbs, host): warps gather whole
 * rows of r floats (r <= 128) at hashed indices over a 65536-row table, eight
 * rows in flight per lane - the roofline of the CSR SpMM, whose factor-row
 * gathers hit L2.  Synchronises the device; allocates 32 MB at most. */
nmf_status nmf_peak_l2_gather(int r, double *gbs);

/* Dense BF16 throughput of this library's tcgen05.mma path in TFLOP/s
 * (*tflops, host) on a contraction wide enough to be bound by the tensor
 * pipe rather than HBM (r = 512): one CTA per SM issues, from shared-memory
 * tiles, pairs of M = 128, N = 256, K = 16 MMAs into all 512 TMEM columns
 * (the descriptors and issue path of nmf_cross), counted as 2 M N K each.
 * The cross term itself is HBM-bound at r <= 128 (2 r / 4 flop per byte of
 * FP32 V); this is the tensor-pipe roofline it sits under.  Synchronises the
 * device; NMF_E_TIMEOUT if the bounded wait for the MMAs ran out (the
 * handle's status word says so, the context stays usable). */
nmf_status nmf_peak_tc_bf16(nmf_handle h, double *tflops);

/* ---- projection onto a fixed basis ----------------------------------------- */

/* E-step alone (Alg. 1 E-step, Alg. 2 first loop) against a fixed basis W
 * (wrows x r) with its rescaled Gram (Qt, d from nmf_gram + nmf_rescale):
 * for each new column j, given as row j of the CSR VnewT (w x wrows),
 * Hnew_j = argmin_{h >= 0} 1/2 ||v_j - W h||^2.  Hnew (w x r) is the warm
 * start on entry (zero for a cold start). */
nmf_status nmf_project(nmf_handle h, const float *Qt, const float *d, const float *W,
                       int64_t wrows, int r, const nmf_csr *VnewT, float *Hnew,
                       const nmf_nnls_opts *opts);

/* ---- projection server: continuous batching -------------------------------- */

/* A server projects incoming blocks of new data columns onto a fixed basis W
 * (the E-step alone, as nmf_project), batching requests continuously: a
 * scheduler thread admits queued requests, in arrival order, into the next
 * free slot while the batch fits the slot and the bytes of all batches in
 * flight stay within hbm_budget; each slot runs its batch (host-to-device
 * copy, SpMM, NNLS, device-to-host copy) on its own CUDA stream, so batches
 * overlap.  A result depends on its own columns only: it is bitwise the same
 * alone and inside any mix of requests. */
typedef struct nmf_server_s *nmf_server_t;

typedef struct {
    int slots;               /* batches in flight, one CUDA stream each (1..64)  */
    int64_t max_batch_cols;  /* new columns per batch (a slot's capacity)        */
    int64_t max_batch_nnz;   /* nonzeros per batch                               */
    size_t hbm_budget;       /* device bytes all batches in flight may hold      */
    nmf_nnls_opts nnls;      /* NNLS options (zeroed: defaults)                   */
} nmf_server_opts_t;

typedef struct {
    int64_t completed;       /* requests finished                                 */
    int64_t completed_cols;  /* new columns finished                              */
    int64_t batches;         /* batches launched                                  */
    int64_t queued;          /* requests waiting for admission now                */
    int64_t max_queue;       /* largest queue seen                                */
    int64_t inflight_bytes;  /* device bytes held by batches in flight now       */
} nmf_server_stats_t;

/* Create a server for basis W (device memory, wrows x r, F32, kept alive by
 * the caller until nmf_server_destroy).  Allocates the slots' device and
 * pinned host buffers and computes the basis' rescaled Gram once. */
nmf_status nmf_server_create(nmf_server_t *out, int device, const float *W, int64_t wrows, int r,
                             const nmf_server_opts_t *opts);
/* Queue a request: w new columns as HOST CSR over the basis rows (rowptr
 * w + 1 entries, colidx/vals nnz entries, copied before returning); `out`
 * (HOST, w x r F32) receives the nonnegative coefficients when the ticket
 * completes.  NMF_E_BUSY if the request exceeds a slot or the budget (it
 * could never be admitted); NMF_E_ARG on malformed CSR. */
nmf_status nmf_server_submit(nmf_server_t s, int64_t w, int64_t nnz, const int64_t *rowptr,
                             const int32_t *colidx, const float *vals, float *out,
                             int64_t *ticket);
/* Wait for a ticket (at most timeout_s seconds: NMF_E_TIMEOUT); latency_ms
 * (optional) receives submit-to-result time. */
nmf_status nmf_server_wait(nmf_server_t s, int64_t ticket, double timeout_s, double *latency_ms);
/* Counters; returns a latched error of the scheduler, if any. */
nmf_status nmf_server_stats(nmf_server_t s, nmf_server_stats_t *st);
/* Finish queued work, then free everything the server holds. */
nmf_status nmf_server_destroy(nmf_server_t s);

/* ---- allocation-free variant ----------------------------------------------- */

/* nmf_gram without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc - code running
 * under an allocator that must own every device byte (a framework's caching
 * allocator or a fixed memory budget reserved up front), real-time or
 * plugin code that may not take the driver's allocation path, and callers
 * that cannot create an nmf_handle (whose workspace is allocated).
 *
 * Computes Q = X^T X + beta I as nmf_gram with NMF_PREC_FP32 does, equal to
 * it within FP32 rounding (the sum is split into at most 63 partial sums,
 * nmf_gram's into up to twice the SM count, so the rounding order differs;
 * relative Frobenius difference below 2e-6 in the tests).  X is rows x r F32
 * (ld >= r), Q is r x r F32; both must be device memory of the CURRENT
 * device, and `cuda_stream` (a cudaStream_t, NULL = legacy default stream)
 * must belong to it.  rows = 0 gives Q = beta I.  Its split-K partial sums
 * use one fixed device array inside the library (about 4.2 MB, room for 63
 * partial r x r slices at r <= 128), which every GPU that loads the library
 * holds until the process exits.
 *
 * Limits and errors: r > 128 returns NMF_E_SHAPE (the array holds r <= 128);
 * NULL pointers, or X or Q not on the current device, NMF_E_ARG; non-F32 X
 * NMF_E_DTYPE; a failed CUDA call NMF_E_CUDA.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use this entry point after a
 * cudaDeviceReset of that device (the kept address belonged to the context
 * the reset destroyed).  Every call shares the one array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. */
nmf_status nmf_gram_noalloc(const nmf_dense *X, float beta, float *Q, void *cuda_stream);

/* ---- fault injection -------------------------------------------------------- */

/* Host-side fault injection, with no counterpart in the paper: the library
 * reads the environment variable NMF_FAULT (a comma-separated list of sites)
 * at each call that can fail there, and fails as if the failure had happened:
 *   alloc    a workspace allocation fails          -> NMF_E_NOMEM
 *   admit    the server refuses a request          -> NMF_E_BUSY
 *   csr      a request's CSR fails validation      -> NMF_E_ARG
 *   barrier  the persistent batched launch's grid barrier gets a deadline
 *            that has already passed: its bounded wait runs out and the
 *            call returns NMF_E_TIMEOUT through the device status word,
 *            the context stays usable (the next call resets the barrier)
 * Nothing injected traps, faults or hangs the GPU.  Returns 1 when `site` is
 * armed now, else 0. */
int nmf_fault_armed(const char *site);

/* ---- instrumentation ------------------------------------------------------- */

/* Kernel classes for nmf_profile_read. */
typedef enum {
    NMF_K_GRAM = 0, NMF_K_CROSS = 1, NMF_K_SPMM = 2, NMF_K_RESCALE = 3, NMF_K_NNLS = 4,
    NMF_K_OBJECTIVE = 5, NMF_K_OTHER = 6
} nmf_kclass;

/* Instrumentation, with no counterpart in the paper: while enabled, every
 * launch is bracketed by two CUDA events on its stream (not inside CUDA-graph
 * capture).  Enabling clears the totals.  Process-wide, one host thread. */
nmf_status nmf_profile_enable(int enable);
/* Device milliseconds and launch count of one kernel class since enabling;
 * waits for the recorded events. */
nmf_status nmf_profile_read(int kclass, double *ms_total, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* NMF_GB300_H */
