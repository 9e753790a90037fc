// Internal declarations shared by the translation units of libnmf.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

#include "../../include/nmf.h"

#define NMF_API extern "C" __attribute__((visibility("default")))

namespace nmfi {

constexpr int kMaxRank = 128;

// Device status word bits (latched until nmf_sync).
constexpr unsigned kStNonFinite = 1u;
constexpr unsigned kStTimeout = 2u;
constexpr unsigned kStBadInput = 4u;   // an argument in device memory broke its contract

void count_launch(int n = 1);

// Host-side fault injection (no counterpart in the paper): true when the
// comma-separated list in the environment variable NMF_FAULT names `site`.
// Sites: "alloc" (workspace allocation fails), "admit" (the server refuses
// admission), "csr" (CSR validation fails), "barrier" (the persistent batched
// kernel's grid-barrier deadline is zero, so its bounded wait runs out).
// Nothing here traps or faults the GPU.
bool fault_armed(const char *site);

// Programmatic dependent launch: a kernel launched with pdl_launch may start
// (prologue, loads of inputs no earlier kernel writes) while the previous
// kernel on the stream drains; it must pass pdl_wait() before it reads that
// kernel's outputs or writes anything an earlier kernel may still read.
// Without the launch attribute both calls are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Per-kernel-class device time (CUDA events around launches while enabled).
enum KClass { KC_GRAM = 0, KC_CROSS, KC_SPMM, KC_RESCALE, KC_NNLS, KC_OBJECTIVE, KC_OTHER,
              KC_COUNT };
void prof_mark(int cls, cudaStream_t s, bool begin);
struct ProfScope {
    int cls;
    cudaStream_t s;
    ProfScope(int c, cudaStream_t st) : cls(c), s(st) { prof_mark(cls, s, true); }
    ~ProfScope() { prof_mark(cls, s, false); }
};
void prof_suspend(bool on);   // no events while a stream is being captured
void prof_thread_off();       // this host thread never records profiler events
bool prof_thread_set_off(bool off);   // set this thread's flag, return the old one

// ---- NNLS (Alg. 3) --------------------------------------------------------
struct NnlsArgs {
    const float *Qt;        // r x r rescaled Gram (row-major, symmetric)
    const float *d;         // r
    const float *C;         // nsplit slices of rows x r, slice stride c_stride
    int nsplit;
    int64_t c_stride;
    int64_t rows;
    int r;
    float alpha;
    float *X;               // rows x r, in: warm start, out: solution
    int max_inner;
    float eps;
    int cd_steps;           // < 0: r
    int maxstop_mode;
    float maxstop;          // threshold for mode 1
    const unsigned *maxstop_dev;   // mode 1: threshold (float bits) in device memory, else null
    int32_t *iters;         // optional per-row counts
    unsigned long long *iter_total;   // optional sum of counts
    unsigned *s_final_max;  // optional: atomicMax of final ||f||^2 bits
    unsigned *status;       // optional device status word
    int lanes;              // lanes per row (0: chosen from r)
    int grad_refresh;       // > 0: recompute the gradient every that many iterations
    // optional epilogue (standalone kernel only): each CTA writes the Gram
    // partial of its rows of the solved X into slice blockIdx of gram_P (r x r)
    // and, if pack_mode >= 0, their columns of the packed operand; the grid
    // is then at most gram_smax CTAs and its size is returned in *grid_out
    float *gram_P;
    int gram_smax;
    int pack_mode;
    void *pack;
    int npad;
    int64_t kp;
    int *grid_out;          // host
    bool grid_query;        // host: only compute the grid into *grid_out
};
cudaError_t launch_nnls(const NnlsArgs &a, cudaStream_t s);
int num_sms();   // SMs of the current device (cached)
int nnls_grid_query(const NnlsArgs &a);   // the grid launch_nnls would use (0 on error)
cudaError_t prepare_nnls(int r, int lanes);
bool nnls_layout(int r, int lanes, int *G, int *J);

// FP32 FFMA throughput of this GPU, measured (TFLOP/s)
cudaError_t measure_fp32_peak(double *tflops);
// L2-resident row-gather bandwidth for rows of r floats (GB/s of gathered data)
cudaError_t measure_l2_gather(int r, double *gbs);
cudaError_t measure_tc_peak(double *tflops, unsigned *status);

// ---- factor preparation (Gram + rescale + tensor-core packing, one launch) --
struct PrepArgs {
    const float *X;         // factor just updated, rows x r (row-major, ld = r)
    int64_t rows;
    int r;
    float beta;             // L2 weight of the next half-step
    float *P;               // partial Gram slices, prep_slice_floats(r) apart (r x r each)
    unsigned *ticket;       // zero before the first launch; left zero
    float *G, *Q;           // optional: X^T X and X^T X + beta I
    float *Qt, *d;          // rescaled Q and its scale
    int pack_mode;          // -1: no packing; else a TcMode
    void *pack;             // packed operand (npad x kp), X3: hi rows then lo rows
    int npad;
    int64_t kp;
    int64_t chunk;          // rows per CTA (set by the launcher)
    int slices;             // > 0: that many partial slices over balanced row ranges
                            // (the NQP kernel's split); 0: 32-row chunks
};
constexpr int kPrepMaxSlices = 512;   // Gram partial slices the finishing kernel sums at most
// floats from one Gram partial slice to the next: r x r rounded up to a
// multiple of 4, so that every slice starts on a 16-byte boundary
__host__ __device__ constexpr int prep_slice_floats(int r) { return (r * r + 3) & ~3; }
cudaError_t launch_factor_prep(const PrepArgs &a, cudaStream_t s);
// the second launch alone, over S partial slices already in a.P (written by
// the NQP kernel's epilogue)
cudaError_t launch_prep_finish(const PrepArgs &a, int S, cudaStream_t s);
// the same on `ctas` CTAs (each walks several 128-element groups), an ordinary
// launch: for a side stream, beside the cross term
cudaError_t launch_prep_finish_narrow(const PrepArgs &a, int S, int ctas, cudaStream_t s);
int prep_slices(int64_t rows);

// ---- Gram / cross term (SIMT FP32) ----------------------------------------
// partial Gram slices: P[s] = X[k0:k1]^T X[k0:k1], s < nsplit, each r x r,
// with the operand arithmetic `mode` (a GramMode)
enum GramMode { GM_FP32 = 0, GM_TF32 = 1, GM_BF16 = 2, GM_BF16X2 = 3 };
cudaError_t launch_gram_partial(const float *X, int64_t rows, int64_t ld, int r, float *P,
                                int nsplit, cudaStream_t s, int mode = GM_FP32);
int gram_splits(int64_t rows);
// partial cross slices: P[s] = A[:, k0:k1] B[k0:k1, :], each M x r; trans: A
// is stored as its transpose (element (m, k) at A[k * lda + m])
cudaError_t launch_cross_dense_f32(const float *A, int64_t M, int64_t K, int64_t lda,
                                   const float *B, int r, float *P, int nsplit,
                                   cudaStream_t s, bool trans = false);
int cross_splits(int64_t M, int64_t K);
// C = sum of nsplit slices (each n elements); accumulate: C += that sum
cudaError_t launch_sum_slices(const float *P, int nsplit, int64_t n, float *out, cudaStream_t s,
                              bool accumulate = false);
// out = A^T (A rows x cols, lda) -> cols x rows
cudaError_t launch_transpose_f32(const float *A, int64_t rows, int64_t cols, int64_t lda,
                                 float *out, cudaStream_t s);

// ---- tensor-core cross term (tcgen05) ---------------------------------------
enum TcMode { TC_TF32 = 0, TC_TF32X3 = 1, TC_BF16 = 2, TC_BF16X2 = 3 };
// operands in BF16 (A and the packed factor); factor packed as [hi; lo]
__host__ __device__ constexpr bool tc_bf16(int mode) { return mode == TC_BF16 || mode == TC_BF16X2; }
__host__ __device__ constexpr bool tc_pair(int mode) { return mode == TC_TF32X3 || mode == TC_BF16X2; }
struct TcArgs {
    int64_t M;
    int r;
    int kblocks;
    int64_t iters;
    int grid;
    int nslices;
    float *P;          // nslices x M x r partial slices
    unsigned *status;
};
struct TcPlan {
    int kblocks = 0, tiles = 0, grid = 0, nslices = 1;
    int64_t iters = 0;
};
int tc_npad(int r);
int64_t tc_kpad(int64_t K, int mode);
size_t tc_pack_bytes(int64_t K, int r, int mode);
bool tc_supported(int64_t lda, int mode, const void *A);
// max_grid > 0 caps the CTAs (SMs left free for work beside the cross term)
TcPlan tc_plan(int64_t M, int64_t K, int r, int mode, int max_grid = 0);
// pack X (K x r row-major FP32) as the B operand of mode `mode`
cudaError_t launch_tc_pack(const float *X, int64_t K, int r, int mode, void *pack, cudaStream_t s);
cudaError_t launch_tc_cross(const void *A, int64_t M, int64_t K, int64_t lda, int r, int mode,
                            const void *pack, float *P, const TcPlan &pl, unsigned *status,
                            cudaStream_t s);

// ---- batched instances (one launch per outer iteration) -------------------
struct BatchInst {
    int64_t m, n;
    int r;
    const float *V, *Vt;
    float *W, *Ht;
    float *gram, *Qt, *d, *Cw, *Ch;
    float alpha_w, alpha_h, beta_w, beta_h;
    // the tensor-core cross phase's copies of V and Vt: the caller's arrays,
    // or row-padded copies whose rows start 16 bytes apart (pitch in floats)
    const float *Vx, *Vtx;
    int64_t ldvx, ldvtx;
};
struct BatchNnls {
    int max_inner;
    float eps;
    int cd_steps;
};
struct BatchArgs {
    const BatchInst *inst;     // device array [count]
    int count;
    const int64_t *item_off;   // device [8][count + 1]: prefix sums of work items
    int phase_begin, phase_end;
    int inst_begin;            // -1: all instances; else one instance
    int nnls_rows;             // rows per NNLS work item
    BatchNnls nnls;
    unsigned long long *iter_total;
    unsigned *status;
    unsigned *bar_count, *bar_gen;
    unsigned long long barrier_ns;   // grid-barrier deadline (kBarrierNs unless injected)
    // per-phase item counters (8): CTAs take items in order from them instead
    // of a fixed stride; null: the fixed stride (one-instance launches)
    unsigned long long *work;
    // cross phases on the tensor cores (3xTF32, tcgen05) instead of FFMA
    int tc;
};
size_t batched_smem_bytes();
int64_t batched_items(int phase, int64_t m, int64_t n, int r, int nnls_mult);
int batched_grid(bool cooperative);
// the tensor-core cross phase's TMEM (256 columns a CTA) fits every CTA an
// SM can hold
bool batched_tc_fits();
cudaError_t launch_batched(const BatchArgs &a, int grid, bool cooperative, cudaStream_t s);

// ---- sparse cross term ----------------------------------------------------
struct SpmmPlan {
    int64_t pieces = 0;     // number of merge-path pieces
    int items_per_piece = 0;
};
SpmmPlan spmm_plan(int64_t rows, int64_t nnz);
size_t spmm_workspace_bytes(const SpmmPlan &p, int r);
cudaError_t launch_spmm_csr(const int64_t *rowptr, const int32_t *colidx, const void *vals,
                            nmf_dtype vdt, int64_t rows, int64_t nnz, const float *B, int r,
                            float *C, const SpmmPlan &plan, void *ws, cudaStream_t s);
// row-per-warp variant: deterministic per row regardless of batch composition
cudaError_t launch_spmm_rowwarp(const int64_t *rowptr, const int32_t *colidx, const void *vals,
                                nmf_dtype vdt, int64_t rows, const float *B, int r, float *C,
                                cudaStream_t s);

// ---- rescale / reductions -------------------------------------------------
// G = sum of nsplit Gram slices; Q = G + beta I; d, Qt (rescaled).  Any output
// pointer may be NULL.
cudaError_t launch_rescale(const float *P, int nsplit, int r, float beta, float *G, float *Q,
                           float *Qt, float *d, cudaStream_t s);
// FP64 trace-identity objective (see nmf_objective)
struct ObjArgs {
    double vv;
    const float *W; int64_t m;
    const float *Ht; int64_t n;
    int r;
    const float *Ch; int nsplit; int64_t ch_stride;
    const float *Gw; const float *Gh;
    float aw, ah, bw, bh;
    double *J;              // device scalar out
    double *hist;           // optional device array, hist[*t] = J
    const int *t;           // device iteration counter (with hist)
    double f_star, gap_target;
    int *done_flag;         // optional: set to 1 when gap <= target
    double *partials;       // workspace: grid doubles x 3
    unsigned *ticket;       // workspace counter (zeroed)
};
cudaError_t launch_objective(const ObjArgs &a, cudaStream_t s);
// FP64 objective from the element-wise residual (dense V)
struct ObjDirectArgs {
    const float *V; int64_t ldv;
    const float *W; int64_t m;
    const float *Ht; int64_t n;
    int r;
    float aw, ah, bw, bh;
    double *J;
    double *partials;       // objective_direct_partials(m, n) doubles
    unsigned *ticket;
};
size_t objective_direct_partials(int64_t m, int64_t n);
cudaError_t launch_objective_direct(const ObjDirectArgs &a, cudaStream_t s);
cudaError_t launch_kkt(const float *Q, const float *C, int64_t rows, int r, float alpha,
                       const float *X, double *out, cudaStream_t s);
cudaError_t launch_sumsq(const void *x, nmf_dtype dt, int64_t n, double *out, double *partials,
                         unsigned *ticket, cudaStream_t s);
cudaError_t launch_f32_to_bf16(const float *x, int64_t n, __nv_bfloat16 *y, cudaStream_t s);

}  // namespace nmfi
