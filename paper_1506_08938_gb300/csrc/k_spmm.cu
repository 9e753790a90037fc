// Sparse cross term C = V B for CSR V (Theorem 2, §4.2: the sparse cost
// O(r S(mn)); the paper exploits sparsity in its Java runs, §5.4).
//
// Work split.  Bag-of-words columns follow a Zipf law, so the CSR of V^T has
// a few rows holding most of the nonzeros.  A warp per row would leave one
// warp with 10^5 gathers while the rest idle; instead the sequence of
// (row ends + nonzeros) is cut into equal pieces by a merge-path search, one
// warp per piece.  A warp writes every row that ends inside its piece and
// leaves the partial sum of the row it stops in as a carry; a second kernel
// adds the carries of each row in piece order, so results are reproducible.
//
// Inner loop: the warp loads 32 (column, value) pairs at once, then gathers
// the r-float rows B[col] of eight pairs at a time with lane-strided,
// coalesced loads (the gathers are latency-bound: eight rows in flight per
// lane) and accumulates them in pair order in FP32 registers (lane l owns
// columns l, l+32, ...).
#include "nmf_internal.cuh"

namespace nmfi {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kItemsPerPiece = 256;

template <typename VT>
__device__ __forceinline__ float to_f(VT v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Merge-path split point of diagonal `diag` between the row-end list
// (rowptr[1..rows]) and the nonzero indices 0..nnz-1: returns the number of
// row ends i consumed; diag - i nonzeros are consumed.
__device__ __forceinline__ int64_t mp_search(const int64_t *__restrict__ rowptr, int64_t rows,
                                             int64_t nnz, int64_t diag)
{
    int64_t lo = diag - nnz > 0 ? diag - nnz : 0;
    int64_t hi = diag < rows ? diag : rows;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (rowptr[mid + 1] <= diag - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// acc += the pairs q .. q+U-1 of the warp's 32 (col, val): U gathers of B
// rows in flight per lane before their FMAs, which run in pair order
template <int U, int J>
__device__ __forceinline__ void gather_pairs(int col, float val, int q,
                                             const float *__restrict__ B, int r, int lane,
                                             float (&acc)[J])
{
    const float *b[U];
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        b[u] = B + (int64_t)__shfl_sync(kFull, col, q + u) * r;
        v[u] = __shfl_sync(kFull, val, q + u);
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        int c = lane + 32 * j;
        if (c < r) {
            float x[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                x[u] = __ldg(b[u] + c);
#pragma unroll
            for (int u = 0; u < U; ++u)
                acc[j] = fmaf(v[u], x[u], acc[j]);
        }
    }
}

// acc += sum_{k in [kb, ke)} vals[k] * B[colidx[k], :], in k order
template <int J, typename VT>
__device__ __forceinline__ void accumulate(const int32_t *__restrict__ colidx,
                                           const VT *__restrict__ vals, int64_t kb, int64_t ke,
                                           const float *__restrict__ B, int r, int lane,
                                           float (&acc)[J])
{
    for (int64_t k = kb; k < ke; k += 32) {
        const int n = ke - k < 32 ? (int)(ke - k) : 32;
        int col = 0;
        float val = 0.f;
        if (lane < n) {
            col = colidx[k + lane];
            val = to_f<VT>(vals[k + lane]);
        }
        int q = 0;
        for (; q + 8 <= n; q += 8)
            gather_pairs<8, J>(col, val, q, B, r, lane, acc);
        if (q + 4 <= n) {
            gather_pairs<4, J>(col, val, q, B, r, lane, acc);
            q += 4;
        }
        for (; q < n; ++q)
            gather_pairs<1, J>(col, val, q, B, r, lane, acc);
    }
}

template <int J, typename VT>
__global__ void __launch_bounds__(256) k_spmm_mp(const int64_t *__restrict__ rowptr,
                                                  const int32_t *__restrict__ colidx,
                                                  const VT *__restrict__ vals, int64_t rows,
                                                  int64_t nnz, const float *__restrict__ B, int r,
                                                  float *__restrict__ C, int64_t pieces,
                                                  int64_t *__restrict__ carry_row,
                                                  float *__restrict__ carry_val)
{
    const int lane = threadIdx.x & 31;
    const int64_t piece = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (piece >= pieces)
        return;
    const int64_t items = rows + nnz;
    const int64_t d0 = piece * kItemsPerPiece;
    const int64_t d1 = d0 + kItemsPerPiece < items ? d0 + kItemsPerPiece : items;
    const int64_t i0 = mp_search(rowptr, rows, nnz, d0);
    const int64_t i1 = mp_search(rowptr, rows, nnz, d1);
    int64_t k = d0 - i0;
    const int64_t k1 = d1 - i1;
    for (int64_t row = i0;; ++row) {
        const int64_t rend = row < i1 ? rowptr[row + 1] : k1;
        float acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j)
            acc[j] = 0.f;
        accumulate<J, VT>(colidx, vals, k, rend, B, r, lane, acc);
        k = rend;
        float *dst;
        if (row < i1) {
            dst = C + row * r;
        } else {
            if (lane == 0)
                carry_row[piece] = row;   // may equal rows: nothing to carry
            dst = carry_val + piece * r;
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            int c = lane + 32 * j;
            if (c < r)
                dst[c] = acc[j];
        }
        if (row >= i1)
            break;
    }
}

// C[row] += carries of that row, in piece order.  One warp per piece; the
// warp whose piece starts a run of equal carry rows sums the whole run.
template <int J>
__global__ void k_spmm_fixup(const int64_t *__restrict__ carry_row,
                             const float *__restrict__ carry_val, int64_t pieces, int64_t rows,
                             int r, float *__restrict__ C)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= pieces)
        return;
    const int64_t R = carry_row[t];
    if (R >= rows || (t > 0 && carry_row[t - 1] == R))
        return;
    // the run [t, end) of pieces carrying row R (carry rows never decrease
    // along the pieces), found 32 entries at a time
    int64_t end = t + 1;
    for (;;) {
        const int64_t u = end + lane;
        const unsigned other = __ballot_sync(kFull, !(u < pieces && carry_row[u] == R));
        if (other) {
            end += __ffs(other) - 1;
            break;
        }
        end += 32;
    }
    float acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        int c = lane + 32 * j;
        acc[j] = c < r ? C[R * r + c] : 0.f;
    }
    // the carries in piece order, eight loaded ahead of their adds (a Zipf
    // head row of V^T spans hundreds of pieces)
    constexpr int U = 8;
    int64_t u = t;
    for (; u + U <= end; u += U) {
        float v[U][J];
#pragma unroll
        for (int q = 0; q < U; ++q)
#pragma unroll
            for (int j = 0; j < J; ++j) {
                int c = lane + 32 * j;
                v[q][j] = c < r ? carry_val[(u + q) * r + c] : 0.f;
            }
#pragma unroll
        for (int q = 0; q < U; ++q)
#pragma unroll
            for (int j = 0; j < J; ++j)
                acc[j] += v[q][j];
    }
    for (; u < end; ++u) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            int c = lane + 32 * j;
            if (c < r)
                acc[j] += carry_val[u * r + c];
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        int c = lane + 32 * j;
        if (c < r)
            C[R * r + c] = acc[j];
    }
}

// One warp per row: the result of a row depends on that row alone.
template <int J, typename VT>
__global__ void __launch_bounds__(256) k_spmm_rowwarp(const int64_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx,
                                                       const VT *__restrict__ vals, int64_t rows,
                                                       const float *__restrict__ B, int r,
                                                       float *__restrict__ C)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rows)
        return;
    float acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j)
        acc[j] = 0.f;
    accumulate<J, VT>(colidx, vals, rowptr[row], rowptr[row + 1], B, r, lane, acc);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        int c = lane + 32 * j;
        if (c < r)
            C[row * r + c] = acc[j];
    }
}

template <int J, typename VT>
cudaError_t spmm_j(const int64_t *rowptr, const int32_t *colidx, const VT *vals, int64_t rows,
                   int64_t nnz, const float *B, int r, float *C, const SpmmPlan &p, void *ws,
                   cudaStream_t s)
{
    int64_t *carry_row = reinterpret_cast<int64_t *>(ws);
    float *carry_val = reinterpret_cast<float *>(carry_row + ((p.pieces + 3) & ~int64_t(3)));
    const int64_t threads = p.pieces * 32;
    k_spmm_mp<J, VT><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        rowptr, colidx, vals, rows, nnz, B, r, C, p.pieces, carry_row, carry_val);
    k_spmm_fixup<J><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(carry_row, carry_val,
                                                                       p.pieces, rows, r, C);
    count_launch(2);
    return cudaGetLastError();
}

template <int J, typename VT>
cudaError_t rowwarp_j(const int64_t *rowptr, const int32_t *colidx, const VT *vals, int64_t rows,
                      const float *B, int r, float *C, cudaStream_t s)
{
    const int64_t threads = rows * 32;
    k_spmm_rowwarp<J, VT><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(rowptr, colidx, vals,
                                                                            rows, B, r, C);
    count_launch();
    return cudaGetLastError();
}

template <typename VT>
cudaError_t spmm_vt(const int64_t *rowptr, const int32_t *colidx, const VT *vals, int64_t rows,
                    int64_t nnz, const float *B, int r, float *C, const SpmmPlan &p, void *ws,
                    cudaStream_t s)
{
    if (r <= 32)
        return spmm_j<1, VT>(rowptr, colidx, vals, rows, nnz, B, r, C, p, ws, s);
    if (r <= 64)
        return spmm_j<2, VT>(rowptr, colidx, vals, rows, nnz, B, r, C, p, ws, s);
    if (r <= 96)
        return spmm_j<3, VT>(rowptr, colidx, vals, rows, nnz, B, r, C, p, ws, s);
    return spmm_j<4, VT>(rowptr, colidx, vals, rows, nnz, B, r, C, p, ws, s);
}

template <typename VT>
cudaError_t rowwarp_vt(const int64_t *rowptr, const int32_t *colidx, const VT *vals,
                       int64_t rows, const float *B, int r, float *C, cudaStream_t s)
{
    if (r <= 32)
        return rowwarp_j<1, VT>(rowptr, colidx, vals, rows, B, r, C, s);
    if (r <= 64)
        return rowwarp_j<2, VT>(rowptr, colidx, vals, rows, B, r, C, s);
    if (r <= 96)
        return rowwarp_j<3, VT>(rowptr, colidx, vals, rows, B, r, C, s);
    return rowwarp_j<4, VT>(rowptr, colidx, vals, rows, B, r, C, s);
}

}  // namespace

SpmmPlan spmm_plan(int64_t rows, int64_t nnz)
{
    SpmmPlan p;
    p.items_per_piece = kItemsPerPiece;
    p.pieces = (rows + nnz + kItemsPerPiece - 1) / kItemsPerPiece;
    if (p.pieces < 1)
        p.pieces = 1;
    return p;
}

size_t spmm_workspace_bytes(const SpmmPlan &p, int r)
{
    return sizeof(int64_t) * (size_t)((p.pieces + 3) & ~int64_t(3)) +
           sizeof(float) * (size_t)p.pieces * r;
}

cudaError_t launch_spmm_csr(const int64_t *rowptr, const int32_t *colidx, const void *vals,
                            nmf_dtype vdt, int64_t rows, int64_t nnz, const float *B, int r,
                            float *C, const SpmmPlan &plan, void *ws, cudaStream_t s)
{
    ProfScope prof_(KC_SPMM, s);
    if (rows <= 0)
        return cudaSuccess;
    if (vdt == NMF_BF16)
        return spmm_vt<__nv_bfloat16>(rowptr, colidx,
                                      reinterpret_cast<const __nv_bfloat16 *>(vals), rows, nnz, B,
                                      r, C, plan, ws, s);
    return spmm_vt<float>(rowptr, colidx, reinterpret_cast<const float *>(vals), rows, nnz, B, r,
                          C, plan, ws, s);
}

cudaError_t launch_spmm_rowwarp(const int64_t *rowptr, const int32_t *colidx, const void *vals,
                                nmf_dtype vdt, int64_t rows, const float *B, int r, float *C,
                                cudaStream_t s)
{
    ProfScope prof_(KC_SPMM, s);
    if (rows <= 0)
        return cudaSuccess;
    if (vdt == NMF_BF16)
        return rowwarp_vt<__nv_bfloat16>(rowptr, colidx,
                                         reinterpret_cast<const __nv_bfloat16 *>(vals), rows, B, r,
                                         C, s);
    return rowwarp_vt<float>(rowptr, colidx, reinterpret_cast<const float *>(vals), rows, B, r, C,
                             s);
}

// ---- L2 gather roof --------------------------------------------------------
// The bandwidth of the SpMM's access pattern when its operand is resident in
// L2: warps gather whole rows of r floats (lane l reads floats l, l + 32, ...)
// at indices spread over a table that fits L2, eight rows in flight per lane,
// as the merge-path kernel does.  The indices are a multiplicative hash of the
// position (a fixed, L2-resident working set; no host randomness).
namespace {

__global__ void __launch_bounds__(256) k_l2_gather_probe(const float *__restrict__ T, int rows,
                                                         int r, int64_t n, float *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float acc = 0.f;
    for (int64_t base = warp * 8; base < n; base += warps * 8) {
        float v[8][4];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t i = (uint32_t)(base + k);
            const int row = (int)((i * 2654435761u) % (uint32_t)rows);
            const float *p = T + (int64_t)row * r;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                v[k][q] = (base + k < n && c < r) ? __ldg(p + c) : 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc += v[k][q];
    }
    if (acc == 12345.678f)   // keeps the loads; never true for the zero table
        out[0] = acc;
}

}  // namespace

cudaError_t measure_l2_gather(int r, double *gbs)
{
    const int rows = 65536;   // 65536 rows of r <= 128 floats: at most 32 MB, inside L2
    float *T = nullptr, *out = nullptr;
    cudaError_t e = cudaMalloc(&T, sizeof(float) * (size_t)rows * r);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&out, sizeof(float))) != cudaSuccess) {
        cudaFree(T);
        return e;
    }
    cudaMemset(T, 0, sizeof(float) * (size_t)rows * r);
    const int64_t n = (int64_t)1 << 22;   // gathered rows per launch
    const int grid = num_sms() * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i = 0; i < 2; ++i)   // warm-up: the table into L2, clocks up
        k_l2_gather_probe<<<grid, 256>>>(T, rows, r, n, out);
    cudaEventRecord(e0);
    const int reps = 5;
    for (int i = 0; i < reps; ++i)
        k_l2_gather_probe<<<grid, 256>>>(T, rows, r, n, out);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(T);
    cudaFree(out);
    if (e != cudaSuccess)
        return e;
    if (cudaGetLastError() != cudaSuccess)
        return cudaErrorLaunchFailure;
    *gbs = (double)reps * n * r * sizeof(float) / (ms * 1e-3) / 1e9;
    return cudaSuccess;
}

}  // namespace nmfi
