// FP32 products of the half-step on CUDA cores (the NMF_PREC_FP32 arithmetic):
//   Gram   Q = X^T X            (Alg. 2 "Q = G^T G", cost O(n r^2) in §4.2)
//   cross  C = A B              (Alg. 2 "Y = F V^T", cost O(m n r))
// Both are split over the long dimension K into `nsplit` FP32 partial slices
// so that a grid covers all SMs; the consumer sums the slices in a fixed
// order, which keeps results bitwise reproducible.
#include "nmf_internal.cuh"

namespace nmfi {
namespace {

constexpr int kThreads = 256;

// ---- cross term: P[s] = A[:, k-range(s)] B[k-range(s), :] -----------------
// CTA tile BM x NB (NB = padded r), K step BK.  Thread (ty, tx) of a 16 x 16
// grid owns rows ty + 16 i (i < BM/16) and columns tx + 16 j (j < NB/16):
// strided ownership keeps the shared-memory reads conflict-free.  TRANS: A
// is stored transposed, element (m, k) at A[k * lda + m] (the product
// V_b^T W_b of a block of rows of V, read along those rows).
template <int NB, bool TRANS>
__global__ void __launch_bounds__(kThreads) k_cross_f32(const float *__restrict__ A, int64_t M,
                                                         int64_t K, int64_t lda,
                                                         const float *__restrict__ B, int r,
                                                         float *__restrict__ P, int64_t kchunk)
{
    constexpr int BM = 128, BK = 16, TM = BM / 16, TN = NB / 16;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][NB];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int64_t kb = (int64_t)blockIdx.y * kchunk;
    const int64_t ke = kb + kchunk < K ? kb + kchunk : K;
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
            acc[i][j] = 0.f;

    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
        // A tile: BM x BK, each warp reads 2 rows x 16 consecutive k (or,
        // transposed, 32 consecutive m of one k)
#pragma unroll
        for (int t = 0; t < BM * BK / kThreads; ++t) {
            int idx = tid + t * kThreads;
            if (TRANS) {
                int mm = idx & (BM - 1), kk = idx / BM;
                int64_t gm = m0 + mm, gk = k0 + kk;
                As[kk][mm] = (gm < M && gk < ke) ? A[gk * lda + gm] : 0.f;
            } else {
                int mm = idx >> 4, kk = idx & 15;
                int64_t gm = m0 + mm, gk = k0 + kk;
                As[kk][mm] = (gm < M && gk < ke) ? A[gm * lda + gk] : 0.f;
            }
        }
#pragma unroll
        for (int t = 0; t < BK * NB / kThreads; ++t) {
            int idx = tid + t * kThreads;
            int kk = idx / NB, nn = idx - kk * NB;
            int64_t gk = k0 + kk;
            Bs[kk][nn] = (nn < r && gk < ke) ? B[gk * r + nn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i)
                a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j)
                b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *Ps = P + (int64_t)blockIdx.y * M * r;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int64_t gm = m0 + ty + 16 * i;
        if (gm >= M)
            continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int n = tx + 16 * j;
            if (n < r)
                Ps[gm * r + n] = acc[i][j];
        }
    }
}

// TF32 value nearest to x (ties to even): keep the sign, the exponent and the
// top 10 of the 23 stored mantissa bits.  Inf and NaN pass unchanged.
__device__ __forceinline__ float round_tf32(float x)
{
    unsigned u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u)
        return x;
    u += 0xfffu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xffffe000u);
}

// ---- Gram: P[s] = X[rows(s)]^T X[rows(s)] ---------------------------------
// Operand arithmetic MODE (a GramMode): FP32 as stored; TF32 or BF16 (each
// element rounded to nearest, products accumulated in FP32); BF16X2 (each
// element split into hi = bf16(x) and lo = bf16(x - hi), and
// hi_a hi_b + hi_a lo_b + lo_a hi_b accumulated in FP32, the lo lo term of
// order 2^-18 dropped).
template <int NB, int MODE>
__global__ void __launch_bounds__(kThreads) k_gram_f32(const float *__restrict__ X, int64_t rows,
                                                        int64_t ld, int r, float *__restrict__ P,
                                                        int64_t chunk)
{
    constexpr int BK = 32, T = NB / 16;
    constexpr int NL = MODE == GM_BF16X2 ? BK : 1;
    __shared__ float Xs[BK][NB];
    __shared__ float Xl[NL][NB];          // low parts (BF16X2 only)
    const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
    const int64_t kb = (int64_t)blockIdx.x * chunk;
    const int64_t ke = kb + chunk < rows ? kb + chunk : rows;
    float acc[T][T];
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b)
            acc[a][b] = 0.f;
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
        for (int idx = tid; idx < BK * NB; idx += kThreads) {
            int kk = idx / NB, c = idx - kk * NB;
            int64_t gk = k0 + kk;
            float v = (c < r && gk < ke) ? X[gk * ld + c] : 0.f;
            if (MODE == GM_TF32) {
                v = round_tf32(v);
            } else if (MODE == GM_BF16) {
                v = __bfloat162float(__float2bfloat16_rn(v));
            } else if (MODE == GM_BF16X2) {
                const float hi = __bfloat162float(__float2bfloat16_rn(v));
                Xl[kk % NL][c] = __bfloat162float(__float2bfloat16_rn(v - hi));
                v = hi;
            }
            Xs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            float xa[T], xb[T];
#pragma unroll
            for (int a = 0; a < T; ++a)
                xa[a] = Xs[kk][ti + 16 * a];
#pragma unroll
            for (int b = 0; b < T; ++b)
                xb[b] = Xs[kk][tj + 16 * b];
            if (MODE == GM_BF16X2) {
                float la[T], lb[T];
#pragma unroll
                for (int a = 0; a < T; ++a)
                    la[a] = Xl[kk % NL][ti + 16 * a];
#pragma unroll
                for (int b = 0; b < T; ++b)
                    lb[b] = Xl[kk % NL][tj + 16 * b];
#pragma unroll
                for (int a = 0; a < T; ++a)
#pragma unroll
                    for (int b = 0; b < T; ++b)
                        acc[a][b] = fmaf(xa[a], xb[b], fmaf(xa[a], lb[b], fmaf(la[a], xb[b],
                                                                               acc[a][b])));
            } else {
#pragma unroll
                for (int a = 0; a < T; ++a)
#pragma unroll
                    for (int b = 0; b < T; ++b)
                        acc[a][b] = fmaf(xa[a], xb[b], acc[a][b]);
            }
        }
        __syncthreads();
    }
    float *Ps = P + (int64_t)blockIdx.x * r * r;
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) {
            int i = ti + 16 * a, j = tj + 16 * b;
            if (i < r && j < r)
                Ps[i * r + j] = acc[a][b];
        }
}

// out[e] = sum_s P[s * n + e].  A block covers 32 consecutive elements; its 8
// warps take interleaved slices (w, w + 8, ...) with coalesced 128-byte loads,
// then warp 0 adds the 8 warp sums in order: a fixed order, so the result is
// reproducible, with 8 x the loads in flight of one thread per element.
__global__ void __launch_bounds__(256) k_sum_slices(const float *__restrict__ P, int nsplit,
                                                    int64_t n, float *__restrict__ out, bool acc)
{
    __shared__ float part[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t e0 = (int64_t)blockIdx.x * 32; e0 < n; e0 += (int64_t)gridDim.x * 32) {
        const int64_t e = e0 + lane;
        float a0 = 0.f, a1 = 0.f;
        if (e < n) {
            int k = w;
            for (; k + 8 < nsplit; k += 16) {
                a0 += P[(int64_t)k * n + e];
                a1 += P[(int64_t)(k + 8) * n + e];
            }
            if (k < nsplit)
                a0 += P[(int64_t)k * n + e];
        }
        part[w][lane] = a0 + a1;
        __syncthreads();
        if (w == 0 && e < n) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                s += part[q][lane];
            out[e] = acc ? out[e] + s : s;
        }
        __syncthreads();
    }
}

__global__ void k_transpose(const float *__restrict__ A, int64_t rows, int64_t cols, int64_t lda,
                            float *__restrict__ out)
{
    __shared__ float t[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int64_t rr = r0 + i, cc = c0 + threadIdx.x;
        t[i][threadIdx.x] = (rr < rows && cc < cols) ? A[rr * lda + cc] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int64_t cc = c0 + i, rr = r0 + threadIdx.x;
        if (cc < cols && rr < rows)
            out[cc * rows + rr] = t[threadIdx.x][i];
    }
}


}  // namespace

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0)
            sms = 1;
    }
    return sms;
}

int gram_splits(int64_t rows)
{
    // 64 rows per CTA: every SM gets work even for K of a few thousand
    int64_t s = (rows + 63) / 64;
    int64_t cap = 2 * (int64_t)num_sms();
    if (s > cap)
        s = cap;
    return s < 1 ? 1 : (int)s;
}

int cross_splits(int64_t M, int64_t K)
{
    int64_t tiles = (M + 127) / 128;
    int64_t target = 2 * (int64_t)num_sms();
    int64_t s = (target + tiles - 1) / tiles;
    int64_t kmax = K / 256;
    if (s > kmax)
        s = kmax;
    if (s > 64)
        s = 64;
    return s < 1 ? 1 : (int)s;
}

template <int MODE>
void gram_launch(const float *X, int64_t rows, int64_t ld, int r, float *P, int64_t chunk,
                 int grid, cudaStream_t s)
{
    if (r <= 32)
        k_gram_f32<32, MODE><<<grid, kThreads, 0, s>>>(X, rows, ld, r, P, chunk);
    else if (r <= 64)
        k_gram_f32<64, MODE><<<grid, kThreads, 0, s>>>(X, rows, ld, r, P, chunk);
    else
        k_gram_f32<128, MODE><<<grid, kThreads, 0, s>>>(X, rows, ld, r, P, chunk);
}

cudaError_t launch_gram_partial(const float *X, int64_t rows, int64_t ld, int r, float *P,
                                int nsplit, cudaStream_t s, int mode)
{
    ProfScope prof_(KC_GRAM, s);
    if (rows <= 0) {
        cudaError_t e = cudaMemsetAsync(P, 0, sizeof(float) * r * r * nsplit, s);
        return e;
    }
    int64_t chunk = (rows + nsplit - 1) / nsplit;
    chunk = (chunk + 31) / 32 * 32;
    int grid = (int)((rows + chunk - 1) / chunk);
    if (grid < 1)
        grid = 1;
    if (grid < nsplit) {   // trailing slices would stay unwritten: clear them
        cudaError_t e = cudaMemsetAsync(P + (int64_t)grid * r * r, 0,
                                        sizeof(float) * r * r * (nsplit - grid), s);
        if (e != cudaSuccess)
            return e;
    }
    switch (mode) {
    case GM_TF32: gram_launch<GM_TF32>(X, rows, ld, r, P, chunk, grid, s); break;
    case GM_BF16: gram_launch<GM_BF16>(X, rows, ld, r, P, chunk, grid, s); break;
    case GM_BF16X2: gram_launch<GM_BF16X2>(X, rows, ld, r, P, chunk, grid, s); break;
    default: gram_launch<GM_FP32>(X, rows, ld, r, P, chunk, grid, s); break;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cross_dense_f32(const float *A, int64_t M, int64_t K, int64_t lda,
                                   const float *B, int r, float *P, int nsplit, cudaStream_t s,
                                   bool trans)
{
    ProfScope prof_(KC_CROSS, s);
    if (M <= 0)
        return cudaSuccess;
    if (K <= 0)
        return cudaMemsetAsync(P, 0, sizeof(float) * M * r * nsplit, s);
    int64_t kchunk = (K + nsplit - 1) / nsplit;
    kchunk = (kchunk + 15) / 16 * 16;
    int gy = (int)((K + kchunk - 1) / kchunk);
    if (gy < 1)
        gy = 1;
    if (gy < nsplit) {
        cudaError_t e = cudaMemsetAsync(P + (int64_t)gy * M * r, 0,
                                        sizeof(float) * M * r * (nsplit - gy), s);
        if (e != cudaSuccess)
            return e;
    }
    dim3 grid((unsigned)((M + 127) / 128), (unsigned)gy);
    if (trans) {
        if (r <= 32)
            k_cross_f32<32, true><<<grid, kThreads, 0, s>>>(A, M, K, lda, B, r, P, kchunk);
        else if (r <= 64)
            k_cross_f32<64, true><<<grid, kThreads, 0, s>>>(A, M, K, lda, B, r, P, kchunk);
        else
            k_cross_f32<128, true><<<grid, kThreads, 0, s>>>(A, M, K, lda, B, r, P, kchunk);
    } else if (r <= 32) {
        k_cross_f32<32, false><<<grid, kThreads, 0, s>>>(A, M, K, lda, B, r, P, kchunk);
    } else if (r <= 64) {
        k_cross_f32<64, false><<<grid, kThreads, 0, s>>>(A, M, K, lda, B, r, P, kchunk);
    } else {
        k_cross_f32<128, false><<<grid, kThreads, 0, s>>>(A, M, K, lda, B, r, P, kchunk);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum_slices(const float *P, int nsplit, int64_t n, float *out, cudaStream_t s,
                              bool accumulate)
{
    ProfScope prof_(KC_OTHER, s);
    if (n <= 0)
        return cudaSuccess;
    int64_t blocks = (n + 31) / 32;
    if (blocks > 8192)
        blocks = 8192;
    k_sum_slices<<<(unsigned)blocks, 256, 0, s>>>(P, nsplit, n, out, accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_transpose_f32(const float *A, int64_t rows, int64_t cols, int64_t lda,
                                 float *out, cudaStream_t s)
{
    ProfScope prof_(KC_OTHER, s);
    if (rows <= 0 || cols <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(A, rows, cols, lda, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace nmfi
