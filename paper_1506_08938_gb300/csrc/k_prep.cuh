// Gram partial and packed operand of a block of factor rows: the shared
// body of the factor-preparation kernel and of the NQP kernel's epilogue
// (which prepares the factor it has just solved, Alg. 2's "H += F_i F_i^T"
// folded into the producer of F_i).
#pragma once
#include "nmf_internal.cuh"

namespace nmfi {
namespace prep_detail {

constexpr int kThreads = 256;      // threads of a CTA running gram_pack_rows
constexpr int kRowsBlock = 32;     // rows staged in shared memory at a time
constexpr int kMaxSlices = kPrepMaxSlices;   // Gram partials at most

// nearest TF32 value (10-bit mantissa)
__device__ __forceinline__ float rn_tf32(float v)
{
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xffffe000u);
}

// NB >= r columns: the Gram partial of rows [k0, k1) of a.X into slice
// `slice` of a.P (r x r, prep_slice_floats(r) floats per slice) and, if
// a.pack_mode >= 0, those rows' columns of the
// packed operand.  Xs: kRowsBlock x (NB + 1) floats of shared memory.  Every
// thread of the (kThreads-thread) CTA calls it; it synchronises the CTA.
template <int NB>
__device__ __forceinline__ void gram_pack_rows(const PrepArgs &a, float (*Xs)[NB + 1], int64_t k0,
                                               int64_t k1, int64_t slice)
{
    constexpr int T = NB / 16;
    const int r = a.r, tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
    float acc[T][T];
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j)
            acc[i][j] = 0.f;

    for (int64_t kb = k0; kb < k1; kb += kRowsBlock) {
        // every load of the block issued before the first store
        constexpr int PER = kRowsBlock * NB / kThreads;
        float v[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * kThreads, kk = idx / NB, c = idx % NB;
            const int64_t gk = kb + kk;
            v[q] = (c < r && gk < k1) ? a.X[gk * r + c] : 0.f;
        }
        __syncthreads();   // the previous block's readers are done with Xs
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * kThreads;
            Xs[idx / NB][idx % NB] = v[q];
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kRowsBlock; ++kk) {
            float xa[T], xb[T];
#pragma unroll
            for (int i = 0; i < T; ++i)
                xa[i] = Xs[kk][ti + 16 * i];
#pragma unroll
            for (int j = 0; j < T; ++j)
                xb[j] = Xs[kk][tj + 16 * j];
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j)
                    acc[i][j] = fmaf(xa[i], xb[j], acc[i][j]);
        }
        // packed operand: row n of the pack holds column n of X along k
        if (a.pack_mode >= 0) {
            for (int idx = tid; idx < a.npad * kRowsBlock; idx += kThreads) {
                const int n = idx / kRowsBlock, kk = idx - n * kRowsBlock;
                const int64_t gk = kb + kk;
                if (gk >= k1)
                    continue;
                const float v = Xs[kk][n];   // zero for n >= r
                const int64_t o = (int64_t)n * a.kp + gk;
                if (a.pack_mode == TC_BF16) {
                    reinterpret_cast<__nv_bfloat16 *>(a.pack)[o] = __float2bfloat16_rn(v);
                } else if (a.pack_mode == TC_BF16X2) {
                    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                    reinterpret_cast<__nv_bfloat16 *>(a.pack)[o] = hi;
                    reinterpret_cast<__nv_bfloat16 *>(a.pack)[(int64_t)a.npad * a.kp + o] =
                        __float2bfloat16_rn(v - __bfloat162float(hi));
                } else if (a.pack_mode == TC_TF32X3) {
                    const float hi = rn_tf32(v);
                    reinterpret_cast<float *>(a.pack)[o] = hi;
                    reinterpret_cast<float *>(a.pack)[(int64_t)a.npad * a.kp + o] =
                        rn_tf32(v - hi);
                } else {
                    reinterpret_cast<float *>(a.pack)[o] = v;
                }
            }
        }
    }
    float *Ps = a.P + slice * prep_slice_floats(r);
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int ii = ti + 16 * i, jj = tj + 16 * j;
            if (ii < r && jj < r)
                Ps[ii * r + jj] = acc[i][j];
        }
}

// columns rows .. kp-1 of the packed operand (the k padding of its last k
// block) set to zero by the calling CTA
__device__ __forceinline__ void zero_pack_padding(const PrepArgs &a)
{
    const int64_t padk = a.kp - a.rows;
    for (int64_t idx = threadIdx.x; idx < (int64_t)a.npad * padk; idx += blockDim.x) {
        const int64_t nn = idx / padk, o = nn * a.kp + a.rows + (idx - nn * padk);
        if (tc_bf16(a.pack_mode)) {
            reinterpret_cast<__nv_bfloat16 *>(a.pack)[o] = __float2bfloat16_rn(0.f);
            if (a.pack_mode == TC_BF16X2)
                reinterpret_cast<__nv_bfloat16 *>(a.pack)[(int64_t)a.npad * a.kp + o] =
                    __float2bfloat16_rn(0.f);
        } else {
            reinterpret_cast<float *>(a.pack)[o] = 0.f;
            if (a.pack_mode == TC_TF32X3)
                reinterpret_cast<float *>(a.pack)[(int64_t)a.npad * a.kp + o] = 0.f;
        }
    }
}

// columns of the staging block for a factor of at most `cols` columns
__host__ __device__ constexpr int stage_cols(int cols) { return cols <= 32 ? 32 : (cols <= 64 ? 64 : 128); }

}  // namespace prep_detail
}  // namespace nmfi
