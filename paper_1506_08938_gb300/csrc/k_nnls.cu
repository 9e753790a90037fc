// Batched NQP solver: Alg. 3 of §3.4 (anti-lopsided exact line search plus
// greedy block coordinate descent) run for many rows that share one rescaled
// Gram matrix Qt.
//
// Layout.  One warp owns one row problem.  Lane l holds the J consecutive
// coordinates l*J .. l*J+J-1 of y (rescaled iterate) and g (gradient) in
// registers, so r <= 32*J.  Qt lives in shared memory, zero-padded to
// RP x RP with RP = 32*J, loaded once per CTA and reused by every row the CTA
// processes.  Qt is symmetric, so the column Qt[:, p] used by the coordinate
// update is read as the contiguous row p.
//
// Reductions: warp shuffles for the sums of the line search and the stop
// rule; the greedy argmax is one redux.sync max over the float bits of the
// (non-negative) gains, a ballot to find the lowest lane holding the maximum,
// and two shuffles to broadcast the winner - the lowest index wins exact ties,
// as in the oracle.
#include "nmf_internal.cuh"

namespace nmfi {
namespace {

constexpr int kWarps = 8;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// load the J floats p[0..J) (p 4*J-byte aligned for J = 2, 4)
template <int J>
__device__ __forceinline__ void ld_seg(const float *p, float (&a)[J])
{
    if constexpr (J == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
    } else if constexpr (J == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        a[0] = t.x; a[1] = t.y;
    } else {
#pragma unroll
        for (int j = 0; j < J; ++j)
            a[j] = p[j];
    }
}

template <int J>
__device__ __forceinline__ void st_seg(float *p, const float (&a)[J])
{
    if constexpr (J == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
    } else if constexpr (J == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(a[0], a[1]);
    } else {
#pragma unroll
        for (int j = 0; j < J; ++j)
            p[j] = a[j];
    }
}

// out = Qt v.  v is distributed over the warp (lane l holds v[l*J..]); it is
// staged in this warp's shared buffer vb and read back as broadcast float4.
// Only the first r4 = roundup(r, 4) columns of Qt are non-zero.
template <int J>
__device__ __forceinline__ void matvec(const float *__restrict__ Qs, float *vb,
                                       const float (&v)[J], float (&out)[J], int lane, int r4)
{
    constexpr int RP = 32 * J;
    st_seg<J>(vb + lane * J, v);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < J; ++j)
        out[j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < r4; k += 4) {
        const float4 vk = *reinterpret_cast<const float4 *>(vb + k);
        const float *q = Qs + k * RP + lane * J;
        float a0[J], a1[J], a2[J], a3[J];
        ld_seg<J>(q, a0);
        ld_seg<J>(q + RP, a1);
        ld_seg<J>(q + 2 * RP, a2);
        ld_seg<J>(q + 3 * RP, a3);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            out[j] = fmaf(a0[j], vk.x, out[j]);
            out[j] = fmaf(a1[j], vk.y, out[j]);
            out[j] = fmaf(a2[j], vk.z, out[j]);
            out[j] = fmaf(a3[j], vk.w, out[j]);
        }
    }
    __syncwarp();
}

// ||P(y, g)||^2 over the warp: the passive set is {y > 0 or g < 0}.
template <int J>
__device__ __forceinline__ float proj_sq(const float (&y)[J], const float (&g)[J])
{
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < J; ++j)
        if (y[j] > 0.f || g[j] < 0.f)
            s = fmaf(g[j], g[j], s);
    return warp_sum(s);
}

template <int J>
__global__ void __launch_bounds__(kWarps * 32, 3) k_nnls(const NnlsArgs a)
{
    constexpr int RP = 32 * J;
    extern __shared__ __align__(16) float smem[];
    float *Qs = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *vb = smem + RP * RP + warp * RP;
    const int r = a.r;
    const int r4 = (r + 3) & ~3;

    for (int idx = threadIdx.x; idx < RP * RP; idx += blockDim.x) {
        int i = idx / RP, j = idx - i * RP;
        Qs[idx] = (i < r && j < r) ? a.Qt[i * r + j] : 0.f;
    }
    __syncthreads();

    // per-lane constants: inverse diagonal, half diagonal, scale d
    float iq[J], hq[J], dd[J];
    bool live[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        int e = lane * J + j;
        float qii = e < r ? Qs[e * RP + e] : 0.f;
        live[j] = qii > 0.f;
        iq[j] = live[j] ? 1.f / qii : 0.f;
        hq[j] = 0.5f * qii;
        dd[j] = (e < r && live[j]) ? a.d[e] : 1.f;
    }
    const int T = a.cd_steps < 0 ? r : a.cd_steps;
    const int64_t wstride = (int64_t)gridDim.x * kWarps;
    unsigned long long my_iters = 0;
    unsigned my_smax = 0;

    for (int64_t row = (int64_t)blockIdx.x * kWarps + warp; row < a.rows; row += wstride) {
        float y[J], g[J];
        bool ok = true;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            int e = lane * J + j;
            float c = 0.f, x0 = 0.f;
            if (e < r) {
                const float *cp = a.C + row * r + e;
                for (int s = 0; s < a.nsplit; ++s)
                    c += cp[s * a.c_stride];
                x0 = a.X[row * r + e];
                ok = ok && isfinite(c) && isfinite(x0);
            }
            // rescaled problem: q = (alpha - c)/d, y = x0 .* d  (Alg. 3 rescale)
            g[j] = live[j] ? (a.alpha - c) / dd[j] : 0.f;
            y[j] = live[j] ? x0 * dd[j] : 0.f;
        }
        if (!__all_sync(kFull, ok)) {
            if (lane == 0 && a.status)
                atomicOr(a.status, kStNonFinite);
            continue;
        }
        {   // gradient f = Qt y + q
            float t[J];
            matvec<J>(Qs, vb, y, t, lane, r4);
#pragma unroll
            for (int j = 0; j < J; ++j)
                g[j] = live[j] ? g[j] + t[j] : 0.f;
        }
        const float s0 = proj_sq<J>(y, g);
        float sk = s0;
        int k = 0;
        if (s0 > 0.f) {
            for (k = 1; k <= a.max_inner; ++k) {
                // ---- exact line search along the masked gradient
                float gb[J];
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    gb[j] = (y[j] > 0.f || g[j] < 0.f) ? g[j] : 0.f;
                    s = fmaf(gb[j], gb[j], s);
                }
                s = warp_sum(s);
                if (s > 0.f) {
                    float u[J];
                    matvec<J>(Qs, vb, gb, u, lane, r4);
                    float den = 0.f;
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        den = fmaf(gb[j], u[j], den);
                    den = warp_sum(den);
                    if (den > 0.f) {
                        const float alpha = s / den;
                        float dl[J];
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            float yn = fmaxf(0.f, y[j] - alpha * gb[j]);
                            dl[j] = yn - y[j];
                            y[j] = yn;
                        }
                        matvec<J>(Qs, vb, dl, u, lane, r4);
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            g[j] += u[j];
                    }
                }
                // ---- greedy coordinate descent
                for (int t = 0; t < T; ++t) {
                    unsigned bkey = 0u;
                    int bj = 0;
                    float bdel = 0.f;
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        float del = fmaxf(0.f, fmaf(-g[j], iq[j], y[j])) - y[j];
                        float gain = -(del * fmaf(hq[j], del, g[j]));
                        unsigned key = __float_as_uint(fmaxf(gain, 0.f)) & 0x7fffffffu;
                        if (key > bkey) {
                            bkey = key;
                            bj = j;
                            bdel = del;
                        }
                    }
                    const unsigned m = __reduce_max_sync(kFull, bkey);
                    if (m == 0u)
                        break;
                    const int src = __ffs(__ballot_sync(kFull, bkey == m)) - 1;
                    const int pj = __shfl_sync(kFull, bj, src);
                    const float dp = __shfl_sync(kFull, bdel, src);
                    const int p = src * J + pj;
                    float col[J];
                    ld_seg<J>(Qs + p * RP + lane * J, col);
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        g[j] = fmaf(col[j], dp, g[j]);
                    if (lane == src) {
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            if (j == pj)
                                y[j] += dp;
                    }
                }
                sk = proj_sq<J>(y, g);
                if (sk <= a.eps * s0)
                    break;
                if (a.maxstop_mode == 1 && sk <= a.maxstop)
                    break;
            }
            if (k > a.max_inner)
                k = a.max_inner;
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            int e = lane * J + j;
            if (e < r)
                a.X[row * r + e] = live[j] ? y[j] / dd[j] : 0.f;
        }
        if (lane == 0) {
            if (a.iters)
                a.iters[row] = k;
            my_iters += (unsigned long long)k;
            unsigned sb = __float_as_uint(sk);
            my_smax = sb > my_smax ? sb : my_smax;
        }
    }
    if (lane == 0) {
        if (a.iter_total && my_iters)
            atomicAdd(a.iter_total, my_iters);
        if (a.s_final_max && my_smax)
            atomicMax(a.s_final_max, my_smax);
    }
}

template <int J>
struct NnlsCfg {
    static int blocks_per_sm, sms;
};
template <int J>
int NnlsCfg<J>::blocks_per_sm = -1;
template <int J>
int NnlsCfg<J>::sms = 0;

// one-time launch configuration (kept out of any stream capture)
template <int J>
cudaError_t prepare_j()
{
    constexpr int RP = 32 * J;
    const size_t smem = sizeof(float) * (size_t)(RP * RP + kWarps * RP);
    int &blocks_per_sm = NnlsCfg<J>::blocks_per_sm, &sms = NnlsCfg<J>::sms;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(k_nnls<J>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_nnls<J>,
                                                          kWarps * 32, smem);
        if (e != cudaSuccess)
            return e;
        if (blocks_per_sm < 1)
            blocks_per_sm = 1;
    }
    return cudaSuccess;
}

template <int J>
cudaError_t launch_j(const NnlsArgs &a, cudaStream_t s)
{
    constexpr int RP = 32 * J;
    const size_t smem = sizeof(float) * (size_t)(RP * RP + kWarps * RP);
    cudaError_t e = prepare_j<J>();
    if (e != cudaSuccess)
        return e;
    const int blocks_per_sm = NnlsCfg<J>::blocks_per_sm, sms = NnlsCfg<J>::sms;
    int64_t need = (a.rows + kWarps - 1) / kWarps;
    int64_t cap = (int64_t)blocks_per_sm * sms;
    int grid = (int)(need < cap ? need : cap);
    if (grid < 1)
        return cudaSuccess;
    k_nnls<J><<<grid, kWarps * 32, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_nnls(int r)
{
    if (r <= 32)
        return prepare_j<1>();
    if (r <= 64)
        return prepare_j<2>();
    if (r <= 96)
        return prepare_j<3>();
    return prepare_j<4>();
}

cudaError_t launch_nnls(const NnlsArgs &a, cudaStream_t s)
{
    ProfScope prof_(KC_NNLS, s);
    if (a.rows <= 0)
        return cudaSuccess;
    if (a.r <= 32)
        return launch_j<1>(a, s);
    if (a.r <= 64)
        return launch_j<2>(a, s);
    if (a.r <= 96)
        return launch_j<3>(a, s);
    return launch_j<4>(a, s);
}

}  // namespace nmfi
