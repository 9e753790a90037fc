// Factor preparation between two half-steps: the factor X just updated
// (rows x r) yields
//   * G = X^T X                  (Gram of Alg. 2, FP32; kept for the objective)
//   * Q = G + beta I             (kept for the KKT check)
//   * Qt = D^-1/2 Q D^-1/2, d    (the rescaled problem of Alg. 3, §3.4)
//   * the packed operand of the next tensor-core cross term (optional).
// Two launches replace four (Gram partials, slice sum, rescale, packing):
//   1. CTAs over row ranges of 32+ rows accumulate Gram partials in registers
//      and write their columns of the packed factor;
//   2. CTAs over 128-element column groups of G sum the partials - 32 warps
//      over interleaved slices, 16-byte loads, then the warp sums in warp order: a fixed
//      order, so the result is reproducible - and the last CTA to finish
//      (ticket counter) rescales and clears the counter.
// Both kernels issue their global loads in batches before using them: a
// load whose value is stored or added right away holds the next load back.
#include "k_prep.cuh"

namespace nmfi {
namespace {

using namespace prep_detail;
constexpr int kSumWarps = 32;      // warps of a reduction CTA

template <int NB>
__global__ void __launch_bounds__(kThreads) k_factor_prep(const PrepArgs a)
{
    __shared__ float Xs[kRowsBlock][NB + 1];
    pdl_trigger();   // the finishing kernel may launch; it waits for these partials
    int64_t k0, k1;
    if (a.slices > 0) {   // the NQP kernel's balanced split
        k0 = (int64_t)blockIdx.x * a.rows / gridDim.x;
        k1 = (int64_t)(blockIdx.x + 1) * a.rows / gridDim.x;
    } else {
        k0 = (int64_t)blockIdx.x * a.chunk;
        k1 = k0 + a.chunk < a.rows ? k0 + a.chunk : a.rows;
    }
    gram_pack_rows<NB>(a, Xs, k0, k1, blockIdx.x);
}

constexpr int kBatch = 8;          // 16-byte loads a thread has in flight

// G[e] = sum_s P[s][e] for groups of 32 float4 columns (128 elements; group
// g on CTA g mod gridDim.x): warp w adds the slices w, w + kSumWarps, ... in
// order, kBatch loads issued before their adds, then the warps' sums are
// added in warp order - a fixed order, so the result is reproducible - and
// the last CTA to finish (ticket counter) forms Q, Qt, d
__global__ void __launch_bounds__(kSumWarps * 32, 1) k_prep_finish(const PrepArgs a, int S)
{
    __shared__ float4 part[kSumWarps][32];
    __shared__ float sd[kMaxRank];
    __shared__ int last;
    pdl_trigger();
    pdl_wait();   // the partials are the previous kernel's output
    const int r = a.r, n = r * r, n4 = prep_slice_floats(r) / 4;
    const float4 *P4 = reinterpret_cast<const float4 *>(a.P);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int g = blockIdx.x; g * 32 < n4; g += gridDim.x) {
        const int c = g * 32 + lane;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k0 = w; k0 < S; k0 += kBatch * kSumWarps) {
            float4 v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int k = k0 + u * kSumWarps;
                v[u] = (c < n4 && k < S) ? P4[(int64_t)k * n4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                acc.x += v[u].x;
                acc.y += v[u].y;
                acc.z += v[u].z;
                acc.w += v[u].w;
            }
        }
        part[w][lane] = acc;
        __syncthreads();
        if (w == 0 && c < n4) {
            float4 t = part[0][lane];
#pragma unroll 4
            for (int q = 1; q < kSumWarps; ++q) {
                const float4 u = part[q][lane];
                t.x += u.x;
                t.y += u.y;
                t.z += u.z;
                t.w += u.w;
            }
            const int e = 4 * c;   // the padding floats past n are dropped
            if (e < n)
                a.G[e] = t.x;
            if (e + 1 < n)
                a.G[e + 1] = t.y;
            if (e + 2 < n)
                a.G[e + 2] = t.z;
            if (e + 3 < n)
                a.G[e + 3] = t.w;
        }
        __syncthreads();   // part is rewritten by the next group
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
        const float qii = a.G[i * r + i] + a.beta;
        sd[i] = qii > 0.f ? sqrtf(qii) : 0.f;
        a.d[i] = qii > 0.f ? sd[i] : 1.f;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        const int i = f / r, j = f - i * r;
        const float g = a.G[f];
        const float q = i == j ? g + a.beta : g;
        if (a.Q)
            a.Q[f] = q;
        float v;
        if (sd[i] == 0.f || sd[j] == 0.f)
            v = 0.f;   // dead coordinate (Q_ii <= 0): held at 0
        else if (i == j)
            v = 1.f;
        else
            v = q / (sd[i] * sd[j]);
        a.Qt[f] = v;
    }
    // zero columns K .. kp-1 of the pack (k padding of the last k block)
    if (a.pack_mode >= 0)
        zero_pack_padding(a);
    if (threadIdx.x == 0)
        *a.ticket = 0u;   // ready for the next launch (graph replays included)
}

// groups of 32 float4 columns (128 elements) of one partial slice
int finish_groups(int r) { return (prep_slice_floats(r) / 4 + 31) / 32; }

}  // namespace

// rows per CTA: 32, more only to keep the partials within kMaxSlices
int64_t prep_chunk(int64_t rows)
{
    int64_t c = (rows + kMaxSlices - 1) / kMaxSlices;
    c = c < kRowsBlock ? kRowsBlock : c;
    return (c + kRowsBlock - 1) / kRowsBlock * kRowsBlock;
}

int prep_slices(int64_t rows)
{
    const int64_t c = prep_chunk(rows);
    const int64_t s = (rows + c - 1) / c;
    return s < 1 ? 1 : (int)s;
}

cudaError_t launch_factor_prep(const PrepArgs &a0, cudaStream_t s)
{
    ProfScope prof_(KC_GRAM, s);
    PrepArgs a = a0;
    if (a.rows <= 0 || a.r < 1 || a.r > kMaxRank || !a.G)
        return cudaErrorInvalidValue;
    a.chunk = prep_chunk(a.rows);
    const int S = a.slices > 0 ? a.slices : prep_slices(a.rows);
    if (S > kMaxSlices)
        return cudaErrorInvalidValue;
    // the partials kernel follows the latency-bound NQP kernel: an ordinary
    // launch; the finishing kernel may start while the partials drain
    if (a.r <= 32)
        k_factor_prep<32><<<S, kThreads, 0, s>>>(a);
    else if (a.r <= 64)
        k_factor_prep<64><<<S, kThreads, 0, s>>>(a);
    else
        k_factor_prep<128><<<S, kThreads, 0, s>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    e = pdl_launch(k_prep_finish, dim3(finish_groups(a.r)), dim3(kSumWarps * 32), 0, s, a, S);
    count_launch();
    return e;
}

cudaError_t launch_prep_finish_narrow(const PrepArgs &a, int S, int ctas, cudaStream_t s)
{
    ProfScope prof_(KC_GRAM, s);
    if (a.rows <= 0 || a.r < 1 || a.r > kMaxRank || !a.G || S < 1 || S > kMaxSlices || ctas < 1)
        return cudaErrorInvalidValue;
    const int groups = finish_groups(a.r);
    k_prep_finish<<<ctas < groups ? ctas : groups, kSumWarps * 32, 0, s>>>(a, S);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_prep_finish(const PrepArgs &a, int S, cudaStream_t s)
{
    ProfScope prof_(KC_GRAM, s);
    if (a.rows <= 0 || a.r < 1 || a.r > kMaxRank || !a.G || S < 1 || S > kMaxSlices)
        return cudaErrorInvalidValue;
    cudaError_t e = pdl_launch(k_prep_finish, dim3(finish_groups(a.r)), dim3(kSumWarps * 32), 0, s, a, S);
    count_launch();
    return e;
}

}  // namespace nmfi
