// Small kernels around the products:
//  * rescale   - anti-lopsided rescaling of the shared Gram (§3.4 Eq. 3)
//  * objective - J by the trace identity, FP64 (Def. 1; Table 4 reports
//                1/2||V - WH||^2), with the L1/L2 terms of §3.5
//  * kkt       - optimality residuals of Eq. 2 (float-float sums, FP64 residuals)
//  * sumsq     - ||V||_F^2 in FP64 (constant term of the trace identity)
// All reductions are two-level with a fixed grid and a last-block finish, so
// their results do not depend on scheduling.
#include "nmf_internal.cuh"

namespace nmfi {
namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide FP64 sum, fixed order (warp tree, then warp 0 over warp sums)
__device__ double block_sum_d(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0)
        sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        t = warp_sum_d(t);
    }
    return t;   // valid in thread 0
}

__global__ void k_rescale(const float *__restrict__ P, int nsplit, int r, float beta,
                          float *__restrict__ G, float *__restrict__ Q, float *__restrict__ Qt,
                          float *__restrict__ dout)
{
    __shared__ float sd[kMaxRank];
    const int n = r * r;
    // diagonal first: d_i = sqrt(Q_ii), 0 marks a dead coordinate
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < nsplit; ++k)
            s += P[(int64_t)k * n + i * r + i];
        const float qii = s + beta;
        sd[i] = qii > 0.f ? sqrtf(qii) : 0.f;
        if (dout)
            dout[i] = qii > 0.f ? sd[i] : 1.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < nsplit; ++k)
            s += P[(int64_t)k * n + e];
        const int i = e / r, j = e - i * r;
        if (G)
            G[e] = s;
        const float q = i == j ? s + beta : s;
        if (Q)
            Q[e] = q;
        if (Qt) {
            float v;
            if (sd[i] == 0.f || sd[j] == 0.f)
                v = 0.f;
            else if (i == j)
                v = 1.f;
            else
                v = q / (sd[i] * sd[j]);
            Qt[e] = v;
        }
    }
}

// J = 1/2 (vv - 2<Ht, Ch> + <Gw, Gh>) + aw sum W + ah sum Ht + bw/2 tr Gw + bh/2 tr Gh
__global__ void __launch_bounds__(kRedThreads) k_objective(const ObjArgs a)
{
    __shared__ double sh[32];
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nh = a.n * a.r, nw = a.m * a.r;
    double dot = 0.0, sw = 0.0, shh = 0.0;
    for (int64_t e = tid; e < nh; e += stride) {
        float c = 0.f;
        for (int s = 0; s < a.nsplit; ++s)
            c += a.Ch[s * a.ch_stride + e];
        const double h = (double)a.Ht[e];
        dot += h * (double)c;
        shh += h;
    }
    for (int64_t e = tid; e < nw; e += stride)
        sw += (double)a.W[e];
    double v0 = block_sum_d(dot, sh);
    double v1 = block_sum_d(sw, sh);
    double v2 = block_sum_d(shh, sh);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        a.partials[blockIdx.x * 3 + 0] = v0;
        a.partials[blockIdx.x * 3 + 1] = v1;
        a.partials[blockIdx.x * 3 + 2] = v2;
        __threadfence();
        unsigned t = atomicAdd(a.ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    // last block: partial sums in block order, then the r x r terms
    double gg = 0.0, trw = 0.0, trh = 0.0;
    const int rr = a.r * a.r;
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        gg += (double)a.Gw[e] * (double)a.Gh[e];
        if (e / a.r == e % a.r) {
            trw += (double)a.Gw[e];
            trh += (double)a.Gh[e];
        }
    }
    gg = block_sum_d(gg, sh);
    trw = block_sum_d(trw, sh);
    trh = block_sum_d(trh, sh);
    if (threadIdx.x == 0) {
        volatile double *pp = a.partials;
        double d = 0.0, s1 = 0.0, s2 = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            d += pp[b * 3 + 0];
            s1 += pp[b * 3 + 1];
            s2 += pp[b * 3 + 2];
        }
        double J = 0.5 * (a.vv - 2.0 * d + gg) + (double)a.aw * s1 + (double)a.ah * s2 +
                   0.5 * (double)a.bw * trw + 0.5 * (double)a.bh * trh;
        *a.J = J;
        if (a.hist && a.t)
            a.hist[*a.t] = J;
        if (a.done_flag && a.f_star > 0.0 && (J - a.f_star) / a.f_star <= a.gap_target)
            *a.done_flag = 1;
        *a.ticket = 0u;   // ready for the next launch
    }
}

// KKT residuals of one factor, FP64.  One warp per row, the row in smem;
// lane j forms (Q x)_j reading Q by columns (Q symmetric), so for each k the
// lanes read one contiguous run of Q instead of 32 separate rows.
// a b added to the float-float sum (hi, lo): the product exactly as p + e
// (one rounding, recovered by an FMA), p added to hi by Knuth's TwoSum, both
// error terms to lo.  The _rn intrinsics keep the compiler from contracting
// or reassociating any of it.
__device__ __forceinline__ void ff_add_prod(float &hi, float &lo, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bv = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

constexpr int kKktRows = 32;   // rows of X per tile
constexpr int kKktRowsPerThread = kKktRows / 4;

// Gradient entries grad_ij = alpha - C_ij + sum_k Q_kj X_ik of one tile of
// 32 rows: thread (ty, tx) owns rows ty*8 .. ty*8+7 and columns tx, tx + 64.
// The sums run over k in order in float-float (products exact, sums
// compensated: about 44 bits), i.e. FP64-grade for FP32 data at FP32
// rates - this part's FP64 pipe runs at 1/64 of the FP32 rate, and a
// double per operand cost two conversions per product there.  The residuals
// and their maxima are FP64.
__global__ void __launch_bounds__(256) k_kkt(const float *__restrict__ Q,
                                             const float *__restrict__ C, int64_t rows, int r,
                                             float alpha, const float *__restrict__ X,
                                             unsigned long long *out)
{
    extern __shared__ float kkt_smem[];
    float *Qs = kkt_smem;            // r x r, as Q
    float *Xs = kkt_smem + r * r;    // kKktRows x r
    __shared__ double red[2][8];
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    for (int i = threadIdx.x; i < r * r; i += blockDim.x)
        Qs[i] = Q[i];
    const bool c0 = tx < r, c1 = tx + 64 < r;
    double m1 = 0.0, m2 = 0.0;
    const int64_t tiles = (rows + kKktRows - 1) / kKktRows;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t row0 = t * kKktRows;
        const int nr = rows - row0 < kKktRows ? (int)(rows - row0) : kKktRows;
        __syncthreads();   // Qs staged; the previous tile's Xs read
        for (int i = threadIdx.x; i < nr * r; i += blockDim.x)
            Xs[i] = X[row0 * r + i];
        for (int i = nr * r + threadIdx.x; i < kKktRows * r; i += blockDim.x)
            Xs[i] = 0.f;   // rows past the end: finite values, results unused
        __syncthreads();
        float hi[kKktRowsPerThread][2], lo[kKktRowsPerThread][2];
#pragma unroll
        for (int i = 0; i < kKktRowsPerThread; ++i) {
            hi[i][0] = hi[i][1] = 0.f;
            lo[i][0] = lo[i][1] = 0.f;
        }
        const float *xr = Xs + ty * kKktRowsPerThread * r;
        for (int k = 0; k < r; ++k) {
            const float q0 = c0 ? Qs[k * r + tx] : 0.f;
            const float q1 = c1 ? Qs[k * r + tx + 64] : 0.f;
#pragma unroll
            for (int i = 0; i < kKktRowsPerThread; ++i) {
                const float xv = xr[i * r + k];   // one address per warp: broadcast
                ff_add_prod(hi[i][0], lo[i][0], q0, xv);
                ff_add_prod(hi[i][1], lo[i][1], q1, xv);
            }
        }
#pragma unroll
        for (int i = 0; i < kKktRowsPerThread; ++i) {
            const int lr = ty * kKktRowsPerThread + i;
            if (lr >= nr)
                continue;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int j = tx + 64 * c;
                if (j >= r)
                    continue;
                const double g = ((double)hi[i][c] + (double)lo[i][c]) + (double)alpha -
                                 (double)C[(row0 + lr) * r + j];
                const double x = (double)xr[i * r + j];
                const double a1 = fabs(x < g ? x : g), a2 = fabs(x * g);
                m1 = a1 > m1 ? a1 : m1;
                m2 = a2 > m2 ? a2 : m2;
            }
        }
    }
    // non-negative doubles order like their bit patterns
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = m1;
        red[1][w] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < 8; ++q) {
            m1 = fmax(m1, red[0][q]);
            m2 = fmax(m2, red[1][q]);
        }
        atomicMax(out, (unsigned long long)__double_as_longlong(m1));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(m2));
    }
}

// J = 1/2 sum_ij (V_ij - W_i . Ht_j)^2 + penalties, the residual formed
// element by element: W_i . Ht_j by an FP32 fma chain over r in order, its
// square summed in FP32 over the thread's 64 elements of a 128 x 128 tile,
// the tile sums in FP64.  Avoids the cancellation of the trace identity.
// One persistent CTA per SM walks the tiles (8 x 8 elements a thread: 64
// FMAs per four 16-byte shared loads); FP64 arithmetic (a small fraction of
// FP32 throughput on this part) is kept to one add per thread per tile.
// Thread (ty, tx) owns rows {ty*4 + i, 64 + ty*4 + i} and columns
// {tx*4 + j, 64 + tx*4 + j} of the tile, so consecutive threads read
// consecutive 16-byte words of the staged factors.  The factors' rows of a
// tile go to shared memory (k-major, 64 columns of r per stage) by cp.async,
// two stages deep: the next stage's copies land while this one is computed.
constexpr int kObjTile = 128, kObjKc = 64, kObjLd = kObjTile + 4;
constexpr size_t kObjSmem = 2 * 2 * kObjKc * kObjLd * sizeof(float);

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    // src-size 0 fills the word with zeros and reads nothing
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

__global__ void __launch_bounds__(256, 1) k_objective_direct(const ObjDirectArgs a)
{
    constexpr int BT = kObjTile, KC = kObjKc, LD = kObjLd;
    extern __shared__ __align__(16) float obj_smem[];
    __shared__ double sh[32];
    __shared__ bool last;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int r = a.r;
    const int64_t tiles_n = (a.n + BT - 1) / BT;
    const int64_t tiles = ((a.m + BT - 1) / BT) * tiles_n;
    const int nch = (r + KC - 1) / KC;   // stages per tile
    const bool v_vec = (a.ldv & 3) == 0 && (reinterpret_cast<uintptr_t>(a.V) & 15) == 0;
    // stage st of this CTA: tile blockIdx.x + (st / nch) gridDim.x, chunk st % nch
    const int64_t my_tiles = blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t stages = my_tiles * nch;
    auto stage_copy = [&](int64_t st) {
        const int64_t tile = blockIdx.x + (st / nch) * gridDim.x;
        const int k0 = (int)(st % nch) * KC;
        const int64_t i0 = (tile / tiles_n) * BT, j0 = (tile % tiles_n) * BT;
        float *Ws = obj_smem + (st & 1) * 2 * KC * LD, *Hs = Ws + KC * LD;
        // element (row rr, column kk) of the stage: consecutive threads take
        // consecutive columns of one row (coalesced), stored k-major
#pragma unroll 4
        for (int idx = tid; idx < BT * KC; idx += 256) {
            const int rr = idx / KC, kk = idx % KC;
            const int gk = k0 + kk;
            const int64_t gi = i0 + rr, gj = j0 + rr;
            const bool wv = gi < a.m && gk < r, hv = gj < a.n && gk < r;
            cp_async4(&Ws[kk * LD + rr], wv ? a.W + gi * r + gk : a.W, wv);
            cp_async4(&Hs[kk * LD + rr], hv ? a.Ht + gj * r + gk : a.Ht, hv);
        }
    };
    double fit = 0.0;
    float vv[8][8], acc[8][8];
    if (stages > 0)
        stage_copy(0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int64_t st = 0; st < stages; ++st) {
        if (st + 1 < stages)
            stage_copy(st + 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // stage st has landed
        __syncthreads();
        const int64_t tile = blockIdx.x + (st / nch) * gridDim.x;
        const int c = (int)(st % nch);
        const int64_t i0 = (tile / tiles_n) * BT, j0 = (tile % tiles_n) * BT;
        if (c == 0) {
            // this thread's 64 elements of V, requested now and used after
            // the products: the loads are in flight while the tile is computed
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t gi = i0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t gj = j0 + h * 64 + tx * 4;
                    if (gi < a.m && v_vec && gj + 3 < a.n) {
                        const float4 q = *reinterpret_cast<const float4 *>(a.V + gi * a.ldv + gj);
                        vv[i][h * 4 + 0] = q.x;
                        vv[i][h * 4 + 1] = q.y;
                        vv[i][h * 4 + 2] = q.z;
                        vv[i][h * 4 + 3] = q.w;
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            vv[i][h * 4 + j] =
                                (gi < a.m && gj + j < a.n) ? a.V[gi * a.ldv + gj + j] : 0.f;
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[i][j] = 0.f;
        }
        const float *Ws = obj_smem + (st & 1) * 2 * KC * LD, *Hs = Ws + KC * LD;
        const int kc = r - c * KC < KC ? r - c * KC : KC;   // columns of this stage
#pragma unroll 2
        for (int kk = 0; kk < kc; ++kk) {
            const float4 wa = *reinterpret_cast<const float4 *>(Ws + kk * LD + ty * 4);
            const float4 wb = *reinterpret_cast<const float4 *>(Ws + kk * LD + 64 + ty * 4);
            const float4 ha = *reinterpret_cast<const float4 *>(Hs + kk * LD + tx * 4);
            const float4 hb = *reinterpret_cast<const float4 *>(Hs + kk * LD + 64 + tx * 4);
            const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
            const float hh[8] = {ha.x, ha.y, ha.z, ha.w, hb.x, hb.y, hb.z, hb.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[i][j] = fmaf(w[i], hh[j], acc[i][j]);
        }
        if (c == nch - 1) {
            float f32 = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t gi = i0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
                if (gi >= a.m)
                    continue;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int64_t gj = j0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
                    if (gj < a.n) {
                        const float e = vv[i][j] - acc[i][j];
                        f32 = fmaf(e, e, f32);
                    }
                }
            }
            fit += (double)f32;
        }
        __syncthreads();   // this buffer is refilled two stages on
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // penalty sums over the factors: FP32 groups of 16, FP64 across groups
    double sw = 0.0, sw2 = 0.0, shh = 0.0, sh2 = 0.0;
    {
        const int64_t gt = (int64_t)blockIdx.x * blockDim.x + tid,
                      gs = (int64_t)gridDim.x * blockDim.x;
        float g1 = 0.f, g2 = 0.f;
        int c = 0;
        for (int64_t e = gt; e < a.m * a.r; e += gs) {
            float v = a.W[e];
            g1 += v;
            g2 = fmaf(v, v, g2);
            if (++c == 16) {
                sw += g1;
                sw2 += g2;
                g1 = g2 = 0.f;
                c = 0;
            }
        }
        sw += g1;
        sw2 += g2;
        g1 = g2 = 0.f;
        c = 0;
        for (int64_t e = gt; e < a.n * a.r; e += gs) {
            float v = a.Ht[e];
            g1 += v;
            g2 = fmaf(v, v, g2);
            if (++c == 16) {
                shh += g1;
                sh2 += g2;
                g1 = g2 = 0.f;
                c = 0;
            }
        }
        shh += g1;
        sh2 += g2;
    }
    double v[5] = {fit, sw, sw2, shh, sh2};
#pragma unroll
    for (int q = 0; q < 5; ++q)
        v[q] = block_sum_d(v[q], sh);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q)
            a.partials[(int64_t)blockIdx.x * 5 + q] = v[q];
        __threadfence();
        last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    volatile double *pp = a.partials;
    double t[5] = {0, 0, 0, 0, 0};
    for (unsigned b = tid; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q)
            t[q] += pp[(int64_t)b * 5 + q];
#pragma unroll
    for (int q = 0; q < 5; ++q)
        t[q] = block_sum_d(t[q], sh);
    if (tid == 0) {
        *a.J = 0.5 * t[0] + (double)a.aw * t[1] + 0.5 * (double)a.bw * t[2] +
               (double)a.ah * t[3] + 0.5 * (double)a.bh * t[4];
        *a.ticket = 0u;
    }
}

template <typename T>
__device__ __forceinline__ float as_f(T v);
template <>
__device__ __forceinline__ float as_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float as_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_sumsq(const T *__restrict__ x, int64_t n,
                                                       double *out, double *partials,
                                                       unsigned *ticket)
{
    __shared__ double sh[32];
    __shared__ bool last;
    // groups of 16 squares in FP32, the groups summed in FP64
    double s = 0.0;
    float g = 0.f;
    int cnt = 0;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // four loads in flight per trip, squared and summed in element order
    for (; e + 3 * st < n; e += 4 * st) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = as_f<T>(x[e + u * st]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            g = fmaf(v[u], v[u], g);
            if (++cnt == 16) {
                s += (double)g;
                g = 0.f;
                cnt = 0;
            }
        }
    }
    for (; e < n; e += st) {
        float v = as_f<T>(x[e]);
        g = fmaf(v, v, g);
        if (++cnt == 16) {
            s += (double)g;
            g = 0.f;
            cnt = 0;
        }
    }
    s += (double)g;
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        volatile double *pp = partials;
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b)
            t += pp[b];
        *out = t;
        *ticket = 0u;
    }
}

__global__ void k_f32_to_bf16(const float *__restrict__ x, int64_t n, __nv_bfloat16 *__restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16_rn(x[e]);
}

}  // namespace

cudaError_t launch_rescale(const float *P, int nsplit, int r, float beta, float *G, float *Q,
                           float *Qt, float *d, cudaStream_t s)
{
    ProfScope prof_(KC_RESCALE, s);
    k_rescale<<<1, 1024, 0, s>>>(P, nsplit, r, beta, G, Q, Qt, d);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_objective(const ObjArgs &a, cudaStream_t s)
{
    ProfScope prof_(KC_OBJECTIVE, s);
    k_objective<<<kRedBlocks, kRedThreads, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

constexpr int kObjBlocks = 4 * 152;   // most persistent CTAs of the direct objective (partials)

size_t objective_direct_partials(int64_t, int64_t) { return (size_t)kObjBlocks * 5; }

cudaError_t launch_objective_direct(const ObjDirectArgs &a, cudaStream_t s)
{
    ProfScope prof_(KC_OBJECTIVE, s);
    const int64_t tiles = ((a.m + kObjTile - 1) / kObjTile) * ((a.n + kObjTile - 1) / kObjTile);
    if (tiles <= 0)
        return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(
            k_objective_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kObjSmem);
        if (e != cudaSuccess)
            return e;
        attr_set = true;
    }
    int64_t grid = num_sms();   // one CTA per SM (64 accumulators a thread)
    grid = grid < kObjBlocks ? grid : kObjBlocks;
    k_objective_direct<<<(unsigned)(tiles < grid ? tiles : grid), 256, kObjSmem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_kkt(const float *Q, const float *C, int64_t rows, int r, float alpha,
                       const float *X, double *out, cudaStream_t s)
{
    ProfScope prof_(KC_OTHER, s);
    cudaMemsetAsync(out, 0, 2 * sizeof(double), s);
    if (rows <= 0)
        return cudaGetLastError();
    if (r < 1 || r > kMaxRank)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)(r * r + kKktRows * r) * sizeof(float);
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_kkt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)((kMaxRank * kMaxRank + kKktRows * kMaxRank) *
                                                         sizeof(float)));
        if (e != cudaSuccess)
            return e;
        attr_set = true;
    }
    const int64_t tiles = (rows + kKktRows - 1) / kKktRows;
    const int64_t cap = 2 * (int64_t)num_sms();
    k_kkt<<<(unsigned)(tiles < cap ? tiles : cap), 256, smem, s>>>(
        Q, C, rows, r, alpha, X, reinterpret_cast<unsigned long long *>(out));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const void *x, nmf_dtype dt, int64_t n, double *out, double *partials,
                         unsigned *ticket, cudaStream_t s)
{
    ProfScope prof_(KC_OTHER, s);
    if (dt == NMF_BF16)
        k_sumsq<__nv_bfloat16><<<kRedBlocks, kRedThreads, 0, s>>>(
            reinterpret_cast<const __nv_bfloat16 *>(x), n, out, partials, ticket);
    else
        k_sumsq<float><<<kRedBlocks, kRedThreads, 0, s>>>(reinterpret_cast<const float *>(x), n,
                                                          out, partials, ticket);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float *x, int64_t n, __nv_bfloat16 *y, cudaStream_t s)
{
    ProfScope prof_(KC_OTHER, s);
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192)
        blocks = 8192;
    if (blocks < 1)
        return cudaSuccess;
    k_f32_to_bf16<<<(unsigned)blocks, 256, 0, s>>>(x, n, y);
    count_launch();
    return cudaGetLastError();
}

}  // namespace nmfi

// ---- FP32 FFMA throughput probe ---------------------------------------------
// Eight independent dependent chains of fmaf per thread, enough warps per SM
// to keep every FMA lane busy; the result is stored only if it equals a value
// the chains never reach, so the compiler keeps the work.
namespace nmfi {
namespace {
__global__ void __launch_bounds__(256) k_ffma_probe(float *out, int iters, float seed)
{
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        a[j] = seed + 1e-3f * (float)(threadIdx.x + j);
    const float mlt = 0.9999999f, add = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            a[j] = fmaf(a[j], mlt, add);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        s += a[j];
    if (s == -1.0f)
        out[blockIdx.x] = s;
}
}  // namespace

cudaError_t measure_fp32_peak(double *tflops)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma_probe, 256, 0);
    if (e != cudaSuccess)
        return e;
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 8192;
    float *out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(float) * grid)) != cudaSuccess)
        return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_ffma_probe<<<grid, 256>>>(out, iters, 1.f);   // warm-up (clocks ramp)
    k_ffma_probe<<<grid, 256>>>(out, iters, 1.f);
    cudaEventRecord(e0);
    const int reps = 5;
    for (int i = 0; i < reps; ++i)
        k_ffma_probe<<<grid, 256>>>(out, iters, 1.f);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess)
        return e;
    const double flops = 2.0 * 8.0 * iters * 256.0 * grid * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return cudaGetLastError();
}
}  // namespace nmfi
