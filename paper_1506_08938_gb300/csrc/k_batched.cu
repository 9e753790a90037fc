// Many independent NMF instances of uneven m, n, r (the paper's computation
// units are independent NQPs, §3.2-3.3; here whole factorisations are
// independent too) advanced by one outer iteration (Alg. 2) per launch.
//
// One outer iteration is eight phases for every instance:
//   0 Gram partials of Ht      1 sum + L2 + rescale -> Qt_W, d_W
//   2 cross C_W = V Ht         3 NNLS of every row of W (Alg. 3)
//   4 Gram partials of W       5 sum + L2 + rescale -> Qt_H, d_H
//   6 cross C_H = V^T W        7 NNLS of every row of Ht
// Each phase is a flat list of work items over all instances (row chunks,
// row tiles, instances); a CTA takes items i, i + grid, ... and maps an item
// to its instance by binary search over per-phase prefix sums.
//
// Persistent mode: one cooperative launch runs all eight phases with grid
// barriers in between (every CTA is resident: the grid is the occupancy
// limit).  Loop mode: the same phase code launched once per instance and
// phase, the baseline whose launch count the persistent form removes.
// Arithmetic is FP32 on CUDA cores; instance ranks r <= 64.
#include "nmf_internal.cuh"

namespace nmfi {
namespace {

constexpr int kT = 256;            // threads per CTA
constexpr int kWarps = kT / 32;
constexpr int kGramRows = 256;     // rows of X per Gram item
constexpr int kCrossRows = 64;     // rows of A per cross item
constexpr unsigned long long kBarrierNs = 2000000000ull;

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded sense-reversing grid barrier; false on timeout
__device__ bool grid_barrier(unsigned *count, volatile unsigned *gen, unsigned nblocks,
                             unsigned *status)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd((unsigned *)gen, 1u);
        } else {
            // a barrier that another CTA gave up on never completes: leave
            // at once instead of waiting out the limit again
            const volatile unsigned *vs = status;
            const unsigned long long dl = gtime() + kBarrierNs;
            while (*gen == g) {
                if ((*vs & kStTimeout) || gtime() > dl) {
                    atomicOr(status, kStTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int find_inst(const int64_t *off, int count, int64_t item)
{
    int lo = 0, hi = count;   // largest i with off[i] <= item
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- phase bodies ----------------------------------------------------------

// Gram partial of rows [k0, k0 + kGramRows) of X (rows x r) into P (r x r)
template <int NB>
__device__ void gram_item(const float *X, int64_t rows, int r, int64_t k0, float *P, float *sm)
{
    constexpr int BK = 32, T = NB / 16;
    float(*Xs)[NB] = reinterpret_cast<float(*)[NB]>(sm);
    const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
    const int64_t ke = k0 + kGramRows < rows ? k0 + kGramRows : rows;
    float acc[T][T];
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b)
            acc[a][b] = 0.f;
    for (int64_t kb = k0; kb < ke; kb += BK) {
        __syncthreads();
        for (int idx = tid; idx < BK * NB; idx += kT) {
            int kk = idx / NB, c = idx - kk * NB;
            int64_t gk = kb + kk;
            Xs[kk][c] = (c < r && gk < ke) ? X[gk * r + c] : 0.f;
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
#pragma unroll
            for (int a = 0; a < T; ++a)
#pragma unroll
                for (int b = 0; b < T; ++b)
                    acc[a][b] = fmaf(xa[a], xb[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) {
            int i = ti + 16 * a, j = tj + 16 * b;
            if (i < r && j < r)
                P[i * r + j] = acc[a][b];
        }
}

// sum the instance's Gram partials, add beta, rescale (Alg. 3 rescale)
__device__ void rescale_item(const float *P, int nparts, int r, float beta, float *Qt, float *d,
                             float *sm)
{
    float *sq = sm;               // r x r
    float *sd = sm + r * r;       // r
    const int n = r * r;
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += kT) {
        float s = 0.f;
        for (int k = 0; k < nparts; ++k)
            s += P[(int64_t)k * n + e];
        const int i = e / r, j = e - i * r;
        sq[e] = i == j ? s + beta : s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += kT) {
        const float q = sq[i * r + i];
        sd[i] = q > 0.f ? sqrtf(q) : 0.f;
        d[i] = q > 0.f ? sd[i] : 1.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += kT) {
        const int i = e / r, j = e - i * r;
        float v;
        if (sd[i] == 0.f || sd[j] == 0.f)
            v = 0.f;
        else if (i == j)
            v = 1.f;
        else
            v = sq[e] / (sd[i] * sd[j]);
        Qt[e] = v;
    }
}

// cross term rows [m0, m0 + kCrossRows) of C = A B (A M x K row-major, B K x r)
template <int NB>
__device__ void cross_item(const float *A, int64_t M, int64_t K, const float *B, int r,
                           int64_t m0, float *C, float *sm)
{
    constexpr int BM = kCrossRows, BK = 16, TM = BM / 16, TN = NB / 16;
    float(*As)[BM + 4] = reinterpret_cast<float(*)[BM + 4]>(sm);
    float(*Bs)[NB] = reinterpret_cast<float(*)[NB]>(sm + BK * (BM + 4));
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
            acc[i][j] = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
#pragma unroll
        for (int t = 0; t < BM * BK / kT; ++t) {
            int idx = tid + t * kT;
            int mm = idx >> 4, kk = idx & 15;
            int64_t gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[gm * K + gk] : 0.f;
        }
        for (int idx = tid; idx < BK * NB; idx += kT) {
            int kk = idx / NB, nn = idx - kk * NB;
            int64_t gk = k0 + kk;
            Bs[kk][nn] = (nn < r && gk < K) ? B[gk * r + nn] : 0.f;
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
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int64_t gm = m0 + ty + 16 * i;
        if (gm >= M)
            continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int n = tx + 16 * j;
            if (n < r)
                C[gm * r + n] = acc[i][j];
        }
    }
}

// Alg. 3 for rows [row0, row0 + kNnlsRows) of X; warp per row, Qt in shared
// memory (the same iteration as the single-instance kernel)
template <int J>
__device__ void nnls_item(const float *Qt, const float *dv, const float *Cm, int64_t rows, int r,
                          float alpha, float *X, int64_t row0, int nrows, const BatchNnls &o,
                          float *sm, unsigned long long *iter_total, unsigned *status)
{
    constexpr int RP = 32 * J;
    float *Qs = sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *vb = sm + RP * RP + warp * RP;
    const int r4 = (r + 3) & ~3;
    __syncthreads();
    for (int idx = threadIdx.x; idx < RP * RP; idx += kT) {
        int i = idx / RP, j = idx - i * RP;
        Qs[idx] = (i < r && j < r) ? Qt[i * r + j] : 0.f;
    }
    __syncthreads();
    float iq[J], hq[J], dd[J];
    bool live[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        int e = lane * J + j;
        float qii = e < r ? Qs[e * RP + e] : 0.f;
        live[j] = qii > 0.f;
        iq[j] = live[j] ? 1.f / qii : 0.f;
        hq[j] = 0.5f * qii;
        dd[j] = (e < r && live[j]) ? dv[e] : 1.f;
    }
    const int T = o.cd_steps < 0 ? r : o.cd_steps;
    auto matvec = [&](const float(&v)[J], float(&out)[J]) {
#pragma unroll
        for (int j = 0; j < J; ++j)
            vb[lane * J + j] = v[j];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < J; ++j)
            out[j] = 0.f;
        for (int k = 0; k < r4; ++k) {
            const float vk = vb[k];
#pragma unroll
            for (int j = 0; j < J; ++j)
                out[j] = fmaf(Qs[k * RP + lane * J + j], vk, out[j]);
        }
        __syncwarp();
    };
    auto proj_sq = [&](const float(&y)[J], const float(&g)[J]) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (y[j] > 0.f || g[j] < 0.f)
                s = fmaf(g[j], g[j], s);
        return warp_sum(s);
    };
    unsigned long long my_iters = 0;
    const int64_t rend = row0 + nrows < rows ? row0 + nrows : rows;
    for (int64_t row = row0 + warp; row < rend; row += kWarps) {
        float y[J], g[J];
        bool ok = true;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            int e = lane * J + j;
            float c = 0.f, x0 = 0.f;
            if (e < r) {
                c = Cm[row * r + e];
                x0 = X[row * r + e];
                ok = ok && isfinite(c) && isfinite(x0);
            }
            g[j] = live[j] ? (alpha - c) / dd[j] : 0.f;
            y[j] = live[j] ? x0 * dd[j] : 0.f;
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0)
                atomicOr(status, kStNonFinite);
            continue;
        }
        {
            float t[J];
            matvec(y, t);
#pragma unroll
            for (int j = 0; j < J; ++j)
                g[j] = live[j] ? g[j] + t[j] : 0.f;
        }
        const float s0 = proj_sq(y, g);
        int k = 0;
        if (s0 > 0.f) {
            for (k = 1; k <= o.max_inner; ++k) {
                float gb[J], s = 0.f;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    gb[j] = (y[j] > 0.f || g[j] < 0.f) ? g[j] : 0.f;
                    s = fmaf(gb[j], gb[j], s);
                }
                s = warp_sum(s);
                if (s > 0.f) {
                    float u[J];
                    matvec(gb, u);
                    float den = 0.f;
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        den = fmaf(gb[j], u[j], den);
                    den = warp_sum(den);
                    if (den > 0.f) {
                        const float al = s / den;
                        float dl[J];
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            float yn = fmaxf(0.f, y[j] - al * gb[j]);
                            dl[j] = yn - y[j];
                            y[j] = yn;
                        }
                        matvec(dl, u);
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            g[j] += u[j];
                    }
                }
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
                    const unsigned mx = __reduce_max_sync(0xffffffffu, bkey);
                    if (mx == 0u)
                        break;
                    const int src = __ffs(__ballot_sync(0xffffffffu, bkey == mx)) - 1;
                    const int pj = __shfl_sync(0xffffffffu, bj, src);
                    const float dp = __shfl_sync(0xffffffffu, bdel, src);
                    const int p = src * J + pj;
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        g[j] = fmaf(Qs[p * RP + lane * J + j], dp, g[j]);
                    if (lane == src) {
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            if (j == pj)
                                y[j] += dp;
                    }
                }
                const float sk = proj_sq(y, g);
                if (sk <= o.eps * s0)
                    break;
            }
            if (k > o.max_inner)
                k = o.max_inner;
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            int e = lane * J + j;
            if (e < r)
                X[row * r + e] = live[j] ? y[j] / dd[j] : 0.f;
        }
        if (lane == 0)
            my_iters += (unsigned long long)k;
    }
    if (lane == 0 && my_iters)
        atomicAdd(iter_total, my_iters);
}

// ---- one phase over its items ---------------------------------------------
__device__ void run_phase(const BatchArgs &a, int phase, int64_t item_begin, int64_t item_end,
                          int64_t stride, float *sm)
{
    const BatchInst *I = a.inst;
    const int64_t *off = a.item_off + (int64_t)phase * (a.count + 1);
    const bool w_update = phase < 4;
    for (int64_t item = item_begin; item < item_end; item += stride) {
        const int i = find_inst(off, a.count, item);
        const int64_t local = item - off[i];
        const BatchInst &b = I[i];
        const int r = b.r;
        switch (phase & 3) {
        case 0: {   // Gram partial of the factor held fixed in this half-step
            const float *X = w_update ? b.Ht : b.W;
            const int64_t rows = w_update ? b.n : b.m;
            float *P = b.gram + local * r * r;
            if (r <= 32)
                gram_item<32>(X, rows, r, local * kGramRows, P, sm);
            else
                gram_item<64>(X, rows, r, local * kGramRows, P, sm);
            break;
        }
        case 1: {
            const int64_t rows = w_update ? b.n : b.m;
            const int parts = (int)((rows + kGramRows - 1) / kGramRows);
            rescale_item(b.gram, parts, r, w_update ? b.beta_w : b.beta_h, b.Qt, b.d, sm);
            break;
        }
        case 2: {
            const float *A = w_update ? b.V : b.Vt;
            const int64_t M = w_update ? b.m : b.n, K = w_update ? b.n : b.m;
            const float *Bm = w_update ? b.Ht : b.W;
            float *C = w_update ? b.Cw : b.Ch;
            if (r <= 32)
                cross_item<32>(A, M, K, Bm, r, local * kCrossRows, C, sm);
            else
                cross_item<64>(A, M, K, Bm, r, local * kCrossRows, C, sm);
            break;
        }
        default: {
            const int64_t rows = w_update ? b.m : b.n;
            const float *C = w_update ? b.Cw : b.Ch;
            float *X = w_update ? b.W : b.Ht;
            const float al = w_update ? b.alpha_w : b.alpha_h;
            if (r <= 32)
                nnls_item<1>(b.Qt, b.d, C, rows, r, al, X, local * a.nnls_rows, a.nnls_rows,
                             a.nnls, sm, a.iter_total, a.status);
            else
                nnls_item<2>(b.Qt, b.d, C, rows, r, al, X, local * a.nnls_rows, a.nnls_rows,
                             a.nnls, sm, a.iter_total, a.status);
            break;
        }
        }
    }
}

__global__ void __launch_bounds__(kT) k_batched_iter(const BatchArgs a)
{
    extern __shared__ __align__(16) float smem[];
    if (*(const volatile unsigned *)a.status & kStTimeout)
        return;   // an earlier launch lost its barrier: the barrier state is stale
    for (int phase = a.phase_begin; phase < a.phase_end; ++phase) {
        const int64_t *off = a.item_off + (int64_t)phase * (a.count + 1);
        const int64_t lo = a.inst_begin >= 0 ? off[a.inst_begin] : 0;
        const int64_t hi = a.inst_begin >= 0 ? off[a.inst_begin + 1] : off[a.count];
        run_phase(a, phase, lo + blockIdx.x, hi, gridDim.x, smem);
        if (phase + 1 < a.phase_end) {
            if (!grid_barrier(a.bar_count, a.bar_gen, gridDim.x, a.status))
                return;
        }
    }
}

}  // namespace

size_t batched_smem_bytes()
{
    // max over phases: NNLS Qt (64 x 64) + staging, Gram tile, cross tiles, rescale
    const size_t nn = sizeof(float) * (64 * 64 + kWarps * 64);
    const size_t gr = sizeof(float) * 32 * 64;
    const size_t cr = sizeof(float) * (16 * (kCrossRows + 4) + 16 * 64);
    const size_t rs = sizeof(float) * (64 * 64 + 64);
    size_t m = nn;
    m = gr > m ? gr : m;
    m = cr > m ? cr : m;
    m = rs > m ? rs : m;
    return m;
}

int64_t batched_items(int phase, int64_t m, int64_t n, int nnls_rows)
{
    const bool w = phase < 4;
    switch (phase & 3) {
    case 0: return ((w ? n : m) + kGramRows - 1) / kGramRows;
    case 1: return 1;
    case 2: return ((w ? m : n) + kCrossRows - 1) / kCrossRows;
    default: return ((w ? m : n) + nnls_rows - 1) / nnls_rows;
    }
}

int batched_grid(bool cooperative)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        const size_t smem = batched_smem_bytes();
        cudaFuncSetAttribute(k_batched_iter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_iter, kT, smem) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    (void)cooperative;
    return per_sm * sms;
}

cudaError_t launch_batched(const BatchArgs &a, int grid, bool cooperative, cudaStream_t s)
{
    ProfScope prof_(KC_OTHER, s);
    const size_t smem = batched_smem_bytes();
    if (grid < 1)
        return cudaSuccess;
    cudaError_t e;
    if (cooperative) {
        void *args[] = {const_cast<BatchArgs *>(&a)};
        e = cudaLaunchCooperativeKernel((const void *)k_batched_iter, dim3(grid), dim3(kT), args,
                                        smem, s);
    } else {
        k_batched_iter<<<grid, kT, smem, s>>>(a);
        e = cudaGetLastError();
    }
    count_launch();
    return e;
}

}  // namespace nmfi
