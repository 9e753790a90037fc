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
// row tiles, instances); a CTA maps an item to its instance by binary search
// over per-phase prefix sums.  Item costs differ by two orders of magnitude
// (K from 100 to 4000, r from 8 to 64), so CTAs take the next item from a
// per-phase counter as they finish one, and the instances are ordered by
// decreasing cost: the large items start first.  An item's result does not
// depend on the CTA that computes it.
//
// Persistent mode: one cooperative launch runs all eight phases with grid
// barriers in between (every CTA is resident: the grid is the occupancy
// limit).  Loop mode: the same phase code launched once per instance and
// phase, the baseline whose launch count the persistent form removes.
// Arithmetic is FP32 on CUDA cores; instance ranks r <= 64.
#include <algorithm>

#include "k_nnls.cuh"

namespace nmfi {
namespace {

constexpr int kT = 256;            // threads per CTA
constexpr int kWarps = kT / 32;
constexpr int kGramRows = 256;     // rows of X per Gram item
constexpr int kCrossRows = 128;    // rows of A per cross item
constexpr unsigned long long kBarrierNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded sense-reversing grid barrier; false on timeout (a CTA that has to
// wait gives up after `limit_ns` of global time)
__device__ bool grid_barrier(unsigned *count, volatile unsigned *gen, unsigned nblocks,
                             unsigned *status, unsigned long long limit_ns)
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
            const unsigned long long dl = gtime() + limit_ns;
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

// cross term rows [m0, m0 + kCrossRows) of C = A B (A M x K row-major, B K x r,
// r <= NB).  Thread (ty, tx) owns rows ty*TM .. ty*TM+TM-1 and columns
// tx*4 .. tx*4+3.  The A tile sits in shared memory transposed (k-major), so
// a thread's TM rows at one k are contiguous: per k one vector load of A, one
// 128-bit load of B and 4 TM FMAs (the row-major tile took TM scalar loads).
// Each output adds its k terms in increasing k, one FMA each.  The next
// 32-wide k tile is loaded into registers while this one is used.
template <int NB>
__device__ void cross_item(const float *A, int64_t M, int64_t K, const float *B, int r,
                           int64_t m0, float *C, float *sm)
{
    constexpr int BM = kCrossRows, BK = 32, TX = NB / 4, TY = kT / TX, TM = BM / TY;
    constexpr int LDT = BM + 4;             // floats per k row of the transposed A tile
    constexpr int AL = BM * BK / kT, BL = (BK * NB + kT - 1) / kT;   // loads per thread
    static_assert(BK * LDT <= BM * (BK + 1) && TM <= 8 && (TM & (TM - 1)) == 0,
                  "tile layout of the cross phase");
    float *As = sm;                         // BK x LDT (A^T of the tile)
    float *Bs = sm + BK * LDT;              // BK x NB (16-byte aligned: BK * LDT % 4 == 0)
    const int tid = threadIdx.x, ty = tid / TX, tx = tid - ty * TX;
    float acc[TM][4];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            acc[i][j] = 0.f;
    float ra[AL], rb[BL];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int idx = tid + kT * q, mm = idx / BK, kk = idx - mm * BK;
            const int64_t gm = m0 + mm, gk = k0 + kk;
            ra[q] = (gm < M && gk < K) ? A[gm * K + gk] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int idx = tid + kT * q, kk = idx / NB, nn = idx - kk * NB;
            const int64_t gk = k0 + kk;
            rb[q] = (idx < BK * NB && nn < r && gk < K) ? B[gk * r + nn] : 0.f;
        }
    };
    fetch(0);
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();   // the previous tile (or item) is no longer read
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int idx = tid + kT * q, mm = idx / BK, kk = idx - mm * BK;
            As[kk * LDT + mm] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int idx = tid + kT * q;
            if (idx < BK * NB)
                Bs[idx] = rb[q];
        }
        __syncthreads();
        if (k0 + BK < K)
            fetch(k0 + BK);
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            const float4 b = *reinterpret_cast<const float4 *>(Bs + kk * NB + tx * 4);
            const float *ap = As + kk * LDT + ty * TM;
            float a[TM];
            if constexpr (TM >= 4) {
#pragma unroll
                for (int i = 0; i < TM; i += 4) {
                    const float4 t = *reinterpret_cast<const float4 *>(ap + i);
                    a[i] = t.x; a[i + 1] = t.y; a[i + 2] = t.z; a[i + 3] = t.w;
                }
            } else if constexpr (TM == 2) {
                const float2 t = *reinterpret_cast<const float2 *>(ap);
                a[0] = t.x; a[1] = t.y;
            } else {
                a[0] = ap[0];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
                acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
                acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
                acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + ty * TM + i;
        if (gm >= M)
            continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = tx * 4 + j;
            if (n < r)
                C[gm * r + n] = acc[i][j];
        }
    }
}

// lanes per row of the grouped NQP solver for rank r <= 64 (J = 8 coordinates
// per lane), and the rows of one NQP work item: `mult` rows per group of
// every warp
__host__ __device__ inline int nnls_lanes(int r) { return r <= 8 ? 1 : r <= 16 ? 2 : r <= 32 ? 4 : 8; }
__host__ __device__ inline int64_t nnls_item_rows(int r, int mult)
{
    return (int64_t)mult * kWarps * (32 / nnls_lanes(r));
}

// Alg. 3 for the rows of one work item (the grouped solver of k_nnls.cuh)
template <int G>
__device__ void nnls_item(const BatchInst &b, bool w_update, int64_t row0, int64_t nrows,
                          const BatchArgs &a, float *sm)
{
    constexpr int RP = nnls_detail::Map<G, 8>::RP;
    float *Qs = sm, *sd = sm + RP * RP;
    const int r = b.r;
    __syncthreads();   // the previous item's warps are done with the shared Qt
    if (!nnls_detail::stage_qt<G, 8>(b.Qt, b.d, r, Qs, sd, a.status))
        return;
    NnlsArgs na{};
    na.Qt = b.Qt;
    na.d = b.d;
    na.C = w_update ? b.Cw : b.Ch;
    na.nsplit = 1;
    na.rows = w_update ? b.m : b.n;
    na.c_stride = na.rows * r;
    na.r = r;
    na.alpha = w_update ? b.alpha_w : b.alpha_h;
    na.X = w_update ? b.W : b.Ht;
    na.max_inner = a.nnls.max_inner;
    na.eps = a.nnls.eps;
    na.cd_steps = a.nnls.cd_steps;
    na.iter_total = a.iter_total;
    na.status = a.status;
    const int64_t end = row0 + nrows < na.rows ? row0 + nrows : na.rows;
    nnls_detail::flush_warp_counters(
        na, nnls_detail::nnls_rows<G, 8>(na, Qs, sd, sd + RP, row0 + (threadIdx.x >> 5), kWarps,
                                         end));
}

// ---- one phase over its items ---------------------------------------------
__device__ void run_phase(const BatchArgs &a, int phase, int64_t item_begin, int64_t item_end,
                          int64_t stride, float *sm)
{
    const BatchInst *I = a.inst;
    const int64_t *off = a.item_off + (int64_t)phase * (a.count + 1);
    const bool w_update = phase < 4;
    __shared__ unsigned long long taken;
    int64_t item = item_begin;
    for (;;) {
        if (a.work) {
            if (threadIdx.x == 0)
                taken = atomicAdd(a.work + phase, 1ull);
            __syncthreads();
            item = item_begin + (int64_t)taken;
            __syncthreads();   // every thread has read it before it is replaced
        }
        if (item >= item_end)
            break;
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
            if (r <= 8)
                cross_item<8>(A, M, K, Bm, r, local * kCrossRows, C, sm);
            else if (r <= 16)
                cross_item<16>(A, M, K, Bm, r, local * kCrossRows, C, sm);
            else if (r <= 32)
                cross_item<32>(A, M, K, Bm, r, local * kCrossRows, C, sm);
            else
                cross_item<64>(A, M, K, Bm, r, local * kCrossRows, C, sm);
            break;
        }
        default: {
            const int64_t nr = nnls_item_rows(r, a.nnls_rows);
            switch (nnls_lanes(r)) {
            case 1: nnls_item<1>(b, w_update, local * nr, nr, a, sm); break;
            case 2: nnls_item<2>(b, w_update, local * nr, nr, a, sm); break;
            case 4: nnls_item<4>(b, w_update, local * nr, nr, a, sm); break;
            default: nnls_item<8>(b, w_update, local * nr, nr, a, sm); break;
            }
            break;
        }
        }
        if (!a.work)
            item += stride;
    }
}

__global__ void __launch_bounds__(kT, 2) k_batched_iter(const BatchArgs a)
{
    extern __shared__ __align__(16) float smem[];
    if (*(const volatile unsigned *)a.status & kStTimeout)
        return;   // an earlier launch lost its barrier: the barrier state is stale
    for (int phase = a.phase_begin; phase < a.phase_end; ++phase) {
        const int64_t *off = a.item_off + (int64_t)phase * (a.count + 1);
        const int64_t lo = a.inst_begin >= 0 ? off[a.inst_begin] : 0;
        const int64_t hi = a.inst_begin >= 0 ? off[a.inst_begin + 1] : off[a.count];
        // the previous phase's counter is free (its phase ended behind a
        // grid barrier or a kernel boundary): zero it for its next use
        if (a.work && blockIdx.x == 0 && threadIdx.x == 0)
            a.work[(phase + 7) & 7] = 0ull;
        run_phase(a, phase, a.work ? lo : lo + blockIdx.x, hi, gridDim.x, smem);
        if (phase + 1 < a.phase_end) {
            if (!grid_barrier(a.bar_count, a.bar_gen, gridDim.x, a.status, a.barrier_ns))
                return;
        }
    }
}

}  // namespace

size_t batched_smem_bytes()
{
    // max over phases: grouped NQP solver (Qt, d, per-group buffers), Gram
    // tile, cross tiles, rescale
    auto nq = [](int rp, size_t pool) { return sizeof(float) * ((size_t)rp * rp + rp + pool); };
    size_t m = nq(8, nnls_detail::pool_floats<1, 8>());
    m = std::max(m, nq(16, nnls_detail::pool_floats<2, 8>()));
    m = std::max(m, nq(32, nnls_detail::pool_floats<4, 8>()));
    m = std::max(m, nq(64, nnls_detail::pool_floats<8, 8>()));
    m = std::max(m, sizeof(float) * 32 * 64);
    m = std::max(m, sizeof(float) * (kCrossRows * 33 + 32 * 64));
    m = std::max(m, sizeof(float) * (64 * 64 + 64));
    return m;
}

int64_t batched_items(int phase, int64_t m, int64_t n, int r, int nnls_mult)
{
    const bool w = phase < 4;
    switch (phase & 3) {
    case 0: return ((w ? n : m) + kGramRows - 1) / kGramRows;
    case 1: return 1;
    case 2: return ((w ? m : n) + kCrossRows - 1) / kCrossRows;
    default: {
        const int64_t nr = nnls_item_rows(r, nnls_mult);
        return ((w ? m : n) + nr - 1) / nr;
    }
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
    // a launch of a single phase is attributed to that phase's kernel class
    static const KClass kPhaseClass[4] = {KC_GRAM, KC_RESCALE, KC_CROSS, KC_NNLS};
    ProfScope prof_(a.phase_end == a.phase_begin + 1 ? kPhaseClass[a.phase_begin & 3] : KC_OTHER, s);
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
