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
// The cross phases run on the tensor cores (3xTF32 tcgen05 MMAs with TMEM
// accumulators, in launches of their own) or, for the FP32_SIMT precision,
// as FFMA on the CUDA cores inside the phase kernel; the other phases are
// FP32 on the CUDA cores.  Instance ranks r <= 64.
#include <algorithm>

#include "k_nnls.cuh"
#include "tc_ptx.cuh"

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

// ---- cross term on the tensor cores ----------------------------------------
// The same rows of C = A B as cross_item, as 3xTF32 tcgen05 MMAs: the tensor
// core reads an FP32 operand as TF32 by dropping its low 13 bits, so the raw
// A and B tiles serve as their own high parts, and the threads write the
// TF32-rounded remainders (A_lo, B_lo) beside them, with a copy of B_hi
// stacked over B_lo; per 8-wide k step one MMA (M 128, N = 2 NP) gives A B_hi
// and A B_lo in two TMEM column regions and a second (N = NP) adds A_lo B_hi
// to the latter.  The tensor core's accumulation rounds
// toward zero, so each 32-wide k block goes to a fresh TMEM buffer and is
// then added into FP32 registers with round-to-nearest adds (two buffers:
// block t accumulates while block t-1 is read).  Rows of A have any pitch,
// so the tiles arrive by 4-byte cp.async (zero-filled outside A and B)
// into a ring of three stages in the K-major 128B-swizzled layout (16-byte
// chunk c of row i at chunk c ^ (i mod 8)); two k blocks are in flight
// while the third is multiplied.
constexpr int kTcStages = 3;
constexpr uint32_t kTcA = 128 * 128;          // A tile: 128 rows x 32 FP32
constexpr uint32_t kTcB = 64 * 128;           // B tile: up to 64 factor columns x 32 FP32
constexpr uint32_t kTcStage = kTcA + kTcB;    // a multiple of 1024 (swizzle atoms)
// ring, then the low parts: A_lo, B_hi stacked over B_lo; + alignment
constexpr size_t kTcSmem = (size_t)kTcStages * kTcStage + kTcA + 2 * kTcB + 1024;
constexpr uint32_t kTcCols = 256;             // TMEM: two buffers of 2 x 64 columns
constexpr uint32_t kTcBufCols = 128;
constexpr unsigned long long kTcWaitNs = 2000000000ull;   // 2 s: an item takes microseconds

// per-CTA tensor-core state of a launch: TMEM base, the MMA-completion
// barriers (one per TMEM buffer) and the parity each thread waits for next
struct TcCtx {
    uint32_t tmem;
    uint64_t *bar;
    uint32_t ph0, ph1;
    volatile int *abort;
};

__device__ __forceinline__ void cp_async4(uint32_t dst, const float *src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}
// 16 bytes (both addresses 16-byte aligned), zero-filled when bytes == 0
__device__ __forceinline__ void cp_async16(uint32_t dst, const float *src, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// offset of element (row i, k) of a K-major 128B-swizzled tile of 32 FP32 per row
__device__ __forceinline__ uint32_t sw128(int i, int k)
{
    return (uint32_t)(i * 128 + ((((k >> 2) ^ (i & 7))) << 4) + (k & 3) * 4);
}

template <int NP>
__device__ bool cross_item_tc(const float *A, int64_t lda, int64_t M, int64_t K, const float *B,
                              int r, int64_t m0, float *C, uint8_t *tsm, TcCtx &tc)
{
    using namespace tcp;
    constexpr int HC = NP / 2;                        // columns per thread per region
    constexpr uint32_t ID = idesc(2u, 128, NP);       // TF32 x TF32 -> F32, M 128, N NP
    constexpr uint32_t ID2 = idesc(2u, 128, 2 * NP);  // the same with N 2 NP
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;      // TMEM lane quadrant, column half
    const int64_t KB = (K + 31) / 32;
    const uint32_t ring = su32(tsm), lo_a = ring + kTcStages * kTcStage, lo_b = lo_a + kTcA;
    const uint64_t dla = sdesc(lo_a), dlb = sdesc(lo_b);   // B_hi rows, then B_lo rows
    const unsigned long long deadline = gtimer() + kTcWaitNs;
    __syncthreads();   // the previous item is done with shared memory

    // Each thread's rows, columns and swizzled chunks are the same in every
    // k block: their offsets are taken once per item.  Rows of A 16-byte
    // aligned (pitch a multiple of 4, A aligned): lane = (row within 4,
    // 16-byte chunk), four 16-byte copies a thread per block; else lane = k,
    // sixteen 4-byte copies (rows warp + 8 q, whose swizzle phase is the
    // warp's).
    const bool vec = (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    const int vrow = (lane >> 3) + 4 * warp, vc = lane & 7;
    const float *pa = vec ? A + (m0 + vrow) * lda + 4 * vc : A + (m0 + warp) * lda + lane;
    const uint32_t da = vec ? (uint32_t)(vrow * 128 + ((vc ^ (vrow & 7)) << 4))
                            : (uint32_t)(warp * 128 + (((lane >> 2) ^ warp) << 4) + (lane & 3) * 4);
    const int64_t left = M - m0;   // rows of this tile inside A
    constexpr int BQ = NP * 32 / kT, BKS = kT / NP;   // B copies a thread, k rows per round
    const int bn = tid % NP, bk = tid / NP;
    const bool bn_in = bn < r;
    const float *pb = B + (int64_t)bk * r + bn;
    auto fetch = [&](int64_t kb, int s) {
        const int64_t k0 = kb * 32;
        const uint32_t a0 = ring + s * kTcStage, b0 = a0 + kTcA;
        if (vec) {
            // a chunk that starts below K is copied whole: K is a multiple of
            // 4, or the rows are a row-padded copy whose pad columns are zero
            const bool kin = k0 + 4 * vc < K;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool in = kin && vrow + 32 * q < left;
                cp_async16(a0 + da + q * 4096, in ? pa + (32 * q) * lda + k0 : A, in ? 16u : 0u);
            }
        } else {
            const bool kin = k0 + lane < K;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const bool in = kin && warp + 8 * q < left;
                cp_async4(a0 + da + q * 1024, in ? pa + (8 * q) * lda + k0 : A, in ? 4u : 0u);
            }
        }
#pragma unroll
        for (int q = 0; q < BQ; ++q) {
            const int k = bk + BKS * q;
            const bool in = bn_in && k0 + k < K;
            cp_async4(b0 + sw128(bn, k), in ? pb + (k0 + BKS * q) * r : B, in ? 4u : 0u);
        }
    };
    auto wait_mma = [&](int b) -> bool {
        uint32_t &ph = b ? tc.ph1 : tc.ph0;
        const bool ok = mbar_wait(tc.bar + b, ph, deadline, tc.abort);
        ph ^= 1u;
        return ok;
    };
    float acc[HC];
#pragma unroll
    for (int j = 0; j < HC; ++j)
        acc[j] = 0.f;
    auto ld_add = [&](uint32_t addr) {
        if constexpr (HC == 32) {
            uint32_t v[32];
            tmem_ld32_nowait(addr, v);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j)
                acc[j] += __uint_as_float(v[j]);
        } else if constexpr (HC == 16) {
            uint32_t v[16];
            tmem_ld16(addr, v);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                acc[j] += __uint_as_float(v[j]);
        } else {
            uint32_t v[8];
            tmem_ld8(addr, v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                acc[j] += __uint_as_float(v[j]);
        }
    };
    auto drain = [&](int b) {
        tc_fence_after();
        const uint32_t base = tc.tmem + b * kTcBufCols + ((uint32_t)(quad * 32) << 16) + half * HC;
        ld_add(base);        // A B_hi
        ld_add(base + NP);   // A B_lo + A_lo B_hi
        tc_fence_before();
    };

    bool ok = true;
    if (KB > 0)
        fetch(0, 0);
    cp_async_commit();
    if (KB > 1)
        fetch(1, 1);
    cp_async_commit();
    for (int64_t t = 0; t < KB; ++t) {
        const int s = (int)(t % kTcStages);
        cp_async_wait<1>();   // this thread's copies of block t have landed
        // MMA t-1 has completed: the low-part buffers and the stage of block
        // t + 2 (last read by MMA t-1) are free, and its TMEM buffer is ready
        if (t > 0 && !__syncthreads_and(wait_mma((int)((t - 1) & 1)))) {
            ok = false;
            break;
        }
        if (t == 0)
            __syncthreads();   // every thread's copies of block t are in place
        {
            const float4 *ha = reinterpret_cast<const float4 *>(tsm + s * kTcStage);
            float4 *la = reinterpret_cast<float4 *>(tsm + kTcStages * kTcStage);
            auto rem = [](float x) {
                return rn_tf32_operand(x - __uint_as_float(__float_as_uint(x) & 0xffffe000u));
            };
#pragma unroll
            for (int q = 0; q < (int)(kTcA / 16 / kT); ++q) {
                const float4 v = ha[tid + kT * q];
                la[tid + kT * q] = make_float4(rem(v.x), rem(v.y), rem(v.z), rem(v.w));
            }
            const float4 *hb = ha + kTcA / 16;
            float4 *lb = la + kTcA / 16;   // NP rows of B_hi, then NP rows of B_lo
            for (int e = tid; e < NP * 8; e += kT) {
                const float4 v = hb[e];
                lb[e] = v;
                lb[NP * 8 + e] = make_float4(rem(v.x), rem(v.y), rem(v.z), rem(v.w));
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t d = tc.tmem + (uint32_t)(t & 1) * kTcBufCols;
            // the tiles are 1024-byte aligned, so the descriptor of the k
            // step 32 kk bytes into a row is the tile's plus 2 kk (16-byte units)
            const uint64_t da0 = sdesc(ring + s * kTcStage), db0 = sdesc(ring + s * kTcStage + kTcA);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc_on = kk > 0 ? 1u : 0u;
                mma<TC_TF32>(d, da0 + 2 * kk, dlb + 2 * kk, ID2, acc_on);
                mma<TC_TF32>(d + NP, dla + 2 * kk, db0 + 2 * kk, ID, 1u);
            }
            mma_commit(tc.bar + (t & 1));
        }
        if (t + 2 < KB)
            fetch(t + 2, (int)((t + 2) % kTcStages));
        cp_async_commit();
        if (t > 0)
            drain((int)((t - 1) & 1));
    }
    cp_async_wait<0>();
    if (ok && KB > 0) {
        if (!__syncthreads_and(wait_mma((int)((KB - 1) & 1))))
            ok = false;
        else
            drain((int)((KB - 1) & 1));
    }
    if (!ok)
        return false;
    const int64_t gm = m0 + quad * 32 + lane;
    if (gm < M) {
#pragma unroll
        for (int j = 0; j < HC; ++j) {
            const int n = half * HC + j;
            if (n < r)
                C[gm * r + n] = acc[j];
        }
    }
    return true;
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

// One cross phase (2 or 6) on the tensor cores, in a launch of its own: the
// streaming tiles want ~97 KB of shared memory a CTA, which in the
// all-phase kernel would leave the NQP phases a small L1.  Items as in
// run_phase: from the phase's counter, or a fixed stride without one.
__global__ void __launch_bounds__(kT, 2) k_batched_cross(const BatchArgs a)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t tc_bar[2];
    __shared__ int tc_abort;
    __shared__ unsigned long long taken;
    if (*(const volatile unsigned *)a.status & kStTimeout)
        return;
    // 256 TMEM columns a CTA; at most two CTAs fit on an SM (shared memory),
    // so the allocation of the SM's 512 columns never has to wait
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tcp::su32(&tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        tcp::mbar_init(&tc_bar[0], 1);
        tcp::mbar_init(&tc_bar[1], 1);
        tc_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tcp::tc_fence_before();
    __syncthreads();
    tcp::tc_fence_after();
    TcCtx tc{tmem_slot, tc_bar, 0u, 0u, &tc_abort};
    // the tiles start at a 1024-byte boundary (the swizzle atom)
    uint8_t *tsm = reinterpret_cast<uint8_t *>(smem) + ((1024u - (tcp::su32(smem) & 1023u)) & 1023u);

    const int phase = a.phase_begin;
    const bool w_update = phase < 4;
    const int64_t *off = a.item_off + (int64_t)phase * (a.count + 1);
    const int64_t lo = a.inst_begin >= 0 ? off[a.inst_begin] : 0;
    const int64_t hi = a.inst_begin >= 0 ? off[a.inst_begin + 1] : off[a.count];
    if (a.work && blockIdx.x == 0 && threadIdx.x == 0)
        a.work[(phase + 7) & 7] = 0ull;
    int64_t item = lo + (a.work ? 0 : blockIdx.x);
    for (;;) {
        if (a.work) {
            if (threadIdx.x == 0)
                taken = atomicAdd(a.work + phase, 1ull);
            __syncthreads();
            item = lo + (int64_t)taken;
            __syncthreads();
        }
        if (item >= hi)
            break;
        const int i = find_inst(off, a.count, item);
        const BatchInst &b = a.inst[i];
        const float *A = w_update ? b.Vx : b.Vtx;
        const int64_t lda = w_update ? b.ldvx : b.ldvtx;
        const int64_t M = w_update ? b.m : b.n, K = w_update ? b.n : b.m;
        const float *Bm = w_update ? b.Ht : b.W;
        float *C = w_update ? b.Cw : b.Ch;
        const int64_t m0 = (item - off[i]) * kCrossRows;
        bool ok;
        if (b.r <= 16)
            ok = cross_item_tc<16>(A, lda, M, K, Bm, b.r, m0, C, tsm, tc);
        else if (b.r <= 32)
            ok = cross_item_tc<32>(A, lda, M, K, Bm, b.r, m0, C, tsm, tc);
        else
            ok = cross_item_tc<64>(A, lda, M, K, Bm, b.r, m0, C, tsm, tc);
        if (!ok) {   // a bounded wait ran out
            if (threadIdx.x == 0)
                atomicOr(a.status, kStTimeout);
            break;
        }
        if (!a.work)
            item += gridDim.x;
    }
    // every MMA this CTA issued has been waited for (or its wait ran out)
    tcp::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tcp::tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem),
                     "r"(kTcCols)
                     : "memory");
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

// CTAs of the tensor-core cross kernel an SM holds (0 on error)
static int cross_per_sm()
{
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaFuncSetAttribute(k_batched_cross, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTcSmem);
        // the whole unified memory as shared memory: two CTAs per SM
        cudaFuncSetAttribute(k_batched_cross, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_cross, kT,
                                                          kTcSmem) != cudaSuccess)
            per_sm = 0;
    }
    return per_sm;
}

bool batched_tc_fits()
{
    // every CTA an SM can hold gets its tensor-memory columns at once: the
    // shared memory of a CTA leaves room for at most two on an SM
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    return cross_per_sm() >= 1 && (size_t)smem_sm < 3 * kTcSmem &&
           2 * (int)kTcCols <= 512;
}

cudaError_t launch_batched(const BatchArgs &a, int grid, bool cooperative, cudaStream_t s)
{
    // a launch of a single phase is attributed to that phase's kernel class
    static const KClass kPhaseClass[4] = {KC_GRAM, KC_RESCALE, KC_CROSS, KC_NNLS};
    ProfScope prof_(a.phase_end == a.phase_begin + 1 ? kPhaseClass[a.phase_begin & 3] : KC_OTHER, s);
    if (grid < 1)
        return cudaSuccess;
    if (a.tc && !batched_tc_fits())
        return cudaErrorInvalidConfiguration;
    const size_t smem = batched_smem_bytes();
    // the phase range in runs: tensor-core cross phases in launches of their
    // own, the phases between them in one (cooperative) launch each
    for (int p0 = a.phase_begin; p0 < a.phase_end;) {
        BatchArgs b = a;
        cudaError_t e;
        if (a.tc && (p0 & 3) == 2) {
            b.phase_begin = p0;
            b.phase_end = p0 + 1;
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            // over all instances: two CTAs per SM (the shared memory of a CTA
            // leaves room for no third), items from the counter; one
            // instance: one CTA per item (the given grid)
            const int g = a.work ? 2 * sms : grid;
            k_batched_cross<<<g, kT, kTcSmem, s>>>(b);
            e = cudaGetLastError();
            ++p0;
        } else {
            int p1 = p0 + 1;
            while (p1 < a.phase_end && !(a.tc && (p1 & 3) == 2))
                ++p1;
            b.phase_begin = p0;
            b.phase_end = p1;
            if (cooperative) {
                void *args[] = {&b};
                e = cudaLaunchCooperativeKernel((const void *)k_batched_iter, dim3(grid), dim3(kT),
                                                args, smem, s);
            } else {
                k_batched_iter<<<grid, kT, smem, s>>>(b);
                e = cudaGetLastError();
            }
            p0 = p1;
        }
        count_launch();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace nmfi
