// Tensor-core cross term C = A B on tcgen05 (sm_103a): A is the data matrix
// (V for the W-update, V^T for the H-update; M x K, K contiguous) and B the
// other factor (K x r).  Alg. 2 "Y = F V^T", the dominant O(mnr) term of
// §4.2.  At r <= 128 the product is bound by the bytes of A, so the design
// goal is to stream A from HBM once at full bandwidth:
//
//  * Work split (stream-K).  The (row tile, 32-wide k block) iterations are
//    cut into equal contiguous ranges, one per CTA, one CTA per SM.  Every SM
//    streams the same number of bytes whatever M and K are.  A CTA writes the
//    accumulator of each row tile it touches into partial slice
//    (CTA - first CTA of that tile); the consumer sums the slices in order.
//  * Pipeline.  Warp 0 (one thread) issues TMA loads of the A tile (128 rows x
//    128 B, 128B swizzle) and the B tile (packed factor, N x 128 B) into a
//    ring of stages tracked by mbarriers.  Warp 1 (one thread) issues
//    tcgen05.mma into a TMEM accumulator (128 lanes x N columns, FP32) and
//    commits each stage back to the producer.  The accumulator is double
//    buffered in TMEM: every chunk of k blocks goes to one buffer while the
//    accumulating warps read the other through tcgen05.ld and add it into
//    FP32 registers (round to nearest), so the tensor core's truncating
//    accumulation never runs over more than one chunk.
//  * Arithmetic.  TF32: one MMA per k step.  TF32X3 (FP32-accurate): the
//    tensor core's TF32 conversion truncates, so the A tile serves as its own
//    high part and warps 2-5 write the TF32-rounded remainder A - trunc(A)
//    to a small ring while warps 6-9 accumulate (the two jobs overlap instead
//    of taking turns); the packed factor stacks its TF32 high part over its
//    TF32 remainder, so one N = 2 NPAD MMA gives A*B_hi and A*B_lo side by
//    side in TMEM and a second (N = NPAD) adds A_lo*B_hi.  BF16: A and B in
//    BF16, kind::f16.  BF16X2: A in BF16, the factor split into a BF16 high
//    part and the BF16 rounding of its remainder, stacked as for TF32X3, so
//    one N = 2 NPAD MMA per k step gives A*B_hi and A*B_lo side by side: the
//    factor enters with ~2^-17 relative error, A with its one BF16 rounding.
//  * Every wait is bounded by a global-timer deadline; on expiry the CTA
//    raises the timeout bit of the status word, drains, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "nmf_internal.cuh"
#include "tc_ptx.cuh"

namespace nmfi {
namespace {

constexpr int kThreads = 384;     // producer, up to 3 MMA issuers, 8 split/accumulate warps
constexpr int kIssuer0 = 1, kIssuer1 = 10, kIssuer2 = 11;   // warps that issue tcgen05.mma
constexpr int kEpi = 256;         // threads of warps 2..9
constexpr int kSplit = 128;       // TF32X3: warps 2..5 split, warps 6..9 accumulate
constexpr uint32_t kABytes = 128 * 128;   // 128 rows x 128 bytes
constexpr unsigned long long kDeadlineNs = 2000000000ull;   // 2 s, a kernel takes < 1 ms
constexpr int kBarBytes = 1024;   // mbarriers, the TMEM address and the abort flag

using namespace tcp;

// CTA that owns iteration x when `iters` iterations are cut into `grid`
// contiguous ranges [floor(c iters/grid), floor((c+1) iters/grid)).
__host__ __device__ inline int owner_of(int64_t x, int64_t iters, int grid)
{
    int64_t c = x * grid / iters;
    while (c + 1 < grid && (c + 1) * iters / grid <= x)
        ++c;
    while (c > 0 && c * iters / grid > x)
        --c;
    return (int)c;
}

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// one k block's position in every ring of the cross kernel: data stage and
// parity, full barrier and parity, low-part slot and parity, low-part full
// barrier and parity, place in the issue window and the window's issuer
struct Ring {
    int stage = 0;
    uint32_t phase = 0;
    int fb = 0;
    uint32_t fph = 0;
    int lo = 0;
    uint32_t lph = 0;
    int lf = 0;
    uint32_t lfph = 0;
    int dc = 0;
    int own = 0;
};

template <int MODE, int NPAD, int STAGES, int NLO, int DRAIN>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_cross(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const TcArgs p)
{
    constexpr bool X3 = MODE == TC_TF32X3;
    constexpr bool BF = MODE == TC_BF16 || MODE == TC_BF16X2;   // A and B in BF16
    constexpr bool PAIR = X3 || MODE == TC_BF16X2;             // B = [B_hi; B_lo]
    // TF32X3 with NPAD <= 64: warps 2-5 split while warps 6-9 accumulate.
    // Wider factors keep all eight warps on both jobs (an accumulating thread
    // could not hold 2 x 128 columns).
    constexpr bool SR = X3 && NPAD <= 64;
    constexpr bool BULK = NPAD <= 64;   // partial tiles leave by bulk copy (see the epilogue)
    constexpr int SPLIT_T = SR ? kSplit : kEpi;   // threads that split
    constexpr int NB = PAIR ? 2 * NPAD : NPAD;                // rows of the packed factor tile
    constexpr uint32_t B_BYTES = NB * 128;
    constexpr uint32_t STAGE_BYTES = kABytes + B_BYTES;
    constexpr uint32_t TX_BYTES = kABytes + B_BYTES;
    constexpr int KSTEP_ELEMS = BF ? 64 : 32;                 // elements per 128-byte row
    constexpr int KMMA = 4;                                   // MMAs of 32 bytes per stage
    constexpr uint32_t BUF_COLS = NB <= 32 ? 32 : (NB <= 64 ? 64 : (NB <= 128 ? 128 : 256));
    // MMA issuers and accumulator buffers: each issuer owns every NISS-th
    // buffer, so the accumulating warps may lag the tensor core by several
    // chunks; three issuers where three buffers fit in TMEM's 512 columns
    constexpr int NISS = 512 / BUF_COLS >= 3 ? 3 : 2;
    constexpr int NACC = NISS == 3 ? 3 : 2;
    // SR: the low parts live in tensor memory (32 columns per k block, one
    // lane per row), read by the A_lo MMAs from there: no shared-memory
    // round trip for them
    constexpr uint32_t LO_COL0 = NACC * BUF_COLS;
    constexpr uint32_t TMEM_USED = NACC * BUF_COLS + (SR ? NLO * 32 : 0);
    static_assert(TMEM_USED <= 512, "tensor memory columns");
    constexpr uint32_t TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 :
                                   TMEM_USED <= 128 ? 128 : TMEM_USED <= 256 ? 256 : 512;
    constexpr uint32_t ID_B = idesc(BF ? 1u : 2u, 128, NB);                  // A x packed tile
    constexpr uint32_t ID_HI = idesc(2u, 128, NPAD);                         // A_lo x B_hi
    // Issuer q owns the k blocks of every NISS-th window of DRAIN consecutive
    // blocks of this CTA (windows are cut at row-tile boundaries into
    // chunks).  An mbarrier wait only tells two consecutive phases apart, so
    // every phase of a barrier must be waited by a thread that waited the one
    // before: the full barriers (NF of them) and the low-part full barriers
    // (NLF) are indexed so that each is only ever waited by one issuer (and
    // by the split warps, which wait every k block in order).
    constexpr int NF = lcm_c(STAGES, DRAIN * NISS);
    constexpr int NLF = NLO > 0 ? lcm_c(NLO, NISS) : 1;
    static_assert(!X3 || DRAIN == 1, "the low-part ring assumes one k block per chunk");
    static_assert((NF + STAGES + NLF + (NLO > 0 ? NLO : 1) + 2 * NACC + 3) * 8 + 8 <= kBarBytes,
                  "barrier area");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    auto A = [&](int s) { return smem + s * STAGE_BYTES; };
    auto B = [&](int s) { return smem + s * STAGE_BYTES + kABytes; };
    // the shared-memory low-part ring (NPAD 128 only; SR keeps it in TMEM)
    constexpr int NLO_SM = SR ? 0 : NLO;
    auto LO = [&](int j) { return smem + STAGES * STAGE_BYTES + j * kABytes; };
    // epilogue staging: 32 (BULK) or 8 rows x NPAD floats per TMEM lane quadrant
    constexpr int STG_ROWS = BULK ? 32 : 8;
    float *stg_all = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES + NLO_SM * kABytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg_all + 4 * STG_ROWS * NPAD);
    uint64_t *full = bars, *empty = bars + NF;
    uint64_t *lo_full = empty + STAGES, *lo_empty = lo_full + NLF;
    uint64_t *acc_full = lo_empty + (NLO > 0 ? NLO : 1), *acc_empty = acc_full + NACC;
    uint64_t *fin = acc_empty + NACC;   // every MMA of issuer q has completed: fin[q]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t it0 = (int64_t)blockIdx.x * p.iters / p.grid;
    const int64_t it1 = (int64_t)(blockIdx.x + 1) * p.iters / p.grid;
    const int KB = p.kblocks;
    // (row tile, k block) of it0; every role then steps both counters (a
    // 64-bit division per iteration would sit on the single-thread paths)
    const int tile0 = (int)(it0 / KB), kb0 = (int)(it0 - (int64_t)tile0 * KB);
    const unsigned long long deadline = gtimer() + kDeadlineNs;
    // every role walks every k block of the CTA through all rings in step
    auto adv = [](Ring &w) {
        if (++w.stage == STAGES) {
            w.stage = 0;
            w.phase ^= 1u;
        }
        if (++w.fb == NF) {
            w.fb = 0;
            w.fph ^= 1u;
        }
        if constexpr (NLO > 0) {
            if (++w.lo == NLO) {
                w.lo = 0;
                w.lph ^= 1u;
            }
            if (++w.lf == NLF) {
                w.lf = 0;
                w.lfph ^= 1u;
            }
        }
        if (++w.dc == DRAIN) {
            w.dc = 0;
            if (++w.own == NISS)
                w.own = 0;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NF; ++s)
            mbar_init(&full[s], 1);
        for (int s = 0; s < STAGES; ++s)
            mbar_init(&empty[s], 1);
        for (int j = 0; j < NLF; ++j)
            mbar_init(&lo_full[j], SPLIT_T);
        for (int j = 0; j < NLO; ++j)
            mbar_init(&lo_empty[j], 1);
        for (int q = 0; q < 3; ++q)
            mbar_init(&fin[q], 1);
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], SR ? kEpi - kSplit : kEpi);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    pdl_trigger();
    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            // A (the data matrix) is written by no earlier kernel: the first
            // stages' A tiles are requested before waiting for the previous
            // kernel, whose output the packed factor B is
            const int64_t pre = it1 - it0 < STAGES ? it1 - it0 : STAGES;
            {
                int tile = tile0, kb = kb0 - 1;
                for (int64_t i = 0; i < pre; ++i) {
                    if (++kb == KB) {
                        kb = 0;
                        ++tile;
                    }
                    mbar_expect_tx(&full[i], TX_BYTES);
                    tma_load_2d(A(i), &tmA, &full[i], kb * KSTEP_ELEMS, tile * 128);
                }
            }
            pdl_wait();
            Ring w{};
            int tile = tile0, kb = kb0 - 1;
            int64_t n = 0;   // positions whose loads were issued
            for (int64_t it = it0; it < it1; ++it, adv(w)) {
                if (++kb == KB) {
                    kb = 0;
                    ++tile;
                }
                if (it - it0 >= pre) {
                    if (!mbar_wait(&empty[w.stage], w.phase ^ 1u, deadline, abort_flag))
                        break;
                    mbar_expect_tx(&full[w.fb], TX_BYTES);
                    tma_load_2d(A(w.stage), &tmA, &full[w.fb], kb * KSTEP_ELEMS, tile * 128);
                }
                tma_load_2d(B(w.stage), &tmB, &full[w.fb], kb * KSTEP_ELEMS, 0);
                n = it - it0 + 1;
            }
            // drain: every load issued must land before the CTA exits; the
            // last use of the slot at position n + s was position n + s - STAGES
            for (int s = 0; s < STAGES; ++s, adv(w)) {
                const int64_t last = n + s - STAGES;
                if (!mbar_wait(&empty[w.stage], w.phase ^ 1u, deadline + kDeadlineNs, abort_flag) &&
                    last >= 0) {
                    // the consumer stopped; wait for the load itself instead
                    mbar_wait_drain(&full[last % NF], (uint32_t)((last / NF) & 1),
                                    deadline + 2 * kDeadlineNs);
                }
            }
        }
    } else if (warp == kIssuer0 || warp == kIssuer1 || warp == kIssuer2) {
        // ---------------- MMA issuers: issuer q takes the k blocks of the
        // windows w with w % NISS == q and accumulates them in buffer q, which
        // only it touches, so one thread's barrier waits and commits overlap
        // the others' MMAs; stage and low-part reuse stay ordered through the
        // producer and split barriers, and tcgen05.commit tracks the MMAs of
        // the thread that issues it.
        const int q = warp == kIssuer0 ? 0 : (warp == kIssuer1 ? 1 : 2);
        if (lane == 0 && q < NISS) {
            Ring w{};
            uint32_t uses = 0;
            const uint32_t d = tmem + q * BUF_COLS;
            int kb = kb0 - 1;
            for (int64_t it = it0; it < it1; ++it, adv(w)) {
                if (++kb == KB)
                    kb = 0;
                if (w.own != q)
                    continue;
                const bool seg_start = it == it0 || kb == 0;
                const bool seg_end = it + 1 == it1 || kb == KB - 1;
                const bool chunk_start = seg_start || w.dc == 0;
                const bool chunk_end = seg_end || w.dc == DRAIN - 1;
                if (chunk_start) {
                    // the accumulating warps have drained the previous use of this buffer
                    const uint32_t u = uses++;
                    if (!mbar_wait(&acc_empty[q], (u & 1u) ^ 1u, deadline, abort_flag))
                        break;
                    tc_fence_after();
                }
                if (!mbar_wait(&full[w.fb], w.fph, deadline, abort_flag))
                    break;
                tc_fence_after();
                const uint32_t a0 = su32(A(w.stage)), b0 = su32(B(w.stage));
                // X3: columns [0, NPAD) get A B_hi, columns [NPAD, 2 NPAD) get
                // A B_lo and (below) A_lo B_hi, both about 2^-11 of A B_hi.  The
                // tensor core's accumulation truncates, and every MMA added to
                // the large columns costs them up to an ulp: keeping the small
                // terms in their own columns leaves four such adds per chunk
                // instead of eight (relative bias 6e-7 -> 1e-7).  These first
                // MMAs need no low part, so they run while the split finishes.
#pragma unroll
                for (int kk = 0; kk < KMMA; ++kk)
                    mma<MODE>(d, sdesc(a0 + 32 * kk), sdesc(b0 + 32 * kk), ID_B,
                              (chunk_start && kk == 0) ? 0u : 1u);
                if constexpr (X3) {
                    if (!mbar_wait(&lo_full[w.lf], w.lfph, deadline, abort_flag))
                        break;   // the final commit below waits for the MMAs issued
                    tc_fence_after();
                    if constexpr (SR) {
                        const uint32_t l0 = tmem + LO_COL0 + w.lo * 32;
#pragma unroll
                        for (int kk = 0; kk < KMMA; ++kk)   // A_lo x B_hi (first NPAD rows)
                            mma_tf32_atmem(d + NPAD, l0 + 8 * kk, sdesc(b0 + 32 * kk), ID_HI, 1u);
                    } else {
                        const uint32_t l0 = su32(LO(w.lo));
#pragma unroll
                        for (int kk = 0; kk < KMMA; ++kk)   // A_lo x B_hi (first NPAD rows)
                            mma<MODE>(d + NPAD, sdesc(l0 + 32 * kk), sdesc(b0 + 32 * kk), ID_HI, 1u);
                    }
                    mma_commit(&lo_empty[w.lo]);
                }
                mma_commit(&empty[w.stage]);
                if (chunk_end)
                    mma_commit(&acc_full[q]);
            }
            // however the loop ended, no MMA may still write TMEM when it is freed
            mma_commit(&fin[q]);
            mbar_wait_drain(&fin[q], 0, deadline + 3 * kDeadlineNs);
        }
    } else if (SR && warp < 6) {
        // ---------------- TF32X3 split: warps 2..5, 128 threads.  The tensor
        // core reads A through its TF32 conversion, which truncates, so A
        // itself acts as the high part and the remainder A - trunc(A),
        // rounded to TF32, goes to the low ring in tensor memory: the thread
        // of TMEM lane `row` reads row `row` of the 128B-swizzled A tile (its
        // 16-byte chunk c sits at chunk c ^ (row mod 8)) and stores its 32
        // low parts along that lane.  The MMA of a stage waits for its low
        // part, so the stage (and A in it) stays valid here.
        const int quad = warp & 3;               // TMEM lane quadrant of this warp
        const int row = quad * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        Ring w{};
        for (int64_t it = it0; it < it1; ++it, adv(w)) {
            // warp-uniform decisions: every lane of the warp continues or none
            if (!__all_sync(0xffffffffu, mbar_wait(&full[w.fb], w.fph, deadline, abort_flag)))
                break;
            if (!__all_sync(0xffffffffu,
                            mbar_wait(&lo_empty[w.lo], w.lph ^ 1u, deadline, abort_flag)))
                break;
            tc_fence_after();
            const uint8_t *ar = A(w.stage) + row * 128;
            uint32_t r[32];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 v = *reinterpret_cast<const float4 *>(ar + 16 * (c ^ (row & 7)));
                r[4 * c + 0] = __float_as_uint(rn_tf32_operand(v.x - __uint_as_float(__float_as_uint(v.x) & 0xffffe000u)));
                r[4 * c + 1] = __float_as_uint(rn_tf32_operand(v.y - __uint_as_float(__float_as_uint(v.y) & 0xffffe000u)));
                r[4 * c + 2] = __float_as_uint(rn_tf32_operand(v.z - __uint_as_float(__float_as_uint(v.z) & 0xffffe000u)));
                r[4 * c + 3] = __float_as_uint(rn_tf32_operand(v.w - __uint_as_float(__float_as_uint(v.w) & 0xffffe000u)));
            }
            tmem_st32(tmem + lane_addr + LO_COL0 + w.lo * 32, r);
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&lo_full[w.lf]);
        }
    } else {
        // ---------------- accumulation: warps 6..9 (SR) or 2..9
        // Thread (quad, lane, half) owns row quad*32 + lane of the tile and
        // columns [half*HC, half*HC + HC) of each accumulator region.  Each
        // chunk of DRAIN k blocks is accumulated by the tensor core in one
        // TMEM buffer, then read here and added into FP32 registers with
        // round-to-nearest adds: the tensor core's own accumulation rounds
        // toward zero, which over a long chain biases the sum low.
        constexpr int HC = SR ? NPAD : NPAD / 2;     // columns per thread per region
        const int quad = warp & 3;                   // TMEM lane quadrant this warp may read
        const int half = SR ? 0 : (warp - 2) >> 2;
        const uint32_t lane_base = ((uint32_t)(quad * 32) << 16) + half * HC;
        float acc[HC];
#pragma unroll
        for (int j = 0; j < HC; ++j)
            acc[j] = 0.f;
        int pending = -1;
        uint32_t drains[NACC] = {};
        Ring w{};
        const int t = threadIdx.x - 64;
        bool ok = true;
        auto ld_add = [&](uint32_t addr) {
            if constexpr (HC % 32 == 0) {
                // every load of the region in flight before one wait
                uint32_t v[HC];
#pragma unroll
                for (int c0 = 0; c0 < HC; c0 += 32)
                    tmem_ld32_nowait(addr + c0, v + c0);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < HC; ++j)
                    acc[j] += __uint_as_float(v[j]);
            } else if constexpr (HC >= 16) {
#pragma unroll
                for (int c0 = 0; c0 < HC; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16(addr + c0, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc[c0 + j] += __uint_as_float(v[j]);
                }
            } else {
                uint32_t v[8];
                tmem_ld8(addr, v);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[j] += __uint_as_float(v[j]);
            }
        };
        auto drain = [&](int b) -> bool {
            const uint32_t n = drains[b];
            if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[b], n & 1u, deadline, abort_flag)))
                return false;
            ++drains[b];
            __syncwarp();
            tc_fence_after();
            ld_add(tmem + b * BUF_COLS + lane_base);
            if constexpr (PAIR)   // A B_lo (and for X3 A_lo B_hi) beside A B_hi
                ld_add(tmem + b * BUF_COLS + NPAD + lane_base);
            tc_fence_before();
            mbar_arrive(&acc_empty[b]);
            return true;
        };
        int tile = tile0, kb = kb0 - 1;
        for (int64_t it = it0; it < it1 && ok; ++it, adv(w)) {
            if (++kb == KB) {
                kb = 0;
                ++tile;
            }
            const bool seg_end = it + 1 == it1 || kb == KB - 1;
            const bool chunk_end = seg_end || w.dc == DRAIN - 1;
            if constexpr (X3 && !SR) {
                // split this stage first (same step as the split warps above)
                if (!__all_sync(0xffffffffu, mbar_wait(&full[w.fb], w.fph, deadline, abort_flag)))
                    break;
                if (!__all_sync(0xffffffffu,
                                mbar_wait(&lo_empty[w.lo], w.lph ^ 1u, deadline, abort_flag)))
                    break;
                const float4 *a4 = reinterpret_cast<const float4 *>(A(w.stage));
                float4 *l4 = reinterpret_cast<float4 *>(LO(w.lo));
#pragma unroll
                for (int q = 0; q < (int)(kABytes / 16 / kEpi); ++q) {
                    const float4 v = a4[t + kEpi * q];
                    float4 r;
                    r.x = rn_tf32_operand(v.x - __uint_as_float(__float_as_uint(v.x) & 0xffffe000u));
                    r.y = rn_tf32_operand(v.y - __uint_as_float(__float_as_uint(v.y) & 0xffffe000u));
                    r.z = rn_tf32_operand(v.z - __uint_as_float(__float_as_uint(v.z) & 0xffffe000u));
                    r.w = rn_tf32_operand(v.w - __uint_as_float(__float_as_uint(v.w) & 0xffffe000u));
                    l4[t + kEpi * q] = r;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&lo_full[w.lf]);
            }
            // drain the previous chunk now that the tensor core has the next one
            if (pending >= 0) {
                ok = drain(pending);
                pending = -1;
                if (!ok)
                    break;
            }
            if (!chunk_end)
                continue;
            const int b = w.own;   // the issuer of this window accumulates in its buffer
            if (!seg_end) {
                pending = b;
                continue;
            }
            if (!(ok = drain(b)))
                break;
            // ---- store this CTA's part of `tile`
            const int64_t first_it = (int64_t)tile * KB, last_it = first_it + KB - 1;
            const int c_first = owner_of(first_it, p.iters, p.grid);
            const int c_last = owner_of(last_it, p.iters, p.grid);
            const int slice = (int)blockIdx.x - c_first;
            // The rows of this quadrant form one contiguous run of the slice
            // (rows of r floats).  NPAD <= 64: the quadrant stages its 32 rows
            // whole in shared memory in that layout and one thread sends them
            // with a bulk copy, so the accumulating warps go back to the next
            // chunk at once (the stores used to hold the drain, and behind it
            // the ring, for several microseconds a launch); wider factors go
            // through in groups of 8 rows with consecutive threads on
            // consecutive floats (a row per thread straight to global memory
            // would cost a separate transaction for every lane of every store).
            const int r = p.r;
            const int64_t row0 = (int64_t)tile * 128 + quad * 32;
            const int64_t left = p.M - row0;
            const int nrow = left <= 0 ? 0 : (left < 32 ? (int)left : 32);
            constexpr int QT = SR ? 32 : 64;                  // threads of a quadrant
            const int qt = SR ? lane : half * 32 + lane;
            auto qsync = [&]() {
                if constexpr (SR)
                    __syncwarp();
                else
                    asm volatile("bar.sync %0, 64;" ::"r"(1 + quad) : "memory");
            };
            float *dst = p.P + (int64_t)slice * p.M * r + row0 * r;
            if constexpr (BULK) {
                float *stg = stg_all + quad * 32 * NPAD;
                if (qt == 0)
                    bulk_wait_read();   // the previous copy has read the buffer
                qsync();
                if (lane < nrow) {
                    float *sr = stg + lane * r + half * HC;
#pragma unroll
                    for (int j = 0; j < HC; ++j)
                        if (half * HC + j < r)
                            sr[j] = acc[j];
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                qsync();
                const int n = nrow * r;
                const int nb = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 ? (n & ~3) : 0;
                if (qt == 0 && nb > 0)
                    bulk_store(dst, stg, (uint32_t)nb * 4u);
                for (int e = nb + qt; e < n; e += QT)
                    dst[e] = stg[e];
            } else {
                float *stg = stg_all + quad * 8 * NPAD;
                for (int g = 0; g < nrow; g += 8) {
                    const int nr = nrow - g < 8 ? nrow - g : 8;
                    if (lane >= g && lane < g + nr) {
                        float *sr = stg + (lane - g) * r + half * HC;
#pragma unroll
                        for (int j = 0; j < HC; ++j)
                            if (half * HC + j < r)
                                sr[j] = acc[j];
                    }
                    qsync();
                    float *d = dst + (int64_t)g * r;
                    for (int e = qt; e < nr * r; e += QT)
                        d[e] = stg[e];
                    qsync();
                }
            }
            // the first part of a tile clears the slices no CTA writes for it
            if (slice == 0) {
                for (int s2 = c_last - c_first + 1; s2 < p.nslices; ++s2) {
                    float *z = p.P + (int64_t)s2 * p.M * r + row0 * r;
                    for (int e = qt; e < nrow * r; e += QT)
                        z[e] = 0.f;
                }
            }
#pragma unroll
            for (int j = 0; j < HC; ++j)
                acc[j] = 0.f;
        }
        // the bulk copies this thread issued complete before the CTA exits
        if constexpr (BULK)
            bulk_wait_all();
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag && p.status)
        atomicOr(p.status, kStTimeout);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---- factor packing: X (K x r, row-major) -> B (NPAD x Kp, K contiguous) --
// mode TF32: raw FP32; TF32X3: 2 NPAD rows, the TF32 high part stacked over
// the TF32 remainder; BF16: round to nearest BF16; BF16X2: 2 NPAD rows, the
// nearest BF16 value over the nearest BF16 value of the remainder.  Rows
// r..NPAD-1 (of each part) and columns K..Kp-1 are zero.
template <int MODE>
__global__ void k_pack_factor(const float *__restrict__ X, int64_t K, int r, int npad, int64_t kp,
                              void *__restrict__ Bhi, void *__restrict__ Blo)
{
    // TF32X3: Bhi rows [0, npad) hold the nearest TF32 value, Blo (= rows
    // [npad, 2 npad) of the same buffer) the nearest TF32 value of the rest
    __shared__ float t[32][33];
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const int n0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t k = k0 + i;
        const int n = n0 + threadIdx.x;
        t[i][threadIdx.x] = (k < K && n < r) ? X[k * r + n] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int n = n0 + i;
        const int64_t k = k0 + threadIdx.x;
        if (n >= npad || k >= kp)
            continue;
        const float v = t[threadIdx.x][i];
        if constexpr (MODE == TC_BF16) {
            reinterpret_cast<__nv_bfloat16 *>(Bhi)[(int64_t)n * kp + k] = __float2bfloat16_rn(v);
        } else if constexpr (MODE == TC_BF16X2) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16 *>(Bhi)[(int64_t)n * kp + k] = hi;
            reinterpret_cast<__nv_bfloat16 *>(Blo)[(int64_t)n * kp + k] =
                __float2bfloat16_rn(v - __bfloat162float(hi));
        } else if constexpr (MODE == TC_TF32X3) {
            const float hi = rn_tf32(v);
            reinterpret_cast<float *>(Bhi)[(int64_t)n * kp + k] = hi;
            reinterpret_cast<float *>(Blo)[(int64_t)n * kp + k] = rn_tf32(v - hi);
        } else {
            reinterpret_cast<float *>(Bhi)[(int64_t)n * kp + k] = v;
        }
    }
}

// ---- host side ----------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

bool make_map(CUtensorMap *m, const void *base, bool bf16, uint64_t inner, uint64_t outer,
              uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer)
{
    auto fn = encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ---- tensor-pipe probe ------------------------------------------------------
// The MMA path of the cross term on a contraction wide enough to be bound by
// the tensor pipe instead of HBM (r = 512): one CTA per SM holds a 128 x 64
// BF16 A tile and a 512 x 64 B tile in shared memory (128B-swizzled, as the
// TMA would leave them) and one thread issues, per 16-wide k step, two
// M = 128, N = 256 MMAs into the two halves of the 512 TMEM columns, cycling
// over the tile's four k steps `iters` times; a commit to an mbarrier (bounded
// wait) ends it.  The tiles hold BF16 values in [0.5, 1.5) from a hash of the
// position.  A launch lasts about a millisecond, too short for the power cap
// to lower the SM clock.
constexpr int kPeakN = 256;
constexpr uint32_t kPeakA = 128 * 128, kPeakB = 2 * kPeakN * 128;   // bytes
constexpr size_t kPeakSmem = 120 * 1024;   // > half the SM's shared memory: one CTA per SM

__global__ void __launch_bounds__(128, 1) k_tc_peak(int iters, unsigned *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    uint8_t *As = smem, *Bs = smem + kPeakA;
    uint64_t *done = reinterpret_cast<uint64_t *>(Bs + kPeakB);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    for (uint32_t i = threadIdx.x; i < (kPeakA + kPeakB) / 4; i += blockDim.x) {
        uint32_t hsh = (i + 1u) * 2654435761u;   // two BF16 values per word
        hsh ^= hsh >> 15;
        const float lo = 0.5f + (float)(hsh & 1023u) * (1.f / 1024.f);
        const float hi = 0.5f + (float)((hsh >> 10) & 1023u) * (1.f / 1024.f);
        const uint32_t w = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
                           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
        reinterpret_cast<uint32_t *>(smem)[i] = w;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        constexpr uint32_t ID = idesc(1u, 128, kPeakN);
        const uint32_t a0 = su32(As), b0 = su32(Bs);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                mma<TC_BF16>(tmem, sdesc(a0 + 32 * kk), sdesc(b0 + 32 * kk), ID, acc);
                mma<TC_BF16>(tmem + kPeakN, sdesc(a0 + 32 * kk),
                             sdesc(b0 + kPeakN * 128 + 32 * kk), ID, acc);
            }
        mma_commit(done);
        const unsigned long long deadline = gtimer() + kDeadlineNs;
        if (!mbar_wait(done, 0, deadline, abort_flag)) {
            if (status)
                atomicOr(status, kStTimeout);
            mbar_wait_drain(done, 0, deadline + kDeadlineNs);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(512u)
                     : "memory");
    }
}

template <int MODE, int NPAD>
struct TcCfg {
    static constexpr int NLO = MODE == TC_TF32X3 ? 3 : 0;       // low-part ring
    // its shared-memory copy: only without the split warps (NPAD 128); with
    // them (NPAD <= 64) the ring is in tensor memory
    static constexpr int NLO_SM = MODE == TC_TF32X3 && NPAD > 64 ? NLO : 0;
    static constexpr int NB = MODE == TC_TF32X3 || MODE == TC_BF16X2 ? 2 * NPAD : NPAD;
    static constexpr int STAGE = kABytes + NB * 128;
    // as many stages as fit: A in flight from HBM is what the ring buys
    // epilogue staging bytes: 32 rows per TMEM lane quadrant (NPAD <= 64), else 8
    static constexpr int STG = 4 * (NPAD <= 64 ? 32 : 8) * NPAD * 4;
    static constexpr int ST0 = (225 * 1024 - NLO_SM * (int)kABytes - STG) / STAGE;
    static constexpr int STAGES = ST0 > 8 ? 8 : ST0;
    static constexpr int DRAIN = MODE == TC_TF32X3 ? 1 : 2;     // k blocks per chunk
    // + 1024 for the 1024-byte alignment of the tiles, + the barrier area
    static constexpr size_t SMEM =
        (size_t)STAGES * STAGE + (size_t)NLO_SM * kABytes + STG + 1024 + kBarBytes;
    static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
};

template <int MODE, int NPAD>
cudaError_t launch_mode(const CUtensorMap &a, const CUtensorMap &b, const TcArgs &p,
                        cudaStream_t s)
{
    using C = TcCfg<MODE, NPAD>;
    auto kern = k_tc_cross<MODE, NPAD, C::STAGES, C::NLO, C::DRAIN>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess)
            return e;
        attr = true;
    }
    cudaError_t e = pdl_launch(kern, dim3(p.grid), dim3(kThreads), C::SMEM, s, a, b, p);
    count_launch();
    return e;
}

template <int MODE>
cudaError_t launch_npad(int npad, const CUtensorMap &a, const CUtensorMap &b, const TcArgs &p,
                        cudaStream_t s)
{
    switch (npad) {
    case 16: return launch_mode<MODE, 16>(a, b, p, s);
    case 32: return launch_mode<MODE, 32>(a, b, p, s);
    case 64: return launch_mode<MODE, 64>(a, b, p, s);
    default: return launch_mode<MODE, 128>(a, b, p, s);
    }
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1)
            n = 1;
    }
    return n;
}

}  // namespace

int tc_npad(int r) { return r <= 16 ? 16 : r <= 32 ? 32 : r <= 64 ? 64 : 128; }

int64_t tc_kpad(int64_t K, int mode) { return tc_bf16(mode) ? (K + 7) / 8 * 8 : (K + 3) / 4 * 4; }

size_t tc_pack_bytes(int64_t K, int r, int mode)
{
    const int64_t kp = tc_kpad(K, mode);
    const size_t e = tc_bf16(mode) ? 2 : 4;
    return (size_t)tc_npad(r) * kp * e * (tc_pair(mode) ? 2 : 1) + 256;
}

cudaError_t launch_tc_pack(const float *X, int64_t K, int r, int mode, void *pack, cudaStream_t s)
{
    ProfScope prof_(KC_OTHER, s);
    const int npad = tc_npad(r);
    const int64_t kp = tc_kpad(K, mode);
    const size_t hb = (size_t)npad * kp * (tc_bf16(mode) ? 2 : 4);
    void *lo = reinterpret_cast<char *>(pack) + hb;   // rows npad.. of the pair modes
    dim3 grid((unsigned)((kp + 31) / 32), (unsigned)((npad + 31) / 32));
    dim3 blk(32, 8);
    if (mode == TC_BF16)
        k_pack_factor<TC_BF16><<<grid, blk, 0, s>>>(X, K, r, npad, kp, pack, nullptr);
    else if (mode == TC_BF16X2)
        k_pack_factor<TC_BF16X2><<<grid, blk, 0, s>>>(X, K, r, npad, kp, pack, lo);
    else if (mode == TC_TF32X3)
        k_pack_factor<TC_TF32X3><<<grid, blk, 0, s>>>(X, K, r, npad, kp, pack, lo);
    else
        k_pack_factor<TC_TF32><<<grid, blk, 0, s>>>(X, K, r, npad, kp, pack, nullptr);
    count_launch();
    return cudaGetLastError();
}

bool tc_supported(int64_t lda, int mode, const void *A)
{
    const int64_t align = tc_bf16(mode) ? 8 : 4;   // 16-byte row pitch
    return (lda % align) == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0 && encode_fn();
}

TcPlan tc_plan(int64_t M, int64_t K, int r, int mode, int max_grid)
{
    TcPlan pl;
    const int kstep = tc_bf16(mode) ? 64 : 32;
    pl.kblocks = (int)((K + kstep - 1) / kstep);
    pl.tiles = (int)((M + 127) / 128);
    pl.iters = (int64_t)pl.tiles * pl.kblocks;
    int g = sm_count();
    if (max_grid > 0 && max_grid < g)
        g = max_grid;
    if (pl.iters < g)
        g = (int)pl.iters;
    pl.grid = g < 1 ? 1 : g;
    int ns = 1;
    for (int t = 0; t < pl.tiles; ++t) {
        const int64_t f = (int64_t)t * pl.kblocks, l = f + pl.kblocks - 1;
        const int n = owner_of(l, pl.iters, pl.grid) - owner_of(f, pl.iters, pl.grid) + 1;
        ns = n > ns ? n : ns;
    }
    pl.nslices = ns;
    return pl;
}

cudaError_t launch_tc_cross(const void *A, int64_t M, int64_t K, int64_t lda, int r, int mode,
                            const void *pack, float *P, const TcPlan &pl, unsigned *status,
                            cudaStream_t s)
{
    ProfScope prof_(KC_CROSS, s);
    if (M <= 0)
        return cudaSuccess;
    const int npad = tc_npad(r);
    const bool bf = tc_bf16(mode);
    const int64_t kp = tc_kpad(K, mode);
    const size_t es = bf ? 2 : 4;
    const uint32_t nb = tc_pair(mode) ? 2 * npad : npad;   // packed rows ([hi; lo] for the pairs)
    CUtensorMap ma, mb;
    const uint32_t box_k = bf ? 64 : 32;
    if (!make_map(&ma, A, bf, (uint64_t)K, (uint64_t)M, (uint64_t)lda * es, box_k, 128) ||
        !make_map(&mb, pack, bf, (uint64_t)kp, (uint64_t)nb, (uint64_t)kp * es, box_k, nb))
        return cudaErrorInvalidValue;
    TcArgs p{};
    p.M = M;
    p.r = r;
    p.kblocks = pl.kblocks;
    p.iters = pl.iters;
    p.grid = pl.grid;
    p.nslices = pl.nslices;
    p.P = P;
    p.status = status;
    if (mode == TC_BF16)
        return launch_npad<TC_BF16>(npad, ma, mb, p, s);
    if (mode == TC_BF16X2)
        return launch_npad<TC_BF16X2>(npad, ma, mb, p, s);
    if (mode == TC_TF32X3)
        return launch_npad<TC_TF32X3>(npad, ma, mb, p, s);
    return launch_npad<TC_TF32>(npad, ma, mb, p, s);
}

// dense BF16 tensor throughput of the MMA path above (TFLOP/s), timed with
// CUDA events over a few launches after a warm-up; TFLOP counted as 2 M N K of
// the MMAs issued
cudaError_t measure_tc_peak(double *tflops, unsigned *status)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_peak, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kPeakSmem);
        if (e != cudaSuccess)
            return e;
        attr = true;
    }
    const int sms = sm_count();
    const int iters = 2048;   // ~1.5 ms a launch at the nominal rate
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    k_tc_peak<<<sms, 128, kPeakSmem>>>(iters, status);   // warm-up
    count_launch();
    const int reps = 5;
    cudaEventRecord(e0);
    for (int i = 0; i < reps; ++i) {
        k_tc_peak<<<sms, 128, kPeakSmem>>>(iters, status);
        count_launch();
    }
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return e;
    const double flop = 2.0 * 128.0 * (2.0 * kPeakN) * 16.0 * 4.0 * iters * sms * reps;
    *tflops = ms > 0.f ? flop / (ms * 1e-3) / 1e12 : 0.0;
    return cudaSuccess;
}

}  // namespace nmfi
