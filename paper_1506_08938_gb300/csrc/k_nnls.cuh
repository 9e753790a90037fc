// Batched NQP solver: Alg. 3 of §3.4 (anti-lopsided rescaled problem, exact
// line search along the masked gradient, then greedy coordinate descent) for
// many rows that share one rescaled Gram matrix Qt.
//
// Qt comes from the rescale step, so its diagonal is exactly 1 on live
// coordinates and its dead rows and columns are zero; the 1-D minimiser of
// coordinate p then moves y_p by del = max(-y_p, -g_p), which lowers the
// objective by -del (g_p + del / 2).  A Qt whose diagonal holds anything but
// 0 or 1 is rejected (status flag, X untouched).
//
// Layout.  A group of G consecutive lanes owns one row problem, so a warp
// works on 32/G rows at once.  Lane li of a group holds J coordinates of the
// gradient g in registers, in chunks of CW = min(J, 4) consecutive
// coordinates: chunk c covers (c*G + li)*CW ... +CW-1, so that the G lanes of
// a group read one contiguous run of any Qt row (no shared-memory bank
// conflicts).  RP = G*J >= r.  The iterate y of each group lives in shared
// memory in coordinate order, where the matrix-vector products read it;
// during the coordinate steps each lane keeps its J entries in registers (a
// step changes one entry, which only its owner lane reads) and writes them
// back after the last step.
// Qt, zero-padded to RP x RP, is loaded once per CTA; it is symmetric, so the
// column Qt[:, p] a coordinate step needs is read as the contiguous row p.
//
// Per coordinate step a lane evaluates the gains of its J coordinates, the
// group takes the maximum key with log2(G) xor-shuffles (one warp-wide
// reduction when G = 32), and a ballot names
// the lowest lane holding it; within a lane the lower index wins, so exact
// ties go to the lowest coordinate, as in the oracle.
//
// Scheduling.  The groups of a warp run in lockstep but on their own rows:
// the warp loops over rounds, each round = (start rows in groups that are
// free) + one iteration of Alg. 3's repeat loop (line search and the
// coordinate steps) for every busy group + the stop test.  A group whose row
// meets the stop rule writes it out and takes the next row of the warp's
// share in the next round, so a row that needs many iterations does not hold
// up its neighbours.  Idle groups ride along with zero steps, which leave
// their state unchanged.  The standalone kernel gives each CTA a balanced
// contiguous range of rows and each warp runs of 32/G consecutive rows of
// it; the line search's matrix-vector products share each Qt load among the
// groups of a warp (matvec_coop).
//
// Epilogue (optional, RP <= 64): each CTA turns its rows of the solved
// factor into one Gram partial and their columns of the packed tensor-core
// operand for the next half-step (k_prep.cuh), so the next half-step's
// preparation needs only the finishing launch.
#pragma once
#include "k_prep.cuh"

namespace nmfi {
namespace nnls_detail {

constexpr int kWarps = 8;
constexpr unsigned kFull = 0xffffffffu;
// keys are the bits of -gain <= 0 read as unsigned: a positive gain maps above
// this value, a zero gain (either sign of zero) to it or below
constexpr unsigned kNoGain = 0x80000000u;

template <int G, int J>
struct Map {
    static constexpr int CW = J < 4 ? J : 4;   // chunk width
    static constexpr int NC = J / CW;          // chunks per lane
    static constexpr int RP = G * J;
    static constexpr int VB = RP + 4;          // per-group buffer stride (16-byte aligned)
    __device__ static __forceinline__ int coord(int li, int j)
    {
        return ((j / CW) * G + li) * CW + (j % CW);
    }
};

// a lane's J values of a length-RP row p (coordinate order)
template <int G, int J>
__device__ __forceinline__ void ld_lane(const float *p, int li, float (&a)[J])
{
    using M = Map<G, J>;
#pragma unroll
    for (int c = 0; c < M::NC; ++c) {
        const float *q = p + (c * G + li) * M::CW;
        if constexpr (M::CW == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(q);
            a[4 * c] = t.x; a[4 * c + 1] = t.y; a[4 * c + 2] = t.z; a[4 * c + 3] = t.w;
        } else {
            const float2 t = *reinterpret_cast<const float2 *>(q);
            a[2 * c] = t.x; a[2 * c + 1] = t.y;
        }
    }
}

template <int G, int J>
__device__ __forceinline__ void st_lane(float *p, int li, const float (&a)[J])
{
    using M = Map<G, J>;
#pragma unroll
    for (int c = 0; c < M::NC; ++c) {
        float *q = p + (c * G + li) * M::CW;
        if constexpr (M::CW == 4)
            *reinterpret_cast<float4 *>(q) =
                make_float4(a[4 * c], a[4 * c + 1], a[4 * c + 2], a[4 * c + 3]);
        else
            *reinterpret_cast<float2 *>(q) = make_float2(a[2 * c], a[2 * c + 1]);
    }
}

// sum over the G lanes of a group (aligned groups: xor offsets < G stay inside)
template <int G>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ unsigned group_max(unsigned v)
{
    if constexpr (G == 32) {
        // one row per warp: a single warp-wide reduction instead of five
        // shuffle-and-max rounds (the maximum of integers: the same value)
        return __reduce_max_sync(kFull, v);
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            unsigned w = __shfl_xor_sync(kFull, v, o);
            v = w > v ? w : v;
        }
        return v;
    }
}

// all G ballot bits of one group set
template <int G>
__host__ __device__ constexpr unsigned group_full()
{
    if constexpr (G == 32)
        return kFull;
    else
        return (1u << G) - 1u;
}

// the G ballot bits of group gi
template <int G>
__device__ __forceinline__ unsigned group_bits(unsigned ballot, int gi)
{
    if constexpr (G == 32)
        return ballot;
    else
        return (ballot >> (gi * G)) & group_full<G>();
}

// out = Qt v for every group of the warp at once, v read from the group's
// buffer vg (coordinate order, broadcast float4); only the first
// r4 = roundup(r, 4) rows of Qt are non-zero.
template <int G, int J>
__device__ __forceinline__ void matvec_buf(const float *__restrict__ Qs, const float *vg,
                                           float (&out)[J], int li, int r4)
{
    constexpr int RP = Map<G, J>::RP;
#pragma unroll
    for (int j = 0; j < J; ++j)
        out[j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < r4; k += 4) {
        const float4 vk = *reinterpret_cast<const float4 *>(vg + k);
        float a0[J], a1[J];
        ld_lane<G, J>(Qs + k * RP, li, a0);
        ld_lane<G, J>(Qs + (k + 1) * RP, li, a1);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            out[j] = fmaf(a0[j], vk.x, out[j]);
            out[j] = fmaf(a1[j], vk.y, out[j]);
        }
        ld_lane<G, J>(Qs + (k + 2) * RP, li, a0);
        ld_lane<G, J>(Qs + (k + 3) * RP, li, a1);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            out[j] = fmaf(a0[j], vk.z, out[j]);
            out[j] = fmaf(a1[j], vk.w, out[j]);
        }
    }
}

// The products of all groups of the warp with each Qt load shared among
// the groups: lane L computes coordinates [L CL, L CL + CL) of every group's
// product (CL = RP / 32), then the products pass through the groups' output
// buffers (stride VB from out0) into the coordinate-step layout.  Inputs are
// read from in0 (group buffers, stride VB; in0 may equal out0).  Each output
// takes its k terms in the order matvec_buf does, so the results agree bit
// for bit; the shared loads cut the shared-memory wavefronts of a product
// about 2.5-fold when a warp holds several groups.
template <int G, int J>
constexpr bool coop_matvec() { return 32 / G >= 2 && Map<G, J>::RP % 32 == 0; }

template <int G, int J>
__device__ __forceinline__ void matvec_coop(const float *__restrict__ Qs, const float *in0,
                                            float *out0, float (&out)[J], int gi, int li, int r4)
{
    using M = Map<G, J>;
    constexpr int RP = M::RP, NG = 32 / G, CL = RP / 32, VB = M::VB;
    const int lane = threadIdx.x & 31;
    float acc[NG][CL];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int i = 0; i < CL; ++i)
            acc[g][i] = 0.f;
    for (int k = 0; k < r4; k += 4) {
        float4 v[NG];
#pragma unroll
        for (int g = 0; g < NG; ++g)
            v[g] = *reinterpret_cast<const float4 *>(in0 + g * VB + k);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const float *qp = Qs + (k + kk) * RP + lane * CL;
            float q[CL];
            if constexpr (CL == 4) {
                const float4 t = *reinterpret_cast<const float4 *>(qp);
                q[0] = t.x; q[1] = t.y; q[2] = t.z; q[3] = t.w;
            } else if constexpr (CL == 2) {
                const float2 t = *reinterpret_cast<const float2 *>(qp);
                q[0] = t.x; q[1] = t.y;
            } else {
                q[0] = qp[0];
            }
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const float vk = kk == 0 ? v[g].x : kk == 1 ? v[g].y : kk == 2 ? v[g].z : v[g].w;
#pragma unroll
                for (int i = 0; i < CL; ++i)
                    acc[g][i] = fmaf(q[i], vk, acc[g][i]);
            }
        }
    }
    __syncwarp();   // every lane has read its inputs
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        float *op = out0 + g * VB + lane * CL;
        if constexpr (CL == 4)
            *reinterpret_cast<float4 *>(op) = make_float4(acc[g][0], acc[g][1], acc[g][2], acc[g][3]);
        else if constexpr (CL == 2)
            *reinterpret_cast<float2 *>(op) = make_float2(acc[g][0], acc[g][1]);
        else
            op[0] = acc[g][0];
    }
    __syncwarp();
    ld_lane<G, J>(out0 + gi * VB, li, out);
    __syncwarp();   // the buffers may be rewritten next
}

// out = Qt v for this lane's group, v in the group buffer vg (the warp's
// group buffers start at v0); products land in the warp's buffers at out0
// when the groups share the loads
template <int G, int J>
__device__ __forceinline__ void matvec_rows(const float *__restrict__ Qs, const float *v0,
                                            const float *vg, float *out0, float (&out)[J],
                                            int gi, int li, int r4)
{
    if constexpr (coop_matvec<G, J>())
        matvec_coop<G, J>(Qs, v0, out0, out, gi, li, r4);
    else
        matvec_buf<G, J>(Qs, vg, out, li, r4);
}

// stage v (a lane's J values) in the group buffer vbg, then out = Qt v
// (vb0: the warp's first group buffer)
template <int G, int J>
__device__ __forceinline__ void matvec(const float *__restrict__ Qs, float *vb0, float *vbg,
                                       const float (&v)[J], float (&out)[J], int gi, int li,
                                       int r4)
{
    st_lane<G, J>(vbg, li, v);
    __syncwarp();
    matvec_rows<G, J>(Qs, vb0, vbg, vb0, out, gi, li, r4);
    __syncwarp();
}

// this lane's part of ||P(y, g)||^2: the passive set is {y > 0 or g < 0}
template <int J>
__device__ __forceinline__ float proj_part(const float (&y)[J], const float (&g)[J])
{
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < J; ++j)
        if (y[j] > 0.f || g[j] < 0.f)
            s = fmaf(g[j], g[j], s);
    return s;
}

// the epilogue that prepares the solved factor (Gram partial, packing) is
// built for RP <= 64, where its accumulators fit the register budget
template <int G, int J>
constexpr bool has_prep_epilogue() { return Map<G, J>::RP <= 64; }

template <int G, int J>
constexpr int stage_floats()
{
    return has_prep_epilogue<G, J>()
               ? prep_detail::kRowsBlock * (prep_detail::stage_cols(Map<G, J>::RP) + 1)
               : 0;
}

template <int G, int J>
constexpr size_t smem_bytes()
{
    using M = Map<G, J>;
    return sizeof(float) * ((size_t)M::RP * M::RP + M::RP + 2 * (size_t)kWarps * (32 / G) * M::VB +
                            stage_floats<G, J>());
}

// CTAs per SM the register budget is sized for
template <int J>
constexpr int min_ctas() { return J >= 16 ? 2 : (J >= 4 ? 3 : 4); }

// Stage Qt (zero-padded to RP x RP) and the scale d (1 for dead and padding
// coordinates) in shared memory; false (and the status flag) if Qt's
// diagonal holds anything but 0 or 1.  All threads of the CTA take part.
template <int G, int J>
__device__ __forceinline__ bool stage_qt(const float *Qt, const float *d, int r, float *Qs,
                                         float *sd, unsigned *status)
{
    constexpr int RP = Map<G, J>::RP;
    constexpr int B = 8;   // loads in flight per thread before their stores
    for (int base = threadIdx.x; base < RP * RP; base += B * blockDim.x) {
        float v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int idx = base + b * blockDim.x, i = idx / RP, j = idx % RP;
            v[b] = (idx < RP * RP && i < r && j < r) ? Qt[i * r + j] : 0.f;
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int idx = base + b * blockDim.x;
            if (idx < RP * RP)
                Qs[idx] = v[b];
        }
    }
    __syncthreads();
    bool bad = false;
    for (int e = threadIdx.x; e < RP; e += blockDim.x) {
        const float qii = Qs[e * RP + e];
        bad = bad || (qii != 0.f && qii != 1.f);
        sd[e] = (e < r && qii > 0.f) ? d[e] : 1.f;
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0 && status)
            atomicOr(status, kStBadInput);
        return false;
    }
    return true;
}

// shared floats behind Qs and sd: per group, a staging buffer and the iterate
template <int G, int J>
constexpr int pool_floats() { return 2 * kWarps * (32 / G) * Map<G, J>::VB; }

// Alg. 3 for this warp's share of the rows, taken in rounds by its groups
// (the layout and schedule of the file header).  The share is the runs of
// `chunk` consecutive rows starting at first, first + stride, first +
// 2 stride, ..., cut at end: its s-th row is first + (s / chunk) stride +
// s % chunk (chunk a power of two, at most stride).  Qs, sd staged by
// stage_qt; pool holds pool_floats<G, J>() floats.  Called by every lane of
// the warp; returns the warp's (inner iterations, largest final ||P||^2
// bits) for the counters of NnlsArgs, which the caller adds.
template <int G, int J>
__device__ __forceinline__ uint2 nnls_rows(const NnlsArgs &a, const float *__restrict__ Qs,
                                          const float *__restrict__ sd, float *pool,
                                          int64_t first, int64_t stride, int64_t end,
                                          int chunk = 1)
{
    using M = Map<G, J>;
    constexpr int RP = M::RP;
    constexpr int NG = 32 / G;            // rows per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gi = lane / G, li = lane - gi * G;
    float *vb0 = pool + warp * NG * M::VB;                               // staging
    float *ys0 = pool + (kWarps * NG + warp * NG) * M::VB;               // iterate y
    float *vbg = vb0 + gi * M::VB, *ysg = ys0 + gi * M::VB;              // this group's
    const int r = a.r;
    const int r4 = (r + 3) & ~3;

    // live coordinates (bit j: this lane's j-th); a dead one keeps y = g = 0
    unsigned live = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int e = M::coord(li, j);
        if (e < r && Qs[e * RP + e] > 0.f)
            live |= 1u << j;
    }
    const int T = a.cd_steps < 0 ? r : a.cd_steps;
    // fast-break threshold (mode 1): from device memory when the previous
    // update of the same factor left it there
    const float mstop = a.maxstop_dev ? __uint_as_float(*a.maxstop_dev) : a.maxstop;
    int64_t taken = 0;      // rows of the share handed out so far
    const int csh = __ffs(chunk) - 1;
    const unsigned below = (1u << (gi * G)) - 1u;          // ballot bits of the groups before gi

    float g[J], zero[J];
#pragma unroll
    for (int j = 0; j < J; ++j)
        g[j] = zero[j] = 0.f;
    st_lane<G, J>(ysg, li, zero);
    int64_t row = -1;
    bool active = false, need = true;
    int k = 0;
    float s0 = 0.f;
    unsigned my_iters = 0;
    unsigned my_smax = 0;

    auto finish = [&](float sk) {
        float y[J];
        ld_lane<G, J>(ysg, li, y);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int e = M::coord(li, j);
            if (e < r)
                a.X[row * r + e] = ((live >> j) & 1u) ? y[j] / sd[e] : 0.f;
        }
        if (li == 0) {
            if (a.iters)
                a.iters[row] = k;
            my_iters += (unsigned)k;
            const unsigned sb = __float_as_uint(sk);
            my_smax = sb > my_smax ? sb : my_smax;
        }
        st_lane<G, J>(ysg, li, zero);
#pragma unroll
        for (int j = 0; j < J; ++j)
            g[j] = 0.f;
    };

    for (;;) {
        // ---- free groups take the next rows of this warp's share, in group order
        const unsigned needb = __ballot_sync(kFull, need && li == 0);
        bool fresh = false;
        if (need) {
            const int64_t sidx = taken + __popc(needb & below);
            const int64_t cand = first + (sidx >> csh) * stride + (sidx & (chunk - 1));
            row = cand < end ? cand : -1;
            fresh = row >= 0;
            need = false;   // busy now, or the share is exhausted: idle for good
        }
        taken += __popc(needb);
        if (!__any_sync(kFull, fresh || active))
            break;

        // ---- start fresh rows: y = x0 .* d, g = Qt y + (alpha - c) ./ d
        if (__any_sync(kFull, fresh)) {
            bool ok = true;
            if (fresh) {
                // every load of a slice issued before the first add (the
                // slices are summed in order, as one scalar chain would)
                float c[J], x0[J], y0[J];
                const float *xr = a.X + row * r, *cr = a.C + row * r;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int e = M::coord(li, j);
                    x0[j] = e < r ? xr[e] : 0.f;
                    c[j] = 0.f;
                }
                for (int s = 0; s < a.nsplit; ++s) {
                    float t[J];
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const int e = M::coord(li, j);
                        t[j] = e < r ? cr[(int64_t)s * a.c_stride + e] : 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        c[j] += t[j];
                }
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int e = M::coord(li, j);
                    if (e < r)
                        ok = ok && isfinite(c[j]) && isfinite(x0[j]);
                    const bool lv = (live >> j) & 1u;
                    g[j] = lv ? (a.alpha - c[j]) / sd[e] : 0.f;   // q staged in g
                    y0[j] = lv ? x0[j] * sd[e] : 0.f;
                }
                st_lane<G, J>(ysg, li, y0);
            }
            const bool gok = group_bits<G>(__ballot_sync(kFull, ok), gi) == group_full<G>();
            __syncwarp();
            float t[J];
            matvec_rows<G, J>(Qs, ys0, ysg, vb0, t, gi, li, r4);   // busy groups' are unused
            __syncwarp();
            if (fresh) {
#pragma unroll
                for (int j = 0; j < J; ++j)
                    g[j] = (gok && ((live >> j) & 1u)) ? g[j] + t[j] : 0.f;
                if (!gok)
                    st_lane<G, J>(ysg, li, zero);
            }
            float y[J];
            ld_lane<G, J>(ysg, li, y);
            const float s0n = group_sum<G>(proj_part<J>(y, g));
            if (fresh) {
                if (!gok) {
                    if (li == 0 && a.status)
                        atomicOr(a.status, kStNonFinite);
                    need = true;   // row skipped, X left as it was
                } else if (s0n > 0.f) {
                    active = true;
                    s0 = s0n;
                    k = 0;
                } else {           // already optimal: k = 0
                    k = 0;
                    finish(s0n);
                    need = true;
                }
            }
        }

        // ---- exact line search along the masked gradient (busy groups)
        {
            float y[J], gb[J];
            ld_lane<G, J>(ysg, li, y);
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                gb[j] = (active && (y[j] > 0.f || g[j] < 0.f)) ? g[j] : 0.f;
                s = fmaf(gb[j], gb[j], s);
            }
            s = group_sum<G>(s);
            if (__any_sync(kFull, s > 0.f)) {
                float u[J];
                matvec<G, J>(Qs, vb0, vbg, gb, u, gi, li, r4);
                float den = 0.f;
#pragma unroll
                for (int j = 0; j < J; ++j)
                    den = fmaf(gb[j], u[j], den);
                den = group_sum<G>(den);
                const float al = (s > 0.f && den > 0.f) ? s / den : 0.f;
                // the projected step; a coordinate the projection clips (its
                // unprojected value t < 0, so it moves to 0) is counted and,
                // if it is the group's only one, its correction -t kept
                unsigned clip = 0;
                float cval = 0.f;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const float t = fmaf(-al, gb[j], y[j]);
                    const float yn = fmaxf(0.f, t);
                    if (t < 0.f) {
                        clip |= 1u << j;
                        cval = -t;
                    }
                    gb[j] = yn - y[j];   // the step actually taken
                    y[j] = yn;
                }
                st_lane<G, J>(ysg, li, y);
                // the gradient moves by Qt dy.  With no clipped coordinate
                // dy = -al gb, so Qt dy = -al u, the product already formed;
                // with one clipped coordinate p, dy = -al gb + c e_p with c =
                // -t_p, so Qt dy = -al u + c Qt[:, p].  Only a group whose step
                // clipped two or more coordinates forms the product of dy.
                const int nclip = (int)group_sum<G>((float)__popc(clip));
                const bool full = nclip > 1;
                if (!full) {
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        g[j] = fmaf(-al, u[j], g[j]);
                }
                if (__any_sync(kFull, full)) {
                    matvec<G, J>(Qs, vb0, vbg, gb, u, gi, li, r4);
                    if (full) {
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            g[j] += u[j];
                    }
                }
                if (__any_sync(kFull, nclip == 1)) {
                    const unsigned wb = group_bits<G>(__ballot_sync(kFull, clip != 0u), gi);
                    const int sli = wb ? __ffs(wb) - 1 : 0;
                    const int src = gi * G + sli;
                    const int pj = __shfl_sync(kFull, clip ? __ffs(clip) - 1 : 0, src);
                    const float c = __shfl_sync(kFull, cval, src);
                    if (nclip == 1) {
                        const int pc = M::coord(sli, pj);
                        float col[J];
                        ld_lane<G, J>(Qs + pc * RP, li, col);
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            g[j] = fmaf(col[j], c, g[j]);
                    }
                }
            }
        }

        // ---- greedy coordinate descent: T steps of the largest decrease.
        // A step changes one coordinate, owned by one lane, and only that
        // lane reads it during the steps: the iterate stays in registers and
        // goes back to shared memory after the last step.
        float yc[J];
        ld_lane<G, J>(ysg, li, yc);
        for (int t = 0; t < T; ++t) {
            const float(&y)[J] = yc;
            unsigned key[J];
            int idx[J];
            float del[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                // dead or padding coordinates have y = g = 0: del = 0, no gain
                del[j] = fmaxf(-y[j], -g[j]);
                key[j] = __float_as_uint(del[j] * fmaf(0.5f, del[j], g[j]));   // = -gain
                idx[j] = j;
            }
#pragma unroll
            for (int s = 1; s < J; s <<= 1)
#pragma unroll
                for (int j = 0; j + s < J; j += 2 * s)
                    if (key[j + s] > key[j]) {   // strict: the lower index keeps ties
                        key[j] = key[j + s];
                        idx[j] = idx[j + s];
                        del[j] = del[j + s];
                    }
            const unsigned bkey = active ? key[0] : 0u;
            const unsigned m = group_max<G>(bkey);
            const bool step = m > kNoGain;
            if (!__any_sync(kFull, step))
                break;
            const unsigned wb = group_bits<G>(__ballot_sync(kFull, bkey == m), gi);
            const int sli = __ffs(wb) - 1;
            const int src = gi * G + sli;
            const int pj = __shfl_sync(kFull, idx[0], src);
            float dp = __shfl_sync(kFull, del[0], src);
            dp = step ? dp : 0.f;   // no positive gain: this group takes no step
            const int p = M::coord(sli, pj);
            float col[J];
            ld_lane<G, J>(Qs + p * RP, li, col);
#pragma unroll
            for (int j = 0; j < J; ++j)
                g[j] = fmaf(col[j], dp, g[j]);
            const unsigned own = (step && lane == src) ? 1u << pj : 0u;
#pragma unroll
            for (int j = 0; j < J; ++j)
                yc[j] = ((own >> j) & 1u) ? yc[j] + dp : yc[j];
        }
        st_lane<G, J>(ysg, li, yc);
        __syncwarp();   // the products below read every group's iterate

        // ---- stop test (Alg. 3): accelerated condition, fast break, cap
        float y[J];
        ld_lane<G, J>(ysg, li, y);
        float sk = group_sum<G>(proj_part<J>(y, g));
        // optional gradient refresh: every grad_refresh-th iteration of a row
        // the gradient carried by updates is replaced by g = Qt y + qt formed
        // afresh (qt from the row's C slices again), so that the rounding the
        // updates accumulate over many iterations does not move the point the
        // iteration converges to; the stop test then uses the fresh gradient
        if (a.grad_refresh > 0) {
            const bool ref = active && (k + 1) % a.grad_refresh == 0;
            if (__any_sync(kFull, ref)) {
                float t[J];
                matvec_rows<G, J>(Qs, ys0, ysg, vb0, t, gi, li, r4);
                __syncwarp();
                if (ref) {
                    const float *cr = a.C + row * r;
                    float c[J];
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        c[j] = 0.f;
                    for (int s = 0; s < a.nsplit; ++s) {
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const int e = M::coord(li, j);
                            c[j] += e < r ? cr[(int64_t)s * a.c_stride + e] : 0.f;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const int e = M::coord(li, j);
                        g[j] = ((live >> j) & 1u) ? (a.alpha - c[j]) / sd[e] + t[j] : 0.f;
                    }
                }
                const float s2 = group_sum<G>(proj_part<J>(y, g));
                sk = ref ? s2 : sk;
            }
        }
        if (active) {
            ++k;
            const bool stop = sk <= a.eps * s0 || (a.maxstop_mode == 1 && sk <= mstop) ||
                              k >= a.max_inner;
            if (stop) {
                finish(sk);
                active = false;
                need = true;
            }
        }
    }
    // the warp's total of inner iterations and largest final ||P||^2 (bits
    // of a non-negative float: unsigned order is float order), in every lane
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_iters += __shfl_xor_sync(kFull, my_iters, o);
        const unsigned t = __shfl_xor_sync(kFull, my_smax, o);
        my_smax = t > my_smax ? t : my_smax;
    }
    return make_uint2(my_iters, my_smax);
}

// the counters of NnlsArgs from per-warp totals: one atomic per warp
__device__ __forceinline__ void flush_warp_counters(const NnlsArgs &a, uint2 t)
{
    if ((threadIdx.x & 31) == 0) {
        if (a.iter_total && t.x)
            atomicAdd(a.iter_total, (unsigned long long)t.x);
        if (a.s_final_max && t.y)
            atomicMax(a.s_final_max, t.y);
    }
}

template <int G, int J>
__global__ void __launch_bounds__(kWarps * 32, min_ctas<J>()) k_nnls(const NnlsArgs a)
{
    constexpr int RP = Map<G, J>::RP;
    extern __shared__ __align__(16) float smem[];
    float *Qs = smem;                     // RP x RP
    float *sd = Qs + RP * RP;             // scale d
    // a dependent launch (the next half-step's cross term) may start on SMs
    // this grid leaves and stream the data matrix, which no NQP writes; it
    // waits for this grid to finish before it reads the packed factor.  The
    // grid is resident at once (at most the CTAs per SM that fit), so its
    // CTAs never wait for SMs the dependent holds.
    pdl_trigger();
    if (!stage_qt<G, J>(a.Qt, a.d, a.r, Qs, sd, a.status))
        return;
    // this CTA's rows: a balanced contiguous range; warp w takes runs of
    // 32 / G rows (one per group) at lo + w * 32 / G, every kWarps runs
    constexpr int NG = 32 / G;
    const int warp = threadIdx.x >> 5;
    const int64_t lo = (int64_t)blockIdx.x * a.rows / gridDim.x;
    const int64_t hi = (int64_t)(blockIdx.x + 1) * a.rows / gridDim.x;
    const uint2 t = nnls_rows<G, J>(a, Qs, sd, sd + RP, lo + (int64_t)warp * NG,
                                    (int64_t)kWarps * NG, hi, NG);
    // one atomic per CTA on each counter (all rows of a launch would
    // otherwise queue on the same two addresses)
    __shared__ uint2 wt[kWarps];
    if ((threadIdx.x & 31) == 0)
        wt[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint2 c = wt[0];
        for (int w = 1; w < kWarps; ++w) {
            c.x += wt[w].x;
            c.y = wt[w].y > c.y ? wt[w].y : c.y;
        }
        flush_warp_counters(a, c);
    }
    // epilogue: this CTA's rows of the solved factor into Gram partial
    // `blockIdx.x` and the packed operand of the next cross term (they are
    // in memory: written by this CTA before the barrier above)
    if constexpr (has_prep_epilogue<G, J>()) {
        if (a.gram_P) {
            constexpr int NBE = prep_detail::stage_cols(RP);
            float(*Xs)[NBE + 1] = reinterpret_cast<float(*)[NBE + 1]>(
                smem + RP * RP + RP + pool_floats<G, J>());
            PrepArgs pa{};
            pa.X = a.X;
            pa.rows = a.rows;
            pa.r = a.r;
            pa.P = a.gram_P;
            pa.pack_mode = a.pack_mode;
            pa.pack = a.pack;
            pa.npad = a.npad;
            pa.kp = a.kp;
            prep_detail::gram_pack_rows<NBE>(pa, Xs, lo, hi, blockIdx.x);
            // CTA 0 zeroes the pack's k padding (columns rows .. kp-1)
            if (blockIdx.x == 0 && a.pack_mode >= 0)
                prep_detail::zero_pack_padding(pa);
        }
    }
}

template <int G, int J>
struct Cfg {
    static int blocks_per_sm, sms;
};
template <int G, int J>
int Cfg<G, J>::blocks_per_sm = -1;
template <int G, int J>
int Cfg<G, J>::sms = 0;

// one-time launch configuration (kept out of any stream capture)
template <int G, int J>
cudaError_t prepare()
{
    const size_t smem = smem_bytes<G, J>();
    int &bps = Cfg<G, J>::blocks_per_sm, &sms = Cfg<G, J>::sms;
    if (bps < 0) {
        cudaError_t e = cudaFuncSetAttribute(k_nnls<G, J>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_nnls<G, J>, kWarps * 32, smem);
        if (e != cudaSuccess)
            return e;
        if (bps < 1)
            bps = 1;
    }
    return cudaSuccess;
}

// Grid of the standalone solver: sms * k CTAs (k <= the CTAs per SM that fit)
// over balanced contiguous row ranges.  The groups of a warp run in lockstep,
// so a warp costs its SM the same issue slots with one busy group as with
// all of them: with w = ceil(rows per CTA / rows per warp) warp-rounds per
// CTA, the busiest SM issues k w warp-rounds (what bounds an issue-bound
// launch) and a warp runs ceil(w / kWarps) rounds in sequence (what bounds a
// latency-bound one).  One round of the dependent chain of Alg. 3's steps
// is taken as worth kLatRounds warp-rounds of issue; the smallest maximum of
// the two wins, then the fewer warp-rounds, then the larger k.
constexpr int64_t kLatRounds = 8;

inline int nnls_grid(int64_t rows, int NG, int sms, int bps)
{
    int best_k = 1;
    int64_t best_cost = -1, best_wr = 0;
    for (int k = 1; k <= bps; ++k) {
        const int64_t g = (int64_t)sms * k;
        const int64_t rpc = (rows + g - 1) / g;
        const int64_t w = (rpc + NG - 1) / NG;
        const int64_t wr = k * w, rounds = (w + kWarps - 1) / kWarps;
        const int64_t cost = wr > kLatRounds * rounds ? wr : kLatRounds * rounds;
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && wr <= best_wr)) {
            best_k = k;
            best_cost = cost;
            best_wr = wr;
        }
    }
    const int64_t g = (int64_t)sms * best_k;
    return (int)(rows < g ? rows : g);
}

template <int G, int J>
cudaError_t launch(const NnlsArgs &a, cudaStream_t s)
{
    cudaError_t e = prepare<G, J>();
    if (e != cudaSuccess)
        return e;
    int grid = nnls_grid(a.rows, 32 / G, Cfg<G, J>::sms, Cfg<G, J>::blocks_per_sm);
    if (a.gram_P) {
        if (!has_prep_epilogue<G, J>() || a.gram_smax < 1)
            return cudaErrorInvalidValue;
        grid = grid < a.gram_smax ? grid : a.gram_smax;
    }
    if (a.grid_out)
        *a.grid_out = grid;
    if (grid < 1 || a.grid_query)
        return cudaSuccess;
    // an ordinary launch: started early beside the tensor-core kernel's tail
    // this latency-bound kernel measured slower, not faster
    k_nnls<G, J><<<grid, kWarps * 32, smem_bytes<G, J>(), s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// all lane counts for one J
template <int J>
cudaError_t dispatch(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s)
{
    switch (G) {
    case 1: return prep_only ? prepare<1, J>() : launch<1, J>(a, s);
    case 2: return prep_only ? prepare<2, J>() : launch<2, J>(a, s);
    case 4: return prep_only ? prepare<4, J>() : launch<4, J>(a, s);
    case 8: return prep_only ? prepare<8, J>() : launch<8, J>(a, s);
    case 16: return prep_only ? prepare<16, J>() : launch<16, J>(a, s);
    case 32: return prep_only ? prepare<32, J>() : launch<32, J>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace nnls_detail

// per-J entry points (one translation unit each)
cudaError_t nnls_dispatch_j2(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s);
cudaError_t nnls_dispatch_j4(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s);
cudaError_t nnls_dispatch_j8(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s);
cudaError_t nnls_dispatch_j16(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s);

}  // namespace nmfi
