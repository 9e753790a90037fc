// One-pass alternating solve with V streamed in row chunks (Alg. 2 as the
// paper writes it, §3.3): the E-step solves the coefficient rows chunk by
// chunk and, while a chunk of V is on the device, adds its contributions
// Y += F_i V_i^T (here C_H += V_b^T W_b) and H += F_i F_i^T (G_W += W_b^T W_b)
// to the M-step's inputs, so every outer iteration reads V exactly once.
//
// V may live in host memory (the limited-internal-memory mode of §1 and
// Table 1: device memory holds kBufs chunk buffers of V, the factors and
// O(r (r + n)) of M-step state per chunk; chunks arrive over NVLink-C2C on a
// copy stream) or in device memory (then the C_H contribution re-reads the
// chunk the W cross term just streamed, from L2).  Per chunk b (rows
// [i0, i1) of V), on worker stream b % kWorkers:
//   C_W,b = V_b Ht       tensor-core cross term (CUDA cores if unaligned)
//   W_b <- Alg. 3        batched NQPs against Qt_W, d_W
//   G_W,b = W_b^T W_b    Gram partial slices of the chunk
//   C_H,b = V_b^T W_b    tensor cores on a transposed copy of the chunk (it
//                        stays in L2: V_b is read from HBM or C2C once), or
//                        CUDA cores reading along V_b's rows when the chunk's
//                        row count is not a multiple of 4
// The chunks are independent problems (Alg. 2's parallel loop), so they run
// side by side; the main stream then sums the C_H,b and the G_W partials in
// chunk order (the result does not depend on which chunk finished first),
// forms Q_H = G_W + b_h I, Qt_H, d_H, solves every row of Ht against C_H,
// forms G_H = Ht^T Ht for the next W-update and J by the FP64 trace identity.
#include <algorithm>
#include <vector>

#include "handle.cuh"

using namespace nmfi;

namespace {

constexpr int kWorkers = 4;   // chunks in flight
constexpr int kBufs = 5;      // chunk buffers of V in host mode (workers + the next copy)

__global__ void k_sum_doubles(const double *x, int n, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            s += x[i];
        *out = s;
    }
}

// events and streams of one call, destroyed on every return path
struct Streams {
    cudaStream_t w[kWorkers] = {};
    cudaStream_t copy = nullptr;
    std::vector<cudaEvent_t> ev;
    ~Streams()
    {
        for (cudaEvent_t e : ev)
            cudaEventDestroy(e);
        for (cudaStream_t s : w)
            if (s)
                cudaStreamDestroy(s);
        if (copy)
            cudaStreamDestroy(copy);
    }
    cudaError_t event(cudaEvent_t *e, bool timing = false)
    {
        cudaError_t r = cudaEventCreateWithFlags(e, timing ? cudaEventDefault
                                                           : cudaEventDisableTiming);
        if (r == cudaSuccess)
            ev.push_back(*e);
        return r;
    }
};

}  // namespace

NMF_API nmf_status nmf_solve_streamed(nmf_handle h, const nmf_dense *V, int r, float *W,
                                      float *Ht, const nmf_solve_opts *opts, int64_t chunk_rows,
                                      nmf_report *rep)
{
    if (!h || !V || !V->data || !W || !Ht || !opts)
        return NMF_E_ARG;
    if (bad_r(r))
        return NMF_E_SHAPE;
    const int64_t m = V->rows, n = V->cols;
    if (m < 1 || n < 1 || V->ld != n || chunk_rows < 1 || opts->outer_iters < 0)
        return NMF_E_SHAPE;
    if (V->dt != NMF_F32)
        return NMF_E_DTYPE;
    if (opts->prec != NMF_PREC_FP32 && opts->prec != NMF_PREC_FP32_SIMT)
        return NMF_E_NOTIMPL;
    nmf_nnls_opts nn = opts_or_default(&opts->nnls);
    if (nn.maxstop_mode != 0 || nn.grad_refresh < 0)
        return NMF_E_NOTIMPL;
    {
        int lg = 0, lj = 0;
        if (!nnls_layout(r, nn.lanes, &lg, &lj))
            return NMF_E_ARG;
    }
    CK(cudaSetDevice(h->device));
    if (is_host_ptr(W) || is_host_ptr(Ht))
        return NMF_E_ARG;   // the factors stay on the device
    const bool host_v = is_host_ptr(V->data);
    const int64_t cr = std::min(chunk_rows, m);
    const int nchunks = (int)((m + cr - 1) / cr);
    // chunk cross terms on tensor cores when the rows allow TMA (chunk buffers
    // and chunk starts are 16-byte aligned when n % 4 == 0)
    const int mode = (opts->prec == NMF_PREC_FP32 && n % 4 == 0 &&
                      (host_v || tc_supported(n, TC_TF32X3, V->data)))
                         ? TC_TF32X3 : -1;
    // ---- workspace
    int max_slices = 1, max_tslices = 1, gw_slices = 0;
    std::vector<TcPlan> plans(nchunks), tplans(nchunks);
    std::vector<int> gsl(nchunks), csl(nchunks), goff(nchunks), tsl(nchunks);
    std::vector<char> ttc(nchunks, 0);   // C_H,b on tensor cores
    for (int b = 0; b < nchunks; ++b) {
        const int64_t rows = std::min(cr, m - (int64_t)b * cr);
        if (mode >= 0) {
            plans[b] = tc_plan(rows, n, r, mode);
            csl[b] = plans[b].nslices;
        } else {
            csl[b] = cross_splits(rows, n);
        }
        ttc[b] = mode >= 0 && rows % 4 == 0;
        if (ttc[b]) {
            tplans[b] = tc_plan(n, rows, r, mode);
            tsl[b] = tplans[b].nslices;
        } else {
            tsl[b] = cross_splits(n, rows);
        }
        max_slices = std::max(max_slices, csl[b]);
        max_tslices = std::max(max_tslices, tsl[b]);
        gsl[b] = gram_splits(rows);
        goff[b] = gw_slices;
        gw_slices += gsl[b];
    }
    const int gh_slices = gram_splits(n);
    const int nbufs = host_v ? std::min(kBufs, nchunks + 1) : 0;
    Sizer z;
    for (int k = 0; k < nbufs; ++k)
        z.add<float>((size_t)cr * n);
    z.add<char>(mode >= 0 ? tc_pack_bytes(n, r, mode) : 16);
    const size_t wpack = mode >= 0 ? tc_pack_bytes(cr, r, mode) : 16;
    for (int w = 0; w < kWorkers; ++w) {
        z.add<float>((size_t)max_slices * cr * r);
        z.add<float>((size_t)max_tslices * n * r);
        z.add<float>(mode >= 0 ? (size_t)cr * n : 4);   // V_b^T
        z.add<char>(wpack);                               // packed W_b
    }
    z.add<float>((size_t)nchunks * n * r);
    z.add<float>((size_t)n * r);
    z.add<float>((size_t)gw_slices * r * r);
    z.add<float>((size_t)gh_slices * r * r);
    for (int i = 0; i < 5; ++i)
        z.add<float>((size_t)r * r);   // Gw, Gh, Qt_W, Qt_H and spare
    z.add<float>(r);
    z.add<float>(r);
    z.add<double>(nchunks);
    z.add<double>(1);
    nmf_status st = ensure_ws(h, z.off);
    if (st)
        return st;
    Arena a(h->ws, h->ws_cap);
    float *vb[kBufs] = {};
    for (int k = 0; k < nbufs; ++k)
        vb[k] = a.take<float>((size_t)cr * n);
    void *pack = a.take<char>(mode >= 0 ? tc_pack_bytes(n, r, mode) : 16);
    float *Pc[kWorkers], *Pt[kWorkers], *VbT[kWorkers];
    void *packW[kWorkers];
    for (int w = 0; w < kWorkers; ++w) {
        Pc[w] = a.take<float>((size_t)max_slices * cr * r);
        Pt[w] = a.take<float>((size_t)max_tslices * n * r);
        VbT[w] = a.take<float>(mode >= 0 ? (size_t)cr * n : 4);
        packW[w] = a.take<char>(wpack);
    }
    float *CHb = a.take<float>((size_t)nchunks * n * r);   // C_H,b of every chunk
    float *CH = a.take<float>((size_t)n * r);
    float *Pgw = a.take<float>((size_t)gw_slices * r * r);
    float *Pgh = a.take<float>((size_t)gh_slices * r * r);
    float *Gw = a.take<float>((size_t)r * r);
    float *Gh = a.take<float>((size_t)r * r);
    float *QtW = a.take<float>((size_t)r * r);
    float *QtH = a.take<float>((size_t)r * r);
    (void)a.take<float>((size_t)r * r);
    float *dW = a.take<float>(r);
    float *dH = a.take<float>(r);
    double *vvb = a.take<double>(nchunks);
    double *Jd = a.take<double>(1);
    CK(prepare_nnls(r, nn.lanes));

    cudaStream_t s = h->stream;
    Streams S;
    for (int w = 0; w < kWorkers; ++w)
        CK(cudaStreamCreateWithFlags(&S.w[w], cudaStreamNonBlocking));
    if (host_v)
        CK(cudaStreamCreateWithFlags(&S.copy, cudaStreamNonBlocking));
    cudaEvent_t e0, e1, ready;
    CK(S.event(&e0, true));
    CK(S.event(&e1, true));
    CK(S.event(&ready));
    cudaEvent_t copied[kBufs] = {}, freed[kBufs] = {}, wdone[kWorkers] = {};
    for (int k = 0; k < nbufs; ++k) {
        CK(S.event(&copied[k]));
        CK(S.event(&freed[k]));
    }
    for (int w = 0; w < kWorkers; ++w)
        CK(S.event(&wdone[w]));

    const float *Vh = static_cast<const float *>(V->data);
    // chunk c of the whole solve (the sum-of-squares pass, then every outer
    // iteration's pass) uses buffer c % nbufs; copies run up to nbufs ahead
    int64_t issued = 0, started = 0;
    const int64_t total_chunks = (int64_t)nchunks * (opts->outer_iters + 1);
    auto issue_copies = [&]() -> cudaError_t {
        while (host_v && issued < total_chunks && issued < started + nbufs) {
            const int k = (int)(issued % nbufs);
            const int b = (int)(issued % nchunks);
            const int64_t i0 = (int64_t)b * cr, rows = std::min(cr, m - i0);
            cudaError_t e = cudaSuccess;
            if (issued >= nbufs)
                e = cudaStreamWaitEvent(S.copy, freed[k], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(vb[k], Vh + i0 * n, sizeof(float) * rows * n,
                                    cudaMemcpyHostToDevice, S.copy);
            if (e == cudaSuccess)
                e = cudaEventRecord(copied[k], S.copy);
            if (e != cudaSuccess)
                return e;
            ++issued;
        }
        return cudaSuccess;
    };
    // the device address of the next chunk on stream `ws` (after its copy)
    auto begin_chunk = [&](int b, cudaStream_t ws) -> const float * {
        if (!host_v)
            return Vh + (int64_t)b * cr * n;
        const int k = (int)(started % nbufs);
        cudaStreamWaitEvent(ws, copied[k], 0);
        return vb[k];
    };
    auto end_chunk = [&](cudaStream_t ws) -> cudaError_t {
        if (!host_v)
            return cudaSuccess;
        const int k = (int)(started % nbufs);
        ++started;
        cudaError_t e = cudaEventRecord(freed[k], ws);
        return e == cudaSuccess ? issue_copies() : e;
    };
    CK(cudaMemsetAsync(h->ctr, 0, sizeof(unsigned long long), s));
    CK(issue_copies());
    // ||V||^2, chunk by chunk on the main stream (one extra pass per solve)
    for (int b = 0; b < nchunks; ++b) {
        const int64_t rows = std::min(cr, m - (int64_t)b * cr);
        const float *Vb = begin_chunk(b, s);
        CK(cudaMemsetAsync(h->tickets + 3, 0, sizeof(unsigned), s));
        CK(launch_sumsq(Vb, NMF_F32, rows * n, vvb + b, h->partials, h->tickets + 3, s));
        CK(end_chunk(s));
    }
    double *vv_dev = h->scal + 12;
    k_sum_doubles<<<1, 32, 0, s>>>(vvb, nchunks, vv_dev);
    count_launch();
    CK(cudaGetLastError());
    double vv = 0.0;
    CK(cudaMemcpyAsync(&vv, vv_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    auto nnls_args = [&](const float *Qt, const float *d, const float *C, int nsplit,
                         int64_t rows, float alpha, float *X) {
        NnlsArgs na{};
        na.Qt = Qt;
        na.d = d;
        na.C = C;
        na.nsplit = nsplit;
        na.c_stride = rows * r;
        na.rows = rows;
        na.r = r;
        na.alpha = alpha;
        na.X = X;
        na.max_inner = nn.max_inner;
        na.eps = (float)nn.eps;
        na.cd_steps = nn.cd_steps;
        na.lanes = nn.lanes;
        na.grad_refresh = nn.grad_refresh;
        na.iter_total = h->ctr;
        na.status = h->status;
        return na;
    };

    // G_H of the initial Ht
    CK(launch_gram_partial(Ht, n, r, r, Pgh, gh_slices, s));
    CK(launch_rescale(Pgh, gh_slices, r, 0.f, Gh, nullptr, nullptr, nullptr, s));
    CK(cudaEventRecord(e0, s));
    int t = 0;
    double J = 0.0;
    for (; t < opts->outer_iters; ++t) {
        // ---- W-update: Q_W = G_H + b_w I, the packed Ht; then the chunks
        CK(launch_rescale(Gh, 1, r, opts->beta_w, nullptr, nullptr, QtW, dW, s));
        if (mode >= 0)
            CK(launch_tc_pack(Ht, n, r, mode, pack, s));
        CK(cudaEventRecord(ready, s));
        for (int w = 0; w < kWorkers; ++w)
            CK(cudaStreamWaitEvent(S.w[w], ready, 0));
        for (int b = 0; b < nchunks; ++b) {
            const int w = b % kWorkers;
            cudaStream_t ws = S.w[w];
            const int64_t i0 = (int64_t)b * cr, rows = std::min(cr, m - i0);
            const float *Vb = begin_chunk(b, ws);
            if (mode >= 0)
                CK(launch_tc_cross(Vb, rows, n, n, r, mode, pack, Pc[w], plans[b], h->status, ws));
            else
                CK(launch_cross_dense_f32(Vb, rows, n, n, Ht, r, Pc[w], csl[b], ws));
            const NnlsArgs na = nnls_args(QtW, dW, Pc[w], csl[b], rows, opts->alpha_w, W + i0 * r);
            CK(launch_nnls(na, ws));
            // the M-step's inputs from this chunk while it is on the device
            CK(launch_gram_partial(W + i0 * r, rows, r, r, Pgw + (size_t)goff[b] * r * r, gsl[b],
                                   ws));
            if (ttc[b]) {
                CK(launch_transpose_f32(Vb, rows, n, n, VbT[w], ws));
                CK(launch_tc_pack(W + i0 * r, rows, r, mode, packW[w], ws));
                CK(launch_tc_cross(VbT[w], n, rows, rows, r, mode, packW[w], Pt[w], tplans[b],
                                   h->status, ws));
            } else {
                CK(launch_cross_dense_f32(Vb, n, rows, n, W + i0 * r, r, Pt[w], tsl[b], ws,
                                          true));
            }
            CK(launch_sum_slices(Pt[w], tsl[b], n * r, CHb + (size_t)b * n * r, ws));
            CK(end_chunk(ws));
        }
        for (int w = 0; w < kWorkers; ++w) {
            CK(cudaEventRecord(wdone[w], S.w[w]));
            CK(cudaStreamWaitEvent(s, wdone[w], 0));
        }
        // ---- H-update: C_H and G_W summed in chunk order; Q_H = G_W + b_h I
        CK(launch_sum_slices(CHb, nchunks, n * r, CH, s));
        CK(launch_rescale(Pgw, gw_slices, r, opts->beta_h, Gw, nullptr, QtH, dH, s));
        CK(launch_nnls(nnls_args(QtH, dH, CH, 1, n, opts->alpha_h, Ht), s));
        CK(launch_gram_partial(Ht, n, r, r, Pgh, gh_slices, s));
        CK(launch_rescale(Pgh, gh_slices, r, 0.f, Gh, nullptr, nullptr, nullptr, s));
        // ---- J by the FP64 trace identity (C_H = V^T W of the new W)
        if (opts->obj_hist || opts->rel_gap_target > 0.0 || t + 1 == opts->outer_iters) {
            CK(cudaMemsetAsync(h->tickets + 0, 0, sizeof(unsigned), s));
            ObjArgs oa{};
            oa.vv = vv;
            oa.W = W;
            oa.m = m;
            oa.Ht = Ht;
            oa.n = n;
            oa.r = r;
            oa.Ch = CH;
            oa.nsplit = 1;
            oa.ch_stride = n * r;
            oa.Gw = Gw;
            oa.Gh = Gh;
            oa.aw = opts->alpha_w;
            oa.ah = opts->alpha_h;
            oa.bw = opts->beta_w;
            oa.bh = opts->beta_h;
            oa.J = Jd;
            oa.partials = h->partials;
            oa.ticket = h->tickets + 0;
            CK(launch_objective(oa, s));
            CK(cudaMemcpyAsync(&J, Jd, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (opts->obj_hist)
                opts->obj_hist[t] = J;
            if (opts->rel_gap_target > 0.0 && opts->f_star > 0.0 &&
                (J - opts->f_star) / opts->f_star <= opts->rel_gap_target) {
                ++t;
                break;
            }
        }
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaStreamSynchronize(s));
    if (host_v)
        CK(cudaStreamSynchronize(S.copy));   // copies issued ahead of the last chunks
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long inner = 0;
    CK(cudaMemcpy(&inner, h->ctr, sizeof(inner), cudaMemcpyDeviceToHost));
    if (rep) {
        *rep = nmf_report{};
        rep->iters_done = t;
        rep->objective = J;
        rep->rel_gap = opts->f_star > 0.0 ? (J - opts->f_star) / opts->f_star : 0.0;
        rep->inner_total = (int64_t)inner;
        rep->kbar = t > 0 ? (double)inner / ((double)t * (double)(m + n)) : 0.0;
        rep->ms_total = ms;
    }
    return nmf_sync(h);
}
