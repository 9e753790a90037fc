// C ABI of libnmf.so: handle, workspace, argument checks and the host side of
// the alternating loop (Alg. 1 / Alg. 2).  Every arithmetic step runs in the
// kernels of the other translation units; this file only validates,
// allocates workspace once, and enqueues launches on the handle's stream.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

#include "handle.cuh"

using namespace nmfi;

namespace nmfi {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool fault_armed(const char *site)
{
    const char *env = getenv("NMF_FAULT");
    if (!env || !site || !*site)
        return false;
    const size_t n = strlen(site);
    for (const char *p = env; *p;) {
        const char *q = strchr(p, ',');
        const size_t len = q ? (size_t)(q - p) : strlen(p);
        if (len == n && strncmp(p, site, n) == 0)
            return true;
        if (!q)
            break;
        p = q + 1;
    }
    return false;
}

// ---- profiler: pairs of events per kernel class --------------------------
namespace {
struct Prof {
    bool on = false;
    int suspended = 0;
    std::vector<cudaEvent_t> pool;     // reusable events
    size_t used = 0;
    struct Pair { int cls; cudaEvent_t b, e; };
    std::vector<Pair> pairs;
    std::vector<int> open_cls;         // stack of classes with a begin pending
    std::vector<cudaEvent_t> open_ev;
    double ms[KC_COUNT] = {0};
    long long n[KC_COUNT] = {0};
    cudaEvent_t get()
    {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess)
                return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void drain()
    {
        for (auto &p : pairs) {
            float t = 0.f;
            if (cudaEventSynchronize(p.e) == cudaSuccess &&
                cudaEventElapsedTime(&t, p.b, p.e) == cudaSuccess) {
                ms[p.cls] += t;
                n[p.cls] += 1;
            }
        }
        pairs.clear();
        used = 0;
    }
};
Prof g_prof;
}  // namespace

thread_local bool tl_prof_off = false;

void prof_suspend(bool on) { g_prof.suspended += on ? 1 : -1; }
void prof_thread_off() { tl_prof_off = true; }
bool prof_thread_set_off(bool off)
{
    const bool was = tl_prof_off;
    tl_prof_off = off;
    return was;
}

void prof_mark(int cls, cudaStream_t s, bool begin)
{
    Prof &P = g_prof;
    if (!P.on || P.suspended > 0 || tl_prof_off)
        return;
    if (begin) {
        if (P.used + 2 > 4096)
            P.drain();   // bound the number of live events
        cudaEvent_t e = P.get();
        if (!e)
            return;
        cudaEventRecord(e, s);
        P.open_cls.push_back(cls);
        P.open_ev.push_back(e);
    } else {
        if (P.open_ev.empty())
            return;
        cudaEvent_t b = P.open_ev.back();
        int c = P.open_cls.back();
        P.open_ev.pop_back();
        P.open_cls.pop_back();
        cudaEvent_t e = P.get();
        if (!e)
            return;
        cudaEventRecord(e, s);
        // nested scopes (a launcher calling another) count once, outermost
        if (P.open_ev.empty())
            P.pairs.push_back({c, b, e});
    }
}
}  // namespace nmfi

NMF_API nmf_status nmf_profile_enable(int enable)
{
    Prof &P = g_prof;
    if (enable) {
        P.drain();
        for (int c = 0; c < KC_COUNT; ++c) {
            P.ms[c] = 0.0;
            P.n[c] = 0;
        }
        P.on = true;
    } else {
        P.on = false;
    }
    return NMF_OK;
}

NMF_API nmf_status nmf_profile_read(int kclass, double *ms_total, int64_t *launches)
{
    if (kclass < 0 || kclass >= KC_COUNT || !ms_total || !launches)
        return NMF_E_ARG;
    g_prof.drain();
    *ms_total = g_prof.ms[kclass];
    *launches = g_prof.n[kclass];
    return NMF_OK;
}

// ---------------------------------------------------------------------------
// handle and workspace
// ---------------------------------------------------------------------------
namespace nmfi {

nmf_status ensure_ws(nmf_handle h, size_t bytes)
{
    if (bytes <= h->ws_cap)
        return NMF_OK;
    if (fault_armed("alloc"))
        return NMF_E_NOMEM;
    CK(cudaStreamSynchronize(h->stream));
    if (h->ws)
        cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_cap = 0;
    size_t cap = bytes + (bytes >> 3) + (1 << 20);
    if (cudaMalloc(&h->ws, cap) != cudaSuccess) {
        cudaGetLastError();
        return NMF_E_NOMEM;
    }
    h->ws_cap = cap;
    return NMF_OK;
}

nmf_nnls_opts opts_or_default(const nmf_nnls_opts *o)
{
    nmf_nnls_opts d;
    nmf_nnls_opts_default(&d);
    if (!o)
        return d;
    nmf_nnls_opts r = *o;
    if (r.max_inner <= 0)
        r.max_inner = d.max_inner;
    if (!(r.eps >= 0.0))
        r.eps = d.eps;
    return r;
}

bool bad_r(int r) { return r < 1 || r > kMaxRank; }

bool is_host_ptr(const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace nmfi

namespace {

nmf_status ensure_stage(nmf_handle h, size_t bytes)
{
    if (bytes <= h->stage_cap)
        return NMF_OK;
    CK(cudaStreamSynchronize(h->stream));
    if (h->stage)
        cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_cap = 0;
    if (cudaMalloc(&h->stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        return NMF_E_NOMEM;
    }
    h->stage_cap = bytes;
    return NMF_OK;
}

}  // namespace

NMF_API const char *nmf_status_string(nmf_status s)
{
    switch (s) {
    case NMF_OK: return "ok";
    case NMF_E_ARG: return "invalid argument";
    case NMF_E_SHAPE: return "invalid shape";
    case NMF_E_DTYPE: return "unsupported dtype";
    case NMF_E_NOMEM: return "out of device memory";
    case NMF_E_CUDA: return "CUDA error";
    case NMF_E_NONFINITE: return "non-finite input";
    case NMF_E_TIMEOUT: return "device wait timed out";
    case NMF_E_BUSY: return "admission refused";
    case NMF_E_NOTIMPL: return "not implemented";
    }
    return "unknown status";
}

NMF_API void nmf_nnls_opts_default(nmf_nnls_opts *o)
{
    if (!o)
        return;
    o->max_inner = 50;
    o->eps = 1e-3;
    o->cd_steps = -1;
    o->maxstop_mode = 0;
    o->maxstop = 0.f;
    o->lanes = 0;
    o->grad_refresh = 0;
}

NMF_API int64_t nmf_launch_count(void) { return g_launches.load(); }

NMF_API int nmf_fault_armed(const char *site) { return fault_armed(site) ? 1 : 0; }

NMF_API nmf_status nmf_create(nmf_handle *out, int device, void *cuda_stream)
{
    if (!out)
        return NMF_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return NMF_E_CUDA;
    }
    CK(cudaSetDevice(device));
    nmf_ctx *h = new nmf_ctx;
    h->device = device;
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    char *aux = nullptr;
    const size_t aux_bytes = 64 * 1024;
    if (cudaMalloc(&aux, aux_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return NMF_E_NOMEM;
    }
    cudaMemset(aux, 0, aux_bytes);
    Arena a(aux, aux_bytes);
    h->status = a.take<unsigned>(4);
    h->tickets = a.take<unsigned>(8);
    h->partials = a.take<double>(3 * 1024);
    h->scal = a.take<double>(16);
    h->ctr = a.take<unsigned long long>(4);
    h->idev = a.take<int>(4);
    h->smax = a.take<unsigned>(4);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(aux);
        delete h;
        return NMF_E_CUDA;
    }
    *out = h;
    return NMF_OK;
}

NMF_API nmf_status nmf_destroy(nmf_handle h)
{
    if (!h)
        return NMF_E_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->ws)
        cudaFree(h->ws);
    if (h->cap)
        cudaStreamDestroy(h->cap);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->ev_fork)
        cudaEventDestroy(h->ev_fork);
    if (h->ev_join)
        cudaEventDestroy(h->ev_join);
    if (h->stage)
        cudaFree(h->stage);
    cudaFree(h->status);   // first allocation of the aux block
    delete h;
    return NMF_OK;
}

NMF_API nmf_status nmf_set_stream(nmf_handle h, void *cuda_stream)
{
    if (!h)
        return NMF_E_ARG;
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return NMF_OK;
}

NMF_API nmf_status nmf_sync(nmf_handle h)
{
    if (!h)
        return NMF_E_ARG;
    CK(cudaStreamSynchronize(h->stream));
    unsigned st = 0;
    CK(cudaMemcpy(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemset(h->status, 0, sizeof(unsigned)));
        if (st & kStTimeout)
            return NMF_E_TIMEOUT;
        if (st & kStBadInput)
            return NMF_E_ARG;
        return NMF_E_NONFINITE;
    }
    return NMF_OK;
}

// ---------------------------------------------------------------------------
// single steps
// ---------------------------------------------------------------------------
namespace {

// Gram into G (r x r, no beta) through `ws`; returns the reduced result in G.
nmf_status gram_into(nmf_handle h, const float *X, int64_t rows, int64_t ld, int r,
                     nmf_prec prec, float *P, int S, float *G)
{
    const int mode = prec == NMF_PREC_TF32 ? GM_TF32 : prec == NMF_PREC_BF16 ? GM_BF16
                     : prec == NMF_PREC_BF16X2 ? GM_BF16X2 : GM_FP32;
    CK(launch_gram_partial(X, rows, ld, r, P, S, h->stream, mode));
    CK(launch_sum_slices(P, S, (int64_t)r * r, G, h->stream));
    return NMF_OK;
}

}  // namespace

NMF_API nmf_status nmf_gram(nmf_handle h, const nmf_dense *X, float beta, nmf_prec prec, float *Q)
{
    if (!h || !X || !Q || (!X->data && X->rows > 0))
        return NMF_E_ARG;
    if (X->rows < 0 || bad_r((int)X->cols) || X->ld < X->cols)
        return NMF_E_SHAPE;
    if (X->dt != NMF_F32)
        return NMF_E_DTYPE;
    if (prec < NMF_PREC_FP32 || prec > NMF_PREC_FP32_SIMT)
        return NMF_E_ARG;
    const int r = (int)X->cols;
    const int S = gram_splits(X->rows);
    Sizer z;
    z.add<float>((size_t)S * r * r);
    z.add<float>((size_t)r * r);
    nmf_status st = ensure_ws(h, z.off);
    if (st)
        return st;
    Arena a(h->ws, h->ws_cap);
    float *P = a.take<float>((size_t)S * r * r);
    float *G = a.take<float>((size_t)r * r);
    st = gram_into(h, (const float *)X->data, X->rows, X->ld, r, prec, P, S, G);
    if (st)
        return st;
    CK(launch_rescale(G, 1, r, beta, nullptr, Q, nullptr, nullptr, h->stream));
    return NMF_OK;
}

NMF_API nmf_status nmf_cross(nmf_handle h, const nmf_matrix *V, const float *B, int r,
                             nmf_prec prec, float *C)
{
    if (!h || !V || !B || !C)
        return NMF_E_ARG;
    if (bad_r(r))
        return NMF_E_SHAPE;
    if (V->is_sparse) {
        const nmf_csr &s = V->s;
        if (s.rows < 0 || s.cols < 0 || s.nnz < 0 || !s.rowptr || (s.nnz > 0 && (!s.colidx || !s.vals)))
            return NMF_E_ARG;
        if (s.dt != NMF_F32 && s.dt != NMF_BF16)
            return NMF_E_DTYPE;
        SpmmPlan p = spmm_plan(s.rows, s.nnz);
        nmf_status st = ensure_ws(h, spmm_workspace_bytes(p, r) + 256);
        if (st)
            return st;
        CK(launch_spmm_csr(s.rowptr, s.colidx, s.vals, s.dt, s.rows, s.nnz, B, r, C, p, h->ws,
                           h->stream));
        return NMF_OK;
    }
    const nmf_dense &d = V->d;
    if (d.rows < 0 || d.cols < 0 || d.ld < d.cols || (!d.data && d.rows > 0))
        return NMF_E_SHAPE;
    int mode = -1;
    if (prec == NMF_PREC_BF16 || prec == NMF_PREC_BF16X2) {
        if (d.dt != NMF_BF16)
            return NMF_E_DTYPE;
        mode = prec == NMF_PREC_BF16 ? TC_BF16 : TC_BF16X2;
        if (!tc_supported(d.ld, mode, d.data))
            return NMF_E_SHAPE;
    } else if (prec == NMF_PREC_TF32 || prec == NMF_PREC_FP32 || prec == NMF_PREC_FP32_SIMT) {
        if (d.dt != NMF_F32)
            return NMF_E_DTYPE;
        const int want = prec == NMF_PREC_TF32 ? TC_TF32 : TC_TF32X3;
        if (prec != NMF_PREC_FP32_SIMT && tc_supported(d.ld, want, d.data))
            mode = want;
        else if (prec == NMF_PREC_TF32)
            return NMF_E_SHAPE;
    } else {
        return NMF_E_NOTIMPL;
    }
    if (mode >= 0) {
        if (d.rows == 0)
            return NMF_OK;
        const TcPlan pl = tc_plan(d.rows, d.cols, r, mode);
        Sizer z;
        z.add<char>(tc_pack_bytes(d.cols, r, mode));
        z.add<float>((size_t)pl.nslices * d.rows * r);
        nmf_status st = ensure_ws(h, z.off);
        if (st)
            return st;
        Arena a(h->ws, h->ws_cap);
        void *pack = a.take<char>(tc_pack_bytes(d.cols, r, mode));
        float *P = pl.nslices == 1 ? C : a.take<float>((size_t)pl.nslices * d.rows * r);
        CK(launch_tc_pack(B, d.cols, r, mode, pack, h->stream));
        CK(launch_tc_cross(d.data, d.rows, d.cols, d.ld, r, mode, pack, P, pl, h->status,
                           h->stream));
        if (pl.nslices > 1)
            CK(launch_sum_slices(P, pl.nslices, d.rows * r, C, h->stream));
        return NMF_OK;
    }
    const int S = cross_splits(d.rows, d.cols);
    if (S == 1) {
        CK(launch_cross_dense_f32((const float *)d.data, d.rows, d.cols, d.ld, B, r, C, 1,
                                  h->stream));
        return NMF_OK;
    }
    nmf_status st = ensure_ws(h, sizeof(float) * (size_t)S * d.rows * r + 256);
    if (st)
        return st;
    float *P = reinterpret_cast<float *>(h->ws);
    CK(launch_cross_dense_f32((const float *)d.data, d.rows, d.cols, d.ld, B, r, P, S, h->stream));
    CK(launch_sum_slices(P, S, d.rows * r, C, h->stream));
    return NMF_OK;
}

NMF_API nmf_status nmf_rescale(nmf_handle h, const float *Q, int r, float *Qt, float *d)
{
    if (!h || !Q || !Qt || !d)
        return NMF_E_ARG;
    if (bad_r(r))
        return NMF_E_SHAPE;
    CK(launch_rescale(Q, 1, r, 0.f, nullptr, nullptr, Qt, d, h->stream));
    return NMF_OK;
}

NMF_API nmf_status nmf_nnls_update(nmf_handle h, const float *Qt, const float *d, const float *C,
                                   int64_t rows, int r, float alpha, float *X,
                                   const nmf_nnls_opts *opts, int32_t *inner_iters)
{
    if (!h || !Qt || !d || (rows > 0 && (!C || !X)))
        return NMF_E_ARG;
    if (rows < 0 || bad_r(r))
        return NMF_E_SHAPE;
    nmf_nnls_opts o = opts_or_default(opts);
    if (o.maxstop_mode < 0 || o.maxstop_mode > 1 || o.grad_refresh < 0)
        return NMF_E_ARG;
    int lg = 0, lj = 0;
    if (!nnls_layout(r, o.lanes, &lg, &lj))
        return NMF_E_ARG;
    NnlsArgs a{};
    a.Qt = Qt;
    a.d = d;
    a.C = C;
    a.nsplit = 1;
    a.c_stride = rows * r;
    a.rows = rows;
    a.r = r;
    a.alpha = alpha;
    a.X = X;
    a.max_inner = o.max_inner;
    a.eps = (float)o.eps;
    a.cd_steps = o.cd_steps;
    a.maxstop_mode = o.maxstop_mode;
    a.maxstop = o.maxstop;
    a.lanes = o.lanes;
    a.grad_refresh = o.grad_refresh;
    a.iters = inner_iters;
    a.status = h->status;
    CK(launch_nnls(a, h->stream));
    return NMF_OK;
}

NMF_API nmf_status nmf_objective(nmf_handle h, double vv, const float *W, int64_t m,
                                 const float *Ht, int64_t n, int r, const float *Ch,
                                 const float *Gw, const float *Gh, float alpha_w, float alpha_h,
                                 float beta_w, float beta_h, double *J_dev)
{
    if (!h || !W || !Ht || !Ch || !Gw || !Gh || !J_dev)
        return NMF_E_ARG;
    if (m < 0 || n < 0 || bad_r(r))
        return NMF_E_SHAPE;
    ObjArgs a{};
    a.vv = vv;
    a.W = W;
    a.m = m;
    a.Ht = Ht;
    a.n = n;
    a.r = r;
    a.Ch = Ch;
    a.nsplit = 1;
    a.ch_stride = n * r;
    a.Gw = Gw;
    a.Gh = Gh;
    a.aw = alpha_w;
    a.ah = alpha_h;
    a.bw = beta_w;
    a.bh = beta_h;
    a.J = J_dev;
    a.partials = h->partials;
    a.ticket = h->tickets + 0;
    CK(launch_objective(a, h->stream));
    return NMF_OK;
}

NMF_API nmf_status nmf_objective_direct(nmf_handle h, const nmf_dense *V, const float *W,
                                        const float *Ht, int r, float alpha_w, float alpha_h,
                                        float beta_w, float beta_h, double *J_dev)
{
    if (!h || !V || !W || !Ht || !J_dev || !V->data)
        return NMF_E_ARG;
    if (V->rows <= 0 || V->cols <= 0 || V->ld < V->cols || bad_r(r))
        return NMF_E_SHAPE;
    if (V->dt != NMF_F32)
        return NMF_E_DTYPE;
    const size_t np = objective_direct_partials(V->rows, V->cols);
    nmf_status st = ensure_ws(h, sizeof(double) * np + 256);
    if (st)
        return st;
    ObjDirectArgs a{};
    a.V = (const float *)V->data;
    a.ldv = V->ld;
    a.W = W;
    a.m = V->rows;
    a.Ht = Ht;
    a.n = V->cols;
    a.r = r;
    a.aw = alpha_w;
    a.ah = alpha_h;
    a.bw = beta_w;
    a.bh = beta_h;
    a.J = J_dev;
    a.partials = reinterpret_cast<double *>(h->ws);
    a.ticket = h->tickets + 2;
    CK(launch_objective_direct(a, h->stream));
    return NMF_OK;
}

NMF_API nmf_status nmf_kkt(nmf_handle h, const float *Q, const float *C, int64_t rows, int r,
                           float alpha, const float *X, double *out_dev)
{
    if (!h || !Q || !out_dev || (rows > 0 && (!C || !X)))
        return NMF_E_ARG;
    if (rows < 0 || bad_r(r))
        return NMF_E_SHAPE;
    CK(launch_kkt(Q, C, rows, r, alpha, X, out_dev, h->stream));
    return NMF_OK;
}

// ---------------------------------------------------------------------------
// whole method
// ---------------------------------------------------------------------------
namespace {

struct HalfStep {
    // operand of the cross term: dense (A, lda) or CSR
    bool sparse;
    const float *A;
    int64_t lda, K;
    const nmf_csr *csr;
    SpmmPlan spplan;
    int64_t rows;       // number of NQPs (rows of the factor updated)
    float *X;           // factor updated (rows x r)
    const float *Xo;    // other factor (K x r)
    int64_t Ko;         // rows of the other factor
    float alpha, beta;
    float *Cs;          // cross slices
    int nsplit;
    float *Q;           // Q = G_other + beta I (kept for KKT)
    unsigned *ms_thr;   // maxStop mode 1: threshold of this update (float bits)
    unsigned *ms_out;   //   and the largest final ||f~||^2 of this update
    int tc_mode;        // -1: CUDA-core FP32 cross term
    const void *Atc;    // tensor-core operand (F32, or the BF16 copy)
    int64_t lda_tc;
    TcPlan plan;        // stream-K plan of the tensor-core cross term
    void *pack;         // packed other factor
    int lanes;          // NQP layout of this half-step (lanes per row)
};

struct Loop {
    int r;
    unsigned *ticket;   // last-CTA counter of the factor preparation
    float *Pg;          // Gram partial slices
    int Pg_slices;      // their capacity
    bool fuse_prep;     // the NQP kernel's epilogue writes the Gram partials
    bool overlap_prep;  // ... and their finishing launch runs beside the cross term
    bool overlap_full;  // no epilogue: the whole preparation runs beside a cross
                        // term that reads the other factor itself (CSR, CUDA cores)
    int S_w, S_h;       // with overlap_prep: partials of W (m rows) and Ht (n rows)
    int gS_w, gS_h;     // gram splits for W (m rows) and Ht (n rows)
    float *Gw, *Gh;     // Grams without beta
    float *Qt, *d;
    void *spws;         // SpMM carries
    HalfStep hw, hh;
    nmf_nnls_opts nn;
    double vv;
    bool direct_obj;
    const float *V; int64_t ldv;   // dense V for the direct objective
    double *obj_partials;
};

// The factor X just updated feeds the next half-step `next`: its Gram G,
// next.Q = G + beta I, the rescaled Qt, d (Alg. 3) and the packed operand of
// next's tensor-core cross term, in one launch.
PrepArgs prep_args(Loop &L, const float *X, int64_t rows, float *G, HalfStep &next)
{
    PrepArgs a{};
    a.X = X;
    a.rows = rows;
    a.r = L.r;
    a.beta = next.beta;
    a.P = L.Pg;
    a.ticket = L.ticket;
    a.G = G;
    a.Q = next.Q;
    a.Qt = L.Qt;
    a.d = L.d;
    a.pack_mode = next.tc_mode;
    a.pack = next.pack;
    if (next.tc_mode >= 0) {
        a.npad = tc_npad(L.r);
        a.kp = tc_kpad(rows, next.tc_mode);
    }
    return a;
}

// The finishing launch of the half-step `s`'s own preparation: G_other,
// s.Q, Qt, d from the Gram partials of its other factor (the packed operand
// is already in place, its padding zeroed by the epilogue that packed it).
PrepArgs finish_args(Loop &L, HalfStep &s, float *G_other)
{
    PrepArgs a = prep_args(L, s.Xo, s.Ko, G_other, s);
    a.pack_mode = -1;
    return a;
}

constexpr int kSideCtas = 8;   // SMs the cross term leaves to the finishing launch

// One half-step: the cross term C = V X_other, every row's NQP (Alg. 3),
// and the preparation of the solved factor for the half-step `next` (Gram G,
// Q, Qt, d, packing).  With fuse_prep the NQP kernel's epilogue writes the
// Gram partials and the packed rows, and the finishing launch (overlap_prep)
// runs at the start of `next` on the side stream beside `next`'s cross term -
// which needs only the packed operand (or the factor itself) and, on tensor
// cores, is planned for the SMs the finishing launch's kSideCtas CTAs leave
// - joining before `next`'s NQP launch.  Without the epilogue, a cross term
// that reads the other factor itself (CSR, CUDA cores) runs beside the whole
// preparation (overlap_full); the tensor-core cross term needs the packed
// operand, so there both launches of the preparation follow the NQP launch.
nmf_status enqueue_half(nmf_handle h, Loop &L, HalfStep &s, float *G, HalfStep &next,
                        float *G_other)
{
    cudaStream_t st = h->stream;
    const bool is_w = &s == &L.hw;
    const bool side = L.overlap_prep || L.overlap_full;
    if (side) {
        CK(cudaEventRecord(h->ev_fork, st));
        CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        if (L.overlap_prep)
            CK(launch_prep_finish_narrow(finish_args(L, s, G_other), is_w ? L.S_h : L.S_w,
                                         kSideCtas, h->side));
        else
            CK(launch_factor_prep(prep_args(L, s.Xo, s.Ko, G_other, s), h->side));
        CK(cudaEventRecord(h->ev_join, h->side));
    }
    // cross term C = V X_other
    if (s.sparse) {
        CK(launch_spmm_csr(s.csr->rowptr, s.csr->colidx, s.csr->vals, s.csr->dt, s.csr->rows,
                           s.csr->nnz, s.Xo, L.r, s.Cs, s.spplan, L.spws, st));
    } else if (s.tc_mode >= 0) {
        CK(launch_tc_cross(s.Atc, s.rows, s.K, s.lda_tc, L.r, s.tc_mode, s.pack, s.Cs, s.plan,
                           h->status, st));
    } else {
        CK(launch_cross_dense_f32(s.A, s.rows, s.K, s.lda, s.Xo, L.r, s.Cs, s.nsplit, st));
    }
    if (side)
        CK(cudaStreamWaitEvent(st, h->ev_join, 0));
    NnlsArgs a{};
    a.Qt = L.Qt;
    a.d = L.d;
    a.C = s.Cs;
    a.nsplit = s.nsplit;
    a.c_stride = s.rows * L.r;
    a.rows = s.rows;
    a.r = L.r;
    a.alpha = s.alpha;
    a.X = s.X;
    a.max_inner = L.nn.max_inner;
    a.eps = (float)L.nn.eps;
    a.cd_steps = L.nn.cd_steps;
    a.maxstop_mode = L.nn.maxstop_mode;
    a.maxstop = 0.f;
    a.lanes = s.lanes;
    a.grad_refresh = L.nn.grad_refresh;
    a.iter_total = h->ctr;
    a.status = h->status;
    if (L.nn.maxstop_mode == 1) {
        // fast break (Alg. 3, reading R11): stop a row once its ||f~||^2 is at
        // most the largest final value of the previous update of this factor
        CK(cudaMemsetAsync(s.ms_out, 0, sizeof(unsigned), st));
        a.maxstop_dev = s.ms_thr;
        a.s_final_max = s.ms_out;
    }
    const PrepArgs pa = prep_args(L, s.X, s.rows, G, next);
    int S = 0;
    if (L.fuse_prep) {
        a.gram_P = pa.P;
        a.gram_smax = L.Pg_slices;
        a.pack_mode = pa.pack_mode;
        a.pack = pa.pack;
        a.npad = pa.npad;
        a.kp = pa.kp;
        a.grid_out = &S;
    }
    CK(launch_nnls(a, st));
    if (L.overlap_prep && S != (is_w ? L.S_w : L.S_h))
        return NMF_E_ARG;   // the partial count the next finishing launch expects
    if (L.nn.maxstop_mode == 1)
        CK(cudaMemcpyAsync(s.ms_thr, s.ms_out, sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
    if (side)
        return NMF_OK;
    if (L.fuse_prep)
        CK(launch_prep_finish(pa, S, st));
    else
        CK(launch_factor_prep(pa, st));
    return NMF_OK;
}

nmf_status enqueue_objective(nmf_handle h, Loop &L, const nmf_solve_opts &o, double f_star,
                             double gap);

nmf_status enqueue_iteration(nmf_handle h, Loop &L, const nmf_solve_opts &o)
{
    (void)o;
    nmf_status s;
    // W-update (E-step): C_W = V Ht against Q_W = Ht^T Ht + b_w I, ready;
    // then G_W = W^T W -> Q_H, Qt, d and packed W for the H-update
    if ((s = enqueue_half(h, L, L.hw, L.Gw, L.hh, L.Gh)))
        return s;
    // H-update (M-step); then G_H = Ht^T Ht -> Q_W, Qt, d and packed Ht for
    // the next W-update
    if ((s = enqueue_half(h, L, L.hh, L.Gh, L.hw, L.Gw)))
        return s;
    return NMF_OK;
}

nmf_status enqueue_objective(nmf_handle h, Loop &L, const nmf_solve_opts &o, double f_star,
                             double gap)
{
    if (L.direct_obj) {
        ObjDirectArgs b{};
        b.V = L.V;
        b.ldv = L.ldv;
        b.W = L.hw.X;
        b.m = L.hw.rows;
        b.Ht = L.hh.X;
        b.n = L.hh.rows;
        b.r = L.r;
        b.aw = o.alpha_w;
        b.ah = o.alpha_h;
        b.bw = o.beta_w;
        b.bh = o.beta_h;
        b.J = h->scal + 0;
        b.partials = L.obj_partials;
        b.ticket = h->tickets + 2;
        CK(launch_objective_direct(b, h->stream));
        return NMF_OK;
    }
    // J(W, H) by the FP64 trace identity.  With the preparation beside the
    // cross term (overlap_prep, overlap_full) G_H = Ht^T Ht is completed at
    // the start of the next W-update; complete it now for the objective (the
    // next W-update writes the same values again)
    if (L.overlap_prep)
        CK(launch_prep_finish(finish_args(L, L.hw, L.Gh), L.S_h, h->stream));
    else if (L.overlap_full)
        CK(launch_factor_prep(prep_args(L, L.hw.Xo, L.hw.Ko, L.Gh, L.hw), h->stream));
    ObjArgs a{};
    a.vv = L.vv;
    a.W = L.hw.X;
    a.m = L.hw.rows;
    a.Ht = L.hh.X;
    a.n = L.hh.rows;
    a.r = L.r;
    a.Ch = L.hh.Cs;
    a.nsplit = L.hh.nsplit;
    a.ch_stride = L.hh.rows * L.r;
    a.Gw = L.Gw;
    a.Gh = L.Gh;
    a.aw = o.alpha_w;
    a.ah = o.alpha_h;
    a.bw = o.beta_w;
    a.bh = o.beta_h;
    a.J = h->scal + 0;
    a.hist = nullptr;
    a.t = nullptr;
    a.f_star = f_star;
    a.gap_target = gap;
    a.done_flag = h->idev + 1;
    a.partials = h->partials;
    a.ticket = h->tickets + 0;
    CK(launch_objective(a, h->stream));
    return NMF_OK;
}

}  // namespace

namespace {
nmf_status solve_device(nmf_handle h, const nmf_matrix *V, const nmf_matrix *Vt, int r, float *W,
                        float *Ht, const nmf_solve_opts *opts, nmf_report *rep);
}

// Host-resident inputs (V, Vt, W, Ht in host memory) are copied to a staging
// area of the handle on its stream, solved there, and W, Ht copied back; the
// copies run at pinned-memory speed when the caller's buffers are pinned.
NMF_API nmf_status nmf_solve(nmf_handle h, const nmf_matrix *V, const nmf_matrix *Vt, int r,
                             float *W, float *Ht, const nmf_solve_opts *opts, nmf_report *rep)
{
    if (!h || !V || !W || !Ht || !opts)
        return NMF_E_ARG;
    if (bad_r(r))
        return NMF_E_SHAPE;
    CK(cudaSetDevice(h->device));
    const bool sp = V->is_sparse != 0;
    const void *probe = sp ? (const void *)V->s.rowptr : V->d.data;
    const bool hv = is_host_ptr(probe), hw = is_host_ptr(W), hh = is_host_ptr(Ht);
    if (!hv && !hw && !hh)
        return solve_device(h, V, Vt, r, W, Ht, opts, rep);
    // sizes
    int64_t m, n;
    size_t vb = 0, vtb = 0;
    if (sp) {
        if (!Vt || !Vt->is_sparse)
            return NMF_E_ARG;
        m = V->s.rows;
        n = V->s.cols;
        const size_t es = V->s.dt == NMF_BF16 ? 2 : 4;
        vb = 8 * (size_t)(m + 1) + 4 * (size_t)V->s.nnz + es * V->s.nnz + 64;
        vtb = 8 * (size_t)(n + 1) + 4 * (size_t)Vt->s.nnz + es * Vt->s.nnz + 64;
    } else {
        m = V->d.rows;
        n = V->d.cols;
        if (V->d.ld != n || V->d.dt != NMF_F32)
            return NMF_E_NOTIMPL;   // staged dense V must be contiguous F32
        vb = sizeof(float) * (size_t)m * n;
        if (Vt)
            vtb = sizeof(float) * (size_t)m * n;
    }
    if (m <= 0 || n <= 0)
        return NMF_E_SHAPE;
    const size_t wb = sizeof(float) * (size_t)m * r, hb = sizeof(float) * (size_t)n * r;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    nmf_status st = ensure_stage(h, al(vb) + al(vtb) + al(wb) + al(hb));
    if (st)
        return st;
    char *p = h->stage;
    cudaStream_t s = h->stream;
    nmf_matrix Vd = *V, Vtd{};
    const nmf_matrix *vtp = Vt;
    if (hv) {
        if (sp) {
            char *q = p;
            CK(cudaMemcpyAsync(q, V->s.rowptr, 8 * (m + 1), cudaMemcpyHostToDevice, s));
            Vd.s.rowptr = (const int64_t *)q;
            q += al(8 * (m + 1));
            CK(cudaMemcpyAsync(q, V->s.colidx, 4 * V->s.nnz, cudaMemcpyHostToDevice, s));
            Vd.s.colidx = (const int32_t *)q;
            q += al(4 * V->s.nnz);
            const size_t es = V->s.dt == NMF_BF16 ? 2 : 4;
            CK(cudaMemcpyAsync(q, V->s.vals, es * V->s.nnz, cudaMemcpyHostToDevice, s));
            Vd.s.vals = q;
            char *t = p + al(vb);
            Vtd = *Vt;
            CK(cudaMemcpyAsync(t, Vt->s.rowptr, 8 * (n + 1), cudaMemcpyHostToDevice, s));
            Vtd.s.rowptr = (const int64_t *)t;
            t += al(8 * (n + 1));
            CK(cudaMemcpyAsync(t, Vt->s.colidx, 4 * Vt->s.nnz, cudaMemcpyHostToDevice, s));
            Vtd.s.colidx = (const int32_t *)t;
            t += al(4 * Vt->s.nnz);
            CK(cudaMemcpyAsync(t, Vt->s.vals, es * Vt->s.nnz, cudaMemcpyHostToDevice, s));
            Vtd.s.vals = t;
            vtp = &Vtd;
        } else {
            CK(cudaMemcpyAsync(p, V->d.data, vb, cudaMemcpyHostToDevice, s));
            Vd.d.data = p;
            if (Vt) {
                Vtd = *Vt;
                CK(cudaMemcpyAsync(p + al(vb), Vt->d.data, vtb, cudaMemcpyHostToDevice, s));
                Vtd.d.data = p + al(vb);
                vtp = &Vtd;
            }
        }
    }
    float *Wd = W, *Hd = Ht;
    char *fp = p + al(vb) + al(vtb);
    if (hw) {
        Wd = (float *)fp;
        CK(cudaMemcpyAsync(Wd, W, wb, cudaMemcpyHostToDevice, s));
    }
    if (hh) {
        Hd = (float *)(fp + al(wb));
        CK(cudaMemcpyAsync(Hd, Ht, hb, cudaMemcpyHostToDevice, s));
    }
    st = solve_device(h, &Vd, vtp, r, Wd, Hd, opts, rep);
    if (st != NMF_OK && st != NMF_E_NONFINITE)
        return st;
    if (hw)
        CK(cudaMemcpyAsync(W, Wd, wb, cudaMemcpyDeviceToHost, s));
    if (hh)
        CK(cudaMemcpyAsync(Ht, Hd, hb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st;
}

namespace {
nmf_status solve_device(nmf_handle h, const nmf_matrix *V, const nmf_matrix *Vt, int r, float *W,
                        float *Ht, const nmf_solve_opts *opts, nmf_report *rep)
{
    if (!h || !V || !W || !Ht || !opts)
        return NMF_E_ARG;
    if (bad_r(r))
        return NMF_E_SHAPE;
    const nmf_solve_opts o = *opts;
    if (o.outer_iters < 0)
        return NMF_E_ARG;
    if (o.prec < NMF_PREC_FP32 || o.prec > NMF_PREC_FP32_SIMT)
        return NMF_E_NOTIMPL;
    Loop L{};
    L.r = r;
    L.nn = opts_or_default(&o.nnls);
    if (L.nn.grad_refresh < 0)
        return NMF_E_ARG;
    if (L.nn.maxstop_mode < 0 || L.nn.maxstop_mode > 1)
        return NMF_E_NOTIMPL;   // mode 2 (sequential, order-dependent) is the oracle's only
    {
        int lg = 0, lj = 0;
        if (!nnls_layout(r, L.nn.lanes, &lg, &lj))
            return NMF_E_ARG;
    }
    int64_t m, n;
    const bool sparse = V->is_sparse != 0;
    if (sparse) {
        if (!Vt || !Vt->is_sparse)
            return NMF_E_ARG;
        m = V->s.rows;
        n = V->s.cols;
        if (Vt->s.rows != n || Vt->s.cols != m || Vt->s.nnz != V->s.nnz)
            return NMF_E_SHAPE;
        if (!V->s.rowptr || !Vt->s.rowptr)
            return NMF_E_ARG;
        if (V->s.dt != Vt->s.dt || (V->s.dt != NMF_F32 && V->s.dt != NMF_BF16))
            return NMF_E_DTYPE;
    } else {
        m = V->d.rows;
        n = V->d.cols;
        if (!V->d.data || V->d.ld < n)
            return NMF_E_ARG;
        if (V->d.dt != NMF_F32)
            return NMF_E_DTYPE;
        if (Vt) {
            if (Vt->is_sparse || Vt->d.rows != n || Vt->d.cols != m || Vt->d.ld < m || !Vt->d.data)
                return NMF_E_SHAPE;
            if (Vt->d.dt != NMF_F32)
                return NMF_E_DTYPE;
        }
    }
    if (m <= 0 || n <= 0)
        return NMF_E_SHAPE;
    CK(cudaSetDevice(h->device));
    // Wide factors of large problems: at r > 64 with tens of thousands of
    // rows in both half-steps, 8 lanes per row (16 coordinates each) beat the
    // default 16 (8 each) by ~20% (fewer instructions per coordinate step
    // when many rounds of rows keep the SMs issue-bound; measured at r = 100
    // on 50000 and 100000 rows).  The layout is fixed for the whole solve.
    if (L.nn.lanes == 0 && r > 64 && (m < n ? m : n) >= 32768)
        L.nn.lanes = 8;
    const int lanes_w = L.nn.lanes, lanes_h = L.nn.lanes;

    // ---- workspace layout
    L.gS_w = gram_splits(m);
    L.gS_h = gram_splits(n);
    int gS = L.gS_w > L.gS_h ? L.gS_w : L.gS_h;
    {
        const int ps = prep_slices(m > n ? m : n);
        gS = ps > gS ? ps : gS;
    }
    // the NQP kernel prepares the factor it solved when its layout carries
    // the epilogue (RP <= 64): one Gram partial per CTA
    {
        int lg = 0, lj = 0, lg2 = 0, lj2 = 0;
        L.fuse_prep = nnls_layout(r, lanes_w, &lg, &lj) && lg * lj <= 64 &&
                      nnls_layout(r, lanes_h, &lg2, &lj2) && lg2 * lj2 <= 64;
        if (L.fuse_prep)
            gS = gS > kPrepMaxSlices ? gS : kPrepMaxSlices;
        L.Pg_slices = kPrepMaxSlices;
    }
    int sw = 1, sh = 1;
    SpmmPlan pw{}, ph{};
    if (sparse) {
        pw = spmm_plan(m, V->s.nnz);
        ph = spmm_plan(n, Vt->s.nnz);
    } else {
        sw = cross_splits(m, n);
        sh = cross_splits(n, m);
    }
    const bool need_vt = !sparse && !Vt;
    // dense cross-term arithmetic: tensor cores when the layouts allow TMA
    int mode = -1;
    if (!sparse) {
        const int64_t vt_ld_req = Vt ? Vt->d.ld : m;
        if (o.prec == NMF_PREC_BF16 || o.prec == NMF_PREC_BF16X2) {
            mode = o.prec == NMF_PREC_BF16 ? TC_BF16 : TC_BF16X2;
            if (n % 8 || m % 8 || !tc_supported(n, mode, V->d.data))
                return NMF_E_NOTIMPL;
        } else if (o.prec != NMF_PREC_FP32_SIMT) {
            const int want = o.prec == NMF_PREC_TF32 ? TC_TF32 : TC_TF32X3;
            if (tc_supported(V->d.ld, want, V->d.data) && vt_ld_req % 4 == 0 &&
                (!Vt || tc_supported(Vt->d.ld, want, Vt->d.data)))
                mode = want;
            else if (o.prec == NMF_PREC_TF32)
                return NMF_E_NOTIMPL;
        }
        // the tensor-core cross term's stream-K plan leaves the finishing
        // launch of the preparation its SMs
        if (mode >= 0) {
            int sms = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int cap = L.fuse_prep && sms > 2 * kSideCtas ? sms - kSideCtas : 0;
            L.hw.plan = tc_plan(m, n, r, mode, cap);
            L.hh.plan = tc_plan(n, m, r, mode, cap);
            sw = L.hw.plan.nslices;
            sh = L.hh.plan.nslices;
        }
    }
    // the preparation beside the cross term: its finishing launch when the NQP
    // epilogue writes the partials; all of it when the cross term reads the
    // other factor itself
    L.overlap_prep = L.fuse_prep;
    L.overlap_full = !L.fuse_prep && (sparse || mode < 0);
    const size_t pack_b = mode >= 0 ? std::max(tc_pack_bytes(n, r, mode), tc_pack_bytes(m, r, mode)) : 0;
    const size_t bf_b = tc_bf16(mode) ? sizeof(__nv_bfloat16) * (size_t)m * n : 0;
    if (o.objective < 0 || o.objective > 1 || (o.objective == 1 && sparse))
        return NMF_E_NOTIMPL;
    L.direct_obj = o.objective == 1;
    const size_t n_objp = L.direct_obj ? objective_direct_partials(m, n) : 0;
    Sizer z;
    z.add<double>(n_objp);
    z.add<float>((size_t)gS * prep_slice_floats(r));
    z.add<unsigned>(4);
    z.add<float>((size_t)r * r);
    z.add<float>((size_t)r * r);
    z.add<float>((size_t)r * r);
    z.add<float>(r);
    z.add<float>((size_t)r * r);
    z.add<float>((size_t)r * r);
    z.add<float>((size_t)sw * m * r);
    z.add<float>((size_t)sh * n * r);
    size_t spb = sparse ? std::max(spmm_workspace_bytes(pw, r), spmm_workspace_bytes(ph, r)) : 0;
    z.add<char>(spb);
    if (need_vt)
        z.add<float>((size_t)m * n);
    z.add<char>(pack_b);
    z.add<char>(bf_b);
    z.add<char>(bf_b);
    nmf_status st = ensure_ws(h, z.off);
    if (st)
        return st;
    Arena a(h->ws, h->ws_cap);
    L.obj_partials = a.take<double>(n_objp);
    if (!sparse) {
        L.V = (const float *)V->d.data;
        L.ldv = V->d.ld;
    }
    L.Pg = a.take<float>((size_t)gS * prep_slice_floats(r));
    L.ticket = a.take<unsigned>(4);
    L.Gw = a.take<float>((size_t)r * r);
    L.Gh = a.take<float>((size_t)r * r);
    L.Qt = a.take<float>((size_t)r * r);
    L.d = a.take<float>(r);
    float *Qw = a.take<float>((size_t)r * r);
    float *Qh = a.take<float>((size_t)r * r);
    float *Cw = a.take<float>((size_t)sw * m * r);
    float *Ch = a.take<float>((size_t)sh * n * r);
    L.spws = a.take<char>(spb);
    const float *vt_data = nullptr;
    int64_t vt_ld = m;
    if (need_vt) {
        float *vtb = a.take<float>((size_t)m * n);
        CK(launch_transpose_f32((const float *)V->d.data, m, n, V->d.ld, vtb, h->stream));
        vt_data = vtb;
    } else if (!sparse) {
        vt_data = (const float *)Vt->d.data;
        vt_ld = Vt->d.ld;
    }
    void *pack = a.take<char>(pack_b);
    __nv_bfloat16 *vbf = a.take<__nv_bfloat16>(bf_b / 2);
    __nv_bfloat16 *vtbf = a.take<__nv_bfloat16>(bf_b / 2);
    if (tc_bf16(mode)) {
        // BF16 copies of V and V^T (contiguous), made once per solve
        CK(launch_f32_to_bf16((const float *)V->d.data, m * n, vbf, h->stream));
        if (vt_ld != m)
            return NMF_E_NOTIMPL;
        CK(launch_f32_to_bf16(vt_data, m * n, vtbf, h->stream));
    }

    // half-step descriptions
    HalfStep &hw = L.hw, &hh = L.hh;
    const TcPlan plan_w = hw.plan, plan_h = hh.plan;
    hw = HalfStep{};
    hh = HalfStep{};
    hw.plan = plan_w;
    hh.plan = plan_h;
    hw.sparse = hh.sparse = sparse;
    hw.rows = m;
    hw.X = W;
    hw.Xo = Ht;
    hw.Ko = n;
    hw.alpha = o.alpha_w;
    hw.beta = o.beta_w;
    hw.Cs = Cw;
    hw.Q = Qw;
    hh.rows = n;
    hh.X = Ht;
    hh.Xo = W;
    hh.Ko = m;
    hh.alpha = o.alpha_h;
    hh.beta = o.beta_h;
    hh.Cs = Ch;
    hh.Q = Qh;
    if (sparse) {
        hw.csr = &V->s;
        hw.spplan = pw;
        hw.nsplit = 1;
        hh.csr = &Vt->s;
        hh.spplan = ph;
        hh.nsplit = 1;
    } else {
        hw.A = (const float *)V->d.data;
        hw.lda = V->d.ld;
        hw.K = n;
        hw.nsplit = sw;
        hh.A = vt_data;
        hh.lda = vt_ld;
        hh.K = m;
        hh.nsplit = sh;
    }
    hw.lanes = lanes_w;
    hh.lanes = lanes_h;
    hw.ms_thr = h->smax + 0;
    hh.ms_thr = h->smax + 1;
    hw.ms_out = h->smax + 2;
    hh.ms_out = h->smax + 3;
    hw.tc_mode = hh.tc_mode = sparse ? -1 : mode;
    hw.pack = hh.pack = pack;
    if (mode >= 0) {
        hw.Atc = tc_bf16(mode) ? (const void *)vbf : (const void *)hw.A;
        hw.lda_tc = tc_bf16(mode) ? n : hw.lda;
        hh.Atc = tc_bf16(mode) ? (const void *)vtbf : (const void *)hh.A;
        hh.lda_tc = tc_bf16(mode) ? m : hh.lda;
    }

    cudaStream_t s = h->stream;
    // ||V||^2 (constant of the trace identity), FP64
    double *vv_dev = h->scal + 1;
    if (sparse)
        CK(launch_sumsq(V->s.vals, V->s.dt, V->s.nnz, vv_dev, h->partials, h->tickets + 1, s));
    else if (V->d.ld == n)
        CK(launch_sumsq(V->d.data, NMF_F32, m * n, vv_dev, h->partials, h->tickets + 1, s));
    else
        return NMF_E_NOTIMPL;   // strided dense V: pass a contiguous V
    CK(cudaMemsetAsync(h->ctr, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->idev, 0, 2 * sizeof(int), s));
    CK(cudaMemsetAsync(L.ticket, 0, 4 * sizeof(unsigned), s));
    CK(cudaMemsetAsync(h->smax, 0, 4 * sizeof(unsigned), s));   // maxStop: 0 before the first update
    CK(cudaMemcpyAsync(&L.vv, vv_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    if (L.overlap_prep) {
        // the NQP launches' grids are the partial counts of the finishing launches
        NnlsArgs q{};
        q.r = r;
        q.lanes = lanes_w;
        q.gram_P = L.Pg;
        q.gram_smax = L.Pg_slices;
        q.rows = m;
        L.S_w = nnls_grid_query(q);
        q.lanes = lanes_h;
        q.rows = n;
        L.S_h = nnls_grid_query(q);
        if (L.S_w < 1 || L.S_h < 1)
            return NMF_E_CUDA;
    }
    if (L.overlap_prep || L.overlap_full) {
        if (!h->side)
            CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        if (!h->ev_fork)
            CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        if (!h->ev_join)
            CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    // G_H = Ht^T Ht, Q_W, Qt, d and packed Ht for the first W-update; with
    // overlap_prep its partials are split as the H-update's NQP launch splits
    // them, since the first W-update's finishing launch sums them again; with
    // overlap_full the first W-update prepares Ht itself
    if (!L.overlap_full) {
        PrepArgs pa = prep_args(L, Ht, n, L.Gh, hw);
        if (L.overlap_prep)
            pa.slices = L.S_h;
        CK(launch_factor_prep(pa, s));
    }

    const bool gap_on = o.rel_gap_target > 0.0 && o.f_star > 0.0;
    const bool adaptive = o.check_every < 0;
    const int check = o.check_every > 0 ? o.check_every : 1;
    // adaptive gap tests: from the last two tests estimate the iterations
    // still needed (gap falls roughly linearly over a few dozen iterations)
    // and test again after 0.6 of them, at most 128 iterations on (on the FP64
    // oracle's trajectory of the dense workload: 17 tests instead of 25 with
    // half the estimate and 64 at most, both without passing the first
    // iteration at the gap)
    int next_check = adaptive ? 4 : check;
    int prev_t = -1;
    double prev_gap = 0.0;
    int n_checks = 0;
    std::vector<double> hist;
    int done_iters = 0;
    double Jlast = NAN;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    long long per_iter_launches = 0;
    CK(prepare_nnls(r, lanes_w));
    CK(prepare_nnls(r, lanes_h));
    if (o.use_graph && o.outer_iters > 0) {
        if (!h->cap)
            CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
        CK(cudaStreamSynchronize(s));
        long long before = nmf_launch_count();
        prof_suspend(true);
        h->stream = h->cap;
        cudaError_t ce = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) {
            h->stream = s;
            prof_suspend(false);
            return cuda_st(ce);
        }
        st = enqueue_iteration(h, L, o);
        cudaGraph_t g2 = nullptr;
        ce = cudaStreamEndCapture(h->cap, &g2);
        h->stream = s;
        prof_suspend(false);
        if (st)
            return st;
        CK(ce);
        graph = g2;
        CK(cudaGraphInstantiate(&gexec, graph, 0));
        per_iter_launches = nmf_launch_count() - before;
        g_launches.fetch_sub(per_iter_launches);
    }
    bool have_j = false;
    for (int t = 0; t < o.outer_iters; ++t) {
        if (gexec) {
            CK(cudaGraphLaunch(gexec, s));
            count_launch((int)per_iter_launches);
        } else {
            st = enqueue_iteration(h, L, o);
            if (st)
                return st;
        }
        ++done_iters;
        const bool last = t + 1 == o.outer_iters;
        const bool check_now = gap_on && (t + 1 >= next_check || last);
        if (o.obj_hist || check_now || (last && rep)) {
            if ((st = enqueue_objective(h, L, o, o.f_star, o.rel_gap_target)))
                return st;
            have_j = true;
        }
        if (o.obj_hist || check_now) {
            double J;
            CK(cudaMemcpyAsync(&J, h->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (o.obj_hist)
                o.obj_hist[t] = J;
            Jlast = J;
            if (check_now) {
                ++n_checks;
                const double gap = (J - o.f_star) / o.f_star;
                if (gap <= o.rel_gap_target)
                    break;
                if (adaptive) {
                    int step = 16;
                    if (prev_t >= 0 && prev_gap > gap) {
                        const double rate = (prev_gap - gap) / (double)(t - prev_t);
                        const double need = (gap - o.rel_gap_target) / rate;
                        step = (int)(0.6 * need);
                    }
                    step = step < 1 ? 1 : (step > 128 ? 128 : step);
                    prev_t = t;
                    prev_gap = gap;
                    next_check = t + 1 + step;
                } else {
                    next_check = t + 1 + check;
                }
            }
        }
    }
    if (!have_j && rep && done_iters > 0) {
        if ((st = enqueue_objective(h, L, o, o.f_star, o.rel_gap_target)))
            return st;
    }
    CK(cudaEventRecord(e1, s));
    if (gexec) {
        cudaGraphExecDestroy(gexec);
        cudaGraphDestroy(graph);
    }

    // report: J, kbar, KKT of the last half-steps' NQPs
    double *kk = h->scal + 4;
    unsigned long long inner = 0;
    if (rep) {
        CK(cudaMemcpyAsync(&Jlast, h->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&inner, h->ctr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        // KKT of the H-update just solved (its Q and C are still in place)
        if (hh.nsplit > 1)
            CK(launch_sum_slices(hh.Cs, hh.nsplit, n * r, hh.Cs, s));
        CK(launch_kkt(hh.Q, hh.Cs, n, r, hh.alpha, Ht, kk, s));
    }
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rep) {
        double kkv[2];
        CK(cudaMemcpy(kkv, kk, sizeof(kkv), cudaMemcpyDeviceToHost));
        rep->iters_done = done_iters;
        rep->objective = Jlast;
        rep->rel_gap = o.f_star > 0.0 ? (Jlast - o.f_star) / o.f_star : 0.0;
        rep->inner_total = (int64_t)inner;
        rep->kbar = done_iters > 0 ? (double)inner / ((double)done_iters * (double)(m + n)) : 0.0;
        rep->kkt_max = kkv[0];
        rep->ms_total = ms;
    }
    return nmf_sync(h);
}

}  // namespace

// ---------------------------------------------------------------------------
// many independent instances
// ---------------------------------------------------------------------------
namespace {

struct BatchPlan {
    BatchInst *dinst = nullptr;   // device array
    int64_t *doff = nullptr;      // device [8][count + 1]
    std::vector<int64_t> hoff;    // host copy
};

nmf_status batch_offsets(std::vector<int64_t> &hoff, const nmf_instance *inst, int count,
                         int nnls_rows)
{
    hoff.assign((size_t)8 * (count + 1), 0);
    for (int ph = 0; ph < 8; ++ph) {
        int64_t acc = 0;
        for (int i = 0; i < count; ++i) {
            hoff[(size_t)ph * (count + 1) + i] = acc;
            acc += batched_items(ph, inst[i].m, inst[i].n, inst[i].r, nnls_rows);
        }
        hoff[(size_t)ph * (count + 1) + count] = acc;
    }
    return NMF_OK;
}

}  // namespace

NMF_API nmf_status nmf_solve_batched(nmf_handle h, int count, const nmf_instance *inst,
                                     const nmf_solve_opts *opts, int mode, nmf_report *reps)
{
    if (!h || !inst || !opts || count < 1 || mode < 0 || mode > 3)
        return NMF_E_ARG;
    if (opts->outer_iters < 0)
        return NMF_E_ARG;
    // FP32 products: 3xTF32 on the tensor cores, or FFMA on the CUDA cores
    if (opts->prec != NMF_PREC_FP32 && opts->prec != NMF_PREC_FP32_SIMT)
        return NMF_E_NOTIMPL;
    for (int i = 0; i < count; ++i) {
        const nmf_instance &b = inst[i];
        if (b.m < 1 || b.n < 1 || b.r < 1 || b.r > 64)
            return NMF_E_SHAPE;
        if (!b.V || !b.Vt || !b.W || !b.Ht)
            return NMF_E_ARG;
    }
    CK(cudaSetDevice(h->device));
    const nmf_nnls_opts nn = opts_or_default(&opts->nnls);
    const bool tc = opts->prec == NMF_PREC_FP32;
    // the tensor-core cross phase copies its tiles 16 bytes at a time: an
    // array whose rows do not start 16 bytes apart gets a row-padded copy
    // (pitch rounded up to 4 floats), made once per call
    auto padded = [](const float *p, int64_t cols) {
        return (cols & 3) != 0 || (reinterpret_cast<uintptr_t>(p) & 15) != 0;
    };
    auto pad4 = [](int64_t c) { return (c + 3) & ~int64_t(3); };
    // ---- workspace: per-instance buffers, then the device tables
    Sizer z;
    for (int i = 0; i < count; ++i) {
        const nmf_instance &b = inst[i];
        const int64_t parts = (std::max(b.m, b.n) + 255) / 256;
        z.add<float>((size_t)parts * b.r * b.r);
        z.add<float>((size_t)b.r * b.r);
        z.add<float>(b.r);
        z.add<float>((size_t)b.m * b.r);
        z.add<float>((size_t)b.n * b.r);
        if (tc && padded(b.V, b.n))
            z.add<float>((size_t)b.m * pad4(b.n));
        if (tc && padded(b.Vt, b.m))
            z.add<float>((size_t)b.n * pad4(b.m));
    }
    z.add<BatchInst>(count);
    z.add<int64_t>((size_t)8 * (count + 1));
    z.add<unsigned long long>(8);
    nmf_status st = ensure_ws(h, z.off);
    if (st)
        return st;
    Arena a(h->ws, h->ws_cap);
    // the device list in decreasing cross-term cost m n r (ties by position):
    // with CTAs taking items in order, the largest instances start first;
    // results do not depend on the order
    std::vector<int> ord(count);
    for (int i = 0; i < count; ++i)
        ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        return (double)inst[x].m * inst[x].n * inst[x].r > (double)inst[y].m * inst[y].n * inst[y].r;
    });
    std::vector<nmf_instance> pinst(count);
    for (int j = 0; j < count; ++j)
        pinst[j] = inst[ord[j]];
    std::vector<BatchInst> hb(count);
    for (int i = 0; i < count; ++i) {
        const nmf_instance &b = pinst[i];
        BatchInst &q = hb[i];
        q.m = b.m;
        q.n = b.n;
        q.r = b.r;
        q.V = b.V;
        q.Vt = b.Vt;
        q.W = b.W;
        q.Ht = b.Ht;
        const int64_t parts = (std::max(b.m, b.n) + 255) / 256;
        q.gram = a.take<float>((size_t)parts * b.r * b.r);
        q.Qt = a.take<float>((size_t)b.r * b.r);
        q.d = a.take<float>(b.r);
        q.Cw = a.take<float>((size_t)b.m * b.r);
        q.Ch = a.take<float>((size_t)b.n * b.r);
        q.alpha_w = opts->alpha_w;
        q.alpha_h = opts->alpha_h;
        q.beta_w = opts->beta_w;
        q.beta_h = opts->beta_h;
        q.Vx = b.V;
        q.ldvx = b.n;
        q.Vtx = b.Vt;
        q.ldvtx = b.m;
        // the pad columns are zeroed: the cross phase copies a row's last
        // 16-byte chunk whole, and the factor rows it meets there are zero
        // (workspace bits left as NaN or Inf would otherwise reach the sums)
        auto pad_copy = [&](const float *src, int64_t rows, int64_t cols) -> float * {
            const int64_t ld = pad4(cols);
            float *c = a.take<float>((size_t)rows * ld);
            if (cudaMemcpy2DAsync(c, ld * sizeof(float), src, cols * sizeof(float),
                                  cols * sizeof(float), rows, cudaMemcpyDeviceToDevice,
                                  h->stream) != cudaSuccess ||
                (ld > cols && cudaMemset2DAsync(c + cols, ld * sizeof(float), 0,
                                                (ld - cols) * sizeof(float), rows,
                                                h->stream) != cudaSuccess))
                return nullptr;
            return c;
        };
        if (tc && padded(b.V, b.n)) {
            if (!(q.Vx = pad_copy(b.V, b.m, b.n)))
                return NMF_E_CUDA;
            q.ldvx = pad4(b.n);
        }
        if (tc && padded(b.Vt, b.m)) {
            if (!(q.Vtx = pad_copy(b.Vt, b.n, b.m)))
                return NMF_E_CUDA;
            q.ldvtx = pad4(b.m);
        }
    }
    BatchInst *dinst = a.take<BatchInst>(count);
    int64_t *doff = a.take<int64_t>((size_t)8 * (count + 1));
    unsigned long long *dwork = a.take<unsigned long long>(8);
    cudaStream_t s = h->stream;
    CK(cudaMemcpyAsync(dinst, hb.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, s));

    BatchArgs ba{};
    ba.inst = dinst;
    ba.count = count;
    ba.item_off = doff;
    ba.nnls.max_inner = nn.max_inner;
    ba.nnls.eps = (float)nn.eps;
    ba.nnls.cd_steps = nn.cd_steps;
    ba.iter_total = h->ctr + 1;
    ba.status = h->status;
    ba.bar_count = reinterpret_cast<unsigned *>(h->idev + 2);
    ba.bar_gen = reinterpret_cast<unsigned *>(h->idev + 3);
    // the barrier's bounded wait: 2 s, or a deadline already passed when the
    // "barrier" fault is injected (the wait runs out, NMF_E_TIMEOUT follows)
    ba.barrier_ns = fault_armed("barrier") ? 0ull : 2000000000ull;
    CK(cudaMemsetAsync(h->ctr + 1, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->idev + 2, 0, 2 * sizeof(int), s));
    CK(cudaMemsetAsync(dwork, 0, 8 * sizeof(unsigned long long), s));
    // the launches over all instances take items from the counters; the
    // one-instance launches of the loop mode keep the fixed stride
    ba.work = mode == 1 ? nullptr : dwork;
    ba.tc = tc ? 1 : 0;
    if (ba.tc && !batched_tc_fits())
        return NMF_E_NOTIMPL;

    std::vector<int64_t> hoff;
    auto set_rows = [&](int rows) -> nmf_status {
        ba.nnls_rows = rows;
        batch_offsets(hoff, pinst.data(), count, rows);
        CK(cudaMemcpyAsync(doff, hoff.data(), sizeof(int64_t) * hoff.size(),
                           cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));   // hoff is reused
        return NMF_OK;
    };
    if ((st = set_rows(1)))
        return st;
    const int max_grid = batched_grid(true);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = max_grid;

    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int t = 0;
    auto one_persistent = [&]() -> nmf_status {
        ba.phase_begin = 0;   // all eight phases, all instances
        ba.phase_end = 8;
        ba.inst_begin = -1;
        CK(launch_batched(ba, grid, true, s));
        return NMF_OK;
    };
    CK(cudaEventRecord(e0, s));
    if (mode == 2) {
        // autotune: each candidate runs one real outer iteration, timed
        const int per_sm_max = std::max(1, max_grid / sms);
        float best = 1e30f;
        int best_grid = max_grid, best_rows = 1;
        const int rows_c[3] = {1, 2, 4};   // rows per group of each warp in an NQP item
        for (int ri = 0; ri < 3 && t < opts->outer_iters; ++ri) {
            if ((st = set_rows(rows_c[ri])))
                return st;
            for (int k = 1; k <= per_sm_max && t < opts->outer_iters; ++k) {
                grid = k * sms;
                cudaEvent_t a0, a1;
                CK(cudaEventCreate(&a0));
                CK(cudaEventCreate(&a1));
                CK(cudaEventRecord(a0, s));
                if ((st = one_persistent()))
                    return st;
                CK(cudaEventRecord(a1, s));
                CK(cudaEventSynchronize(a1));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a0, a1);
                cudaEventDestroy(a0);
                cudaEventDestroy(a1);
                ++t;
                if (ms < best) {
                    best = ms;
                    best_grid = grid;
                    best_rows = rows_c[ri];
                }
            }
        }
        grid = best_grid;
        if ((st = set_rows(best_rows)))
            return st;
    }
    if (mode == 0 || mode == 2) {
        ba.phase_begin = 0;
        ba.phase_end = 8;
        ba.inst_begin = -1;
        cudaGraphExec_t gexec = nullptr;
        int graph_kernels = 0;
        if (opts->use_graph && t < opts->outer_iters) {
            if (!h->cap)
                CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
            CK(cudaStreamSynchronize(s));
            prof_suspend(true);
            cudaGraph_t g = nullptr;
            const long long l0 = g_launches.load();
            bool ok = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) ==
                      cudaSuccess;
            if (ok) {
                ok = launch_batched(ba, grid, true, h->cap) == cudaSuccess;
                ok = (cudaStreamEndCapture(h->cap, &g) == cudaSuccess) && ok;
            }
            prof_suspend(false);
            // kernels per iteration: one cooperative launch, or three around
            // the two tensor-core cross launches
            graph_kernels = (int)(g_launches.load() - l0);
            g_launches.fetch_sub(graph_kernels);
            if (!(ok && g && cudaGraphInstantiate(&gexec, g, 0) == cudaSuccess)) {
                gexec = nullptr;   // capture of a cooperative launch refused: launch directly
                cudaGetLastError();
            }
            if (g)
                cudaGraphDestroy(g);
        }
        for (; t < opts->outer_iters; ++t) {
            if (gexec) {
                CK(cudaGraphLaunch(gexec, s));
                count_launch(graph_kernels);
            } else if ((st = one_persistent())) {
                return st;
            }
        }
        if (gexec)
            cudaGraphExecDestroy(gexec);
    } else if (mode == 3) {
        // one launch per phase over all instances: stream order separates
        // the phases, no grid barrier
        ba.inst_begin = -1;
        for (; t < opts->outer_iters; ++t)
            for (int ph = 0; ph < 8; ++ph) {
                ba.phase_begin = ph;
                ba.phase_end = ph + 1;
                CK(launch_batched(ba, grid, false, s));
            }
    } else {
        for (; t < opts->outer_iters; ++t)
            for (int ph = 0; ph < 8; ++ph)
                for (int i = 0; i < count; ++i) {
                    ba.phase_begin = ph;
                    ba.phase_end = ph + 1;
                    ba.inst_begin = i;
                    const int64_t items = hoff[(size_t)ph * (count + 1) + i + 1] -
                                          hoff[(size_t)ph * (count + 1) + i];
                    CK(launch_batched(ba, (int)items, false, s));
                }
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    unsigned long long inner = 0;
    CK(cudaMemcpy(&inner, h->ctr + 1, sizeof(inner), cudaMemcpyDeviceToHost));
    if (reps) {
        double rows_total = 0.0;
        for (int i = 0; i < count; ++i)
            rows_total += (double)(inst[i].m + inst[i].n);
        for (int i = 0; i < count; ++i) {
            nmf_dense Vd{inst[i].m, inst[i].n, inst[i].n, NMF_F32, inst[i].V};
            double *Jd = h->scal + 8;
            nmf_status e = nmf_objective_direct(h, &Vd, inst[i].W, inst[i].Ht, inst[i].r,
                                                opts->alpha_w, opts->alpha_h, opts->beta_w,
                                                opts->beta_h, Jd);
            if (e)
                return e;
            double J = 0.0;
            CK(cudaMemcpyAsync(&J, Jd, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            reps[i] = nmf_report{};
            reps[i].iters_done = opts->outer_iters;
            reps[i].objective = J;
            reps[i].ms_total = ms;
            reps[i].inner_total = (int64_t)inner;
            reps[i].kbar = opts->outer_iters > 0 ? (double)inner / (opts->outer_iters * rows_total)
                                                 : 0.0;
        }
    }
    return nmf_sync(h);
}

NMF_API nmf_status nmf_peak_fp32(double *tflops)
{
    if (!tflops)
        return NMF_E_ARG;
    CK(measure_fp32_peak(tflops));
    return NMF_OK;
}

NMF_API nmf_status nmf_peak_tc_bf16(nmf_handle h, double *tflops)
{
    if (!h || !tflops)
        return NMF_E_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaMemset(h->status, 0, sizeof(unsigned)));
    CK(measure_tc_peak(tflops, h->status));
    unsigned st = 0;
    CK(cudaMemcpy(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    return (st & kStTimeout) ? NMF_E_TIMEOUT : NMF_OK;
}

NMF_API nmf_status nmf_peak_l2_gather(int r, double *gbs)
{
    if (!gbs)
        return NMF_E_ARG;
    if (bad_r(r))
        return NMF_E_SHAPE;
    CK(measure_l2_gather(r, gbs));
    return NMF_OK;
}

// ---------------------------------------------------------------------------
// projection onto a fixed basis
// ---------------------------------------------------------------------------
NMF_API nmf_status nmf_project(nmf_handle h, const float *Qt, const float *d, const float *W,
                               int64_t wrows, int r, const nmf_csr *VnewT, float *Hnew,
                               const nmf_nnls_opts *opts)
{
    if (!h || !Qt || !d || !W || !VnewT || !Hnew)
        return NMF_E_ARG;
    if (bad_r(r) || wrows < 0 || VnewT->rows < 0 || VnewT->cols != wrows)
        return NMF_E_SHAPE;
    if (!VnewT->rowptr || (VnewT->nnz > 0 && (!VnewT->colidx || !VnewT->vals)))
        return NMF_E_ARG;
    if (VnewT->dt != NMF_F32 && VnewT->dt != NMF_BF16)
        return NMF_E_DTYPE;
    const int64_t w = VnewT->rows;
    if (w == 0)
        return NMF_OK;
    nmf_status st = ensure_ws(h, sizeof(float) * (size_t)w * r + 256);
    if (st)
        return st;
    float *C = reinterpret_cast<float *>(h->ws);
    CK(launch_spmm_rowwarp(VnewT->rowptr, VnewT->colidx, VnewT->vals, VnewT->dt, w, W, r, C,
                           h->stream));
    return nmf_nnls_update(h, Qt, d, C, w, r, 0.f, Hnew, opts, nullptr);
}
