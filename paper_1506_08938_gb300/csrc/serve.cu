// Projection server: continuous batching of E-step requests (Alg. 1 E-step /
// the first loop of Alg. 2) against a fixed, device-resident basis W.
//
// A request is a block of w new data columns given as host CSR (one CSR row
// per new column, over the basis rows).  The scheduler thread:
//   * admits queued requests in arrival order into the next free slot while
//     the batch fits the slot (columns, nonzeros) and the bytes held by all
//     batches in flight stay within the HBM budget - requests that arrive
//     while others run are admitted as slots and memory free up;
//   * packs the admitted CSR blocks into one batch (rebased row pointers) in
//     pinned staging memory and enqueues, on the slot's own stream: the
//     host-to-device copies, the row-per-warp SpMM C = Vnew W, the NNLS
//     solve of every new column against the rescaled basis Gram, and the
//     device-to-host copy of the results;
//   * polls slot events, copies each request's rows to its output buffer,
//     stamps its latency (submit -> result in host memory) and frees the
//     slot.
// Several slots are in flight at once, so batches overlap on the device.
// Each new column's result depends on that column alone (row-per-warp SpMM,
// warp-per-row NNLS), so it is the same alone and inside any mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nmf_internal.cuh"

using namespace nmfi;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    int64_t w, nnz;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colidx;
    std::vector<float> vals;
    float *out;                 // host, w x r
    Clock::time_point t_submit;
    size_t bytes;               // device footprint while in flight
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    char *dev = nullptr;        // device buffer
    char *host = nullptr;       // pinned staging (inputs, then outputs)
    bool busy = false;
    std::vector<Request> reqs;
    int64_t cols = 0, nnz = 0;
    size_t bytes = 0;
};

}  // namespace

struct nmf_server_s {
    int device = 0;
    int r = 0;
    int64_t wrows = 0;
    const float *W = nullptr;
    float *Qt = nullptr, *d = nullptr, *gram_ws = nullptr;
    nmf_server_opts_t o{};
    std::vector<Slot> slots;
    size_t slot_bytes = 0, host_bytes = 0;
    std::deque<Request> queue;
    std::unordered_map<int64_t, double> done_ms;   // ticket -> latency
    int64_t next_ticket = 1;
    size_t inflight_bytes = 0;
    int64_t completed = 0, completed_cols = 0, batches = 0, max_queue = 0;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    bool stop = false;
    nmf_status error = NMF_OK;
    std::thread worker;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t batch_bytes(int64_t cols, int64_t nnz, int r)
{
    return align256(8 * (size_t)(cols + 1)) + align256(4 * (size_t)nnz) +
           align256(4 * (size_t)nnz) + 2 * align256(4 * (size_t)cols * r);
}

// enqueue the whole pipeline of one batch on its slot's stream
nmf_status launch_batch(nmf_server_s *S, Slot &sl)
{
    const int r = S->r;
    const int64_t cols = sl.cols, nnz = sl.nnz;
    // pack inputs into pinned staging: rowptr | colidx | vals
    char *hp = sl.host;
    int64_t *rp = reinterpret_cast<int64_t *>(hp);
    int32_t *ci = reinterpret_cast<int32_t *>(hp + align256(8 * (cols + 1)));
    float *va = reinterpret_cast<float *>(reinterpret_cast<char *>(ci) + align256(4 * nnz));
    int64_t row0 = 0, nz0 = 0;
    rp[0] = 0;
    for (auto &q : sl.reqs) {
        for (int64_t i = 0; i < q.w; ++i)
            rp[row0 + i + 1] = nz0 + q.rowptr[i + 1];
        std::memcpy(ci + nz0, q.colidx.data(), 4 * q.nnz);
        std::memcpy(va + nz0, q.vals.data(), 4 * q.nnz);
        row0 += q.w;
        nz0 += q.nnz;
    }
    const size_t in_bytes = align256(8 * (cols + 1)) + align256(4 * nnz) + align256(4 * nnz);
    char *dp = sl.dev;
    int64_t *drp = reinterpret_cast<int64_t *>(dp);
    int32_t *dci = reinterpret_cast<int32_t *>(dp + align256(8 * (cols + 1)));
    float *dva = reinterpret_cast<float *>(reinterpret_cast<char *>(dci) + align256(4 * nnz));
    float *C = reinterpret_cast<float *>(dp + in_bytes);
    float *H = reinterpret_cast<float *>(dp + in_bytes + align256(4 * (size_t)cols * r));
    cudaStream_t st = sl.stream;
    if (cudaMemcpyAsync(dp, hp, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return NMF_E_CUDA;
    if (cudaMemsetAsync(H, 0, 4 * (size_t)cols * r, st) != cudaSuccess)
        return NMF_E_CUDA;
    if (launch_spmm_rowwarp(drp, dci, dva, NMF_F32, cols, S->W, r, C, st) != cudaSuccess)
        return NMF_E_CUDA;
    NnlsArgs a{};
    a.Qt = S->Qt;
    a.d = S->d;
    a.C = C;
    a.nsplit = 1;
    a.c_stride = cols * r;
    a.rows = cols;
    a.r = r;
    a.alpha = 0.f;
    a.X = H;
    a.max_inner = S->o.nnls.max_inner;
    a.eps = (float)S->o.nnls.eps;
    a.cd_steps = S->o.nnls.cd_steps;
    a.lanes = S->o.nnls.lanes;
    a.grad_refresh = S->o.nnls.grad_refresh;
    if (launch_nnls(a, st) != cudaSuccess)
        return NMF_E_CUDA;
    if (cudaMemcpyAsync(sl.host, H, 4 * (size_t)cols * r, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return NMF_E_CUDA;
    if (cudaEventRecord(sl.done, st) != cudaSuccess)
        return NMF_E_CUDA;
    return NMF_OK;
}

void worker_loop(nmf_server_s *S)
{
    cudaSetDevice(S->device);
    prof_thread_off();
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // 1. completions
        for (auto &sl : S->slots) {
            if (!sl.busy)
                continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady)
                continue;
            const auto now = Clock::now();
            if (q != cudaSuccess) {
                S->error = NMF_E_CUDA;
                cudaGetLastError();
            }
            const float *res = reinterpret_cast<const float *>(sl.host);
            int64_t off = 0;
            for (auto &rq : sl.reqs) {
                std::memcpy(rq.out, res + off * S->r, 4 * (size_t)rq.w * S->r);
                off += rq.w;
                const double ms =
                    std::chrono::duration<double, std::milli>(now - rq.t_submit).count();
                S->done_ms[rq.ticket] = ms;
                ++S->completed;
                S->completed_cols += rq.w;
            }
            S->inflight_bytes -= sl.bytes;
            sl.reqs.clear();
            sl.busy = false;
            S->cv_done.notify_all();
        }
        // 2. admission: fill free slots from the queue head
        for (auto &sl : S->slots) {
            if (sl.busy || S->queue.empty())
                continue;
            sl.cols = sl.nnz = 0;
            sl.bytes = 0;
            while (!S->queue.empty()) {
                Request &q = S->queue.front();
                const int64_t c2 = sl.cols + q.w, z2 = sl.nnz + q.nnz;
                const size_t b2 = batch_bytes(c2, z2, S->r);
                if (c2 > S->o.max_batch_cols || b2 > S->slot_bytes ||
                    S->inflight_bytes + b2 > S->o.hbm_budget)
                    break;
                sl.cols = c2;
                sl.nnz = z2;
                sl.bytes = b2;
                sl.reqs.push_back(std::move(q));
                S->queue.pop_front();
            }
            if (sl.reqs.empty())
                break;   // head waits for memory to free up
            S->inflight_bytes += sl.bytes;
            sl.busy = true;
            ++S->batches;
            nmf_status e = launch_batch(S, sl);
            if (e != NMF_OK)
                S->error = e;
        }
        bool any_busy = false;
        for (auto &sl : S->slots)
            any_busy = any_busy || sl.busy;
        if (S->stop && !any_busy && S->queue.empty())
            break;
        if (any_busy) {
            // poll completions without holding the lock
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

NMF_API nmf_status nmf_server_create(nmf_server_t *out, int device, const float *W, int64_t wrows,
                                     int r, const nmf_server_opts_t *opts)
{
    if (!out || !W || !opts)
        return NMF_E_ARG;
    *out = nullptr;
    if (r < 1 || r > kMaxRank || wrows < 1)
        return NMF_E_SHAPE;
    if (opts->slots < 1 || opts->slots > 64 || opts->max_batch_cols < 1 ||
        opts->max_batch_nnz < 1 || opts->hbm_budget == 0)
        return NMF_E_ARG;
    if (cudaSetDevice(device) != cudaSuccess)
        return NMF_E_CUDA;
    auto *S = new nmf_server_s;
    S->device = device;
    S->r = r;
    S->wrows = wrows;
    S->W = W;
    S->o = *opts;
    if (S->o.nnls.max_inner <= 0)
        nmf_nnls_opts_default(&S->o.nnls);
    {
        int lg = 0, lj = 0;
        if (!nnls_layout(r, S->o.nnls.lanes, &lg, &lj)) {
            delete S;
            return NMF_E_ARG;
        }
    }
    S->slot_bytes = batch_bytes(opts->max_batch_cols, opts->max_batch_nnz, r);
    S->host_bytes = S->slot_bytes;
    // basis Gram, rescaled once: Qt and d (the E-step's shared Q, Alg. 2)
    const int gs = gram_splits(wrows);
    size_t gbytes = sizeof(float) * ((size_t)gs * r * r + 2 * (size_t)r * r + r) + 1024;
    if (cudaMalloc(&S->gram_ws, gbytes) != cudaSuccess) {
        delete S;
        return NMF_E_NOMEM;
    }
    float *P = S->gram_ws, *G = P + (size_t)gs * r * r;
    S->Qt = G + (size_t)r * r;
    S->d = S->Qt + (size_t)r * r;
    if (launch_gram_partial(W, wrows, r, r, P, gs, nullptr) != cudaSuccess ||
        launch_sum_slices(P, gs, (int64_t)r * r, G, nullptr) != cudaSuccess ||
        launch_rescale(G, 1, r, 0.f, nullptr, nullptr, S->Qt, S->d, nullptr) != cudaSuccess ||
        prepare_nnls(r, S->o.nnls.lanes) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(S->gram_ws);
        delete S;
        return NMF_E_CUDA;
    }
    S->slots.resize(opts->slots);
    for (auto &sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&sl.dev, S->slot_bytes) != cudaSuccess ||
            cudaMallocHost(&sl.host, S->host_bytes) != cudaSuccess) {
            nmf_server_destroy(S);
            return NMF_E_NOMEM;
        }
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return NMF_OK;
}

NMF_API nmf_status nmf_server_submit(nmf_server_t S, int64_t w, int64_t nnz, const int64_t *rowptr,
                                     const int32_t *colidx, const float *vals, float *out,
                                     int64_t *ticket)
{
    if (!S || !rowptr || !out || !ticket || w < 1 || nnz < 0 || (nnz > 0 && (!colidx || !vals)))
        return NMF_E_ARG;
    if (rowptr[0] != 0 || rowptr[w] != nnz || fault_armed("csr"))
        return NMF_E_ARG;
    for (int64_t i = 0; i < nnz; ++i)
        if (colidx[i] < 0 || colidx[i] >= S->wrows)
            return NMF_E_ARG;
    const size_t b = batch_bytes(w, nnz, S->r);
    // a request that could never be admitted is refused up front
    if (w > S->o.max_batch_cols || b > S->slot_bytes || b > S->o.hbm_budget ||
        fault_armed("admit"))
        return NMF_E_BUSY;
    Request q;
    q.w = w;
    q.nnz = nnz;
    q.rowptr.assign(rowptr, rowptr + w + 1);
    q.colidx.assign(colidx, colidx + nnz);
    q.vals.assign(vals, vals + nnz);
    q.out = out;
    q.bytes = b;
    q.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->error != NMF_OK)
            return S->error;
        q.ticket = S->next_ticket++;
        *ticket = q.ticket;
        S->queue.push_back(std::move(q));
        if ((int64_t)S->queue.size() > S->max_queue)
            S->max_queue = (int64_t)S->queue.size();
    }
    S->cv.notify_one();
    return NMF_OK;
}

NMF_API nmf_status nmf_server_wait(nmf_server_t S, int64_t ticket, double timeout_s,
                                   double *latency_ms)
{
    if (!S || ticket < 1)
        return NMF_E_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (!S->done_ms.count(ticket)) {
        if (S->error != NMF_OK)
            return S->error;
        if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
            !S->done_ms.count(ticket))
            return NMF_E_TIMEOUT;
    }
    if (latency_ms)
        *latency_ms = S->done_ms[ticket];
    return NMF_OK;
}

NMF_API nmf_status nmf_server_stats(nmf_server_t S, nmf_server_stats_t *st)
{
    if (!S || !st)
        return NMF_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    st->completed = S->completed;
    st->completed_cols = S->completed_cols;
    st->batches = S->batches;
    st->queued = (int64_t)S->queue.size();
    st->max_queue = S->max_queue;
    st->inflight_bytes = (int64_t)S->inflight_bytes;
    return S->error;
}

NMF_API nmf_status nmf_server_destroy(nmf_server_t S)
{
    if (!S)
        return NMF_E_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable())
        S->worker.join();
    cudaSetDevice(S->device);
    for (auto &sl : S->slots) {
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
        if (sl.done)
            cudaEventDestroy(sl.done);
        if (sl.dev)
            cudaFree(sl.dev);
        if (sl.host)
            cudaFreeHost(sl.host);
    }
    if (S->gram_ws)
        cudaFree(S->gram_ws);
    delete S;
    return NMF_OK;
}
