// The handle and the workspace helpers shared by the host-side translation
// units of the C ABI (api.cu, stream.cu).
#pragma once

#include "nmf_internal.cuh"

struct nmf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;          // arena
    size_t ws_cap = 0;
    // small fixed device buffers
    unsigned *status = nullptr;  // latched device status
    unsigned *tickets = nullptr; // 8 reduction tickets
    double *partials = nullptr;  // 3 * 256 doubles
    double *scal = nullptr;      // 16 doubles of scalar outputs
    unsigned long long *ctr = nullptr;  // 4 counters
    int *idev = nullptr;         // 4 ints (iteration index, done flag)
    unsigned *smax = nullptr;    // 2 words (maxStop bits per factor)
    cudaStream_t cap = nullptr;  // private stream for graph capture (the
                                 // legacy default stream cannot be captured)
    cudaStream_t side = nullptr; // second stream of the solve (work beside the cross term)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    char *stage = nullptr;       // device copies of host-resident solve inputs
    size_t stage_cap = 0;
};

namespace nmfi {

struct Arena {
    char *base;
    size_t off = 0, cap;
    Arena(char *b, size_t c) : base(b), cap(c) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += sizeof(T) * count;
        return p;
    }
};

// Bytes a sequence of take() calls needs: replay them on a null arena.
struct Sizer {
    size_t off = 0;
    template <typename T>
    void add(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        off += sizeof(T) * count;
    }
};

inline nmf_status cuda_st(cudaError_t e)
{
    if (e == cudaSuccess)
        return NMF_OK;
    if (e == cudaErrorMemoryAllocation)
        return NMF_E_NOMEM;
    return NMF_E_CUDA;
}

#define CK(expr)                                  \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess)                    \
            return cuda_st(_e);                   \
    } while (0)

nmf_status ensure_ws(nmf_handle h, size_t bytes);
nmf_nnls_opts opts_or_default(const nmf_nnls_opts *o);
bool bad_r(int r);
// true when p is host memory (pinned or pageable) rather than device memory
bool is_host_ptr(const void *p);

}  // namespace nmfi
