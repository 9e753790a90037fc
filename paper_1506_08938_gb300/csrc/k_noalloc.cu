// nmf_gram_noalloc: the Gram matrix Q = X^T X + beta I computed without any
// device allocation, for callers that cannot call cudaMalloc.
//
// Its split-K partial sums live in one file-scope device array of fixed size
// (gScratch below, about 4.2 MB), which every GPU that loads this library
// keeps until the process exits.  Host code cannot use the array's name as a
// device address, so the address is looked up once per device with
// cudaGetSymbolAddress (on the first call made while that device is current)
// and passed to the kernels.
#include <mutex>

#include "nmf_internal.cuh"

namespace {

constexpr int kMaxSlices = 63;                       // partial Gram slices
constexpr size_t kScratchFloats =
    (size_t)(kMaxSlices + 1) * nmfi::kMaxRank * nmfi::kMaxRank;   // slices + reduced G

__device__ __align__(256) float gScratch[kScratchFloats];

constexpr int kMaxDevices = 64;
float *g_addr[kMaxDevices] = {nullptr};
std::mutex g_mu;

// true when p is device (or managed) memory usable from device `dev`
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged)
        return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// device address of gScratch on device `dev`, the current device (looked up
// once per device; a device reset ends the context the cached address
// belongs to)
cudaError_t scratch_address(int dev, float **out)
{
    cudaError_t e = cudaSuccess;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, gScratch);
        if (e != cudaSuccess)
            return e;
        g_addr[dev] = static_cast<float *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

NMF_API nmf_status nmf_gram_noalloc(const nmf_dense *X, float beta, float *Q, void *cuda_stream)
{
    if (!X || !Q || (!X->data && X->rows > 0))
        return NMF_E_ARG;
    if (X->rows < 0 || X->cols < 1 || X->ld < X->cols)
        return NMF_E_SHAPE;
    if (X->cols > nmfi::kMaxRank)   // the scratch holds r <= 128 only
        return NMF_E_SHAPE;
    if (X->dt != NMF_F32)
        return NMF_E_DTYPE;
    const int r = (int)X->cols;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return NMF_E_CUDA;
    }
    // the kernels run on the current device: X and Q must live there
    if ((X->rows > 0 && !on_device(X->data, dev)) || !on_device(Q, dev))
        return NMF_E_ARG;
    int S = nmfi::gram_splits(X->rows);
    if (S > kMaxSlices)
        S = kMaxSlices;
    float *scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) {
        cudaGetLastError();
        return NMF_E_CUDA;
    }
    float *P = scratch;                                   // S slices of r x r
    float *G = scratch + (size_t)kMaxSlices * nmfi::kMaxRank * nmfi::kMaxRank;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    // no profiler events on this thread meanwhile: creating them would allocate
    const bool prof_was_off = nmfi::prof_thread_set_off(true);
    cudaError_t e = nmfi::launch_gram_partial((const float *)X->data, X->rows, X->ld, r, P, S, s);
    if (e == cudaSuccess)
        e = nmfi::launch_sum_slices(P, S, (int64_t)r * r, G, s);
    if (e == cudaSuccess)
        e = nmfi::launch_rescale(G, 1, r, beta, nullptr, Q, nullptr, nullptr, s);
    nmfi::prof_thread_set_off(prof_was_off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NMF_E_CUDA;
    }
    return NMF_OK;
}
