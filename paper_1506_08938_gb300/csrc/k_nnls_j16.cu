// Instantiations of the grouped NQP solver (k_nnls.cuh) for J = 16
// coordinates per lane and every group width G.
#include "k_nnls.cuh"

namespace nmfi {

cudaError_t nnls_dispatch_j16(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s)
{
    return nnls_detail::dispatch<16>(a, G, prep_only, s);
}

}  // namespace nmfi
