// Instantiations of the grouped NQP solver (k_nnls.cuh) for J = 4
// coordinates per lane and every group width G.
#include "k_nnls.cuh"

namespace nmfi {

cudaError_t nnls_dispatch_j4(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s)
{
    return nnls_detail::dispatch<4>(a, G, prep_only, s);
}

}  // namespace nmfi
