// Instantiations of the grouped NQP solver (k_nnls.cuh) for J = 2
// coordinates per lane and every group width G.
#include "k_nnls.cuh"

namespace nmfi {

cudaError_t nnls_dispatch_j2(const NnlsArgs &a, int G, bool prep_only, cudaStream_t s)
{
    return nnls_detail::dispatch<2>(a, G, prep_only, s);
}

}  // namespace nmfi
