// Launch-shape choice of the grouped NQP solver (Alg. 3, k_nnls.cuh): G lanes
// per row and J = RP / G coordinates per lane.
#include "k_nnls.cuh"

namespace nmfi {

// G: explicit (1, 2, 4, ..., 32) or, for lanes == 0, the fewest lanes that
// keep J <= 8 (fewest shuffles per coordinate step); J: the smallest of
// 2, 4, 8, 16 with G * J >= r and G * J >= 4.  Depends on r and lanes only,
// so a row's result never depends on how many rows share the launch.
bool nnls_layout(int r, int lanes, int *G, int *J)
{
    int g = lanes;
    if (g == 0) {
        const int need = (r + 7) / 8;
        g = 1;
        while (g < need)
            g <<= 1;
    }
    if (g < 1 || g > 32 || (g & (g - 1)))
        return false;
    for (int j = 2; j <= 16; j <<= 1)
        if (g * j >= r && g * j >= 4) {
            *G = g;
            *J = j;
            return true;
        }
    return false;
}

static cudaError_t nnls_go(const NnlsArgs &a, int r, int lanes, bool prep_only, cudaStream_t s)
{
    int G = 0, J = 0;
    if (!nnls_layout(r, lanes, &G, &J))
        return cudaErrorInvalidValue;
    switch (J) {
    case 2: return nnls_dispatch_j2(a, G, prep_only, s);
    case 4: return nnls_dispatch_j4(a, G, prep_only, s);
    case 8: return nnls_dispatch_j8(a, G, prep_only, s);
    default: return nnls_dispatch_j16(a, G, prep_only, s);
    }
}

cudaError_t prepare_nnls(int r, int lanes)
{
    NnlsArgs a{};
    return nnls_go(a, r, lanes, true, nullptr);
}

int nnls_grid_query(const NnlsArgs &a0)
{
    NnlsArgs a = a0;
    int g = 0;
    a.grid_query = true;
    a.grid_out = &g;
    if (a.rows <= 0 || nnls_go(a, a.r, a.lanes, false, nullptr) != cudaSuccess)
        return 0;
    return g;
}

cudaError_t launch_nnls(const NnlsArgs &a, cudaStream_t s)
{
    ProfScope prof_(KC_NNLS, s);
    if (a.rows <= 0)
        return cudaSuccess;
    return nnls_go(a, a.r, a.lanes, false, s);
}

}  // namespace nmfi
