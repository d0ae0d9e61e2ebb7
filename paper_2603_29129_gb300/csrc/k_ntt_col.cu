// k_ntt_col.cu -- column-pass instantiations (one kernel per column length
// 2^m1, m1 = 1..10) for both directions; the kernels are described in
// ntt_impl.cuh.  Plans with a tensor map take the TMA kernels of
// k_ntt_col_tma.cu for m1 >= 4.
#include "ntt_impl.cuh"

namespace oz {

cudaError_t launch_ntt_fwd_col(const NttGeom& g, uint32_t* data, const uint2* tw, cudaStream_t s)
{
    if (g.nvec == 0 || g.m1 == 0) return cudaSuccess;
    cudaError_t e;
    if (launch_col_tma(false, g, tw, s, &e)) return e;
    switch (g.m1) {
    case 1: return launch_col_m<false, 1>(g, data, tw, s);
    case 2: return launch_col_m<false, 2>(g, data, tw, s);
    case 3: return launch_col_m<false, 3>(g, data, tw, s);
    case 4: return launch_col_m<false, 4>(g, data, tw, s);
    case 5: return launch_col_m<false, 5>(g, data, tw, s);
    case 6: return launch_col_m<false, 6>(g, data, tw, s);
    case 7: return launch_col_m<false, 7>(g, data, tw, s);
    case 8: return launch_col_m<false, 8>(g, data, tw, s);
    case 9: return launch_col_m<false, 9>(g, data, tw, s);
    case 10: return launch_col_m<false, 10>(g, data, tw, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ntt_inv_col(const NttGeom& g, uint32_t* data, const uint2* tw, cudaStream_t s)
{
    if (g.nvec == 0 || g.m1 == 0) return cudaSuccess;
    cudaError_t e;
    if (launch_col_tma(true, g, tw, s, &e)) return e;
    switch (g.m1) {
    case 1: return launch_col_m<true, 1>(g, data, tw, s);
    case 2: return launch_col_m<true, 2>(g, data, tw, s);
    case 3: return launch_col_m<true, 3>(g, data, tw, s);
    case 4: return launch_col_m<true, 4>(g, data, tw, s);
    case 5: return launch_col_m<true, 5>(g, data, tw, s);
    case 6: return launch_col_m<true, 6>(g, data, tw, s);
    case 7: return launch_col_m<true, 7>(g, data, tw, s);
    case 8: return launch_col_m<true, 8>(g, data, tw, s);
    case 9: return launch_col_m<true, 9>(g, data, tw, s);
    case 10: return launch_col_m<true, 10>(g, data, tw, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace oz
