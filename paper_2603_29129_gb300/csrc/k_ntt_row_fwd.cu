// k_ntt_row_fwd.cu -- forward row-pass instantiations (one kernel per local
// length 2^m2, m2 = 0..14); the kernels are described in ntt_impl.cuh.
#include "ntt_impl.cuh"

namespace oz {

cudaError_t launch_ntt_fwd_row(const NttGeom& g, uint32_t* data, const uint2* tw, cudaStream_t s)
{
    if (g.nvec == 0) return cudaSuccess;
    switch (g.m2) {
    case 0: return launch_row_m<false, false, 0>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 1: return launch_row_m<false, false, 1>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 2: return launch_row_m<false, false, 2>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 3: return launch_row_m<false, false, 3>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 4: return launch_row_m<false, false, 4>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 5: return launch_row_m<false, false, 5>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 6: return launch_row_m<false, false, 6>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 7: return launch_row_m<false, false, 7>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 8: return launch_row_m<false, false, 8>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 9: return launch_row_m<false, false, 9>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 10: return launch_row_m<false, false, 10>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 11: return launch_row_m<false, false, 11>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 12: return launch_row_m<false, false, 12>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 13: return launch_row_m<false, false, 13>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    case 14: return launch_row_m<false, false, 14>(g, data, tw, MacSrc{nullptr, nullptr}, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace oz
