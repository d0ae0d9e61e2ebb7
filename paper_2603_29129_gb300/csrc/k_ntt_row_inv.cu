// k_ntt_row_inv.cu -- inverse row-pass instantiations, with the fused
// multiply-accumulate (one kernel per local length 2^m2, m2 = 0..14); the
// kernels are described in ntt_impl.cuh.
#include "ntt_impl.cuh"

namespace oz {

cudaError_t launch_ntt_inv_row(const NttGeom& g, uint32_t* data, const uint2* tw, MacSrc mac, cudaStream_t s)
{
    if (g.nvec == 0) return cudaSuccess;
    switch (g.m2) {
    case 0: return launch_row_m<true, true, 0>(g, data, tw, mac, s);
    case 1: return launch_row_m<true, true, 1>(g, data, tw, mac, s);
    case 2: return launch_row_m<true, true, 2>(g, data, tw, mac, s);
    case 3: return launch_row_m<true, true, 3>(g, data, tw, mac, s);
    case 4: return launch_row_m<true, true, 4>(g, data, tw, mac, s);
    case 5: return launch_row_m<true, true, 5>(g, data, tw, mac, s);
    case 6: return launch_row_m<true, true, 6>(g, data, tw, mac, s);
    case 7: return launch_row_m<true, true, 7>(g, data, tw, mac, s);
    case 8: return launch_row_m<true, true, 8>(g, data, tw, mac, s);
    case 9: return launch_row_m<true, true, 9>(g, data, tw, mac, s);
    case 10: return launch_row_m<true, true, 10>(g, data, tw, mac, s);
    case 11: return launch_row_m<true, true, 11>(g, data, tw, mac, s);
    case 12: return launch_row_m<true, true, 12>(g, data, tw, mac, s);
    case 13: return launch_row_m<true, true, 13>(g, data, tw, mac, s);
    case 14: return launch_row_m<true, true, 14>(g, data, tw, mac, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace oz
