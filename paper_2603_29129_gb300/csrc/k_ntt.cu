// k_ntt.cu -- host-side geometry of the batched NTTs (ntt_impl.cuh): how a
// length N = 2^m transform is cut into a column pass (stages 0..m1-1) and a row
// pass (stages m1..m-1), and the forward transform as the two launches.
#include "ntt_impl.cuh"

namespace oz {

void ntt_configure(NttGeom& g, int64_t N)
{
    g.N = N;
    int lg = 0;
    while ((int64_t(1) << lg) < N) ++lg;
    g.lgN = lg;
    if (lg <= TILE_LOG) {          // one pass: whole vectors in a CTA tile
        g.m1 = 0;
        g.m2 = lg;
    } else {                       // rows of 2^12 (2^13, 2^14 for N = 2^23, 2^24), columns of the rest
        g.m2 = TILE_LOG;
        g.m1 = lg - TILE_LOG;
        if (g.m1 > 10) { g.m1 = 10; g.m2 = lg - 10; }
    }
    g.T = g.m1 > 0 ? (1 << col_log_t(g.m1)) : 0;
    g.rows_per_cta = g.m2 <= TILE_LOG ? (1 << (TILE_LOG - g.m2)) : 1;
}

bool ntt_configure_split(NttGeom& g, int64_t N, int m2)
{
    ntt_configure(g, N);
    const int lg = g.lgN;
    // row kernels exist for 2^0 .. 2^14 residues, column kernels for 2^1 .. 2^10 rows
    if (m2 < 0 || m2 > 14 || m2 > lg || (lg - m2 > 10) || (lg - m2 > 0 && m2 < 5)) return false;
    g.m2 = m2;
    g.m1 = lg - m2;
    g.T = g.m1 > 0 ? (1 << col_log_t(g.m1)) : 0;
    if (g.m1 > 0 && g.T > (1 << g.m2)) return false;  // a column tile wider than a row
    g.rows_per_cta = g.m2 <= TILE_LOG ? (1 << (TILE_LOG - g.m2)) : 1;
    return true;
}

int64_t ntt_launches(const NttGeom& g) { return g.m1 > 0 ? 2 : 1; }

cudaError_t launch_ntt_forward(const NttGeom& g, uint32_t* X, const uint2* tw, cudaStream_t s)
{
    cudaError_t e = launch_ntt_fwd_col(g, X, tw, s);
    return e != cudaSuccess ? e : launch_ntt_fwd_row(g, X, tw, s);
}

}  // namespace oz
