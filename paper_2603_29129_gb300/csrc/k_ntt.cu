// k_ntt.cu -- batched 32-bit NTTs (§3.3) for libozfft on sm_103a.
//
// Forward transforms are radix-2 decimation-in-frequency (Gentleman-Sande):
// natural-order input, output in bit-reversed order (position bitrev(k) holds
// X(k)).  Inverse transforms are decimation-in-time on bit-reversed input,
// natural-order output; they run the forward stages backwards with w^-1 and
// omit the 1/N, which the plan folds into the w~* spectra.  The pointwise
// products of Alg. 8 are order-agnostic, so no bit reversal is ever done.
//
// A length N = 2^m transform runs in one or two passes over HBM:
//   column pass -- global stages 0..m1-1; a CTA holds T adjacent columns
//                  j2 of the N1 x N2 view (j = j1*N2 + j2, N1 = 2^m1), loaded
//                  row by row (coalesced), and transforms each column over j1
//                  with the full-length twiddles w_N^((j mod h_s) 2^s);
//   row pass    -- global stages m1..m-1, which act inside contiguous blocks
//                  of N2 = 2^m2 elements; a CTA holds TILE/N2 blocks.
// Inside a pass the stages run in rounds of up to three: each thread loads
// 2^r elements of one column from shared memory, does r radix-2 stages in
// registers, and stores them back.
//
// The inverse's first pass (the row pass) builds its input on the fly:
// Z(f) = sum over the flush group of X_s(f) * Ym_t(f) mod p (Montgomery,
// Ym = Y * N^-1 * 2^32 mod p), i.e. the NTT-domain accumulation of Alg. 8
// is fused into the load, and Z never goes to HBM.
#include "oz_common.cuh"
#include "oz_kernels.h"

namespace oz {

__device__ __forceinline__ int pad_idx(int i) { return i + (i >> 5); }

// DIF butterfly: (a, b) -> (a + b, (a - b) w)
__device__ __forceinline__ void bfly_dif(uint32_t& a, uint32_t& b, uint2 w, uint32_t p)
{
    uint32_t s = mod_add(a, b, p);
    uint32_t d = a - b + p;                 // (0, 2p)
    b = shoup(d, w.x, w.y, p);
    a = s;
}
// DIT butterfly: (a, b) -> (a + b w, a - b w)
__device__ __forceinline__ void bfly_dit(uint32_t& a, uint32_t& b, uint2 w, uint32_t p)
{
    uint32_t t = shoup(b, w.x, w.y, p);
    b = mod_sub(a, t, p);
    a = mod_add(a, t, p);
}

// Twiddle source of a round: the table of prime pi is tw_all + pi * (N/2).
// With pvar set, column c uses prime (pi0 + c) mod P (rows that are whole
// vectors of alternating primes); otherwise every column uses pi0.
struct TwSel {
    const uint2* __restrict__ tw_all;
    int64_t stride;   // N / 2
    int pi0, P;
    bool pvar;
};

// One round of R = 2^RL elements per thread on `cols` columns of M = 2^mloc
// elements held in shared memory.  Stages s0 .. s0+RL-1 (local numbering).
// Element i of column c is at sm[pad_idx(c * cstride + i * istride)].
// Twiddle exponent of a butterfly with top element i at stage s:
//   e = ((i mod h_s) * estride + c * ecol + ebase) << s,  h_s = M >> (s+1).
template <bool INV, int RL>
__device__ __forceinline__ void ntt_round(uint32_t* sm, int mloc, int s0, int cols, int cstride, int istride,
                                          int estride, int ebase, int ecol, TwSel ts, bool col_fast)
{
    constexpr int R = 1 << RL;
    const int lg_hlast = mloc - s0 - RL;
    const int hlast = 1 << lg_hlast;
    const int gpc = (1 << mloc) >> RL;   // groups per column
    const int ngroups = gpc * cols;
    for (int gid = threadIdx.x; gid < ngroups; gid += blockDim.x) {
        int c, g;
        if (col_fast) { c = gid % cols; g = gid / cols; }
        else { g = gid & (gpc - 1); c = gid >> (mloc - RL); }
        const int pi = ts.pvar ? (ts.pi0 + c) % ts.P : ts.pi0;
        const uint32_t p = prime_of(pi);
        const uint2* __restrict__ tw = ts.tw_all + pi * ts.stride;
        const int blk = g >> lg_hlast;
        const int low = g & (hlast - 1);
        const int base = (blk << (mloc - s0)) + low;
        const int a0 = c * cstride;
        uint32_t v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = sm[pad_idx(a0 + (base + t * hlast) * istride)];
        const int e0 = low * estride + ebase + c * ecol;
        const int estep = hlast * estride;
        if (!INV) {
#pragma unroll
            for (int j = 0; j < RL; ++j) {
                const int half = R >> (j + 1);
                const int sh = s0 + j;
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    if (t & half) continue;
                    const int e = (e0 + (t & (half - 1)) * estep) << sh;
                    bfly_dif(v[t], v[t + half], __ldg(&tw[e]), p);
                }
            }
        } else {
#pragma unroll
            for (int j = RL - 1; j >= 0; --j) {
                const int half = R >> (j + 1);
                const int sh = s0 + j;
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    if (t & half) continue;
                    const int e = (e0 + (t & (half - 1)) * estep) << sh;
                    bfly_dit(v[t], v[t + half], __ldg(&tw[e]), p);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < R; ++t) sm[pad_idx(a0 + (base + t * hlast) * istride)] = v[t];
    }
}

// all stages of a pass, in rounds of 3 (DIF ascending / DIT descending)
template <bool INV>
__device__ void ntt_stages(uint32_t* sm, int mloc, int cols, int cstride, int istride, int estride, int ebase,
                           int ecol, TwSel ts, bool col_fast)
{
    const int nfull = mloc / 3, rem = mloc % 3;
    if (!INV) {
        for (int r = 0; r < nfull; ++r) {
            ntt_round<false, 3>(sm, mloc, 3 * r, cols, cstride, istride, estride, ebase, ecol, ts, col_fast);
            __syncthreads();
        }
        if (rem == 2) ntt_round<false, 2>(sm, mloc, 3 * nfull, cols, cstride, istride, estride, ebase, ecol, ts, col_fast);
        if (rem == 1) ntt_round<false, 1>(sm, mloc, 3 * nfull, cols, cstride, istride, estride, ebase, ecol, ts, col_fast);
        if (rem) __syncthreads();
    } else {
        if (rem == 2) ntt_round<true, 2>(sm, mloc, 3 * nfull, cols, cstride, istride, estride, ebase, ecol, ts, col_fast);
        if (rem == 1) ntt_round<true, 1>(sm, mloc, 3 * nfull, cols, cstride, istride, estride, ebase, ecol, ts, col_fast);
        if (rem) __syncthreads();
        for (int r = nfull - 1; r >= 0; --r) {
            ntt_round<true, 3>(sm, mloc, 3 * r, cols, cstride, istride, estride, ebase, ecol, ts, col_fast);
            __syncthreads();
        }
    }
}

// vector activity: forward vectors [B][2][K][P] are live when k < kcnt[b][v];
// inverse vectors [B][4][G][P] when g < ngroups of (b, conv).
__device__ __forceinline__ bool fwd_live(const NttGeom& g, int64_t vec)
{
    int64_t bv = vec / (g.P * g.K);
    int k = (int)((vec / g.P) % g.K);
    return k < g.kcnt[bv];
}
__device__ __forceinline__ bool inv_live(const NttGeom& g, int64_t vec)
{
    int64_t bc = vec / (g.P * g.G);
    int grp = (int)((vec / g.P) % g.G);
    return grp < g.sched[bc].ngroups;
}

// ---------------------------------------------------------------- column pass
template <bool INV>
__global__ void __launch_bounds__(512) ntt_col_kernel(NttGeom g, uint32_t* __restrict__ data,
                                                      const uint2* __restrict__ tw_all)
{
    extern __shared__ uint32_t sm[];
    const int N1 = 1 << g.m1, N2 = 1 << g.m2, T = g.T;
    const int tpv = N2 / T;
    const int64_t vec = blockIdx.x / tpv;
    const int col0 = (blockIdx.x % tpv) * T;
    if (INV ? !inv_live(g, vec) : !fwd_live(g, vec)) return;
    const int pi = (int)(vec % g.P);
    uint32_t* v = data + vec * g.N;
    const int tile = N1 * T;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int row = idx / T, c = idx % T;
        sm[pad_idx(idx)] = v[(int64_t)row * N2 + col0 + c];
    }
    __syncthreads();
    // columns c < T, element i at row i: sm[pad(i*T + c)]
    const TwSel ts{tw_all, g.N >> 1, pi, g.P, false};
    ntt_stages<INV>(sm, g.m1, T, 1, T, N2, col0, 1, ts, true);
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int row = idx / T, c = idx % T;
        v[(int64_t)row * N2 + col0 + c] = sm[pad_idx(idx)];
    }
}

// ------------------------------------------------------------------- row pass
// MAC: build the inverse input from the forward spectra X and the plan's w~*
// spectra Ym according to the flush schedule.
template <bool INV, bool MAC>
__global__ void __launch_bounds__(512) ntt_row_kernel(NttGeom g, uint32_t* __restrict__ data,
                                                      const uint2* __restrict__ tw_all, MacSrc mac)
{
    extern __shared__ uint32_t sm[];
    const int M = 1 << g.m2;
    const int64_t rows_total = g.nvec * (g.N >> g.m2);
    const int rpc = g.rows_per_cta;
    const int64_t row0 = (int64_t)blockIdx.x * rpc;
    const int rows = (int)min((int64_t)rpc, rows_total - row0);
    // skip when no row of this CTA belongs to a live vector
    {
        const int64_t vfirst = (row0 * M) >> g.lgN, vlast = ((row0 + rows) * M - 1) >> g.lgN;
        bool any = false;
        for (int64_t vv = vfirst; vv <= vlast && !any; ++vv) any = INV ? inv_live(g, vv) : fwd_live(g, vv);
        if (!any) return;
    }
    const int nel = rows * M;
    const int64_t gbase = row0 * M;
    for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
        const int64_t gi = gbase + idx;
        uint32_t val;
        if (MAC) {
            const int64_t vec = gi >> g.lgN;
            const int64_t j = gi & (g.N - 1);
            const int pi = (int)(vec % g.P);
            const int grp = (int)((vec / g.P) % g.G);
            const int64_t bc = vec / ((int64_t)g.P * g.G);
            const int conv = (int)(bc & 3);
            const int64_t b = bc >> 2;
            const Sched& S = g.sched[bc];
            const uint32_t p = prime_of(pi), pn = pneg_inv_of(pi);
            const int vx = (conv == 0 || conv == 3) ? 0 : 1;   // RR, RI use Re x'; II, IR use Im x'
            const int vw = (conv == 0 || conv == 2) ? 0 : 1;   // RR, IR use Re w*; II, RI use Im w*
            uint32_t acc = 0;
            if (grp < S.ngroups) {
                const int sz = S.size[grp];
                for (int m = 0; m < sz; ++m) {
                    const int pr = S.pair[grp][m];
                    const int s = pr >> 4, t = pr & 15;
                    const uint32_t xv = mac.X[(((b * 2 + vx) * g.K + s) * g.P + pi) * g.N + j];
                    const uint32_t yv = mac.Ym[(((int64_t)vw * g.K + t) * g.P + pi) * g.N + j];
                    acc = mod_add(acc, mont_mul(xv, yv, p, pn), p);
                }
            }
            val = acc;
        } else {
            val = data[gi];
        }
        sm[pad_idx(idx)] = val;
    }
    __syncthreads();
    {
        // each row is a column of M elements at sm[pad(r*M + i)]; rows that are
        // whole vectors (N = M) alternate primes
        const int64_t vec0 = gbase >> g.lgN;
        const bool pvar = (g.N >> g.m2) < rpc && g.P > 1;
        const TwSel ts{tw_all, g.N >> 1, (int)(vec0 % g.P), g.P, pvar};
        ntt_stages<INV>(sm, g.m2, rows, M, 1, 1 << g.m1, 0, 0, ts, false);
    }
    for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) data[gbase + idx] = sm[pad_idx(idx)];
}

}  // namespace oz

// --------------------------------------------------------------------- host
namespace oz {

static constexpr int TILE_LOG = 13;

void ntt_configure(NttGeom& g, int64_t N)
{
    g.N = N;
    int lg = 0;
    while ((int64_t(1) << lg) < N) ++lg;
    g.lgN = lg;
    if (lg <= TILE_LOG) {
        g.m1 = 0;
        g.m2 = lg;
    } else {
        g.m2 = TILE_LOG;
        g.m1 = lg - TILE_LOG;
        if (g.m1 > 10) { g.m1 = 10; g.m2 = lg - 10; }
    }
    if (g.m1 > 0) {
        int T = (1 << TILE_LOG) >> g.m1;
        if (T < 32) T = 32;
        if (T > (1 << g.m2)) T = 1 << g.m2;
        g.T = T;
    } else {
        g.T = 0;
    }
    g.rows_per_cta = g.m2 <= TILE_LOG ? (1 << (TILE_LOG - g.m2)) : 1;
}

int64_t ntt_launches(const NttGeom& g) { return g.m1 > 0 ? 2 : 1; }

static int threads_for(int64_t tile) { return tile <= (1 << TILE_LOG) ? 256 : 512; }
static size_t smem_for(int64_t tile) { return (size_t)(tile + tile / 32) * sizeof(uint32_t); }

template <typename K>
static cudaError_t prep(K kernel, size_t smem)
{
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <bool INV>
static cudaError_t launch_col(const NttGeom& g, uint32_t* data, const uint2* tw, cudaStream_t s)
{
    const int64_t tile = (int64_t(1) << g.m1) * g.T;
    const size_t smem = smem_for(tile);
    cudaError_t e = prep(ntt_col_kernel<INV>, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = g.nvec * ((int64_t(1) << g.m2) / g.T);
    ntt_col_kernel<INV><<<(unsigned)grid, threads_for(tile), smem, s>>>(g, data, tw);
    return cudaGetLastError();
}

template <bool INV, bool MAC>
static cudaError_t launch_row(const NttGeom& g, uint32_t* data, const uint2* tw, MacSrc mac, cudaStream_t s)
{
    const int64_t tile = (int64_t(1) << g.m2) * g.rows_per_cta;
    const size_t smem = smem_for(tile);
    cudaError_t e = prep(ntt_row_kernel<INV, MAC>, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows_total = g.nvec * (g.N >> g.m2);
    const int64_t grid = (rows_total + g.rows_per_cta - 1) / g.rows_per_cta;
    ntt_row_kernel<INV, MAC><<<(unsigned)grid, threads_for(tile), smem, s>>>(g, data, tw, mac);
    return cudaGetLastError();
}

cudaError_t launch_ntt_fwd_col(const NttGeom& g, uint32_t* X, const uint2* tw, cudaStream_t s)
{
    return (g.nvec == 0 || g.m1 == 0) ? cudaSuccess : launch_col<false>(g, X, tw, s);
}
cudaError_t launch_ntt_fwd_row(const NttGeom& g, uint32_t* X, const uint2* tw, cudaStream_t s)
{
    return g.nvec == 0 ? cudaSuccess : launch_row<false, false>(g, X, tw, MacSrc{nullptr, nullptr}, s);
}
cudaError_t launch_ntt_inv_row(const NttGeom& g, uint32_t* Z, const uint2* twinv, MacSrc mac, cudaStream_t s)
{
    return g.nvec == 0 ? cudaSuccess : launch_row<true, true>(g, Z, twinv, mac, s);
}
cudaError_t launch_ntt_inv_col(const NttGeom& g, uint32_t* Z, const uint2* twinv, cudaStream_t s)
{
    return (g.nvec == 0 || g.m1 == 0) ? cudaSuccess : launch_col<true>(g, Z, twinv, s);
}
cudaError_t launch_ntt_forward(const NttGeom& g, uint32_t* X, const uint2* tw, cudaStream_t s)
{
    cudaError_t e = launch_ntt_fwd_col(g, X, tw, s);
    return e != cudaSuccess ? e : launch_ntt_fwd_row(g, X, tw, s);
}

}  // namespace oz
