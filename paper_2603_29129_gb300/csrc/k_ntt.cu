// k_ntt.cu -- batched 32-bit NTTs (§3.3) for libozfft on sm_103a.
//
// Forward transforms are radix-2 Cooley-Tukey on natural-order input with the
// output in bit-reversed order (position bitrev(k) holds X(k)); inverse
// transforms are Gentleman-Sande on bit-reversed input with natural-order
// output and no 1/N (the plan folds N^-1 into the w~* spectra).  The pointwise
// products of Alg. 8 do not care about the order, so nothing is ever permuted.
//
// Twiddles are per block: at stage s (2^s blocks of 2t = N/2^s elements) every
// butterfly of block i uses tw[2^s + i] = w^((N/2^(s+1)) * bitrev_s(i)), so a
// stage needs 2^s table entries, contiguous in memory.  The butterflies are
//   forward:  (a, b) -> (a + b W, a - b W)
//   inverse:  (a, b) -> (a + b, (a - b) W^-1)
// with residues kept canonical in [0, p) and Shoup products (oz_common.cuh).
//
// A length N = 2^m transform takes one or two passes over HBM:
//   column pass -- stages 0..m1-1.  With j = j1*N2 + j2 (N1 = 2^m1, N2 = 2^m2)
//                  these stages act on each column j2 exactly as a length-N1
//                  transform with the same table entries, so a CTA loads T
//                  adjacent columns (row segments, coalesced) and transforms
//                  them in shared memory;
//   row pass    -- stages m1..m-1 act inside contiguous rows of N2 elements;
//                  for row r, local stage s and local block i the twiddle is
//                  tw[((2^m1 + r) << s) + i].
// Inside a pass, stages run in rounds of up to four: a thread loads 2^RL
// elements of one column from shared memory, does RL stages in registers
// (2^j contiguous twiddles at the j-th), and stores them back.
//
// The inverse's first pass (the row pass) builds its input on the fly:
// Z(f) = sum over the flush group of X_s(f) * Ym_t(f) mod p (Montgomery,
// Ym = Y * N^-1 * 2^32 mod p): the NTT-domain accumulation of Alg. 8 is fused
// into the load, and Z never goes to HBM.
#include "oz_common.cuh"
#include "oz_kernels.h"

namespace oz {

constexpr int NTT_THREADS = 512;
constexpr int TILE_LOG = 13;

__device__ __forceinline__ int pad_idx(int i) { return i + (i >> 5); }

__device__ __forceinline__ void bfly_ct(uint32_t& a, uint32_t& b, uint2 w, uint32_t p)
{
    const uint32_t t = shoup(b, w.x, w.y, p);
    b = mod_sub(a, t, p);
    a = mod_add(a, t, p);
}
__device__ __forceinline__ void bfly_gs(uint32_t& a, uint32_t& b, uint2 w, uint32_t p)
{
    const uint32_t s = mod_add(a, b, p);
    b = shoup(a - b + p, w.x, w.y, p);
    a = s;
}

// RL stages on v[0 .. 2^RL) in registers; the stage-j twiddles are
// tw[(B0 << j) + q], q < 2^j (q = sub-block of the element).
template <bool INV, int RL>
__device__ __forceinline__ void radix_group(uint32_t (&v)[1 << RL], const uint2* __restrict__ tw, int B0, uint32_t p)
{
    constexpr int R = 1 << RL;
#pragma unroll
    for (int jj = 0; jj < RL; ++jj) {
        const int j = INV ? RL - 1 - jj : jj;
        const int half = R >> (j + 1);
        uint2 w[1 << (RL - 1)];
        const uint2* base = tw + (B0 << j);
        if (j == 0) {
            w[0] = __ldg(base);
        } else {
#pragma unroll
            for (int q = 0; q < (1 << j); q += 2) {
                const uint4 t = __ldg(reinterpret_cast<const uint4*>(base + q));
                w[q] = make_uint2(t.x, t.y);
                w[q + 1] = make_uint2(t.z, t.w);
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (u & half) continue;
            const int q = u >> (RL - j);
            if (INV) bfly_gs(v[u], v[u + half], w[q], p);
            else bfly_ct(v[u], v[u + half], w[q], p);
        }
    }
}

// One round: stages s0 .. s0+RL-1 of an M = 2^mloc point transform on `cols`
// columns held in shared memory; element l of column c is at
// sm[pad_idx((c << cshift) + (l << ishift))].  Column c's table row is
// R0(c) = rbase + c * rstep, its prime pi0 (or (pi0 + c) mod P with pvar).
struct RoundCfg {
    int mloc, cols, cshift, ishift;
    int rbase, rstep;
    const uint2* tw_all;
    int64_t tw_stride;
    int pi0, P;
    bool pvar, col_fast;
};

template <bool INV, int RL>
__device__ __forceinline__ void ntt_round(uint32_t* sm, const RoundCfg& rc, int s0)
{
    constexpr int R = 1 << RL;
    const int lg_h = rc.mloc - s0 - RL;
    const int h = 1 << lg_h;
    const int lg_gpc = rc.mloc - RL;        // groups per column = 2^lg_gpc
    const int ngroups = rc.cols << lg_gpc;
    const int lg_cols = 31 - __clz(rc.cols);
    for (int gid = threadIdx.x; gid < ngroups; gid += blockDim.x) {
        int c, grp;
        if (rc.col_fast) { c = gid & (rc.cols - 1); grp = gid >> lg_cols; }
        else { grp = gid & ((1 << lg_gpc) - 1); c = gid >> lg_gpc; }
        const int blk = grp >> lg_h;
        const int low = grp & (h - 1);
        const int base = (blk << (rc.mloc - s0)) + low;
        const int cbase = c << rc.cshift;
        int pi = rc.pi0;
        if (rc.pvar) pi = (int)((unsigned)(rc.pi0 + c) % (unsigned)rc.P);
        const uint32_t p = prime_of(pi);
        const uint2* __restrict__ tw = rc.tw_all + pi * rc.tw_stride;
        const int B0 = ((rc.rbase + c * rc.rstep) << s0) + blk;
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = sm[pad_idx(cbase + ((base + (u << lg_h)) << rc.ishift))];
        radix_group<INV, RL>(v, tw, B0, p);
#pragma unroll
        for (int u = 0; u < R; ++u) sm[pad_idx(cbase + ((base + (u << lg_h)) << rc.ishift))] = v[u];
    }
}

// all stages of a pass in rounds of at most four, sizes as equal as possible
template <bool INV>
__device__ void ntt_pass_stages(uint32_t* sm, const RoundCfg& rc)
{
    const int m = rc.mloc;
    if (m == 0) return;
    const int nr = (m + 3) / 4;
    for (int rr = 0; rr < nr; ++rr) {
        const int r = INV ? nr - 1 - rr : rr;
        const int size = m / nr + (r < m % nr ? 1 : 0);
        const int start = r * (m / nr) + min(r, m % nr);
        switch (size) {
        case 1: ntt_round<INV, 1>(sm, rc, start); break;
        case 2: ntt_round<INV, 2>(sm, rc, start); break;
        case 3: ntt_round<INV, 3>(sm, rc, start); break;
        default: ntt_round<INV, 4>(sm, rc, start); break;
        }
        __syncthreads();
    }
}

// vector activity: forward vectors [B][2][K][P] are live when k < kcnt[b][v];
// inverse vectors [B][4][G][P] when g < ngroups of (b, conv).
__device__ __forceinline__ bool fwd_live(const NttGeom& g, unsigned vec)
{
    const unsigned bv = vec / (unsigned)(g.P * g.K);
    const int k = (int)((vec / (unsigned)g.P) % (unsigned)g.K);
    return k < g.kcnt[bv];
}
__device__ __forceinline__ bool inv_live(const NttGeom& g, unsigned vec)
{
    const unsigned bc = vec / (unsigned)(g.P * g.G);
    const int grp = (int)((vec / (unsigned)g.P) % (unsigned)g.G);
    return grp < g.sched[bc].ngroups;
}

// ---------------------------------------------------------------- column pass
template <bool INV>
__global__ void __launch_bounds__(NTT_THREADS, 2) ntt_col_kernel(NttGeom g, uint32_t* __restrict__ data,
                                                              const uint2* __restrict__ tw_all)
{
    extern __shared__ uint32_t sm[];
    const int lgT = 31 - __clz(g.T);
    const int lg_tpv = g.m2 - lgT;                     // tiles per vector = N2 / T
    const unsigned vec = blockIdx.x >> lg_tpv;
    const int col0 = (int)(blockIdx.x & ((1u << lg_tpv) - 1)) << lgT;
    if (INV ? !inv_live(g, vec) : !fwd_live(g, vec)) return;
    const int pi = (int)(vec % (unsigned)g.P);
    uint32_t* v = data + (int64_t)vec * g.N;
    const int tile4 = (g.T << g.m1) >> 2;              // uint4 per tile
    const int lgT4 = lgT - 2;
    for (int q = threadIdx.x; q < tile4; q += blockDim.x) {
        const int row = q >> lgT4, c = (q & ((1 << lgT4) - 1)) << 2;
        const uint4 t = *reinterpret_cast<const uint4*>(v + ((int64_t)row << g.m2) + col0 + c);
        const int a = (row << lgT) + c;
        sm[pad_idx(a)] = t.x; sm[pad_idx(a + 1)] = t.y; sm[pad_idx(a + 2)] = t.z; sm[pad_idx(a + 3)] = t.w;
    }
    __syncthreads();
    const RoundCfg rc{g.m1, g.T, 0, lgT, 1, 0, tw_all, g.N, pi, g.P, false, true};
    ntt_pass_stages<INV>(sm, rc);
    for (int q = threadIdx.x; q < tile4; q += blockDim.x) {
        const int row = q >> lgT4, c = (q & ((1 << lgT4) - 1)) << 2;
        const int a = (row << lgT) + c;
        *reinterpret_cast<uint4*>(v + ((int64_t)row << g.m2) + col0 + c) =
            make_uint4(sm[pad_idx(a)], sm[pad_idx(a + 1)], sm[pad_idx(a + 2)], sm[pad_idx(a + 3)]);
    }
}

// ------------------------------------------------------------------- row pass
// Decoded flush group of one inverse vector (for the fused MAC): X_s lives at
// xbase + s * step and Ym_t at ybase + t * step (step = P N elements).
struct MacVec {
    int n;                     // products (0: empty group)
    uint32_t st[2];            // (s, t) nibbles of up to 8 products
    int64_t xbase, ybase, step;
    uint32_t p, pn;
};

__device__ __forceinline__ MacVec mac_decode(const NttGeom& g, unsigned vec)
{
    MacVec m;
    const int pi = (int)(vec % (unsigned)g.P);
    const unsigned rest = vec / (unsigned)g.P;
    const int grp = (int)(rest % (unsigned)g.G);
    const unsigned bc = rest / (unsigned)g.G;
    const int conv = (int)(bc & 3u);
    const unsigned b = bc >> 2;
    const Sched& S = g.sched[bc];
    const int vx = (conv == 0 || conv == 3) ? 0 : 1;   // RR, RI use Re x'; II, IR use Im x'
    const int vw = (conv == 0 || conv == 2) ? 0 : 1;   // RR, IR use Re w*; II, RI use Im w*
    m.n = grp < S.ngroups ? S.size[grp] : 0;
    m.st[0] = m.st[1] = 0u;
    for (int k = 0; k < m.n; ++k) m.st[k >> 2] |= (uint32_t)(S.pair[grp][k] & 0xff) << (8 * (k & 3));
    m.step = (int64_t)g.P * g.N;
    m.xbase = (((int64_t)b * 2 + vx) * g.K * g.P + pi) * g.N;
    m.ybase = ((int64_t)vw * g.K * g.P + pi) * g.N;
    m.p = prime_of(pi);
    m.pn = pneg_inv_of(pi);
    return m;
}

__device__ __forceinline__ void mac_offsets(const MacVec& m, int k, int64_t& xo, int64_t& yo)
{
    const uint32_t pr = (m.st[k >> 2] >> (8 * (k & 3))) & 0xffu;
    xo = m.xbase + (int64_t)(pr >> 4) * m.step;
    yo = m.ybase + (int64_t)(pr & 15u) * m.step;
}

__device__ __forceinline__ uint4 mac_load4(const MacVec& m, const MacSrc& mac, int64_t j)
{
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
    for (int k = 0; k < m.n; ++k) {
        int64_t xo, yo;
        mac_offsets(m, k, xo, yo);
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(mac.X + xo + j));
        const uint4 y = __ldg(reinterpret_cast<const uint4*>(mac.Ym + yo + j));
        acc[0] = mod_add(acc[0], mont_mul(x.x, y.x, m.p, m.pn), m.p);
        acc[1] = mod_add(acc[1], mont_mul(x.y, y.y, m.p, m.pn), m.p);
        acc[2] = mod_add(acc[2], mont_mul(x.z, y.z, m.p, m.pn), m.p);
        acc[3] = mod_add(acc[3], mont_mul(x.w, y.w, m.p, m.pn), m.p);
    }
    return make_uint4(acc[0], acc[1], acc[2], acc[3]);
}

__device__ __forceinline__ uint32_t mac_load1(const MacVec& m, const MacSrc& mac, int64_t j)
{
    uint32_t acc = 0u;
    for (int k = 0; k < m.n; ++k) {
        int64_t xo, yo;
        mac_offsets(m, k, xo, yo);
        acc = mod_add(acc, mont_mul(__ldg(mac.X + xo + j), __ldg(mac.Ym + yo + j), m.p, m.pn), m.p);
    }
    return acc;
}

template <bool INV, bool MAC>
__global__ void __launch_bounds__(NTT_THREADS, 2) ntt_row_kernel(NttGeom g, uint32_t* __restrict__ data,
                                                              const uint2* __restrict__ tw_all, MacSrc mac)
{
    extern __shared__ uint32_t sm[];
    const int M = 1 << g.m2;
    const int lg_rpv = g.lgN - g.m2;                   // rows per vector = 2^lg_rpv
    const int64_t rows_total = (int64_t)g.nvec << lg_rpv;
    const int rpc = g.rows_per_cta;
    const int64_t row0 = (int64_t)blockIdx.x * rpc;
    const int rows = (int)min((int64_t)rpc, rows_total - row0);
    const int nel = rows << g.m2;
    const int64_t gbase = row0 << g.m2;
    const bool one_vec = lg_rpv >= 31 - __clz(rpc);    // every row of the CTA in one vector
    if (one_vec) {
        const unsigned vec = (unsigned)(row0 >> lg_rpv);
        if (INV ? !inv_live(g, vec) : !fwd_live(g, vec)) return;
        const int pi = (int)(vec % (unsigned)g.P);
        const int64_t j0 = gbase - ((int64_t)vec << g.lgN);   // offset inside the vector
        if (nel >= 4) {
            if (MAC) {
                const MacVec mv = mac_decode(g, vec);
                for (int q = threadIdx.x; q < (nel >> 2); q += blockDim.x) {
                    const uint4 t = mac_load4(mv, mac, j0 + 4 * q);
                    const int a = 4 * q;
                    sm[pad_idx(a)] = t.x; sm[pad_idx(a + 1)] = t.y; sm[pad_idx(a + 2)] = t.z; sm[pad_idx(a + 3)] = t.w;
                }
            } else {
                for (int q = threadIdx.x; q < (nel >> 2); q += blockDim.x) {
                    const uint4 t = *reinterpret_cast<const uint4*>(data + gbase + 4 * q);
                    const int a = 4 * q;
                    sm[pad_idx(a)] = t.x; sm[pad_idx(a + 1)] = t.y; sm[pad_idx(a + 2)] = t.z; sm[pad_idx(a + 3)] = t.w;
                }
            }
        } else {
            const MacVec mv = MAC ? mac_decode(g, vec) : MacVec{};
            for (int i = threadIdx.x; i < nel; i += blockDim.x)
                sm[pad_idx(i)] = MAC ? mac_load1(mv, mac, j0 + i) : data[gbase + i];
        }
        __syncthreads();
        const int rin0 = (int)(row0 & ((int64_t(1) << lg_rpv) - 1));
        const RoundCfg rc{g.m2, rows, g.m2, 0, (1 << g.m1) + rin0, 1, tw_all, g.N, pi, g.P, false, false};
        ntt_pass_stages<INV>(sm, rc);
    } else {
        // rows are whole vectors (N = M < tile): vector row0 + r, primes alternate
        bool any = false;
        for (int r = 0; r < rows && !any; ++r)
            any = INV ? inv_live(g, (unsigned)(row0 + r)) : fwd_live(g, (unsigned)(row0 + r));
        if (!any) return;
        for (int r = 0; r < rows; ++r) {
            const unsigned vec = (unsigned)(row0 + r);
            if (MAC) {
                const MacVec mv = mac_decode(g, vec);
                for (int l = threadIdx.x; l < M; l += blockDim.x) sm[pad_idx((r << g.m2) + l)] = mac_load1(mv, mac, l);
            } else {
                for (int l = threadIdx.x; l < M; l += blockDim.x)
                    sm[pad_idx((r << g.m2) + l)] = data[((int64_t)vec << g.lgN) + l];
            }
        }
        __syncthreads();
        const RoundCfg rc{g.m2, rows, g.m2, 0, 1, 0, tw_all, g.N, (int)(row0 % g.P), g.P, g.P > 1, false};
        ntt_pass_stages<INV>(sm, rc);
    }
    if ((nel & 3) == 0) {
        for (int q = threadIdx.x; q < (nel >> 2); q += blockDim.x) {
            const int a = 4 * q;
            *reinterpret_cast<uint4*>(data + gbase + a) =
                make_uint4(sm[pad_idx(a)], sm[pad_idx(a + 1)], sm[pad_idx(a + 2)], sm[pad_idx(a + 3)]);
        }
    } else {
        for (int i = threadIdx.x; i < nel; i += blockDim.x) data[gbase + i] = sm[pad_idx(i)];
    }
}

}  // namespace oz

// --------------------------------------------------------------------- host
namespace oz {

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

static size_t smem_for(int64_t tile) { return (size_t)(tile + tile / 32) * sizeof(uint32_t); }

template <typename Kern>
static cudaError_t prep(Kern kernel, size_t smem)
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
    ntt_col_kernel<INV><<<(unsigned)grid, NTT_THREADS, smem, s>>>(g, data, tw);
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
    ntt_row_kernel<INV, MAC><<<(unsigned)grid, NTT_THREADS, smem, s>>>(g, data, tw, mac);
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
