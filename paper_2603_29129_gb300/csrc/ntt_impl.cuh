// ntt_impl.cuh -- batched 32-bit NTTs (§3.3) for libozfft on sm_103a.
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
// Inside a pass the stages run in rounds of up to four: a thread loads 2^RL
// elements of one column from shared memory, does RL stages in registers
// (2^j contiguous twiddles at the j-th), and stores them back.  The kernels are
// instantiated per local transform size, so every shared-memory address of a
// group is its base plus a compile-time offset: with one pad word per 32,
// element u of a group with stride S sits at pad(base) + u*S + floor(u*S/32).
//
// The inverse's first pass (the row pass) builds its input on the fly:
// Z(f) = sum over the flush group of X_s(f) * Ym_t(f) mod p (Montgomery,
// Ym = Y * N^-1 * 2^32 mod p): the NTT-domain accumulation of Alg. 8 is fused
// into the load, and Z never goes to HBM.
#pragma once
#include "oz_common.cuh"
#include "oz_kernels.h"

namespace oz {

constexpr int NTT_THREADS = 128;   // 8 (column pass) or 10 (row pass) CTAs per SM overlap load, compute, store
constexpr int TILE_LOG = 12;   // CTA tile of 4096 residues: ~13 CTAs fit an SM by shared memory

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
// the same with W = 1 (block 0 of a stage): (a - b) mod p, the value the Shoup
// product by 1 gives
__device__ __forceinline__ void bfly_gs_unit(uint32_t& a, uint32_t& b, uint32_t p)
{
    const uint32_t s = mod_add(a, b, p);
    b = mod_sub(a, b, p);
    a = s;
}

// RL stages on v[0 .. 2^RL) in registers; the stage-j twiddles are
// tw[(B0 << j) + q], q < 2^j (q = sub-block of the element).  All 2^RL - 1 of
// them are loaded before the first butterfly so their latencies overlap.
template <bool INV, int RL>
__device__ __forceinline__ void radix_group(uint32_t (&v)[1 << RL], const uint2* __restrict__ tw, int B0, uint32_t p)
{
    constexpr int R = 1 << RL;
    uint2 w[R];                      // w[(1 << j) + q]: stage j, sub-block q (w[0] unused)
    w[1] = __ldg(tw + B0);
#pragma unroll
    for (int j = 1; j < RL; ++j)
#pragma unroll
        for (int q = 0; q < (1 << j); q += 2) {
            const uint4 t = __ldg(reinterpret_cast<const uint4*>(tw + (B0 << j) + q));
            w[(1 << j) + q] = make_uint2(t.x, t.y);
            w[(1 << j) + q + 1] = make_uint2(t.z, t.w);
        }
#pragma unroll
    for (int jj = 0; jj < RL; ++jj) {
        const int j = INV ? RL - 1 - jj : jj;
        const int half = R >> (j + 1);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (u & half) continue;
            const int q = u >> (RL - j);
            if (INV) bfly_gs(v[u], v[u + half], w[(1 << j) + q], p);
            else bfly_ct(v[u], v[u + half], w[(1 << j) + q], p);
        }
    }
}

// radix_group with the table read by plain loads from any address space (a
// copy of the table's first rows in shared memory, 16-byte aligned)
template <bool INV, int RL>
__device__ __forceinline__ void radix_group_tab(uint32_t (&v)[1 << RL], const uint2* tab, int B0, uint32_t p)
{
    constexpr int R = 1 << RL;
    uint2 w[R];
    w[1] = tab[B0];
#pragma unroll
    for (int j = 1; j < RL; ++j)
#pragma unroll
        for (int q = 0; q < (1 << j); q += 2) {
            const uint4 t = *reinterpret_cast<const uint4*>(tab + (B0 << j) + q);
            w[(1 << j) + q] = make_uint2(t.x, t.y);
            w[(1 << j) + q + 1] = make_uint2(t.z, t.w);
        }
#pragma unroll
    for (int jj = 0; jj < RL; ++jj) {
        const int j = INV ? RL - 1 - jj : jj;
        const int half = R >> (j + 1);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (u & half) continue;
            const int q = u >> (RL - j);
            if (INV) bfly_gs(v[u], v[u + half], w[(1 << j) + q], p);
            else bfly_ct(v[u], v[u + half], w[(1 << j) + q], p);
        }
    }
}

// load, transform and store one group whose elements are S words apart
// (PAD = false: a dense tile without the pad words, as the tensor-memory-access
// column pass keeps it)
template <bool INV, int RL, int S, bool PAD = true>
__device__ __forceinline__ void group_bfly(uint32_t* smp, const uint2* __restrict__ tw, int B0, uint32_t p)
{
    constexpr int R = 1 << RL;
    uint32_t v[R];
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = smp[PAD ? u * S + (u * S) / 32 : u * S];
    radix_group<INV, RL>(v, tw, B0, p);
#pragma unroll
    for (int u = 0; u < R; ++u) smp[PAD ? u * S + (u * S) / 32 : u * S] = v[u];
}

// round partition of an M = 2^ML point pass: ceil(ML/4) rounds, sizes equal
// up to one, the larger rounds last (fewer bank conflicts, e.g. 3,3,3,4 for 13)
template <int ML>
struct Part {
    static constexpr int NR = (ML + 3) / 4;
    static constexpr int EXTRA = NR ? ML % NR : 0;
    static constexpr int size(int r) { return ML / NR + (r >= NR - EXTRA ? 1 : 0); }
    static constexpr int start(int r) { return r * (ML / NR) + (r > NR - EXTRA ? r - (NR - EXTRA) : 0); }
};

// runtime facts of a pass: number of columns (rows of a row pass), table row
// of column c = rbase + c * rstep, prime of column c = pi0 or (pi0 + c) mod P
struct PassArgs {
    int cols, rbase, rstep;
    const uint2* tw_all;
    int64_t tw_stride;
    int pi0, P;
    bool pvar;
};

__device__ __forceinline__ const uint2* table_of(const PassArgs& a, int c, uint32_t& p)
{
    int pi = a.pi0;
    if (a.pvar) pi = (int)((unsigned)(a.pi0 + c) % (unsigned)a.P);
    p = prime_of(pi);
    return a.tw_all + pi * a.tw_stride;
}

// row pass round: element l of row c at sm[pad((c << ML) + l)]
template <bool INV, int ML, int S0, int RL>
__device__ __forceinline__ void row_round(uint32_t* sm, const PassArgs& a)
{
    constexpr int LOG_H = ML - S0 - RL, H = 1 << LOG_H, LOG_GPC = ML - RL;
    // stride-16 rounds: adjacent blocks lie 2^(ML-S0) words (+ pad) apart, which
    // puts the two half-warps on overlapping banks; pairing block b with b + 2^D
    // (D = 9 - (ML - S0)), by swapping bits 0 and D of the block index, puts them
    // 16 banks apart
    constexpr bool PERM = LOG_H == 4 && ML - S0 >= 6 && ML - S0 <= 8;
    constexpr int D = 9 - (ML - S0);
    const int ngroups = a.cols << LOG_GPC;
    for (int gid = threadIdx.x; gid < ngroups; gid += blockDim.x) {
        int grp = gid & ((1 << LOG_GPC) - 1);
        if constexpr (PERM) {
            const int b = grp >> 4;
            const int sw = (b ^ (b >> D)) & 1;             // bits 0 and D differ: flip both
            grp ^= (sw | (sw << D)) << 4;
        }
        const int c = gid >> LOG_GPC;
        const int blk = grp >> LOG_H;
        const int base = (c << ML) + (blk << (ML - S0)) + (grp & (H - 1));
        uint32_t p;
        const uint2* tw = table_of(a, c, p);
        group_bfly<INV, RL, H>(sm + pad_idx(base), tw, ((a.rbase + c * a.rstep) << S0) + blk, p);
    }
}

// column pass round: element l of column c at sm[pad((l << LOG_T) + c)]
template <bool INV, int ML, int S0, int RL, int LOG_T, bool PAD = true>
__device__ __forceinline__ void col_round(uint32_t* sm, const PassArgs& a)
{
    constexpr int LOG_H = ML - S0 - RL, H = 1 << LOG_H, LOG_GPC = ML - RL;
    constexpr int T = 1 << LOG_T;
    for (int gid = threadIdx.x; gid < (T << LOG_GPC); gid += blockDim.x) {
        const int c = gid & (T - 1);
        const int grp = gid >> LOG_T;
        const int blk = grp >> LOG_H;
        const int l0 = (blk << (ML - S0)) + (grp & (H - 1));
        uint32_t p;
        const uint2* tw = table_of(a, 0, p);
        const int at = (l0 << LOG_T) + c;
        group_bfly<INV, RL, H * T, PAD>(sm + (PAD ? pad_idx(at) : at), tw, (1 << S0) + blk, p);
    }
}

template <bool INV, bool COL, int ML, int LOG_T, int I, bool PAD = true>
__device__ __forceinline__ void run_rounds(uint32_t* sm, const PassArgs& a)
{
    if constexpr (I < Part<ML>::NR) {
        constexpr int R_ = INV ? Part<ML>::NR - 1 - I : I;
        constexpr int S0 = Part<ML>::start(R_), RL = Part<ML>::size(R_);
        if constexpr (COL) col_round<INV, ML, S0, RL, LOG_T, PAD>(sm, a);
        else row_round<INV, ML, S0, RL>(sm, a);
        __syncthreads();
        run_rounds<INV, COL, ML, LOG_T, I + 1, PAD>(sm, a);
    }
}

// vector activity: forward vectors [B][2][K][P] are live when k < kcnt[b][v];
// inverse vectors [B][4][G][P] when g < ngroups of (b, conv).
__device__ __forceinline__ bool fwd_live(const NttGeom& g, unsigned vec)
{
    const unsigned vp = udiv_small(vec, (unsigned)g.P);       // vec / P
    const unsigned bv = udiv_small(vp, (unsigned)g.K);        // vec / (P K)
    const int k = (int)(vp - bv * (unsigned)g.K);
    if (g.redo && !g.redo[bv]) return false;   // transformed already by the fused split
    return k < g.kcnt[bv];
}
__device__ __forceinline__ bool inv_live(const NttGeom& g, unsigned vec)
{
    const unsigned bc = vec / (unsigned)(g.P * g.G);
    const int grp = (int)((vec / (unsigned)g.P) % (unsigned)g.G);
    return grp < g.sched[bc].ngroups;
}

// columns per column-pass tile: 2^(12 - m1) up to m1 = 6 (4096-residue tiles), then 64
// columns (256-byte row segments) up to m1 = 8, then 32
constexpr int col_log_t(int m1) { return m1 <= 6 ? ((TILE_LOG - m1) > 5 ? (TILE_LOG - m1) : 5) : (m1 <= 8 ? 6 : 5); }

// ---------------------------------------------------------------- column pass
template <bool INV, int M1>
__global__ void __launch_bounds__(NTT_THREADS, 8) ntt_col_kernel(NttGeom g, uint32_t* __restrict__ data,
                                                                 const uint2* __restrict__ tw_all)
{
    extern __shared__ uint32_t sm[];
    constexpr int LOG_T = col_log_t(M1), T = 1 << LOG_T;
    const int lg_tpv = g.m2 - LOG_T;                   // tiles per vector = N2 / T
    const unsigned vec = blockIdx.x >> lg_tpv;
    const int col0 = (int)(blockIdx.x & ((1u << lg_tpv) - 1)) << LOG_T;
    if (INV ? !inv_live(g, vec) : !fwd_live(g, vec)) return;
    const int pi = (int)(vec - udiv_small(vec, (unsigned)g.P) * (unsigned)g.P);
    uint32_t* v = data + (int64_t)vec * g.N + col0;
    constexpr int TILE4 = (T << M1) >> 2;
    static_assert(TILE4 % (8 * NTT_THREADS) == 0, "column tile");
    // eight 16-byte loads in flight per thread before the shared-memory stores
    for (int q0 = 0; q0 < TILE4; q0 += 8 * NTT_THREADS) {
        uint4 t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int q = q0 + k * NTT_THREADS + threadIdx.x;
            const int row = q >> (LOG_T - 2), c = (q & ((T >> 2) - 1)) << 2;
            t[k] = *reinterpret_cast<const uint4*>(v + ((int64_t)row << g.m2) + c);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int q = q0 + k * NTT_THREADS + threadIdx.x;
            const int row = q >> (LOG_T - 2), c = (q & ((T >> 2) - 1)) << 2;
            uint32_t* s = sm + pad_idx((row << LOG_T) + c);
            s[0] = t[k].x; s[1] = t[k].y; s[2] = t[k].z; s[3] = t[k].w;
        }
    }
    __syncthreads();
    const PassArgs a{T, 1, 0, tw_all, g.N, pi, g.P, false};
    run_rounds<INV, true, M1, LOG_T, 0>(sm, a);
    for (int q = threadIdx.x; q < TILE4; q += blockDim.x) {
        const int row = q >> (LOG_T - 2), c = (q & ((T >> 2) - 1)) << 2;
        const uint32_t* s = sm + pad_idx((row << LOG_T) + c);
        *reinterpret_cast<uint4*>(v + ((int64_t)row << g.m2) + c) = make_uint4(s[0], s[1], s[2], s[3]);
    }
}

// ------------------------------------------------------------------- row pass
// Decoded flush group of one inverse vector (for the fused MAC): X_s lives at
// xbase + s * step and Ym_t at ybase + t * step (step = P N elements); Ym is
// shared by the batch, or per signal (ym_stride apart) in a plan over uneven
// lengths.  In a merged schedule a group holds products of both convolutions
// of one output part (RR and II, or IR and RI): each product names its
// convolution, which picks Re or Im of x~' and of w~* (vstride apart), and
// the II products enter with a minus sign.
struct MacVec {
    int n;                     // products (0: empty group)
    uint32_t st0, st1;         // (s, t) bytes of products 0..3 and 4..7
    uint32_t cv;               // merged groups: convolution of each product, 2 bits each
    int64_t xbase, ybase, step, vstride;
    uint32_t p, pn;
    bool merged;
};

__device__ __forceinline__ MacVec mac_decode(const NttGeom& g, unsigned vec, int64_t ym_stride)
{
    MacVec m;
    const int pi = (int)(vec % (unsigned)g.P);
    const unsigned rest = vec / (unsigned)g.P;
    const int grp = (int)(rest % (unsigned)g.G);
    const unsigned bc = rest / (unsigned)g.G;
    const int conv = (int)(bc & 3u);
    const unsigned b = bc >> 2;
    const Sched& S = g.sched[bc];
    m.merged = g.merged != 0;
    const int vx = m.merged ? 0 : ((conv == 0 || conv == 3) ? 0 : 1);   // RR, RI use Re x'; II, IR use Im x'
    const int vw = m.merged ? 0 : ((conv == 0 || conv == 2) ? 0 : 1);   // RR, IR use Re w*; II, RI use Im w*
    m.n = grp < S.ngroups ? S.size[grp] : 0;
    m.st0 = m.st1 = m.cv = 0u;
    for (int k = 0; k < m.n; ++k) {
        const int32_t pr = S.pair[grp][k];
        const uint32_t byte = (uint32_t)(pr & 0xff) << (8 * (k & 3));
        if (k < 4) m.st0 |= byte;
        else m.st1 |= byte;
        m.cv |= (uint32_t)((pr >> 8) & 3) << (2 * k);
    }
    m.step = (int64_t)g.P * g.N;
    m.vstride = (int64_t)g.K * g.P * g.N;
    m.xbase = (((int64_t)b * 2 + vx) * g.K * g.P + pi) * g.N;
    m.ybase = ((int64_t)vw * g.K * g.P + pi) * g.N + (int64_t)b * ym_stride;
    m.p = prime_of(pi);
    m.pn = pneg_inv_of(pi);
    return m;
}

// offsets of product k's X_s and Ym_t; in a merged group also the Re/Im choice
// of its convolution, and whether it enters with a minus sign (II)
template <bool MERGED>
__device__ __forceinline__ bool mac_offsets(const MacVec& m, int k, int64_t& xo, int64_t& yo)
{
    const uint32_t pr = ((k < 4 ? m.st0 : m.st1) >> (8 * (k & 3))) & 0xffu;
    xo = m.xbase + (int64_t)(pr >> 4) * m.step;
    yo = m.ybase + (int64_t)(pr & 15u) * m.step;
    if (!MERGED) return false;
    const uint32_t c = (m.cv >> (2 * k)) & 3u;
    if (c == 1u || c == 2u) xo += m.vstride;   // II, IR: Im x'
    if (c == 1u || c == 3u) yo += m.vstride;   // II, RI: Im w*
    return c == 1u;                            // II enters the real part with a minus sign
}

template <bool MERGED>
__device__ __forceinline__ uint4 mac_sum4(const MacVec& m, const MacSrc& mac, int64_t j)
{
    uint32_t a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u;
    if (!MERGED && m.n > 0) {   // the first product sets the sums (no add of zero)
        int64_t xo, yo;
        mac_offsets<false>(m, 0, xo, yo);
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(mac.X + xo + j));
        const uint4 y = __ldg(reinterpret_cast<const uint4*>(mac.Ym + yo + j));
        a0 = mont_mul(x.x, y.x, m.p, m.pn); a1 = mont_mul(x.y, y.y, m.p, m.pn);
        a2 = mont_mul(x.z, y.z, m.p, m.pn); a3 = mont_mul(x.w, y.w, m.p, m.pn);
    }
    for (int k = (!MERGED && m.n > 0) ? 1 : 0; k < m.n; ++k) {
        int64_t xo, yo;
        const bool neg = mac_offsets<MERGED>(m, k, xo, yo);
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(mac.X + xo + j));
        const uint4 y = __ldg(reinterpret_cast<const uint4*>(mac.Ym + yo + j));
        const uint32_t t0 = mont_mul(x.x, y.x, m.p, m.pn), t1 = mont_mul(x.y, y.y, m.p, m.pn);
        const uint32_t t2 = mont_mul(x.z, y.z, m.p, m.pn), t3 = mont_mul(x.w, y.w, m.p, m.pn);
        if (MERGED && neg) {
            a0 = mod_sub(a0, t0, m.p); a1 = mod_sub(a1, t1, m.p);
            a2 = mod_sub(a2, t2, m.p); a3 = mod_sub(a3, t3, m.p);
        } else {
            a0 = mod_add(a0, t0, m.p); a1 = mod_add(a1, t1, m.p);
            a2 = mod_add(a2, t2, m.p); a3 = mod_add(a3, t3, m.p);
        }
    }
    return make_uint4(a0, a1, a2, a3);
}

__device__ __forceinline__ uint4 mac_load4(const MacVec& m, const MacSrc& mac, int64_t j)
{
    return m.merged ? mac_sum4<true>(m, mac, j) : mac_sum4<false>(m, mac, j);
}

// one product (L = 1, unmerged: the only unmerged schedules whose sums are
// formed in registers): Z = X_s Ym_t, for a live vector
__device__ __forceinline__ uint4 mac_one4(const MacVec& m, const MacSrc& mac, int64_t j)
{
    int64_t xo, yo;
    mac_offsets<false>(m, 0, xo, yo);
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(mac.X + xo + j));
    const uint4 y = __ldg(reinterpret_cast<const uint4*>(mac.Ym + yo + j));
    return make_uint4(mont_mul(x.x, y.x, m.p, m.pn), mont_mul(x.y, y.y, m.p, m.pn), mont_mul(x.z, y.z, m.p, m.pn),
                      mont_mul(x.w, y.w, m.p, m.pn));
}

template <bool MERGED>
__device__ __forceinline__ uint32_t mac_sum1(const MacVec& m, const MacSrc& mac, int64_t j)
{
    uint32_t acc = 0u;
    for (int k = 0; k < m.n; ++k) {
        int64_t xo, yo;
        const bool neg = mac_offsets<MERGED>(m, k, xo, yo);
        const uint32_t t = mont_mul(__ldg(mac.X + xo + j), __ldg(mac.Ym + yo + j), m.p, m.pn);
        acc = (MERGED && neg) ? mod_sub(acc, t, m.p) : mod_add(acc, t, m.p);
    }
    return acc;
}

__device__ __forceinline__ uint32_t mac_load1(const MacVec& m, const MacSrc& mac, int64_t j)
{
    return m.merged ? mac_sum1<true>(m, mac, j) : mac_sum1<false>(m, mac, j);
}

// middle rounds I = 1 .. NR - 2 of the inverse row pass
template <int ML, int I>
__device__ __forceinline__ void inv_middle_rounds(uint32_t* sm, const PassArgs& a)
{
    if constexpr (I < Part<ML>::NR - 1) {
        constexpr int R_ = Part<ML>::NR - 1 - I;
        row_round<true, ML, Part<ML>::start(R_), Part<ML>::size(R_)>(sm, a);
        __syncthreads();
        inv_middle_rounds<ML, I + 1>(sm, a);
    }
}

// Twiddles of the inverse row pass's middle and last rounds staged in shared
// memory (one row per CTA and three rounds): the 2^S0 blocks of the middle
// round take 2^RL - 1 table entries each, the last round's single block
// 2^RL0 - 1, laid out per block in radix_group's order w[1], w[2..3], w[4..7],
// w[8..15]; the CTA copies them while its first round forms the Alg. 8 sums.
#ifndef OZ_TW_STAGE
#define OZ_TW_STAGE 1
#endif
template <int ML>
struct InvTw {
    static constexpr int NR = Part<ML>::NR;
    static constexpr bool ON = OZ_TW_STAGE && NR == 3;
    static constexpr int S0M = Part<ML>::start(1), RLM = Part<ML>::size(1), RL0 = Part<ML>::size(0);
    static constexpr int PER = (1 << RLM) - 1, MID = (1 << S0M) * PER, TOTAL = MID + (1 << RL0) - 1;
};

template <int ML>
__device__ __forceinline__ void stage_inv_tw(uint2* tws, const uint2* __restrict__ tw, int rbase)
{
    using T = InvTw<ML>;
    for (int e = threadIdx.x; e < T::TOTAL; e += NTT_THREADS) {
        const bool mid = e < T::MID;
        const int blk = mid ? e / T::PER : 0;
        const int k = (mid ? e - blk * T::PER : e - T::MID) + 1;   // radix_group's index (1 << j) + q
        const int j = 31 - __clz(k);
        const int B0 = mid ? (rbase << T::S0M) + blk : rbase;
        tws[e] = __ldg(tw + (B0 << j) + (k - (1 << j)));
    }
}

template <int RL>
__device__ __forceinline__ void radix_group_inv_staged(uint32_t (&v)[1 << RL], const uint2* tws, uint32_t p)
{
    constexpr int R = 1 << RL;
    uint2 w[R];
#pragma unroll
    for (int k = 1; k < R; ++k) w[k] = tws[k - 1];
#pragma unroll
    for (int j = RL - 1; j >= 0; --j) {
        const int half = R >> (j + 1);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (u & half) continue;
            bfly_gs(v[u], v[u + half], w[(1 << j) + (u >> (RL - j))], p);
        }
    }
}

// the middle round of a one-row tile with staged twiddles (row_round's map)
template <int ML>
__device__ __forceinline__ void inv_middle_round_staged(uint32_t* sm, const uint2* tws, uint32_t p)
{
    using T = InvTw<ML>;
    constexpr int S0 = T::S0M, RL = T::RLM, R = 1 << RL;
    constexpr int LOG_H = ML - S0 - RL, H = 1 << LOG_H, LOG_GPC = ML - RL;
    constexpr bool PERM = LOG_H == 4 && ML - S0 >= 6 && ML - S0 <= 8;
    constexpr int D = 9 - (ML - S0);
#pragma unroll 1
    for (int gid = threadIdx.x; gid < (1 << LOG_GPC); gid += NTT_THREADS) {
        int grp = gid;
        if constexpr (PERM) {
            const int b = grp >> 4;
            const int sw = (b ^ (b >> D)) & 1;
            grp ^= (sw | (sw << D)) << 4;
        }
        const int blk = grp >> LOG_H;
        uint32_t* smp = sm + pad_idx((blk << (ML - S0)) + (grp & (H - 1)));
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = smp[u * H + (u * H) / 32];
        radix_group_inv_staged<RL>(v, tws + blk * T::PER, p);
#pragma unroll
        for (int u = 0; u < R; ++u) smp[u * H + (u * H) / 32] = v[u];
    }
}

// The inverse row pass of a full tile of ROWS rows of one vector with the MAC
// in registers: the first round's groups are 2^RL contiguous residues, so each
// thread forms their Alg. 8 sums straight from X and Ym; the last round (the
// stages of stride H = 2^(ML - RL)) stores straight to global memory, with
// consecutive lanes on consecutive addresses.  Two shared-memory passes and two
// barriers fewer than loading, transforming and storing separately.
template <int ML, int ROWS, bool ONE>
__device__ __forceinline__ void row_inv_mac(uint32_t* sm, uint32_t* __restrict__ out, const uint2* __restrict__ tw_all,
                                            int pi, int64_t tw_stride, int rbase, const MacVec& mv, const MacSrc& mac,
                                            int64_t j0, uint2* tws)
{
    using PT = Part<ML>;
    const uint2* tw = tw_all + (int64_t)pi * tw_stride;
    const uint32_t p = prime_of(pi);
    constexpr bool STAGED = ROWS == 1 && InvTw<ML>::ON;   // tws: InvTw<ML>::TOTAL entries
    if constexpr (STAGED) stage_inv_tw<ML>(tws, tw, rbase);   // visible after the first round's barrier
    {
        constexpr int R_ = PT::NR - 1, S0 = PT::start(R_), RL = PT::size(R_), R = 1 << RL, LOG_GPC = ML - RL;
        static_assert(S0 + RL == ML && RL >= 2 && RL <= 4, "first inverse round: contiguous groups");
        constexpr int NG = ROWS << LOG_GPC;
#pragma unroll 1
        for (int gid = threadIdx.x; gid < NG; gid += NTT_THREADS) {
            const int grp = gid & ((1 << LOG_GPC) - 1), c = gid >> LOG_GPC;
            const int base = (c << ML) + (grp << RL);
            uint32_t v[R];
#pragma unroll
            for (int q = 0; q < R; q += 4) {
                const uint4 t = ONE ? mac_one4(mv, mac, j0 + base + q) : mac_load4(mv, mac, j0 + base + q);
                v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
            }
            radix_group<true, RL>(v, tw, ((rbase + c) << S0) + grp, p);
            uint32_t* smp = sm + pad_idx(base);
#pragma unroll
            for (int u = 0; u < R; ++u) smp[u] = v[u];
        }
    }
    __syncthreads();
    if constexpr (STAGED) {
        inv_middle_round_staged<ML>(sm, tws, p);
        __syncthreads();
    } else {
        const PassArgs a{ROWS, rbase, 1, tw_all, tw_stride, pi, 1, false};
        inv_middle_rounds<ML, 1>(sm, a);
    }
    {
        constexpr int RL = PT::size(0), R = 1 << RL, LOG_H = ML - RL, H = 1 << LOG_H;
        constexpr int NG = ROWS << LOG_H;
#pragma unroll 1
        for (int gid = threadIdx.x; gid < NG; gid += NTT_THREADS) {
            const int l0 = gid & (H - 1), c = gid >> LOG_H;
            const int base = (c << ML) + l0;
            uint32_t v[R];
            const uint32_t* smp = sm + pad_idx(base);
#pragma unroll
            for (int u = 0; u < R; ++u) v[u] = smp[u * H + (u * H) / 32];
            if constexpr (STAGED) radix_group_inv_staged<RL>(v, tws + InvTw<ML>::MID, p);
            else radix_group<true, RL>(v, tw, rbase + c, p);
#pragma unroll
            for (int u = 0; u < R; ++u) out[base + u * H] = v[u];
        }
    }
}

// ----------------------------------------------- inverse row pass, V vectors
// The same inverse row pass (MAC in registers, a full tile of ROWS rows) on V
// vectors that use one prime: every twiddle a thread loads serves the V
// vectors' groups at once, and the V groups' butterflies give the scheduler
// V independent chains.  V = 2 halves the twiddle loads and the index work per
// residue (the vectors' tiles sit TW words apart in shared memory).
template <int RL, int V>
__device__ __forceinline__ void radix_group_inv_v(uint32_t (&x)[V][1 << RL], const uint2* __restrict__ tw, int B0,
                                                  uint32_t p)
{
    constexpr int R = 1 << RL;
    uint2 w[R];
    w[1] = __ldg(tw + B0);
#pragma unroll
    for (int j = 1; j < RL; ++j)
#pragma unroll
        for (int q = 0; q < (1 << j); q += 2) {
            const uint4 t = __ldg(reinterpret_cast<const uint4*>(tw + (B0 << j) + q));
            w[(1 << j) + q] = make_uint2(t.x, t.y);
            w[(1 << j) + q + 1] = make_uint2(t.z, t.w);
        }
#pragma unroll
    for (int j = RL - 1; j >= 0; --j) {
        const int half = R >> (j + 1);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (u & half) continue;
            const int q = u >> (RL - j);
#pragma unroll
            for (int i = 0; i < V; ++i) bfly_gs(x[i][u], x[i][u + half], w[(1 << j) + q], p);
        }
    }
}

// the same with the twiddles from shared memory (stage_inv_tw's layout)
template <int RL, int V>
__device__ __forceinline__ void radix_group_inv_v_staged(uint32_t (&x)[V][1 << RL], const uint2* tws, uint32_t p)
{
    constexpr int R = 1 << RL;
    uint2 w[R];
#pragma unroll
    for (int k = 1; k < R; ++k) w[k] = tws[k - 1];
#pragma unroll
    for (int j = RL - 1; j >= 0; --j) {
        const int half = R >> (j + 1);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (u & half) continue;
#pragma unroll
            for (int i = 0; i < V; ++i) bfly_gs(x[i][u], x[i][u + half], w[(1 << j) + (u >> (RL - j))], p);
        }
    }
}

// middle round of the inverse row pass on V tiles (the row_round index map)
template <int ML, int S0, int RL, int V, int TW, int ROWS, bool STG = false>
__device__ __forceinline__ void row_round_inv_v(uint32_t* sm, int rbase, const uint2* __restrict__ tw, uint32_t p,
                                                const uint2* tws = nullptr)
{
    constexpr int LOG_H = ML - S0 - RL, H = 1 << LOG_H, LOG_GPC = ML - RL, R = 1 << RL;
    constexpr bool PERM = LOG_H == 4 && ML - S0 >= 6 && ML - S0 <= 8;
    constexpr int D = 9 - (ML - S0);
    constexpr int ngroups = ROWS << LOG_GPC;
#pragma unroll 1
    for (int gid = threadIdx.x; gid < ngroups; gid += NTT_THREADS) {
        int grp = ROWS == 1 ? gid : gid & ((1 << LOG_GPC) - 1);
        if constexpr (PERM) {
            const int b = grp >> 4;
            const int sw = (b ^ (b >> D)) & 1;
            grp ^= (sw | (sw << D)) << 4;
        }
        const int c = ROWS == 1 ? 0 : gid >> LOG_GPC;
        const int blk = grp >> LOG_H;
        const int base = (c << ML) + (blk << (ML - S0)) + (grp & (H - 1));
        uint32_t x[V][R];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const uint32_t* s = sm + i * TW + pad_idx(base);
#pragma unroll
            for (int u = 0; u < R; ++u) x[i][u] = s[u * H + (u * H) / 32];
        }
        if constexpr (STG) radix_group_inv_v_staged<RL, V>(x, tws + blk * ((1 << RL) - 1), p);
        else radix_group_inv_v<RL, V>(x, tw, ((rbase + c) << S0) + blk, p);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            uint32_t* s = sm + i * TW + pad_idx(base);
#pragma unroll
            for (int u = 0; u < R; ++u) s[u * H + (u * H) / 32] = x[i][u];
        }
    }
}

template <int ML, int V, int TW, int ROWS, int I>
__device__ __forceinline__ void inv_middle_rounds_v(uint32_t* sm, int rbase, const uint2* tw, uint32_t p)
{
    if constexpr (I < Part<ML>::NR - 1) {
        constexpr int R_ = Part<ML>::NR - 1 - I;
        row_round_inv_v<ML, Part<ML>::start(R_), Part<ML>::size(R_), V, TW, ROWS>(sm, rbase, tw, p);
        __syncthreads();
        inv_middle_rounds_v<ML, V, TW, ROWS, I + 1>(sm, rbase, tw, p);
    }
}

// one CTA: rows [row0, row0 + RPC) of two vectors of one prime and one flush
// group index: those of convolutions RR and RI (both products of Re x~'
// slices) or of II and IR (Im x~'), which in the usual schedule read the same
// X_s row, so the second vector's X loads hit L1 as its twiddles do
constexpr int INV_PAIR_V = 2;
template <int M2, bool MERGED>
__global__ void __launch_bounds__(NTT_THREADS, 6) ntt_inv_row_v_kernel(NttGeom g, uint32_t* __restrict__ data,
                                                                      const uint2* __restrict__ tw_all, MacSrc mac)
{
    constexpr int V = INV_PAIR_V;
    static_assert(V == 2, "pairs of convolutions (RR, RI) and (II, IR)");
    constexpr int RPC = 1 << (TILE_LOG - M2);
    constexpr int TW = (RPC << M2) + ((RPC << M2) >> 5);      // words of one vector's padded tile
    using PT = Part<M2>;
    extern __shared__ uint32_t sm[];
    const int lg_rb = g.lgN - TILE_LOG;                     // row blocks per vector = 2^lg_rb
    const unsigned k = blockIdx.x >> lg_rb;
    const int row0 = (int)(blockIdx.x & ((1u << lg_rb) - 1)) * RPC;
    const unsigned P = (unsigned)g.P, GP = (unsigned)g.G * P;
    // k enumerates (signal, pair type, group, prime); vectors are [signal][conv][group][prime]
    const int pi = (int)(k % P);
    const unsigned grp = (k / P) % (unsigned)g.G, pt = (k / GP) & 1u, sig = k / (2 * GP);
    const unsigned vec_of[V] = {((4 * sig + pt) * g.G + grp) * P + pi, ((4 * sig + 3 - pt) * g.G + grp) * P + pi};
    const uint32_t p = prime_of(pi);
    const uint2* tw = tw_all + (int64_t)pi * g.N;
    const int rbase = (1 << g.m1) + row0;
    const int64_t j0 = (int64_t)row0 << M2;
    MacVec mv[V];
    bool live[V];
    bool any = false;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const unsigned vec = vec_of[i];
        live[i] = inv_live(g, vec);
        any = any || live[i];
        mv[i] = mac_decode(g, vec, mac.ym_stride);
    }
    if (!any) return;
    constexpr bool STAGED = RPC == 1 && InvTw<M2>::ON;
    __shared__ uint2 tws[STAGED ? InvTw<M2>::TOTAL : 1];
    if constexpr (STAGED) stage_inv_tw<M2>(tws, tw, rbase);   // visible after the first round's barrier
    {   // first round: groups of 2^RL contiguous residues, the Alg. 8 sums formed from X and Ym
        constexpr int R_ = PT::NR - 1, S0 = PT::start(R_), RL = PT::size(R_), R = 1 << RL, LOG_GPC = M2 - RL;
        static_assert(S0 + RL == M2 && RL >= 2 && RL <= 4, "first inverse round: contiguous groups");
#pragma unroll 1
        for (int gid = threadIdx.x; gid < (RPC << LOG_GPC); gid += NTT_THREADS) {
            const int grp = RPC == 1 ? gid : gid & ((1 << LOG_GPC) - 1), c = RPC == 1 ? 0 : gid >> LOG_GPC;
            const int base = (c << M2) + (grp << RL);
            uint32_t x[V][R];
#pragma unroll
            for (int i = 0; i < V; ++i)
#pragma unroll
                for (int q = 0; q < R; q += 4) {
                    uint4 t = make_uint4(0u, 0u, 0u, 0u);
                    if (live[i]) t = MERGED ? mac_sum4<true>(mv[i], mac, j0 + base + q) : mac_one4(mv[i], mac, j0 + base + q);
                    x[i][q] = t.x; x[i][q + 1] = t.y; x[i][q + 2] = t.z; x[i][q + 3] = t.w;
                }
            radix_group_inv_v<RL, V>(x, tw, ((rbase + c) << S0) + grp, p);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                uint32_t* s = sm + i * TW + pad_idx(base);
#pragma unroll
                for (int u = 0; u < R; ++u) s[u] = x[i][u];
            }
        }
    }
    __syncthreads();
    if constexpr (STAGED) {
        row_round_inv_v<M2, InvTw<M2>::S0M, InvTw<M2>::RLM, V, TW, RPC, true>(sm, rbase, tw, p, tws);
        __syncthreads();
    } else {
        inv_middle_rounds_v<M2, V, TW, RPC, 1>(sm, rbase, tw, p);
    }
    {   // last round: stride 2^(M2 - RL), stored straight to HBM
        constexpr int RL = PT::size(0), R = 1 << RL, LOG_H = M2 - RL, H = 1 << LOG_H;
#pragma unroll 1
        for (int gid = threadIdx.x; gid < (RPC << LOG_H); gid += NTT_THREADS) {
            const int l0 = RPC == 1 ? gid : gid & (H - 1), c = RPC == 1 ? 0 : gid >> LOG_H;
            const int base = (c << M2) + l0;
            uint32_t x[V][R];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const uint32_t* s = sm + i * TW + pad_idx(base);
#pragma unroll
                for (int u = 0; u < R; ++u) x[i][u] = s[u * H + (u * H) / 32];
            }
            if constexpr (STAGED) radix_group_inv_v_staged<RL, V>(x, tws + InvTw<M2>::MID, p);
            else radix_group_inv_v<RL, V>(x, tw, rbase + c, p);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if (!live[i]) continue;
                uint32_t* out = data + ((int64_t)vec_of[i] << g.lgN) + j0 + base;
#pragma unroll
                for (int u = 0; u < R; ++u) out[u * H] = x[i][u];
            }
        }
    }
}

// 10 CTAs per SM (48 registers); the inverse pass with the MAC in registers
// needs 56 (9 CTAs) to stay free of spills
template <bool INV, bool MAC, int M2>
__global__ void __launch_bounds__(NTT_THREADS, (INV && MAC) ? 9 : 10) ntt_row_kernel(NttGeom g, uint32_t* __restrict__ data,
                                                                 const uint2* __restrict__ tw_all, MacSrc mac)
{
    extern __shared__ uint32_t sm[];
    constexpr int M = 1 << M2;
    constexpr int RPC = M2 <= TILE_LOG ? (1 << (TILE_LOG - M2)) : 1;   // rows per CTA
    const int lg_rpv = g.lgN - M2;                     // rows per vector = 2^lg_rpv
    const int64_t rows_total = (int64_t)g.nvec << lg_rpv;
    const int64_t row0 = (int64_t)blockIdx.x * RPC;
    const int rows = (int)min((int64_t)RPC, rows_total - row0);
    const int nel = rows << M2;
    const int64_t gbase = row0 << M2;
    if ((1 << lg_rpv) >= RPC) {
        // every row of the CTA belongs to one vector
        const unsigned vec = (unsigned)(row0 >> lg_rpv);
        if (INV ? !inv_live(g, vec) : !fwd_live(g, vec)) return;
        const int pi = (int)(vec % (unsigned)g.P);
        const int64_t j0 = gbase - ((int64_t)vec << g.lgN);   // offset inside the vector
        if constexpr (INV && MAC && Part<M2>::NR >= 2 && M2 <= TILE_LOG) {
            if (rows == RPC && g.mac_reg) {   // groups of several products keep the coalesced staged loads
                const MacVec mv = mac_decode(g, vec, mac.ym_stride);
                const int rin0 = (int)(row0 & ((int64_t(1) << lg_rpv) - 1));
                __shared__ uint2 tws[RPC == 1 && InvTw<M2>::ON ? InvTw<M2>::TOTAL : 1];
                // one unmerged product per group (L = 1): the MAC without the product loop
                // (one-row tiles; with several rows per CTA the second variant spills)
                if (RPC == 1 && !mv.merged && mv.n == 1)
                    row_inv_mac<M2, RPC, RPC == 1>(sm, data + gbase, tw_all, pi, g.N, (1 << g.m1) + rin0, mv, mac,
                                                   j0, tws);
                else
                    row_inv_mac<M2, RPC, false>(sm, data + gbase, tw_all, pi, g.N, (1 << g.m1) + rin0, mv, mac, j0,
                                                tws);
                return;
            }
        }
        if (nel >= 4) {
            if (MAC) {
                const MacVec mv = mac_decode(g, vec, mac.ym_stride);
                if (!mv.merged && mv.n == 1 && (nel >> 2) % (2 * NTT_THREADS) == 0) {
                    // one product (L = 1): two iterations' loads in flight per thread
                    int64_t xo, yo;
                    mac_offsets<false>(mv, 0, xo, yo);
                    const uint4* xp = reinterpret_cast<const uint4*>(mac.X + xo + j0);
                    const uint4* yp = reinterpret_cast<const uint4*>(mac.Ym + yo + j0);
                    for (int q0 = threadIdx.x; q0 < (nel >> 2); q0 += 2 * NTT_THREADS) {
                        const uint4 x0 = __ldg(xp + q0), y0 = __ldg(yp + q0);
                        const uint4 x1 = __ldg(xp + q0 + NTT_THREADS), y1 = __ldg(yp + q0 + NTT_THREADS);
                        uint32_t* s = sm + pad_idx(4 * q0);
                        s[0] = mont_mul(x0.x, y0.x, mv.p, mv.pn); s[1] = mont_mul(x0.y, y0.y, mv.p, mv.pn);
                        s[2] = mont_mul(x0.z, y0.z, mv.p, mv.pn); s[3] = mont_mul(x0.w, y0.w, mv.p, mv.pn);
                        s = sm + pad_idx(4 * (q0 + NTT_THREADS));
                        s[0] = mont_mul(x1.x, y1.x, mv.p, mv.pn); s[1] = mont_mul(x1.y, y1.y, mv.p, mv.pn);
                        s[2] = mont_mul(x1.z, y1.z, mv.p, mv.pn); s[3] = mont_mul(x1.w, y1.w, mv.p, mv.pn);
                    }
                } else
                for (int q = threadIdx.x; q < (nel >> 2); q += blockDim.x) {
                    const uint4 t = mac_load4(mv, mac, j0 + 4 * q);
                    uint32_t* s = sm + pad_idx(4 * q);
                    s[0] = t.x; s[1] = t.y; s[2] = t.z; s[3] = t.w;
                }
            } else if ((nel >> 2) % (8 * NTT_THREADS) == 0) {
                // eight 16-byte loads in flight per thread before the shared-memory stores
                for (int q0 = 0; q0 < (nel >> 2); q0 += 8 * NTT_THREADS) {
                    uint4 t[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        t[k] = *reinterpret_cast<const uint4*>(data + gbase + 4 * (q0 + k * NTT_THREADS + threadIdx.x));
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        uint32_t* s = sm + pad_idx(4 * (q0 + k * NTT_THREADS + threadIdx.x));
                        s[0] = t[k].x; s[1] = t[k].y; s[2] = t[k].z; s[3] = t[k].w;
                    }
                }
            } else {
                for (int q = threadIdx.x; q < (nel >> 2); q += blockDim.x) {
                    const uint4 t = *reinterpret_cast<const uint4*>(data + gbase + 4 * q);
                    uint32_t* s = sm + pad_idx(4 * q);
                    s[0] = t.x; s[1] = t.y; s[2] = t.z; s[3] = t.w;
                }
            }
        } else {
            const MacVec mv = MAC ? mac_decode(g, vec, mac.ym_stride) : MacVec{};
            for (int i = threadIdx.x; i < nel; i += blockDim.x)
                sm[pad_idx(i)] = MAC ? mac_load1(mv, mac, j0 + i) : data[gbase + i];
        }
        __syncthreads();
        const int rin0 = (int)(row0 & ((int64_t(1) << lg_rpv) - 1));
        const PassArgs a{rows, (1 << g.m1) + rin0, 1, tw_all, g.N, pi, g.P, false};
        run_rounds<INV, false, M2, 0, 0>(sm, a);
    } else {
        // rows are whole vectors (N = M < tile): vector row0 + r, primes alternate
        bool any = false;
        for (int r = 0; r < rows && !any; ++r)
            any = INV ? inv_live(g, (unsigned)(row0 + r)) : fwd_live(g, (unsigned)(row0 + r));
        if (!any) return;
        for (int r = 0; r < rows; ++r) {
            const unsigned vec = (unsigned)(row0 + r);
            if (MAC) {
                const MacVec mv = mac_decode(g, vec, mac.ym_stride);
                for (int l = threadIdx.x; l < M; l += blockDim.x) sm[pad_idx((r << M2) + l)] = mac_load1(mv, mac, l);
            } else {
                for (int l = threadIdx.x; l < M; l += blockDim.x)
                    sm[pad_idx((r << M2) + l)] = data[((int64_t)vec << g.lgN) + l];
            }
        }
        __syncthreads();
        const PassArgs a{rows, 1, 0, tw_all, g.N, (int)(row0 % g.P), g.P, g.P > 1};
        run_rounds<INV, false, M2, 0, 0>(sm, a);
    }
    if ((nel & 3) == 0) {
        for (int q = threadIdx.x; q < (nel >> 2); q += blockDim.x) {
            const uint32_t* s = sm + pad_idx(4 * q);
            *reinterpret_cast<uint4*>(data + gbase + 4 * q) = make_uint4(s[0], s[1], s[2], s[3]);
        }
    } else {
        for (int i = threadIdx.x; i < nel; i += blockDim.x) data[gbase + i] = sm[pad_idx(i)];
    }
}

// ------------------------------------------------------------------ launches
static inline size_t ntt_smem_for(int64_t tile) { return (size_t)(tile + tile / 32) * sizeof(uint32_t); }

template <typename Kern>
static cudaError_t ntt_prep(Kern kernel, size_t smem)
{
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <bool INV, int M1>
cudaError_t launch_col_m(const NttGeom& g, uint32_t* data, const uint2* tw, cudaStream_t s)
{
    constexpr int64_t tile = (int64_t(1) << col_log_t(M1)) << M1;
    const size_t smem = ntt_smem_for(tile);
    cudaError_t e = ntt_prep(ntt_col_kernel<INV, M1>, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = g.nvec * ((int64_t(1) << g.m2) >> col_log_t(M1));
    ntt_col_kernel<INV, M1><<<(unsigned)grid, NTT_THREADS, smem, s>>>(g, data, tw);
    return cudaGetLastError();
}

// the V-vector inverse row pass applies to full tiles of one vector (2^12 <= N,
// rows of 2^5 .. 2^12 residues) with the MAC in registers and whole groups of
// V vectors per prime
inline bool inv_row_v_ok(const NttGeom& g, int M2)
{
    return g.mac_reg && M2 >= 5 && M2 <= TILE_LOG && g.lgN >= TILE_LOG && g.nvec % (4 * g.G * g.P) == 0;
}

template <int M2>
cudaError_t launch_inv_row_v(const NttGeom& g, uint32_t* data, const uint2* tw, MacSrc mac, cudaStream_t s)
{
    const size_t smem = (size_t)INV_PAIR_V * ntt_smem_for(int64_t(1) << TILE_LOG);
    const int64_t grid = (g.nvec / INV_PAIR_V) << (g.lgN - TILE_LOG);
    if (g.merged) {
        cudaError_t e = ntt_prep(ntt_inv_row_v_kernel<M2, true>, smem);
        if (e != cudaSuccess) return e;
        ntt_inv_row_v_kernel<M2, true><<<(unsigned)grid, NTT_THREADS, smem, s>>>(g, data, tw, mac);
    } else {
        cudaError_t e = ntt_prep(ntt_inv_row_v_kernel<M2, false>, smem);
        if (e != cudaSuccess) return e;
        ntt_inv_row_v_kernel<M2, false><<<(unsigned)grid, NTT_THREADS, smem, s>>>(g, data, tw, mac);
    }
    return cudaGetLastError();
}

template <bool INV, bool MAC, int M2>
cudaError_t launch_row_m(const NttGeom& g, uint32_t* data, const uint2* tw, MacSrc mac, cudaStream_t s)
{
    if constexpr (INV && MAC && M2 >= 5 && M2 <= TILE_LOG) {
        if (g.inv_vecs_per_cta == INV_PAIR_V && inv_row_v_ok(g, M2)) return launch_inv_row_v<M2>(g, data, tw, mac, s);
    }
    constexpr int RPC = M2 <= TILE_LOG ? (1 << (TILE_LOG - M2)) : 1;
    constexpr int64_t tile = (int64_t(1) << M2) * RPC;
    const size_t smem = ntt_smem_for(tile);
    cudaError_t e = ntt_prep(ntt_row_kernel<INV, MAC, M2>, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows_total = g.nvec * (g.N >> M2);
    const int64_t grid = (rows_total + RPC - 1) / RPC;
    ntt_row_kernel<INV, MAC, M2><<<(unsigned)grid, NTT_THREADS, smem, s>>>(g, data, tw, mac);
    return cudaGetLastError();
}

}  // namespace oz
