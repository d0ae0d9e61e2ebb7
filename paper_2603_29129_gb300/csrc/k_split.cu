// k_split.cu -- chirp table, Bluestein pre-multiply and the Ozaki split for
// libozfft (sm_103a).
//
//   chirp_kernel   w(j) = exp(-i pi j^2 / n) (Alg. 1), correctly rounded to
//                  binary64 from a double-word evaluation (plan time);
//   wstar_kernel   w~* = ZeroPad+-(conj w, N) (§3.2) (plan time);
//   premul_kernel  x~'(j) = x(j) w(j) for j < n, 0 up to N (Alg. 1 step 1);
//   split_kernel   one level k of Alg. 3 on every real vector of the batch.
//
// Each real vector v (Re or Im of a signal) is a contiguous row r[v][0..N).
// Its per-level maxima mu[v][k] = ||r^(k)||_inf are reduced with integer max and
// atomicMax on the binary64 bit pattern (non-negative doubles order like their
// bits); a
// kernel boundary separates level k's reduction from level k+1's use, which is
// the grid-wide dependency Alg. 3 has between mu^(k) and sigma^(k).
#include "oz_common.cuh"
#include "oz_kernels.h"
#include "ntt_impl.cuh"

namespace oz {

// ----------------------------------------------------- double-word sin / cos
struct dw { double h, l; };

__device__ __forceinline__ dw dw_norm(double a, double b)
{
    dw r;
    fast_two_sum(a, b, r.h, r.l);
    return r;
}
__device__ __forceinline__ dw dw_mul(dw a, dw b)
{
    double p = __dmul_rn(a.h, b.h);
    double e = __fma_rn(a.h, b.h, -p);
    e = __fma_rn(a.h, b.l, e);
    e = __fma_rn(a.l, b.h, e);
    return dw_norm(p, e);
}
__device__ __forceinline__ dw dw_div_d(dw a, double d)
{
    double q1 = __ddiv_rn(a.h, d);
    double p = __dmul_rn(q1, d);
    double pe = __fma_rn(q1, d, -p);                 // q1 d = p + pe exactly
    double r = __dadd_rn(__dsub_rn(__dsub_rn(a.h, p), pe), a.l);
    double q2 = __ddiv_rn(r, d);
    return dw_norm(q1, q2);
}
__device__ __forceinline__ dw dw_one_minus(dw a)
{
    double s, e;
    two_sum(1.0, -a.h, s, e);
    return dw_norm(s, __dsub_rn(e, a.l));
}

// sin(pi a/d), cos(pi a/d) for 0 <= a/d <= 1/4, Taylor series in Horner form
// on x = pi a/d in double-word arithmetic (truncation below 1e-40).
__device__ void sincospi_small(int64_t a, int64_t d, double& s_out, double& c_out)
{
    if (a == 0) { s_out = 0.0; c_out = 1.0; return; }
    const dw pi = {3.141592653589793116e+00, 1.224646799147353207e-16};
    double ad = (double)a, dd = (double)d;
    double t1 = __ddiv_rn(ad, dd);
    double rem = __fma_rn(-t1, dd, ad);              // exact remainder
    dw t = dw_norm(t1, __ddiv_rn(rem, dd));
    dw x = dw_mul(pi, t);
    dw x2 = dw_mul(x, x);
    dw s = {1.0, 0.0}, c = {1.0, 0.0};
    for (int k = 17; k >= 1; --k) {
        s = dw_one_minus(dw_div_d(dw_mul(x2, s), (double)((2 * k) * (2 * k + 1))));
        c = dw_one_minus(dw_div_d(dw_mul(x2, c), (double)((2 * k - 1) * (2 * k))));
    }
    s = dw_mul(x, s);
    s_out = __dadd_rn(s.h, s.l);
    c_out = __dadd_rn(c.h, c.l);
}

// sin, cos of pi a/d for 0 <= a/d < 2: exact integer octant reduction, then
// the small-angle evaluation.
__device__ void sincospi_frac(int64_t a, int64_t d, double& s, double& c)
{
    bool neg_s = false, neg_c = false, swap = false;
    if (a >= d) { a -= d; neg_s = !neg_s; neg_c = !neg_c; }
    if (2 * a > d) { a = d - a; neg_c = !neg_c; }
    if (4 * a > d) { a = d - 2 * a; d = 2 * d; swap = true; }
    double sv, cv;
    sincospi_small(a, d, sv, cv);
    if (swap) { double t = sv; sv = cv; cv = t; }
    s = neg_s ? -sv : sv;
    c = neg_c ? -cv : cv;
}

__global__ void chirp_kernel(double2* w, int64_t n)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r = ((uint64_t)j * (uint64_t)j) % (uint64_t)(2 * n);   // j < n <= 2^24
        double s, c;
        sincospi_frac((int64_t)r, n, s, c);
        w[j] = make_double2(c == 0.0 ? 0.0 : c, s == 0.0 ? 0.0 : -s);   // zero components are +0
    }
}

// chunking: a CTA works on CHUNK consecutive elements of one vector
constexpr int SPLIT_THREADS = 256;
constexpr int CHUNK = 4096;

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// block-wide max of non-negative binary64 bit patterns, then atomicMax into *dst
__device__ __forceinline__ void block_umax_to(uint64_t* dst, uint64_t v)
{
    __shared__ uint64_t redu[32];
    for (int o = 16; o > 0; o >>= 1) v = umax64(v, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) redu[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? redu[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) v = umax64(v, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o));
        if (lane == 0 && v) atomicMax((unsigned long long*)dst, (unsigned long long)v);
    }
}

// w~* of every signal: vector v = 2 b + part holds Re (part 0) or Im (part 1)
// of ZeroPad+-(conj w_b, N) (cyclic, w~* = conj w, when N = n)
__global__ void __launch_bounds__(SPLIT_THREADS) wstar_kernel(const double2* __restrict__ w, int64_t n, int64_t N,
                                                              const SigDesc* __restrict__ sd,
                                                              double* __restrict__ r, uint64_t* __restrict__ mu, int K)
{
    const int64_t chunks = (N + CHUNK - 1) / CHUNK;
    const int64_t v = blockIdx.x / chunks;
    const int part = (int)(v & 1);
    const int64_t j0 = (blockIdx.x % chunks) * CHUNK;
    const int64_t j1 = min(N, j0 + CHUNK);
    int64_t nb = n;
    if (sd) {
        const SigDesc d = sd[v >> 1];
        nb = d.n;
        w += d.chirp_off;
    }
    uint64_t m = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        int64_t src = -1;
        if (j < nb) src = j;
        else if (N != nb && j >= N - nb + 1) src = N - j;
        double val = 0.0;
        if (src >= 0) {
            const double2 ws = w[src];
            val = part == 0 ? ws.x : -ws.y;   // conj(w)
        }
        r[v * N + j] = val;
        m = umax64(m, (uint64_t)__double_as_longlong(val) & 0x7fffffffffffffffull);
    }
    block_umax_to(&mu[v * (K + 1) + 0], m);
}

__global__ void __launch_bounds__(SPLIT_THREADS) premul_kernel(const double2* __restrict__ x,
                                                               const double2* __restrict__ w, int64_t n, int64_t N,
                                                               int conj_in, const SigDesc* __restrict__ sd,
                                                               const IoPtrs* __restrict__ io, double* __restrict__ r,
                                                               uint64_t* __restrict__ mu, int K, int* status)
{
    const int64_t chunks = (N + CHUNK - 1) / CHUNK;
    const int64_t b = blockIdx.x / chunks;
    const int64_t j0 = (blockIdx.x % chunks) * CHUNK;
    const int64_t j1 = min(N, j0 + CHUNK);
    if (io) x = io->in;
    int64_t nb = n;
    if (sd) {
        const SigDesc d = sd[b];
        nb = d.n;
        x += d.io_off;
        w += d.chirp_off;
    } else {
        x += b * n;
    }
    uint64_t mr = 0, mi = 0;   // bit patterns of |.|: non-negative doubles order like their bits
    bool bad = false;
    double* rr = r + (2 * b) * N;
    double* ri = rr + N;
    for (int64_t jb = j0 + threadIdx.x; jb < j1; jb += 4 * (int64_t)blockDim.x) {
        double2 xv[4], wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {   // four elements' loads in flight before the arithmetic
            const int64_t j = jb + u * (int64_t)blockDim.x;
            if (j < j1 && j < nb) {
                xv[u] = __ldg(x + j);
                wv[u] = __ldg(w + j);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t j = jb + u * (int64_t)blockDim.x;
            if (j >= j1) break;
            double re = 0.0, im = 0.0;
            if (j < nb) {   // integer sign flip and finiteness test: the binary64 pipe is kept for the product
                const uint64_t bx = (uint64_t)__double_as_longlong(xv[u].x);
                const uint64_t by = (uint64_t)__double_as_longlong(xv[u].y);
                if ((~bx & 0x7ff0000000000000ull) == 0 || (~by & 0x7ff0000000000000ull) == 0) bad = true;
                const double xi = __longlong_as_double((long long)(by ^ ((uint64_t)(conj_in != 0) << 63)));
                cmul(xv[u].x, xi, wv[u].x, wv[u].y, re, im);
            }
            rr[j] = re;
            ri[j] = im;
            mr = umax64(mr, (uint64_t)__double_as_longlong(re) & 0x7fffffffffffffffull);
            mi = umax64(mi, (uint64_t)__double_as_longlong(im) & 0x7fffffffffffffffull);
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    block_umax_to(&mu[(2 * b) * (K + 1)], mr);
    __syncthreads();
    block_umax_to(&mu[(2 * b + 1) * (K + 1)], mi);
}

__global__ void set_io_kernel(IoPtrs* io, const double2* in, double2* out)
{
    io->in = in;
    io->out = out;
}

// One level of Alg. 3 on one element, from its bit pattern, in integer
// arithmetic only (binary64 throughput is low on this part).  With
// sigma = 2^(e + rho), |r| <= 2^e and rho >= 1, r + sigma stays in the binade
// [sigma, 2 sigma) for r >= 0 and [sigma/2, sigma) for r < 0, whose spacing is
// 2^g with g = e + rho - 52 (resp. - 53), never below 2^-1074.  Hence
//   s = fl(fl(r + sigma) - sigma) = 2^g * round_half_even(r / 2^g),
// the residual r - s is exact, and q = s / 2^(e - alpha) = s * 2^(alpha - e).
// "Even" is the parity of round(r / 2^g) because sigma / 2^g is even.
__device__ __forceinline__ void split_level_int(uint64_t rb, int e, int alpha, long long& q, uint64_t& rnb)
{
    const int rho = 53 - alpha;
    const bool neg = (rb >> 63) != 0;
    const int Eb = (int)((rb >> 52) & 0x7ff);
    uint64_t m = rb & ((1ull << 52) - 1);
    if (Eb == 0 && m == 0) { q = 0; rnb = rb; return; }
    int E = -1074;
    if (Eb) { m |= 1ull << 52; E = Eb - 1075; }          // r = +-m 2^E
    const int g = max(neg ? e + rho - 53 : e + rho - 52, -1074);
    uint64_t k;
    long long d;                                           // residual in units 2^E
    if (g <= E) {
        k = m << (E - g);
        d = 0;
    } else {
        const int sh = g - E;
        if (sh >= 64) {
            k = 0;
            d = (long long)m;
        } else {
            k = m >> sh;
            const uint64_t rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
            if (rem > half || (rem == half && (k & 1))) ++k;
            d = (long long)m - (long long)(k << sh);
        }
    }
    q = (long long)(k << (g - (e - alpha)));
    if (neg) { q = -q; d = -d; }
    if (d == 0) { rnb = 0; return; }                      // r - s == 0 is +0
    const uint64_t a = (uint64_t)(d < 0 ? -d : d);
    const int pb = 63 - __clzll((long long)a);            // leading bit of |d|
    uint64_t bits;
    if (E + pb >= -1022) {
        const uint64_t mant = pb <= 52 ? (a << (52 - pb)) : (a >> (pb - 52));
        bits = ((uint64_t)(E + pb + 1023) << 52) | (mant & ((1ull << 52) - 1));
    } else {
        bits = a << (E + 1074);                            // subnormal
    }
    rnb = bits | (d < 0 ? (1ull << 63) : 0ull);
}

// Level k of Alg. 3 for every vector: q = s 2^(alpha - e) with |q| <= 2^alpha,
// residues q mod p written per prime, the residual written back for the next
// level and its maximum reduced into mu[v][k+1].
template <bool SD>
__global__ void __launch_bounds__(SPLIT_THREADS) split_kernel(int k, double* __restrict__ r,
                                                              uint64_t* __restrict__ mu, int64_t N, int K,
                                                              int alpha, const SigDesc* __restrict__ sd, int P,
                                                              uint32_t* __restrict__ X, int write_r, int* status)
{
    const int64_t chunks = (N + CHUNK - 1) / CHUNK;
    const int64_t v = blockIdx.x / chunks;
    if (SD) alpha = sd[v >> 1].alpha;                     // vector v = 2 b + part
    const int64_t j0 = (blockIdx.x % chunks) * CHUNK;
    const int64_t j1 = min(N, j0 + CHUNK);
    const uint64_t mub = mu[v * (K + 1) + k];
    if (mub == 0) return;                                 // level empty: mu^(k) = 0 ends the split
    const int e = ceil_log2_pos(__longlong_as_double((long long)mub));
    if (e + 53 - alpha > 1023) {
        if (threadIdx.x == 0) atomicOr(status, ST_RANGE);
        return;
    }
    uint64_t* rv = reinterpret_cast<uint64_t*>(r + v * N);
    uint32_t* xk = X + ((v * K + k) * P) * N;
    uint64_t m = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        long long q;
        uint64_t rn;
        split_level_int(rv[j], e, alpha, q, rn);
#pragma unroll
        for (int pi = 0; pi < MAX_PRIMES; ++pi) {
            if (pi >= P) break;
            const long long p = (long long)prime_of(pi);
            long long a = alpha <= 30 ? q : q % p;   // |q| <= 2^alpha < p when alpha <= 30
            if (a < 0) a += p;
            xk[pi * N + j] = (uint32_t)a;
        }
        if (write_r) rv[j] = rn;
        m = umax64(m, rn & 0x7fffffffffffffffull);
    }
    if (k + 1 <= K) block_umax_to(&mu[v * (K + 1) + k + 1], m);
}

// One level of Alg. 3 on an element held as sign, integer magnitude and the
// fixed exponent of its binary64 input: r = (-1)^neg a 2^E with a < 2^53 and
// E the weight of the input's last mantissa bit.  The level's grid is 2^g
// (g as in split_level_int); with sh = g - E the level keeps
// kq = round_half_even(a / 2^sh) grid units and leaves the exact residual
// (a - kq 2^sh) 2^E, which stays in the same units, so nothing is renormalised
// between levels.  q = +-kq 2^(g - (e - alpha)).
__device__ __forceinline__ long long split_level_fixed(uint64_t& a, bool& neg, int E, int e, int alpha)
{
    if (a == 0) return 0;
    const int g = max(neg ? e - alpha : e + 1 - alpha, -1074);
    const int sh = g - E;
    uint64_t kq;
    long long d;
    if (sh <= 0) {                       // the grid is at least as fine as the input: all of it is kept
        kq = a << (-sh);
        d = 0;
    } else if (sh >= 64) {               // a < 2^53 <= 2^(sh - 1): rounds to zero
        kq = 0;
        d = (long long)a;
    } else {
        kq = a >> sh;
        const uint64_t rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (kq & 1))) ++kq;
        d = (long long)a - (long long)(kq << sh);
    }
    long long q = (long long)(kq << (g - (e - alpha)));
    if (neg) q = -q;
    neg = neg != (d < 0);
    a = (uint64_t)(d < 0 ? -d : d);
    return q;
}

// The same level for alpha <= 30 (|q| <= 2^alpha fits 32 bits): the rounding
// of a / 2^sh to nearest, ties to even, as one add and one shift,
// (a + 2^(sh-1) - 1 + odd) >> sh with odd the last bit of a >> sh (a remainder
// above half carries, one below does not, exactly half carries when the
// quotient is odd), then the exact residual a - kq 2^sh.  Bit-identical to
// split_level_fixed (which handles any alpha).
__device__ __forceinline__ int32_t split_level_fixed32(uint64_t& a, bool& neg, int E, int e, int alpha)
{
    if (a == 0) return 0;
    const int g = max(neg ? e - alpha : e + 1 - alpha, -1074);
    const int sh = g - E;
    uint32_t kq;
    int64_t d;
    if (sh <= 0) {                       // the grid is at least as fine as the input: all of it is kept
        kq = (uint32_t)(a << (-sh));
        d = 0;
    } else if (sh >= 55) {               // a < 2^53 < 2^(sh - 2): rounds to zero
        kq = 0;
        d = (int64_t)a;
    } else {
        const uint64_t k64 = (a + ((1ull << (sh - 1)) - 1) + ((a >> sh) & 1ull)) >> sh;
        kq = (uint32_t)k64;
        d = (int64_t)a - (int64_t)(k64 << sh);
    }
    int32_t q = (int32_t)(kq << (g - (e - alpha)));
    if (neg) q = -q;
    neg = neg != (d < 0);
    a = (uint64_t)(d < 0 ? -d : d);
    return q;
}

// ceil(log2(a 2^E)) for a > 0
__device__ __forceinline__ int ceil_log2_fixed(uint64_t a, int E)
{
    return E + (a == 1 ? 0 : 64 - __clzll((long long)(a - 1)));
}

// binary64 bit pattern of 2^c (-1074 <= c <= 1023)
__device__ __forceinline__ uint64_t pow2_bits(int c)
{
    return c >= -1022 ? (uint64_t)(c + 1023) << 52 : 1ull << (c + 1074);
}

// All K levels of Alg. 3 in one pass over the vectors, the exponent of level
// k >= 1 taken as e_k = e_0 - k alpha.  Level k rounds to a grid of 2^(e_k + 1
// - alpha) (2^(e_k - alpha) for negative r), so its residual stays within
// 2^(e_k - alpha) and e_(k+1) = ceil_log2 mu^(k+1) can only be that or smaller;
// it is smaller only when no residual of the whole vector reaches half the
// bound.  Alg. 3 uses mu^(k) only through ceil_log2 mu^(k), and ceil_log2 of a
// maximum is the maximum of the ceil_log2, so mu[v][k] (k >= 1) receives
// 2^ceil_log2 of the largest residual (0 when all are zero);
// split_fix_kernel then redoes every vector whose exponents contradict the
// guess, so the slices are those of Alg. 3 either way.  Residuals are not
// written back (r keeps r^(0)).  KM bounds K at compile time (the per-level
// maxima stay in registers).
template <bool SD, int KM, bool A30>
__global__ void __launch_bounds__(SPLIT_THREADS) split_spec_kernel(const double* __restrict__ r,
                                                                   uint64_t* __restrict__ mu, int64_t N, int K,
                                                                   int alpha, const SigDesc* __restrict__ sd, int P,
                                                                   uint32_t* __restrict__ X, int* status)
{
    const int64_t chunks = (N + CHUNK - 1) / CHUNK;
    const int64_t v = blockIdx.x / chunks;
    if (SD) alpha = sd[v >> 1].alpha;
    const int64_t j0 = (blockIdx.x % chunks) * CHUNK;
    const int64_t j1 = min(N, j0 + CHUNK);
    const uint64_t mub = mu[v * (K + 1)];
    if (mub == 0) return;                                 // every level empty
    const int e0 = ceil_log2_pos(__longlong_as_double((long long)mub));
    if (e0 + 53 - alpha > 1023) {
        if (threadIdx.x == 0) atomicOr(status, ST_RANGE);
        return;
    }
    const uint64_t* rv = reinterpret_cast<const uint64_t*>(r + v * N);
    uint32_t* xv = X + (v * K) * P * N;
    int cmax[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) cmax[k] = -2000;
    uint64_t rb_next = j0 + threadIdx.x < j1 ? rv[j0 + threadIdx.x] : 0ull;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const uint64_t rb = rb_next;   // the next element's load in flight during this one's levels
        if (j + blockDim.x < j1) rb_next = rv[j + blockDim.x];
        bool neg = (rb >> 63) != 0;
        const int Eb = (int)((rb >> 52) & 0x7ff);
        uint64_t a = rb & ((1ull << 52) - 1);
        int E = -1074;
        if (Eb) { a |= 1ull << 52; E = Eb - 1075; }
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if (k >= K) break;
            if constexpr (A30) {                  // |q| <= 2^alpha < p
                const int32_t q = split_level_fixed32(a, neg, E, e0 - k * alpha, alpha);
#pragma unroll
                for (int pi = 0; pi < MAX_PRIMES; ++pi) {
                    if (pi >= P) break;
                    const uint32_t p = prime_of(pi);
                    xv[(k * P + pi) * N + j] = q < 0 ? (uint32_t)(q + (int32_t)p) : (uint32_t)q;
                }
            } else {
                const long long q = split_level_fixed(a, neg, E, e0 - k * alpha, alpha);
#pragma unroll
                for (int pi = 0; pi < MAX_PRIMES; ++pi) {
                    if (pi >= P) break;
                    long long t = q % (long long)prime_of(pi);
                    if (t < 0) t += prime_of(pi);
                    xv[(k * P + pi) * N + j] = (uint32_t)t;
                }
            }
            if (a) cmax[k] = max(cmax[k], ceil_log2_fixed(a, E));
        }
    }
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (k >= K) break;
        block_umax_to(&mu[v * (K + 1) + k + 1], cmax[k] > -2000 ? pow2_bits(cmax[k]) : 0ull);
        __syncthreads();
    }
}

// One CTA per vector: keep the speculative split when every nonzero mu[v][k]
// (k = 1 .. K-1) has ceil_log2 = e_0 - k alpha; otherwise run Alg. 3 level by
// level from r^(0), residuals in place, and rewrite mu[v][1..K] (as powers of
// two, like the one-pass kernel).
constexpr int FIX_THREADS = 512;
template <bool SD>
__global__ void __launch_bounds__(FIX_THREADS) split_fix_kernel(double* __restrict__ r, uint64_t* __restrict__ mu,
                                                                int64_t N, int K, int alpha,
                                                                const SigDesc* __restrict__ sd, int P,
                                                                uint32_t* __restrict__ X, int32_t* __restrict__ redo)
{
    const int64_t v = blockIdx.x;
    if (SD) alpha = sd[v >> 1].alpha;
    uint64_t* mv = mu + v * (K + 1);
    if (redo && threadIdx.x == 0) redo[v] = 0;
    if (mv[0] == 0) return;
    const int e0 = ceil_log2_pos(__longlong_as_double((long long)mv[0]));
    if (e0 + 53 - alpha > 1023) return;                   // flagged by the speculative pass
    bool ok = true;
    for (int k = 1; k < K && ok; ++k) {
        if (mv[k] == 0) break;                            // r^(k) = 0: the rest is zero under any exponent
        ok = ceil_log2_pos(__longlong_as_double((long long)mv[k])) == e0 - k * alpha;
    }
    if (ok) return;
    if (redo && threadIdx.x == 0) redo[v] = 1;            // its residues are rewritten untransformed
    __syncthreads();                                      // every thread has read mu before it changes
    __shared__ uint64_t redu[32];
    uint64_t* rv = reinterpret_cast<uint64_t*>(r + v * N);
    for (int k = 0; k < K; ++k) {
        const uint64_t mk = mv[k];
        if (mk == 0) {                                    // level k empty: so are the rest
            if (threadIdx.x == 0)
                for (int l = k + 1; l <= K; ++l) mv[l] = 0;
            return;
        }
        const int e = ceil_log2_pos(__longlong_as_double((long long)mk));
        uint32_t* xk = X + ((v * K + k) * P) * N;
        uint64_t m = 0;
        for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
            long long q;
            uint64_t rn;
            split_level_int(rv[j], e, alpha, q, rn);
            for (int pi = 0; pi < P; ++pi) {
                const long long p = (long long)prime_of(pi);
                long long a = alpha <= 30 ? q : q % p;
                if (a < 0) a += p;
                xk[pi * N + j] = (uint32_t)a;
            }
            if (k + 1 < K) rv[j] = rn;
            m = umax64(m, rn & 0x7fffffffffffffffull);
        }
        for (int o = 16; o > 0; o >>= 1) m = umax64(m, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)m, o));
        if ((threadIdx.x & 31) == 0) redu[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = umax64(t, redu[w]);
            mv[k + 1] = t ? pow2_bits(ceil_log2_pos(__longlong_as_double((long long)t))) : 0ull;
        }
        __syncthreads();                                  // mu[v][k + 1] and r^(k + 1) before the next level
    }
}

// ------------------------------- split fused with the forward column pass
// One CTA takes T = 2^(11 - m1) adjacent columns x all 2^m1 rows of one real
// vector (2048 elements, j = row 2^m2 + col), runs every level of Alg. 3 on
// them with the guessed exponents of split_spec_kernel (the level maxima
// reduced into mu for split_fix_kernel's check), writes each level's residues
// per prime into a dense shared-memory tile [row][T], transforms the columns of
// all K P tiles (stages 0..m1-1 of the forward NTT, as the column pass does) and
// stores them into X.  The untransformed residues never reach HBM: against
// the split and the column pass apart, X is written once instead of written,
// read and written again.  Consecutive lanes take consecutive columns of a
// row, so the dense tiles need no pad words for T >= 32 (T = 16 for m1 = 7
// leaves some 2-way conflicts).
constexpr int SC_THREADS = 256;
constexpr int SC_TILE_LOG = 11;
constexpr int SC_TILE = 1 << SC_TILE_LOG;     // elements per tile

template <int ML, int S0, int RL, int LOG_T>
__device__ __forceinline__ void sc_round(uint32_t* sm, int ntiles, int P, const uint2* __restrict__ tw_all, int64_t N)
{
    constexpr int LOG_H = ML - S0 - RL, H = 1 << LOG_H, LOG_GPC = ML - RL, T = 1 << LOG_T;
    constexpr int LOG_GPT = LOG_T + LOG_GPC;     // groups per tile = T 2^LOG_GPC
    for (int gid = threadIdx.x; gid < (ntiles << LOG_GPT); gid += SC_THREADS) {
        const int tile = gid >> LOG_GPT;
        const int gg = gid & ((1 << LOG_GPT) - 1);
        const int c = gg & (T - 1), grp = gg >> LOG_T;
        const int blk = grp >> LOG_H;
        const int l0 = (blk << (ML - S0)) + (grp & (H - 1));
        // prime of tile k P + pi without a division (tile < 9): tile / 3 = (11 tile) >> 5
        const int pi = P == 1 ? 0 : (P == 2 ? (tile & 1) : tile - 3 * ((tile * 11) >> 5));
        group_bfly<false, RL, H * T, false>(sm + tile * SC_TILE + (l0 << LOG_T) + c, tw_all + pi * N, (1 << S0) + blk,
                                            prime_of(pi));
    }
}

template <int ML, int LOG_T, int I>
__device__ __forceinline__ void sc_rounds(uint32_t* sm, int ntiles, int P, const uint2* tw_all, int64_t N)
{
    if constexpr (I < Part<ML>::NR) {
        sc_round<ML, Part<ML>::start(I), Part<ML>::size(I), LOG_T>(sm, ntiles, P, tw_all, N);
        __syncthreads();
        sc_rounds<ML, LOG_T, I + 1>(sm, ntiles, P, tw_all, N);
    }
}

template <bool SD, int M1, int KM, bool A30>
__global__ void __launch_bounds__(SC_THREADS) split_col_kernel(const double* __restrict__ r, uint64_t* __restrict__ mu,
                                                               int64_t N, int m2, int K, int alpha,
                                                               const SigDesc* __restrict__ sd, int P,
                                                               uint32_t* __restrict__ X, const uint2* __restrict__ tw_all,
                                                               int* status)
{
    constexpr int LOG_T = SC_TILE_LOG - M1, T = 1 << LOG_T;
    static_assert(T >= 8, "16-byte row segments");
    extern __shared__ __align__(16) uint32_t sct[];      // K P tiles of SC_TILE words
    const int lg_tpv = m2 - LOG_T;
    const int64_t v = blockIdx.x >> lg_tpv;
    const int c0 = (int)(blockIdx.x & ((1u << lg_tpv) - 1)) << LOG_T;
    if (SD) alpha = sd[v >> 1].alpha;
    const uint64_t mub = mu[v * (K + 1)];
    if (mub == 0) return;                                 // every level empty
    const int e0 = ceil_log2_pos(__longlong_as_double((long long)mub));
    if (e0 + 53 - alpha > 1023) {
        if (threadIdx.x == 0) atomicOr(status, ST_RANGE);
        return;
    }
    const uint64_t* rv = reinterpret_cast<const uint64_t*>(r + v * N);
    int cmax[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) cmax[k] = -2000;
#pragma unroll 2
    for (int e = threadIdx.x; e < SC_TILE; e += SC_THREADS) {
        const uint64_t rb = rv[((int64_t)(e >> LOG_T) << m2) + c0 + (e & (T - 1))];
        bool neg = (rb >> 63) != 0;
        const int Eb = (int)((rb >> 52) & 0x7ff);
        uint64_t a = rb & ((1ull << 52) - 1);
        int E = -1074;
        if (Eb) { a |= 1ull << 52; E = Eb - 1075; }
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if (k >= K) break;
            if constexpr (A30) {                          // |q| <= 2^alpha < p
                const int32_t q = split_level_fixed32(a, neg, E, e0 - k * alpha, alpha);
#pragma unroll
                for (int pi = 0; pi < MAX_PRIMES; ++pi) {
                    if (pi >= P) break;
                    const uint32_t p = prime_of(pi);
                    sct[(k * P + pi) * SC_TILE + e] = q < 0 ? (uint32_t)(q + (int32_t)p) : (uint32_t)q;
                }
            } else {
                const long long q = split_level_fixed(a, neg, E, e0 - k * alpha, alpha);
#pragma unroll
                for (int pi = 0; pi < MAX_PRIMES; ++pi) {
                    if (pi >= P) break;
                    long long t = q % (long long)prime_of(pi);
                    if (t < 0) t += prime_of(pi);
                    sct[(k * P + pi) * SC_TILE + e] = (uint32_t)t;
                }
            }
            if (a) cmax[k] = max(cmax[k], ceil_log2_fixed(a, E));
        }
    }
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (k >= K) break;
        block_umax_to(&mu[v * (K + 1) + k + 1], cmax[k] > -2000 ? pow2_bits(cmax[k]) : 0ull);
        __syncthreads();                                  // also: every residue tile is complete
    }
    sc_rounds<M1, LOG_T, 0>(sct, K * P, P, tw_all, N);
    // store: 16-byte row segments of each tile (vector (v K + k) P + pi of X)
    constexpr int Q = SC_TILE / 4;
    for (int q = threadIdx.x; q < K * P * Q; q += SC_THREADS) {
        const int tile = q / Q, w = q - tile * Q;
        const int row = w >> (LOG_T - 2), c = (w & ((T >> 2) - 1)) << 2;
        const uint4 val = *reinterpret_cast<const uint4*>(sct + tile * SC_TILE + (row << LOG_T) + c);
        *reinterpret_cast<uint4*>(X + (v * K * P + tile) * N + ((int64_t)row << m2) + c0 + c) = val;
    }
}

// ------------------------------------------------------------------ launchers
static unsigned grid_for(int64_t nvec, int64_t N) { return (unsigned)(nvec * ((N + CHUNK - 1) / CHUNK)); }

cudaError_t launch_chirp(double2* w, int64_t n, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    chirp_kernel<<<(unsigned)blocks, 256, 0, s>>>(w, n);
    return cudaGetLastError();
}

cudaError_t launch_wstar(const double2* w, int64_t n, int64_t N, int64_t B, const SigDesc* sd, double* r, uint64_t* mu,
                         int K, int*, cudaStream_t s)
{
    wstar_kernel<<<grid_for(2 * B, N), SPLIT_THREADS, 0, s>>>(w, n, N, sd, r, mu, K);
    return cudaGetLastError();
}

cudaError_t launch_premul(const double2* x, const double2* w, int64_t n, int64_t N, int64_t B, int conj_in,
                          const SigDesc* sd, const IoPtrs* io, double* r, uint64_t* mu, int K, int* status,
                          cudaStream_t s)
{
    premul_kernel<<<grid_for(B, N), SPLIT_THREADS, 0, s>>>(x, w, n, N, conj_in, sd, io, r, mu, K, status);
    return cudaGetLastError();
}

cudaError_t launch_split_level(int k, double* r, const uint64_t*, uint64_t* mu, int64_t N, int64_t nvec, int K,
                               int alpha, const SigDesc* sd, int P, uint32_t* X, int write_r, int* status,
                               cudaStream_t s)
{
    if (sd) split_kernel<true><<<grid_for(nvec, N), SPLIT_THREADS, 0, s>>>(k, r, mu, N, K, alpha, sd, P, X, write_r, status);
    else split_kernel<false><<<grid_for(nvec, N), SPLIT_THREADS, 0, s>>>(k, r, mu, N, K, alpha, sd, P, X, write_r, status);
    return cudaGetLastError();
}

cudaError_t launch_split_spec(double* r, uint64_t* mu, int64_t N, int64_t nvec, int K, int alpha, const SigDesc* sd,
                              int P, uint32_t* X, int* status, cudaStream_t s)
{
    const unsigned grid = grid_for(nvec, N);
    // alpha of every signal <= 30 (the plan's largest for a length class): 32-bit digits
    const bool a30 = alpha <= 30;
#define OZ_SPLIT_SPEC(SDV, KMV, A30V) \
    split_spec_kernel<SDV, KMV, A30V><<<grid, SPLIT_THREADS, 0, s>>>(r, mu, N, K, alpha, sd, P, X, status)
    if (sd) {
        if (K <= 4) { if (a30) OZ_SPLIT_SPEC(true, 4, true); else OZ_SPLIT_SPEC(true, 4, false); }
        else { if (a30) OZ_SPLIT_SPEC(true, MAX_K, true); else OZ_SPLIT_SPEC(true, MAX_K, false); }
        split_fix_kernel<true><<<(unsigned)nvec, FIX_THREADS, 0, s>>>(r, mu, N, K, alpha, sd, P, X, nullptr);
    } else {
        if (K <= 4) { if (a30) OZ_SPLIT_SPEC(false, 4, true); else OZ_SPLIT_SPEC(false, 4, false); }
        else { if (a30) OZ_SPLIT_SPEC(false, MAX_K, true); else OZ_SPLIT_SPEC(false, MAX_K, false); }
        split_fix_kernel<false><<<(unsigned)nvec, FIX_THREADS, 0, s>>>(r, mu, N, K, alpha, sd, P, X, nullptr);
    }
#undef OZ_SPLIT_SPEC
    return cudaGetLastError();
}

bool split_col_supported(int K, int P, int m1, int m2)
{
    return K >= 1 && K <= 4 && K * P <= 9 && m1 >= 5 && m1 <= 8 && m2 >= SC_TILE_LOG - m1;
}

template <bool SD, int M1>
static cudaError_t launch_split_col_m(double* r, uint64_t* mu, int64_t N, int m2, int64_t nvec, int K, int alpha,
                                      const SigDesc* sd, int P, uint32_t* X, const uint2* tw, int* status,
                                      cudaStream_t s)
{
    const size_t smem = (size_t)K * P * SC_TILE * sizeof(uint32_t);
    const unsigned grid = (unsigned)(nvec << (m2 - (SC_TILE_LOG - M1)));
    cudaError_t e;
    if (alpha <= 30) {
        e = cudaFuncSetAttribute(split_col_kernel<SD, M1, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        split_col_kernel<SD, M1, 4, true><<<grid, SC_THREADS, smem, s>>>(r, mu, N, m2, K, alpha, sd, P, X, tw, status);
    } else {
        e = cudaFuncSetAttribute(split_col_kernel<SD, M1, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        split_col_kernel<SD, M1, 4, false><<<grid, SC_THREADS, smem, s>>>(r, mu, N, m2, K, alpha, sd, P, X, tw, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_col(double* r, uint64_t* mu, int64_t N, int m1, int m2, int64_t nvec, int K, int alpha,
                             const SigDesc* sd, int P, uint32_t* X, const uint2* tw, int32_t* redo, int* status,
                             cudaStream_t s)
{
    if (!split_col_supported(K, P, m1, m2)) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    switch (m1) {
    case 5: e = sd ? launch_split_col_m<true, 5>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s)
                   : launch_split_col_m<false, 5>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s); break;
    case 6: e = sd ? launch_split_col_m<true, 6>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s)
                   : launch_split_col_m<false, 6>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s); break;
    case 7: e = sd ? launch_split_col_m<true, 7>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s)
                   : launch_split_col_m<false, 7>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s); break;
    case 8: e = sd ? launch_split_col_m<true, 8>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s)
                   : launch_split_col_m<false, 8>(r, mu, N, m2, nvec, K, alpha, sd, P, X, tw, status, s); break;
    default: break;
    }
    if (e != cudaSuccess) return e;
    // the check: vectors whose guessed exponents fail are redone level by level,
    // untransformed, and flagged for the column pass
    if (sd) split_fix_kernel<true><<<(unsigned)nvec, FIX_THREADS, 0, s>>>(r, mu, N, K, alpha, sd, P, X, redo);
    else split_fix_kernel<false><<<(unsigned)nvec, FIX_THREADS, 0, s>>>(r, mu, N, K, alpha, sd, P, X, redo);
    return cudaGetLastError();
}

cudaError_t launch_set_io(IoPtrs* io, const void* in, void* out, cudaStream_t s)
{
    set_io_kernel<<<1, 1, 0, s>>>(io, (const double2*)in, (double2*)out);
    return cudaGetLastError();
}

}  // namespace oz
