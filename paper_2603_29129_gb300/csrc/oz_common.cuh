// oz_common.cuh -- shared device definitions of libozfft (sm_103a).
//
// Modular arithmetic for the 32-bit NTTs (§3.3): every residue is kept
// canonical in [0, p) with p < 2^31, so a + b and a - b + p never exceed 2^32.
// Constant multiplications (NTT twiddles, Garner's inverse) use Shoup's
// precomputed quotient; products of two variable residues (the pointwise
// products of Alg. 8) use Montgomery multiplication with R = 2^32.
// The paper's CPU code uses the same two reductions (§5.5).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace oz {

constexpr int MAX_PRIMES = 3;
constexpr int MAX_K = 8;                      // split levels per vector
constexpr int MAX_GROUPS = MAX_K * MAX_K;     // flush groups per real convolution
constexpr int MAX_L = 8;                      // products per flush group

// data-dependent status bits (ozfft_get_status)
constexpr int ST_NONFINITE = 1;
constexpr int ST_RANGE = 2;
constexpr int ST_TIMEOUT = 4;   // a bounded device-side wait gave up
constexpr int ST_LEVELS = 8;    // K = infinity: a vector's residual is nonzero after MAX_K levels

struct PrimeInfo {
    uint32_t p;
    uint32_t pneg_inv;   // -p^-1 mod 2^32 (Montgomery)
};

// Flush schedule of one real convolution of one signal (Alg. 8); the layout is
// part of the debug-dump ABI: int32 ngroups, S[64], size[64], pair[64][8].
struct Sched {
    int32_t ngroups;
    int32_t S[MAX_GROUPS];           // s_x + s_y: the group's products carry 1/(c_x c_y) = 2^-S
    int32_t size[MAX_GROUPS];        // products in the group (<= L)
    int32_t pair[MAX_GROUPS][MAX_L]; // s * 16 + t; merged schedules add conv * 256
};

// The moduli: p0, p1 of §5.1 and a third NTT-friendly prime 15 * 2^27 + 1.
// N-th roots of unity exist for N up to 2^24, 2^25, 2^27 respectively.
constexpr uint32_t PRIME0 = 2130706433u;   // 127 * 2^24 + 1
constexpr uint32_t PRIME1 = 2113929217u;   //  63 * 2^25 + 1
constexpr uint32_t PRIME2 = 2013265921u;   //  15 * 2^27 + 1

__host__ __device__ __forceinline__ uint32_t prime_of(int pi)
{
    return pi == 0 ? PRIME0 : (pi == 1 ? PRIME1 : PRIME2);
}
// -p^-1 mod 2^32: for p = c 2^s + 1 with 2s >= 32 this is c 2^s - 1
// (the plan verifies p * pneg_inv == -1 mod 2^32 at creation)
__host__ __device__ __forceinline__ uint32_t pneg_inv_of(int pi)
{
    return pi == 0 ? PRIME0 - 2u : (pi == 1 ? PRIME1 - 2u : PRIME2 - 2u);
}

// ------------------------------------------------ division by small divisors
// x / d for a divisor 1 <= d <= SMALL_DIV_MAX that is the same in every thread (the
// number of primes, levels or flush groups of a vector index) and any 32-bit x,
// by multiplication with a precomputed reciprocal (division by invariant integers,
// Granlund and Montgomery 1994): M = floor(2^64 / d) + 1 (2^64 / d for a power
// of two), floor(x M / 2^64) = floor(x / d) since x (M d - 2^64) < 2^64.  A few
// integer instructions instead of the generic division sequence.
constexpr int SMALL_DIV_MAX = 512;
struct SmallRcp {
    unsigned long long v[SMALL_DIV_MAX + 1];
};
constexpr SmallRcp make_small_rcp()
{
    SmallRcp t{};
    for (int d = 2; d <= SMALL_DIV_MAX; ++d) t.v[d] = 0xffffffffffffffffull / (unsigned)d + 1ull;
    return t;
}
static __constant__ SmallRcp c_small_rcp = make_small_rcp();

__device__ __forceinline__ uint32_t udiv_small(uint32_t x, uint32_t d)
{
    if (d <= 1u) return x;
    if (d > (uint32_t)SMALL_DIV_MAX) return x / d;   // not reached: primes, levels and groups are below it
    const unsigned long long m = c_small_rcp.v[d];
    // the high word of x * m without the 64 x 64 product: x m_hi + high(x m_lo)
    const unsigned long long t = (unsigned long long)x * (uint32_t)(m >> 32) + __umulhi(x, (uint32_t)m);
    return (uint32_t)(t >> 32);
}

// ---------------------------------------------------------------- modular ops
__device__ __forceinline__ uint32_t mod_add(uint32_t a, uint32_t b, uint32_t p)
{
    uint32_t s = a + b;
    return min(s, s - p);
}
__device__ __forceinline__ uint32_t mod_sub(uint32_t a, uint32_t b, uint32_t p)
{
    uint32_t d = a - b + p;
    return min(d, d - p);
}
// Shoup: x * w mod p for a constant w < p with wq = floor(w 2^32 / p); any
// x < 2^32.  Lazy result in [0, 2p).
__device__ __forceinline__ uint32_t shoup_lazy(uint32_t x, uint32_t w, uint32_t wq, uint32_t p)
{
    uint32_t q = __umulhi(x, wq);
    return x * w - q * p;
}
__device__ __forceinline__ uint32_t shoup(uint32_t x, uint32_t w, uint32_t wq, uint32_t p)
{
    uint32_t r = shoup_lazy(x, w, wq, p);
    return min(r, r - p);
}
// Montgomery: a * b * 2^-32 mod p for a, b < p.
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t p, uint32_t pneg_inv)
{
    uint64_t t = (uint64_t)a * b;
    uint32_t m = (uint32_t)t * pneg_inv;
    uint32_t u = (uint32_t)((t + (uint64_t)m * p) >> 32);
    return min(u, u - p);
}

// ------------------------------------------------------------ binary64 helpers
// ceil(log2(mu)) for finite mu > 0, from the bit pattern: mu = 1.f * 2^(E-1023)
// gives E-1023 when f == 0 and E-1022 otherwise; subnormals likewise.
__device__ __forceinline__ int ceil_log2_pos(double mu)
{
    uint64_t b = (uint64_t)__double_as_longlong(mu);
    int E = (int)(b >> 52) & 0x7ff;
    uint64_t f = b & ((1ull << 52) - 1);
    if (E != 0) return f == 0 ? E - 1023 : E - 1022;
    // subnormal: mu = f * 2^-1074
    int fl = 63 - __clzll((long long)f);            // floor(log2 f)
    return ((f & (f - 1)) == 0 ? fl : fl + 1) - 1074;
}

// error-free transformations (no contraction: explicit round-to-nearest ops)
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    e = __dsub_rn(b, __dsub_rn(s, a));
}
// Double-word + double-word, AccurateDWPlusDW (Joldes, Muller, Popescu,
// ACM TOMS 2017, Alg. 6): relative error below 3u^2.
__device__ __forceinline__ void dw_add(double& xh, double& xl, double yh, double yl)
{
    double sh, sl, th, tl, vh, vl;
    two_sum(xh, yh, sh, sl);
    two_sum(xl, yl, th, tl);
    double c = __dadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    double w = __dadd_rn(tl, vl);
    fast_two_sum(vh, w, xh, xl);
}
// complex product, re = fma(a,c,-(b d)), im = fma(a,d,b c)
__device__ __forceinline__ void cmul(double a, double b, double c, double d, double& re, double& im)
{
    double bd = __dmul_rn(b, d);
    double bc = __dmul_rn(b, c);
    re = __fma_rn(a, c, -bd);
    im = __fma_rn(a, d, bc);
}

}  // namespace oz
