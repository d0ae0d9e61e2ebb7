// k_crt.cu -- Garner CRT, exact accumulation, rounding and the Bluestein
// post-multiply for libozfft (sm_103a).
//
// For every output y(k), k < n, of every signal: each flush group g of the
// four real convolutions (RR, II, IR, RI, §4.5) contributes the CRT integer z'
// of its inverse NTTs (Garner with symmetric digits, Eq. (1), §3.3) times
// 1/(c_x c_y) = 2^-S_g (Alg. 8).  The real part of y' is the exact sum of the
// RR terms minus the II terms and the imaginary part the exact sum of the IR and
// RI terms, each rounded once to nearest binary64; then y = y' w (Alg. 1).  The
// inverse direction conjugates and divides by n (Eq. (4)); the adjoint of the
// forward transform (+2) only conjugates, that of the inverse (-2) only divides.
//
// The exact sums use integer arithmetic only (binary64 throughput is low on
// this part), in three kernels by signal:
//   crt_fast_kernel  two primes, every convolution's group scales non-increasing
//                    in schedule order (always, unless split levels have gaps)
//                    and spanning <= FAST_SPAN bits: Horner's rule on a 192-bit
//                    integer, groups taken from the smallest scale up, so a
//                    change of scale is one left shift and every term a plain
//                    add-with-carry;
//   crt_reg_body     (inside crt_fast_kernel's launch) the other two-prime
//                    signals whose scales span at most
//                    REG_LIMBS - 5 limbs: int64 limbs in registers, each holding
//                    a sum of 32-bit digits in units of 2^-max(S); a term
//                    z * 2^(max S - S_g) is split into digits and added to
//                    consecutive limbs without carries;
//   crt_fast3_kernel three primes, the same conditions (span <= FAST3_SPAN):
//                    Horner's rule with 128-bit CRT integers;
//   crt_wide_kernel  the rest (wide spans, scales out of order with three
//                    primes): the same limbs as a column per thread in shared
//                    memory.
// One carry pass and an integer round-to-nearest-even at the end produce the
// binary64 bit pattern.
#include <mutex>

#include "ntt_impl.cuh"
#include "ts_arith.cuh"

namespace oz {

struct GarnerConst {
    uint32_t inv01, inv01q;   // p0^-1 mod p1 and its Shoup quotient
    uint32_t inv2, inv2q;     // (p0 p1)^-1 mod p2 and its Shoup quotient
    uint32_t p0_mod2;         // p0 mod p2
};

__constant__ GarnerConst c_garner;

constexpr uint32_t P0 = PRIME0, P1 = PRIME1, P2 = PRIME2;

// 128-bit two's complement integer as (hi, lo)
struct i128p { long long hi; unsigned long long lo; };

__device__ __forceinline__ i128p garner(const uint32_t* z, int P)
{
    // z'_0: symmetric representative of z0 mod p0
    long long v0 = (long long)z[0];
    if (v0 > (long long)(P0 - 1) / 2) v0 -= P0;
    // digit 1: ((z1 - z'_0) p0^-1) mod p1, symmetric
    long long t = (long long)z[1] - v0;
    if (t < 0) t += P1;
    else if (t >= (long long)P1) t -= P1;
    long long d1 = (long long)shoup((uint32_t)t, c_garner.inv01, c_garner.inv01q, P1);
    if (d1 > (long long)(P1 - 1) / 2) d1 -= P1;
    const long long z1 = v0 + d1 * (long long)P0;     // |z1| < p0 p1 / 2 < 2^62
    i128p r;
    if (P == 2) {
        r.hi = z1 < 0 ? -1 : 0;
        r.lo = (unsigned long long)z1;
        return r;
    }
    // digit 2: ((z2 - z'_1) (p0 p1)^-1) mod p2, symmetric
    const long long v0m = v0 < 0 ? v0 + P2 : v0;
    const long long d1m = d1 < 0 ? d1 + P2 : d1;
    const long long zm = (v0m + (d1m * (long long)c_garner.p0_mod2) % P2) % P2;   // z'_1 mod p2
    long long t2 = (long long)z[2] - zm;
    if (t2 < 0) t2 += P2;
    long long d2 = (long long)shoup((uint32_t)t2, c_garner.inv2, c_garner.inv2q, P2);
    if (d2 > (long long)(P2 - 1) / 2) d2 -= P2;
    // z'_2 = z'_1 + d2 p0 p1 in 128 bits
    const unsigned long long p01 = (unsigned long long)P0 * P1;
    const unsigned long long ad = (unsigned long long)(d2 < 0 ? -d2 : d2);
    unsigned long long plo = ad * p01, phi = __umul64hi(ad, p01);
    if (d2 < 0) {
        plo = ~plo + 1ull;
        phi = ~phi + (plo == 0 ? 1ull : 0ull);
    }
    const unsigned long long zlo = (unsigned long long)z1;
    const unsigned long long zhi = z1 < 0 ? ~0ull : 0ull;
    r.lo = plo + zlo;
    r.hi = (long long)(phi + zhi + (r.lo < plo ? 1ull : 0ull));
    return r;
}

// acc[col + l*stride] += digits of z * 2^sh, l = sh/32 .. sh/32+3
__device__ __forceinline__ void add_term(long long* acc, int stride, i128p z, int sh)
{
    const int q = sh >> 5, b = sh & 31;
    const unsigned long long t0 = z.lo << b;
    const unsigned long long t1 = b ? (((unsigned long long)z.hi << b) | (z.lo >> (64 - b))) : (unsigned long long)z.hi;
    long long* a = acc + q * stride;
    a[0] += (long long)(uint32_t)t0;
    a[stride] += (long long)(uint32_t)(t0 >> 32);
    a[2 * stride] += (long long)(uint32_t)t1;
    a[3 * stride] += (long long)(int32_t)(uint32_t)(t1 >> 32);
}

// Round the integer sum of nl limbs (value = sum acc[l] 2^(32 l) 2^unit) to the
// nearest binary64, ties to even, from integer operations only.
__device__ double limbs_to_double(long long* acc, int stride, int nl, int unit)
{
    // carry pass: 32-bit digits in place (two's complement, the top digit signed)
    long long carry = 0;
    for (int l = 0; l < nl; ++l) {
        const long long v = acc[l * stride] + carry;
        acc[l * stride] = (long long)(uint32_t)v;
        carry = v >> 32;
    }
    const bool neg = (acc[(nl - 1) * stride] >> 31) & 1;
    if (neg) {   // magnitude by two's complement negation
        unsigned long long c = 1;
        for (int l = 0; l < nl; ++l) {
            const unsigned long long s = (unsigned long long)(uint32_t)~(uint32_t)acc[l * stride] + c;
            acc[l * stride] = (long long)(uint32_t)s;
            c = s >> 32;
        }
    }
    int top = nl - 1;
    while (top >= 0 && (uint32_t)acc[top * stride] == 0) --top;
    if (top < 0) return 0.0;
    const uint32_t dt = (uint32_t)acc[top * stride];
    const int lz = __clz(dt);
    // 96-bit window from digits top, top-1, top-2, leading one moved to bit 63
    const uint32_t d1 = top >= 1 ? (uint32_t)acc[(top - 1) * stride] : 0u;
    const uint32_t d2 = top >= 2 ? (uint32_t)acc[(top - 2) * stride] : 0u;
    const unsigned long long hi64 = ((unsigned long long)dt << 32) | d1;
    const unsigned long long w = lz ? (hi64 << lz) | ((unsigned long long)d2 >> (32 - lz)) : hi64;
    bool sticky = lz ? ((d2 << lz) != 0u) : (d2 != 0u);
    for (int l = top - 3; l >= 0 && !sticky; --l) sticky = (uint32_t)acc[l * stride] != 0u;
    const int lead = unit + 32 * top + 31 - lz;           // exponent of the leading one
    const int eulp = max(lead - 52, -1074);
    if (eulp > 971) return neg ? -__longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0x7ff0000000000000ll);
    const int kb = lead - eulp + 1;                         // kept bits (<= 53)
    unsigned long long qv;
    bool rb;
    if (kb >= 1) {
        qv = w >> (64 - kb);
        rb = (w >> (63 - kb)) & 1ull;
        sticky = sticky || (kb < 63 && (w << (kb + 1)) != 0ull);
    } else if (kb == 0) {
        qv = 0;
        rb = true;                                          // the leading one is the round bit
        sticky = sticky || (w << 1) != 0ull;
    } else {
        qv = 0;
        rb = false;
        sticky = true;
    }
    if (rb && (sticky || (qv & 1ull))) qv += 1;
    const unsigned long long bits = ((unsigned long long)(eulp + 1074) << 52) + qv;
    const double r = __longlong_as_double((long long)bits);
    return neg ? -r : r;
}

// ---------------------------------------------------------------- fast path
// Two-prime Garner in 32-bit arithmetic: z'_0 = z0 symmetric, the digit
// d = ((z1 - z'_0) p0^-1) mod p1 symmetric, z' = z'_0 + d p0 (|z'| < p0 p1 / 2).
__device__ __forceinline__ long long garner2(uint32_t z0, uint32_t z1)
{
    const int32_t v0 = (int32_t)(z0 > (P0 - 1) / 2 ? z0 - P0 : z0);
    const uint32_t vm = v0 < 0 ? (uint32_t)(v0 + (int32_t)P1) : (uint32_t)v0;   // z'_0 mod p1
    const uint32_t d = shoup(mod_sub(z1, vm, P1), c_garner.inv01, c_garner.inv01q, P1);
    const int32_t ds = (int32_t)(d > (P1 - 1) / 2 ? d - P1 : d);
    return (long long)v0 + (long long)ds * (long long)P0;
}

// The same without centering z0, valid when every convolution value obeys
// |z| < p0 p1 / 2 - p0 (the host checks L n 4^alpha against that bound).  With
// u = z0 + e p0 in [0, p0 p1) (e = ((z1 - z0) p0^-1) mod p1): z >= 0 gives
// u = z, so e p0 <= z < p0 p1 / 2 - p0 and e < (p1 - 1) / 2; z < 0 gives
// u = z + p0 p1 > p0 p1 / 2 + p0, so e p0 > p0 p1 / 2 and e > (p1 - 1) / 2.
// Taking e symmetric therefore yields z0 + e p0 = z in both cases.
__device__ __forceinline__ long long garner2u(uint32_t z0, uint32_t z1)
{
    const uint32_t t = min(z0, z0 - P1);   // z0 mod p1 (z0 < p0 < 2 p1)
    const uint32_t e = shoup(mod_sub(z1, t, P1), c_garner.inv01, c_garner.inv01q, P1);
    const int32_t es = (int32_t)(e > (P1 - 1) / 2 ? e - P1 : e);
    return (long long)es * (long long)P0 + (long long)z0;
}

template <bool UC>
__device__ __forceinline__ long long garner2x(uint32_t z0, uint32_t z1)
{
    return UC ? garner2u(z0, z1) : garner2(z0, z1);
}

// acc[q..q+2] += digits of z * 2^b for a signed z with |z 2^b| < 2^95: two
// unsigned low digits and a signed top digit; q is uniform across the warp, so
// the switch selects fixed registers without divergence.
template <int NL>
__device__ __forceinline__ void acc_add3(long long (&acc)[NL], long long z, int sh)
{
    const int q = sh >> 5, b = sh & 31;
    const unsigned long long lo = (unsigned long long)z << b;
    const long long hi = b ? (z >> (64 - b)) : (z >> 63);   // bits 64.. of z 2^b, sign-extended
    const long long c0 = (long long)(uint32_t)lo, c1 = (long long)(uint32_t)(lo >> 32);
    const long long c2 = (long long)(int32_t)(uint32_t)hi;
#define OZ_ADD3(Q)                                   \
    case Q:                                          \
        if (Q + 2 < NL) {                            \
            acc[Q] += c0;                            \
            acc[Q + 1] += c1;                        \
            acc[Q + 2] += c2;                        \
        }                                            \
        break;
    switch (q) {
        OZ_ADD3(0) OZ_ADD3(1) OZ_ADD3(2) OZ_ADD3(3) OZ_ADD3(4) OZ_ADD3(5) OZ_ADD3(6) OZ_ADD3(7)
    default: break;
    }
#undef OZ_ADD3
}

// round sum acc[l] 2^(32 l) 2^unit to the nearest binary64, ties to even
template <int NL>
__device__ __forceinline__ double acc_to_double(long long (&acc)[NL], int unit)
{
    uint32_t d[NL];
    long long carry = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const long long v = acc[l] + carry;
        d[l] = (uint32_t)v;
        carry = v >> 32;
    }
    const bool neg = (d[NL - 1] >> 31) != 0;
    if (neg) {
        unsigned long long c = 1;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const unsigned long long t = (unsigned long long)(uint32_t)~d[l] + c;
            d[l] = (uint32_t)t;
            c = t >> 32;
        }
    }
    int top = -1;
    uint32_t dt = 0, d1 = 0, d2 = 0;
    bool low_nz = false;   // any digit below top-2
    // scan from the top digit down (unrolled, no dynamic register indexing)
#pragma unroll
    for (int l = NL - 1; l >= 0; --l) {
        if (top < 0) {
            if (d[l]) { top = l; dt = d[l]; }
        } else if (l == top - 1) {
            d1 = d[l];
        } else if (l == top - 2) {
            d2 = d[l];
        } else {
            low_nz = low_nz || d[l] != 0u;
        }
    }
    if (top < 0) return 0.0;
    const int lz = __clz(dt);
    const unsigned long long hi64 = ((unsigned long long)dt << 32) | d1;
    const unsigned long long w = lz ? (hi64 << lz) | ((unsigned long long)d2 >> (32 - lz)) : hi64;
    bool sticky = low_nz || (lz ? ((d2 << lz) != 0u) : (d2 != 0u));
    const int lead = unit + 32 * top + 31 - lz;
    const int eulp = max(lead - 52, -1074);
    if (eulp > 971) return neg ? -__longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0x7ff0000000000000ll);
    const int kb = lead - eulp + 1;
    unsigned long long qv;
    bool rb;
    if (kb >= 1) {
        qv = w >> (64 - kb);
        rb = (w >> (63 - kb)) & 1ull;
        sticky = sticky || (w << (kb + 1)) != 0ull;
    } else if (kb == 0) {
        qv = 0;
        rb = true;
        sticky = sticky || (w << 1) != 0ull;
    } else {
        qv = 0;
        rb = false;
        sticky = true;
    }
    if (rb && (sticky || (qv & 1ull))) qv += 1;
    const double r = __longlong_as_double((long long)(((unsigned long long)(eulp + 1074) << 52) + qv));
    return neg ? -r : r;
}

constexpr int REG_LIMBS = 10;   // register accumulator: spans up to 8 limbs of shift

constexpr int FAST_THREADS = 128;
constexpr int WIDE_LIMBS = 144;
constexpr int WIDE_THREADS = 32;
constexpr int CRT_CHUNK = 256;

// limbs needed for a signal's scale span
__device__ __forceinline__ int limbs_for(int smin, int smax) { return ((smax - smin) >> 5) + 5; }

__device__ __forceinline__ void load_res(const CrtArgs& a, const Sched* sc, int part, int i, int n0, int64_t b,
                                         int64_t j, uint32_t (&z)[3], int& S, bool& negate)
{
    const int c = i < n0 ? 2 * part : 2 * part + 1;
    const int g = i < n0 ? i : i - n0;
    const uint32_t* zp = a.Z + (((b * 4 + c) * a.G + g) * a.P) * a.N + j;
    z[0] = __ldg(zp);
    z[1] = __ldg(zp + a.N);
    z[2] = a.P > 2 ? __ldg(zp + 2 * a.N) : 0u;
    S = sc[c].S[g];
    negate = c == 1;   // II enters the real part with a minus sign
}

// signals whose exact sums fit the register accumulator (two primes, scale
// span of at most REG_LIMBS - 5 limbs) take the register path; the rest the
// shared-memory path
__device__ __forceinline__ bool reg_path(const CrtArgs& a, int64_t b)
{
    return a.P == 2 && limbs_for(a.span[b * 3], a.span[b * 3 + 1]) <= REG_LIMBS;
}

// signals for crt_fast_kernel: two primes, scales non-increasing in group order
// and spanning at most FAST_SPAN bits (every signal whose split levels have no
// gaps); crt_reg_body takes the other register-path signals
constexpr int FAST_SPAN = 120;
__device__ __forceinline__ bool fast_path(const CrtArgs& a, int64_t b)
{
    return a.P == 2 && (a.span[b * 3 + 2] & 2) && a.span[b * 3 + 1] - a.span[b * 3] <= FAST_SPAN;
}
// the same for three primes (|z'| < 2^92): crt_fast3_kernel
constexpr int FAST3_SPAN = 90;
__device__ __forceinline__ bool fast3_path(const CrtArgs& a, int64_t b)
{
    return a.P == 3 && (a.span[b * 3 + 2] & 2) && a.span[b * 3 + 1] - a.span[b * 3] <= FAST3_SPAN;
}

// a signal's length, chirp table and output row: the plan's (plain plans, the
// kernel parameters themselves) or the signal's descriptor (uneven lengths)
struct SigOut {
    int64_t n;
    const double2* w;
    double2* out;
};

template <bool SD>
__device__ __forceinline__ SigOut sig_out(const CrtArgs& a, int64_t b)
{
    if (SD) {
        double2* out = a.io ? a.io->out : a.out;
        const SigDesc d = a.sd[b];
        return {d.n, a.w + d.chirp_off, out + d.io_off};
    }
    return {a.n, a.w, a.out + b * a.n};
}

__device__ __forceinline__ void post_store(const CrtArgs& a, const SigOut& so, int64_t j, double yr, double yi)
{
    const double2 w = so.w[j];
    double re, im;
    cmul(yr, yi, w.x, w.y, re, im);
    if (a.direction > 0) im = -im;                      // inverse, adjoint: conj
    if (a.direction == 1 || a.direction == -2) {        // inverse, adjoint of the inverse: / n
        re = __ddiv_rn(re, (double)so.n);
        im = __ddiv_rn(im, (double)so.n);
    }
    so.out[j] = make_double2(re, im);
}

// register path: one output element per thread, integer-only accumulation
template <bool SD, bool UC>
__device__ __forceinline__ void crt_reg_body(const CrtArgs& a)
{
    const int64_t chunks = (a.n + CRT_CHUNK - 1) / CRT_CHUNK;
    const int64_t b = blockIdx.x / chunks;
    if (!reg_path(a, b) || fast_path(a, b)) return;
    const SigOut so = sig_out<SD>(a, b);
    const int64_t j0 = (blockIdx.x % chunks) * (int64_t)CRT_CHUNK;
    const int64_t j1 = min(so.n, j0 + CRT_CHUNK);
    const Sched* sc = a.sched + b * 4;
    const int smax = a.span[b * 3 + 1], any = a.span[b * 3 + 2] & 1;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        double yp[2] = {0.0, 0.0};
        if (any) {
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                long long acc[REG_LIMBS];
#pragma unroll
                for (int l = 0; l < REG_LIMBS; ++l) acc[l] = 0;
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int c = 2 * part + cc;
                    const Sched& S = sc[c];
                    const uint32_t* zp = a.Z + ((b * 4 + c) * a.G) * 2 * a.N + j;
                    const int ng = S.ngroups;
                    uint32_t z0 = 0, z1 = 0;
                    if (ng > 0) { z0 = __ldg(zp); z1 = __ldg(zp + a.N); }
                    for (int g = 0; g < ng; ++g) {
                        const uint32_t c0 = z0, c1 = z1;
                        if (g + 1 < ng) {   // prefetch the next group
                            z0 = __ldg(zp + (int64_t)(g + 1) * 2 * a.N);
                            z1 = __ldg(zp + (int64_t)(g + 1) * 2 * a.N + a.N);
                        }
                        long long z = garner2x<UC>(c0, c1);
                        if (c == 1 && !a.merged) z = -z;   // II enters the real part with a minus sign
                        acc_add3(acc, z, smax - S.S[g]);
                    }
                }
                yp[part] = acc_to_double(acc, -smax);
            }
        }
        post_store(a, so, j, yp[0], yp[1]);
    }
}

// ------------------------------------------------------------ Horner path
// A 192-bit two's complement integer in six 32-bit words (w[0] least
// significant), with carry-chain arithmetic in inline PTX.
struct Acc192 {
    uint32_t w[6];
};

__device__ __forceinline__ void acc192_add64(Acc192& A, long long z)   // A += z, z sign-extended
{
    const uint32_t lo = (uint32_t)z, hi = (uint32_t)((unsigned long long)z >> 32), ext = (uint32_t)(z >> 63);
    asm("add.cc.u32 %0, %0, %6;\n\t"
        "addc.cc.u32 %1, %1, %7;\n\t"
        "addc.cc.u32 %2, %2, %8;\n\t"
        "addc.cc.u32 %3, %3, %8;\n\t"
        "addc.cc.u32 %4, %4, %8;\n\t"
        "addc.u32 %5, %5, %8;"
        : "+r"(A.w[0]), "+r"(A.w[1]), "+r"(A.w[2]), "+r"(A.w[3]), "+r"(A.w[4]), "+r"(A.w[5])
        : "r"(lo), "r"(hi), "r"(ext));
}

__device__ __forceinline__ void acc192_sub64(Acc192& A, long long z)   // A -= z, z sign-extended
{
    const uint32_t lo = (uint32_t)z, hi = (uint32_t)((unsigned long long)z >> 32), ext = (uint32_t)(z >> 63);
    asm("sub.cc.u32 %0, %0, %6;\n\t"
        "subc.cc.u32 %1, %1, %7;\n\t"
        "subc.cc.u32 %2, %2, %8;\n\t"
        "subc.cc.u32 %3, %3, %8;\n\t"
        "subc.cc.u32 %4, %4, %8;\n\t"
        "subc.u32 %5, %5, %8;"
        : "+r"(A.w[0]), "+r"(A.w[1]), "+r"(A.w[2]), "+r"(A.w[3]), "+r"(A.w[4]), "+r"(A.w[5])
        : "r"(lo), "r"(hi), "r"(ext));
}

__device__ __forceinline__ void acc192_add(Acc192& A, const Acc192& B)   // A += B
{
    asm("add.cc.u32 %0, %0, %6;\n\t"
        "addc.cc.u32 %1, %1, %7;\n\t"
        "addc.cc.u32 %2, %2, %8;\n\t"
        "addc.cc.u32 %3, %3, %9;\n\t"
        "addc.cc.u32 %4, %4, %10;\n\t"
        "addc.u32 %5, %5, %11;"
        : "+r"(A.w[0]), "+r"(A.w[1]), "+r"(A.w[2]), "+r"(A.w[3]), "+r"(A.w[4]), "+r"(A.w[5])
        : "r"(B.w[0]), "r"(B.w[1]), "r"(B.w[2]), "r"(B.w[3]), "r"(B.w[4]), "r"(B.w[5]));
}

__device__ __forceinline__ void acc192_add128(Acc192& A, i128p z)   // A += z, z sign-extended
{
    const unsigned long long lo = z.lo, hi = (unsigned long long)z.hi;
    const uint32_t ext = (uint32_t)(z.hi >> 63);
    asm("add.cc.u32 %0, %0, %6;\n\t"
        "addc.cc.u32 %1, %1, %7;\n\t"
        "addc.cc.u32 %2, %2, %8;\n\t"
        "addc.cc.u32 %3, %3, %9;\n\t"
        "addc.cc.u32 %4, %4, %10;\n\t"
        "addc.u32 %5, %5, %10;"
        : "+r"(A.w[0]), "+r"(A.w[1]), "+r"(A.w[2]), "+r"(A.w[3]), "+r"(A.w[4]), "+r"(A.w[5])
        : "r"((uint32_t)lo), "r"((uint32_t)(lo >> 32)), "r"((uint32_t)hi), "r"((uint32_t)(hi >> 32)), "r"(ext));
}

// A <<= d for a shift d that is the same in every thread (0 <= d < 192)
__device__ __forceinline__ void acc192_shl(Acc192& A, int d)
{
    for (; d >= 32; d -= 32) {   // whole words
        A.w[5] = A.w[4]; A.w[4] = A.w[3]; A.w[3] = A.w[2]; A.w[2] = A.w[1]; A.w[1] = A.w[0]; A.w[0] = 0u;
    }
    if (d) {
#pragma unroll
        for (int i = 5; i >= 1; --i) A.w[i] = __funnelshift_l(A.w[i - 1], A.w[i], d);
        A.w[0] <<= d;
    }
}

// Round the 192-bit two's complement integer A (in units of 2^unit) to the
// nearest binary64, ties to even: magnitude, leading 64-bit word, a 64-bit
// window with the leading one at bit 63 and a sticky flag for the rest.  Not
// inlined: inside the Horner kernels' register budget it would spill.
__device__ __noinline__ double acc192_to_double(Acc192 A, int unit)
{
    const bool neg = (int32_t)A.w[5] < 0;
    if (neg) {
        const uint32_t zero = 0u;
        asm("sub.cc.u32 %0, %6, %0;\n\t"
            "subc.cc.u32 %1, %6, %1;\n\t"
            "subc.cc.u32 %2, %6, %2;\n\t"
            "subc.cc.u32 %3, %6, %3;\n\t"
            "subc.cc.u32 %4, %6, %4;\n\t"
            "subc.u32 %5, %6, %5;"
            : "+r"(A.w[0]), "+r"(A.w[1]), "+r"(A.w[2]), "+r"(A.w[3]), "+r"(A.w[4]), "+r"(A.w[5])
            : "r"(zero));
    }
    const unsigned long long h = ((unsigned long long)A.w[5] << 32) | A.w[4];
    const unsigned long long m = ((unsigned long long)A.w[3] << 32) | A.w[2];
    const unsigned long long l = ((unsigned long long)A.w[1] << 32) | A.w[0];
    unsigned long long hi, mid;
    bool low;
    int top;
    if (h) { top = 2; hi = h; mid = m; low = l != 0ull; }
    else if (m) { top = 1; hi = m; mid = l; low = false; }
    else if (l) { top = 0; hi = l; mid = 0ull; low = false; }
    else return 0.0;
    const int lz = __clzll((long long)hi);
    const unsigned long long w = lz ? (hi << lz) | (mid >> (64 - lz)) : hi;
    bool sticky = low || (mid << lz) != 0ull;
    const int lead = unit + 64 * top + 63 - lz;            // exponent of the leading one
    const int eulp = max(lead - 52, -1074);
    if (eulp > 971) return neg ? -__longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0x7ff0000000000000ll);
    const int kb = lead - eulp + 1;                         // kept bits (<= 53)
    unsigned long long qv;
    bool rb;
    if (kb >= 1) {
        qv = w >> (64 - kb);
        rb = (w >> (63 - kb)) & 1ull;
        sticky = sticky || (w << (kb + 1)) != 0ull;
    } else if (kb == 0) {
        qv = 0;
        rb = true;                                          // the leading one is the round bit
        sticky = sticky || (w << 1) != 0ull;
    } else {
        qv = 0;
        rb = false;
        sticky = true;
    }
    if (rb && (sticky || (qv & 1ull))) qv += 1;
    const double r = __longlong_as_double((long long)(((unsigned long long)(eulp + 1074) << 52) + qv));
    return neg ? -r : r;
}

// Exact accumulation by Horner's rule: a convolution's groups run from the
// last (smallest scale S, largest terms) to the first, so every change of
// scale multiplies the running sum by 2^(S_new - S_old) >= 1, a left shift;
// terms are then added as plain integers.  The running sum of a convolution
// ends in units of 2^-S of its first group and is shifted to the signal's
// 2^-max S; at most 2^62 * 64 * 2^FAST_SPAN in magnitude, inside 192 bits.
template <bool SD, bool UC>
__global__ void __launch_bounds__(FAST_THREADS, 10) crt_fast_kernel(CrtArgs a)
{
    const int64_t chunks = (a.n + CRT_CHUNK - 1) / CRT_CHUNK;
    const int64_t b = blockIdx.x / chunks;
    if (!fast_path(a, b)) {   // the signal's CTAs take the limb path instead (one launch for both)
        crt_reg_body<SD, UC>(a);
        return;
    }
    if (a.fused) return;      // done by the fused column pass (colcrt_kernel)
    const SigOut so = sig_out<SD>(a, b);
    const int64_t j0 = (blockIdx.x % chunks) * (int64_t)CRT_CHUNK;
    const int64_t j1 = min(so.n, j0 + CRT_CHUNK);
    const Sched* sc = a.sched + b * 4;
    const int smax = a.span[b * 3 + 1], any = a.span[b * 3 + 2] & 1;
    __shared__ int s_S[4][MAX_GROUPS], s_ng[4];   // the signal's group scales, read once per CTA
    for (int i = threadIdx.x; i < 4 * MAX_GROUPS; i += blockDim.x)
        s_S[i / MAX_GROUPS][i % MAX_GROUPS] = sc[i / MAX_GROUPS].S[i % MAX_GROUPS];
    if (threadIdx.x < 4) s_ng[threadIdx.x] = sc[threadIdx.x].ngroups;
    __syncthreads();
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        double yp[2] = {0.0, 0.0};
        if (any) {
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                Acc192 A = {{0u, 0u, 0u, 0u, 0u, 0u}};
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int c = 2 * part + cc;
                    const int ng = s_ng[c];
                    const int* SS = s_S[c];
                    if (ng == 0) continue;
                    const uint32_t* zp = a.Z + ((b * 4 + c) * a.G) * 2 * a.N + j;
                    Acc192 T = {{0u, 0u, 0u, 0u, 0u, 0u}};
                    int scur = SS[ng - 1];
                    constexpr int PF = 9;
                    if (ng <= PF) {   // every group's residues in flight at once
                        uint32_t r0[PF], r1[PF];
#pragma unroll
                        for (int q = 0; q < PF; ++q)
                            if (q < ng) {
                                r0[q] = __ldg(zp + (int64_t)q * 2 * a.N);
                                r1[q] = __ldg(zp + (int64_t)q * 2 * a.N + a.N);
                            }
#pragma unroll
                        for (int q = PF - 1; q >= 0; --q)
                            if (q < ng) {
                                const int sg = SS[q];
                                if (sg != scur) {
                                    acc192_shl(T, sg - scur);
                                    scur = sg;
                                }
                                long long z = garner2x<UC>(r0[q], r1[q]);
                                if (c == 1 && !a.merged) z = -z;
                                acc192_add64(T, z);
                            }
                        acc192_shl(T, smax - scur);
                        acc192_add(A, T);
                        continue;
                    }
                    uint32_t z0 = __ldg(zp + (int64_t)(ng - 1) * 2 * a.N);
                    uint32_t z1 = __ldg(zp + (int64_t)(ng - 1) * 2 * a.N + a.N);
                    for (int g = ng - 1; g >= 0; --g) {
                        const uint32_t c0 = z0, c1 = z1;
                        if (g > 0) {   // prefetch the previous group
                            z0 = __ldg(zp + (int64_t)(g - 1) * 2 * a.N);
                            z1 = __ldg(zp + (int64_t)(g - 1) * 2 * a.N + a.N);
                        }
                        const int sg = SS[g];
                        if (sg != scur) {
                            acc192_shl(T, sg - scur);
                            scur = sg;
                        }
                        long long z = garner2x<UC>(c0, c1);
                        if (c == 1 && !a.merged) z = -z;   // II enters the real part with a minus sign
                        acc192_add64(T, z);
                    }
                    acc192_shl(T, smax - scur);
                    acc192_add(A, T);
                }
                yp[part] = acc192_to_double(A, -smax);
            }
        }
        post_store(a, so, j, yp[0], yp[1]);
    }
}

// Horner's rule for three primes: the same scheme with the 128-bit CRT
// integers of the three-digit Garner form (|z'| < 2^92, so spans of at most
// FAST3_SPAN bits stay inside 192 bits).
template <bool SD>
__global__ void __launch_bounds__(FAST_THREADS) crt_fast3_kernel(CrtArgs a)
{
    const int64_t chunks = (a.n + CRT_CHUNK - 1) / CRT_CHUNK;
    const int64_t b = blockIdx.x / chunks;
    if (!fast3_path(a, b)) return;
    const SigOut so = sig_out<SD>(a, b);
    const int64_t j0 = (blockIdx.x % chunks) * (int64_t)CRT_CHUNK;
    const int64_t j1 = min(so.n, j0 + CRT_CHUNK);
    const Sched* sc = a.sched + b * 4;
    const int smax = a.span[b * 3 + 1], any = a.span[b * 3 + 2] & 1;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        double yp[2] = {0.0, 0.0};
        if (any) {
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                Acc192 A = {{0u, 0u, 0u, 0u, 0u, 0u}};
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int c = 2 * part + cc;
                    const Sched& S = sc[c];
                    const int ng = S.ngroups;
                    if (ng == 0) continue;
                    const uint32_t* zp = a.Z + ((b * 4 + c) * a.G) * 3 * a.N + j;
                    Acc192 T = {{0u, 0u, 0u, 0u, 0u, 0u}};
                    int scur = S.S[ng - 1];
                    uint32_t z[3] = {__ldg(zp + (int64_t)(ng - 1) * 3 * a.N), __ldg(zp + (int64_t)(ng - 1) * 3 * a.N + a.N),
                                     __ldg(zp + (int64_t)(ng - 1) * 3 * a.N + 2 * a.N)};
                    for (int g = ng - 1; g >= 0; --g) {
                        const uint32_t cz[3] = {z[0], z[1], z[2]};
                        if (g > 0) {   // prefetch the previous group
                            const uint32_t* q = zp + (int64_t)(g - 1) * 3 * a.N;
                            z[0] = __ldg(q);
                            z[1] = __ldg(q + a.N);
                            z[2] = __ldg(q + 2 * a.N);
                        }
                        const int sg = S.S[g];
                        if (sg != scur) {
                            acc192_shl(T, sg - scur);
                            scur = sg;
                        }
                        i128p v = garner(cz, 3);
                        if (c == 1 && !a.merged) {   // II enters the real part with a minus sign
                            v.lo = ~v.lo + 1ull;
                            v.hi = (long long)(~(unsigned long long)v.hi + (v.lo == 0 ? 1ull : 0ull));
                        }
                        acc192_add128(T, v);
                    }
                    acc192_shl(T, smax - scur);
                    acc192_add(A, T);
                }
                yp[part] = acc192_to_double(A, -smax);
            }
        }
        post_store(a, so, j, yp[0], yp[1]);
    }
}

// shared-memory path: any prime count and scale span, one limb column per thread
template <bool SD>
__global__ void __launch_bounds__(WIDE_THREADS) crt_wide_kernel(CrtArgs a)
{
    extern __shared__ long long acc_dyn[];
    const int chunks = (int)((a.n + CRT_CHUNK - 1) / CRT_CHUNK);
    const int64_t work = a.B * chunks;
    for (int64_t item = blockIdx.x; item < work; item += gridDim.x) {
        const int64_t b = item / chunks;
        if (reg_path(a, b) || fast3_path(a, b)) {   // skip the signal
            item += ((chunks - 1 - item % chunks) / gridDim.x) * gridDim.x;
            continue;
        }
        const SigOut so = sig_out<SD>(a, b);
        const int64_t j0 = (item % chunks) * (int64_t)CRT_CHUNK;
        const int64_t j1 = min(so.n, j0 + CRT_CHUNK);
        const Sched* sc = a.sched + b * 4;
        const int smin = a.span[b * 3 + 0], smax = a.span[b * 3 + 1], any = a.span[b * 3 + 2] & 1;
        const int nl = limbs_for(smin, smax);
        if (nl > WIDE_LIMBS) {   // cannot happen for finite inputs that passed the split's range check
            if (threadIdx.x == 0) atomicOr(a.status, ST_RANGE);
            continue;
        }
        long long* col = acc_dyn + threadIdx.x;
        const int stride = blockDim.x;
        for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            double yp[2] = {0.0, 0.0};
            if (any) {
                for (int part = 0; part < 2; ++part) {
                    for (int l = 0; l < nl; ++l) col[l * stride] = 0;
                    for (int c = 2 * part; c < 2 * part + 2; ++c) {
                        const Sched& S = sc[c];
                        for (int g = 0; g < S.ngroups; ++g) {
                            const uint32_t* zp = a.Z + (((b * 4 + c) * a.G + g) * a.P) * a.N + j;
                            uint32_t z[3];
                            z[0] = zp[0];
                            z[1] = zp[a.N];
                            z[2] = a.P > 2 ? zp[2 * a.N] : 0u;
                            i128p v = garner(z, a.P);
                            if (c == 1 && !a.merged) {   // II enters the real part with a minus sign
                                v.lo = ~v.lo + 1ull;
                                v.hi = (long long)(~(unsigned long long)v.hi + (v.lo == 0 ? 1ull : 0ull));
                            }
                            add_term(col, stride, v, smax - S.S[g]);
                        }
                    }
                    yp[part] = limbs_to_double(col, stride, nl, -smax);
                }
            }
            post_store(a, so, j, yp[0], yp[1]);
        }
    }
}

// Per-device state: the __constant__ Garner constants and the wide kernel's
// shared-memory attribute belong to each device's copy of the module, so each
// device is set up once, under a mutex (plans may be created from several
// threads and on several devices).
constexpr int CRT_MAX_DEVICES = 64;
static bool s_garner_ready[CRT_MAX_DEVICES] = {};
static bool s_wide_attr[CRT_MAX_DEVICES] = {};
static std::mutex s_crt_mutex;

static uint64_t host_powmod(uint64_t b, uint64_t e, uint64_t m)
{
    unsigned __int128 r = 1 % m, x = b % m;
    while (e) {
        if (e & 1) r = r * x % m;
        x = x * x % m;
        e >>= 1;
    }
    return (uint64_t)r;
}

int crt_launches() { return 2; }

cudaError_t crt_init()
{
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return de;
    if (dev < 0 || dev >= CRT_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(s_crt_mutex);
    if (!s_garner_ready[dev]) {
        GarnerConst gc;
        gc.inv01 = (uint32_t)host_powmod(P0 % P1, P1 - 2, P1);
        gc.inv01q = (uint32_t)(((uint64_t)gc.inv01 << 32) / P1);
        const uint64_t p01m2 = (uint64_t)((unsigned __int128)P0 * P1 % P2);
        gc.inv2 = (uint32_t)host_powmod(p01m2, P2 - 2, P2);
        gc.inv2q = (uint32_t)(((uint64_t)gc.inv2 << 32) / P2);
        gc.p0_mod2 = P0 % P2;
        cudaError_t e = cudaMemcpyToSymbol(c_garner, &gc, sizeof(gc));
        if (e != cudaSuccess) return e;
        s_garner_ready[dev] = true;
    }
    if (!s_wide_attr[dev]) {
        // crt_wide_kernel's limb columns exceed the default 48 KiB of dynamic shared memory
        const int smem = (int)(sizeof(long long) * WIDE_LIMBS * WIDE_THREADS);
        cudaError_t e = cudaFuncSetAttribute(crt_wide_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(crt_wide_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        s_wide_attr[dev] = true;
    }
    return cudaSuccess;
}

// ------------------------------------- inverse column pass fused with the CRT
// For the signals of crt_fast_kernel (two primes, monotone group scales, span
// <= FAST_SPAN) the inverse NTT's column stages and the exact accumulation run
// in one kernel, so the inverse-NTT residues never return to HBM.  A CTA owns
// T adjacent columns x all 2^m1 rows (1024 positions j = row 2^m2 + col) of
// one signal and walks the flush groups of both output parts, two per step:
// it copies their four column tiles (two groups x two primes) into shared
// memory with cp.async (the next step's copies in flight during this step's
// arithmetic), runs the column rounds of the Gentleman-Sande inverse on all
// four between the same barriers, and every thread adds the Garner integers
// of its four positions to a 192-bit Horner sum.  With up to six column
// stages the last two run in registers: each thread transforms the four
// positions it accumulates (one column group, both primes) and feeds them to
// Garner directly, one shared-memory pass and one barrier fewer per step.  The groups of a part's two convolutions (RR and II, or
// IR and RI) are taken in one merged order of increasing scale, so one
// accumulator per position serves the whole part (II with a minus sign); the
// real part is rounded before the imaginary part starts.  Signals off that
// path get the column pass only, stored back for the other CRT kernels.  In
// a merged schedule a part's groups fill the slots of its two convolutions,
// each slot in scale order, with II's sign already applied by the MAC.
//
// Shared-memory tiles are [row][T] with T pad words after every 16 rows
// (T < 32): the column rounds then touch 32 distinct banks per warp.
constexpr int FC_THREADS = 256;
constexpr int FC_TILE = 1024;                         // positions per tile (per prime)
constexpr int FC_E = FC_TILE / FC_THREADS;            // positions per thread
constexpr int FC_STAGES = 2;

template <int LOG_T>
__host__ __device__ constexpr int fc_words() { return FC_TILE + (LOG_T < 5 ? (FC_TILE >> (LOG_T + 4)) << LOG_T : 0); }
template <int LOG_T>
__device__ __forceinline__ int fc_pad(int i) { return LOG_T < 5 ? i + ((i >> (LOG_T + 4)) << LOG_T) : i; }

// one column round over NT tiles (PW words apart; even tiles prime 0, odd
// tiles prime 1): 2^RL-point groups of stride H rows; element u of a group
// sits at the group's base plus the compile-time offset u H T + T floor(u H /
// 16) (a group never straddles a 16-row bucket except at multiples of H)
// STG: 0 the table from global memory, 1 the REG01 round's staged layout (stw),
// 2 tw0 / tw1 are copies of the table's first 2^ML entries in shared memory
template <int ML, int S0, int RL, int LOG_T, int NT, int STG = 0>
__device__ __forceinline__ void fc_round(uint32_t* st, const uint2* __restrict__ tw0, const uint2* __restrict__ tw1,
                                         const uint2* stw = nullptr)
{
    constexpr int LOG_H = ML - S0 - RL, H = 1 << LOG_H, LOG_GPC = ML - RL, T = 1 << LOG_T, R = 1 << RL;
    constexpr int GPT = T << LOG_GPC, PW = fc_words<LOG_T>();
    for (int gid = threadIdx.x; gid < NT * GPT; gid += FC_THREADS) {
        const int tile = gid / GPT, pr = tile & 1;
        const int gg = gid - tile * GPT;
        const int c = gg & (T - 1), grp = gg >> LOG_T;
        const int blk = grp >> LOG_H;
        const int l0 = (blk << (ML - S0)) + (grp & (H - 1));
        uint32_t* base = st + tile * PW + (l0 << LOG_T) + c + (LOG_T < 5 ? ((l0 >> 4) << LOG_T) : 0);
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = base[u * H * T + (LOG_T < 5 ? ((u * H) >> 4) << LOG_T : 0)];
        if constexpr (STG == 1)   // staged: [prime][block][2^RL - 1] in radix_group's order
            radix_group_inv_staged<RL>(v, stw + (pr << S0) * (R - 1) + blk * (R - 1), pr ? P1 : P0);
        else if constexpr (STG == 2)
            radix_group_tab<true, RL>(v, pr ? tw1 : tw0, (1 << S0) + blk, pr ? P1 : P0);
        else
            radix_group<true, RL>(v, pr ? tw1 : tw0, (1 << S0) + blk, pr ? P1 : P0);
#pragma unroll
        for (int u = 0; u < R; ++u) base[u * H * T + (LOG_T < 5 ? ((u * H) >> 4) << LOG_T : 0)] = v[u];
    }
}

template <int ML, int LOG_T, int NT, int I>
__device__ __forceinline__ void fc_rounds(uint32_t* st, const uint2* tw0, const uint2* tw1)
{
    if constexpr (I < Part<ML>::NR) {
        constexpr int R_ = Part<ML>::NR - 1 - I;   // the inverse takes the rounds last to first
        fc_round<ML, Part<ML>::start(R_), Part<ML>::size(R_), LOG_T, NT, 2>(st, tw0, tw1);
        __syncthreads();
        fc_rounds<ML, LOG_T, NT, I + 1>(st, tw0, tw1);
    }
}

// the column rounds for stages 2 .. ML-1 in one round (ML <= 6); stages 0 and
// 1 then run in registers in colcrt_kernel
template <int ML, int LOG_T, int NT>
__device__ __forceinline__ void fc_rounds_hi(uint32_t* st, const uint2* tw0, const uint2* tw1, const uint2* stw)
{
    static_assert(ML - 2 >= 1 && ML - 2 <= 4, "one shared-memory round");
    fc_round<ML, 2, ML - 2, LOG_T, NT, 1>(st, tw0, tw1, stw);
    __syncthreads();
}

// the twiddles of that round (4 blocks of stage 2's table rows, 2^(ML-2) - 1
// entries each, both primes) copied once per CTA: every flush group of the CTA
// uses the same ones
template <int ML>
struct FcTw {
    static constexpr int PER = (1 << (ML - 2)) - 1, TOTAL = 2 * 4 * PER;
};
template <int ML>
__device__ __forceinline__ void fc_stage_tw(uint2* stw, const uint2* __restrict__ tw0, const uint2* __restrict__ tw1)
{
    constexpr int PER = FcTw<ML>::PER;
    for (int e = threadIdx.x; e < FcTw<ML>::TOTAL; e += FC_THREADS) {
        const int pr = e / (4 * PER), rest = e - pr * 4 * PER;
        const int blk = rest / PER, k = rest - blk * PER + 1;     // radix_group's index (1 << j) + q
        const int j = 31 - __clz(k);
        stw[e] = __ldg((pr ? tw1 : tw0) + ((4 + blk) << j) + (k - (1 << j)));
    }
}

template <bool B>
struct FcBool {
    static constexpr bool value = B;
};

struct FcTerm {
    int64_t off;     // Z offset of the group's prime-0 vector
    int16_t sh;      // left shift of the running sum before the term
    int16_t neg;     // II: subtract
};

// TB flush groups per step (their 2 TB tiles transformed between the same
// barriers)
template <bool SD, int M1, int TB, bool UC>
__global__ void __launch_bounds__(FC_THREADS, 4) colcrt_kernel(CrtArgs a, int m2, const uint2* __restrict__ tw_all)
{
    constexpr int LOG_T = 10 - M1, T = 1 << LOG_T;
    constexpr int PW = fc_words<LOG_T>(), SW = 2 * TB * PW;
    static_assert((1 << M1) * T == FC_TILE && T >= 4, "column tile");
    extern __shared__ __align__(16) uint32_t fc_sm[];
    __shared__ FcTerm terms[4 * MAX_GROUPS];
    __shared__ int s_pstart[3], s_fsh[2];
    const int tiles = (1 << m2) >> LOG_T;
    const int64_t b = blockIdx.x / tiles;
    const int c0 = (int)(blockIdx.x % tiles) << LOG_T;
    const bool fast = fast_path(a, b);
    const Sched* sc = a.sched + b * 4;
    const int smax = a.span[b * 3 + 1];
    if (threadIdx.x == 0) {   // both parts' groups, each part merged in increasing scale
        int n = 0;
        for (int part = 0; part < 2; ++part) {
            s_pstart[part] = n;
            const Sched& A = sc[2 * part];
            const Sched& B = sc[2 * part + 1];
            int ia = A.ngroups - 1, ib = B.ngroups - 1, scur = 0;
            bool first = true;
            while (ia >= 0 || ib >= 0) {
                const bool takeA = ib < 0 || (ia >= 0 && A.S[ia] <= B.S[ib]);
                const int c = takeA ? 2 * part : 2 * part + 1, g = takeA ? ia-- : ib--;
                const int S = takeA ? A.S[g] : B.S[g];
                FcTerm t;
                t.off = ((b * 4 + c) * a.G + g) * 2 * a.N;
                t.sh = (int16_t)(first ? 0 : S - scur);
                t.neg = (int16_t)(c == 1 && !a.merged);
                terms[n++] = t;
                scur = S;
                first = false;
            }
            s_fsh[part] = first ? 0 : smax - scur;
        }
        s_pstart[2] = n;
    }
    __syncthreads();
    const int nterms = s_pstart[2], nsteps = (nterms + TB - 1) / TB;
    // up to 6 column stages: stages 2.. in shared memory, then each thread runs
    // stages 1 and 0 of one column group (four positions, rows fl0 + u HB of
    // column fcl) for both primes in registers and accumulates those positions;
    // otherwise all rounds in shared memory, positions threadIdx.x + e FC_THREADS
    constexpr bool REG01 = M1 <= 6;
    constexpr int HB = 1 << (M1 - 2);                     // stride of stages 0 and 1 in rows
    static_assert(!REG01 || (T * HB == FC_THREADS && FC_E == 4), "one column group of four positions per thread");
    const int fcl = threadIdx.x & (T - 1), fl0 = threadIdx.x >> LOG_T;
    const uint2* tw0 = tw_all;
    const uint2* tw1 = tw_all + a.N;
    // chunk q of a tile pair: prime q / 256, row and 16-byte column group
    auto issue = [&](int i) {
#pragma unroll
        for (int tb = 0; tb < TB; ++tb) {
            const int ti = i * TB + tb;
            if (ti < nterms) {
                uint32_t* st = fc_sm + (i % FC_STAGES) * SW + tb * 2 * PW;
                const uint32_t* zb = a.Z + terms[ti].off + c0;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int q = threadIdx.x + k * FC_THREADS;
                    const int pr = q >> 8, w = q & 255;
                    const int row = w >> (LOG_T - 2), cw = (w & ((T >> 2) - 1)) << 2;
                    const uint32_t* src = zb + pr * a.N + ((int64_t)row << m2) + cw;
                    const uint32_t dst =
                        (uint32_t)__cvta_generic_to_shared(st + pr * PW + fc_pad<LOG_T>((row << LOG_T) + cw));
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    static_assert(FC_STAGES == 2, "the copies of step i + 1 go to the buffer step i - 1 used");
    issue(0);
    // the twiddles of the shared-memory rounds, copied once per CTA (every flush
    // group uses the same ones): the REG01 round's entries, or the first 2^M1
    // entries of both primes' tables (the column transform's whole table)
    __shared__ __align__(16) uint2 fc_tw[REG01 ? FcTw<(M1 < 3 ? 3 : M1)>::TOTAL : 2 << M1];
    if constexpr (REG01) {
        fc_stage_tw<M1>(fc_tw, tw0, tw1);   // visible after the first step's barrier
    } else {
        for (int e = threadIdx.x; e < (2 << M1); e += FC_THREADS)
            fc_tw[e] = __ldg((e >> M1 ? tw1 : tw0) + (e & ((1 << M1) - 1)));
    }
    // stages 1 and 0 (the register round): table entries 1 and 2 are 1 (block 0
    // of stages 0 and 1), entry 3 is w^(N/4), the same for every step
    const uint2 w3_0 = __ldg(tw0 + 3), w3_1 = __ldg(tw1 + 3);
    Acc192 acc[FC_E];
    __shared__ double s_yr[FC_E][FC_THREADS];           // the real parts, kept out of the registers
#pragma unroll
    for (int e = 0; e < FC_E; ++e) {
        acc[e] = Acc192{{0u, 0u, 0u, 0u, 0u, 0u}};
        s_yr[e][threadIdx.x] = 0.0;
    }
    // the step loop, instantiated for signals on the Horner path and for the others
    // (column pass only), so that neither carries the other's code and registers
    auto run_steps = [&](auto fast_c) {
    constexpr bool FAST = decltype(fast_c)::value;
    for (int i = 0; i < nsteps; ++i) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();                                  // step i's tiles are in shared memory, and every
                                                          // thread is done with step i - 1's buffer
        issue(i + 1);                                     // into that buffer, during this step's arithmetic
        uint32_t* st = fc_sm + (i % FC_STAGES) * SW;
        if constexpr (REG01) fc_rounds_hi<M1, LOG_T, 2 * TB>(st, tw0, tw1, fc_tw);   // ends with a barrier
        else fc_rounds<M1, LOG_T, 2 * TB, 0>(st, fc_tw, fc_tw + (1 << M1));
#pragma unroll
        for (int tb = 0; tb < TB; ++tb) {
            const int ti = i * TB + tb;
            if (ti >= nterms) break;
            const FcTerm t = terms[ti];
            const uint32_t* sp = st + tb * 2 * PW;
            uint32_t v0[FC_E], v1[FC_E];                  // the thread's positions, prime 0 and prime 1
            if constexpr (REG01) {
                const uint32_t* gp = sp + (fl0 << LOG_T) + fcl + (LOG_T < 5 ? ((fl0 >> 4) << LOG_T) : 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int o = u * HB * T + (LOG_T < 5 ? ((u * HB) >> 4) << LOG_T : 0);
                    v0[u] = gp[o];
                    v1[u] = gp[PW + o];
                }
                // stage 1: (0, 1) with entry 2 = 1, (2, 3) with entry 3; stage 0: (0, 2) and
                // (1, 3) with entry 1 = 1 (a unit twiddle: the difference reduced mod p)
                bfly_gs_unit(v0[0], v0[1], P0); bfly_gs(v0[2], v0[3], w3_0, P0);
                bfly_gs_unit(v1[0], v1[1], P1); bfly_gs(v1[2], v1[3], w3_1, P1);
                bfly_gs_unit(v0[0], v0[2], P0); bfly_gs_unit(v0[1], v0[3], P0);
                bfly_gs_unit(v1[0], v1[2], P1); bfly_gs_unit(v1[1], v1[3], P1);
            } else {
#pragma unroll
                for (int e = 0; e < FC_E; ++e) {
                    const int p = fc_pad<LOG_T>(threadIdx.x + e * FC_THREADS);
                    v0[e] = sp[p];
                    v1[e] = sp[PW + p];
                }
            }
            if constexpr (FAST) {
                if (t.sh) {                               // the same shift for every position
#pragma unroll
                    for (int e = 0; e < FC_E; ++e) acc192_shl(acc[e], t.sh);
                }
                if (t.neg) {                              // II: subtracted (uniform branch)
#pragma unroll
                    for (int e = 0; e < FC_E; ++e) acc192_sub64(acc[e], garner2x<UC>(v0[e], v1[e]));
                } else {
#pragma unroll
                    for (int e = 0; e < FC_E; ++e) acc192_add64(acc[e], garner2x<UC>(v0[e], v1[e]));
                }
                if (ti + 1 == s_pstart[1]) {              // the real part is complete
#pragma unroll
                    for (int e = 0; e < FC_E; ++e) {
                        acc192_shl(acc[e], s_fsh[0]);
                        s_yr[e][threadIdx.x] = acc192_to_double(acc[e], -smax);
                        acc[e] = Acc192{{0u, 0u, 0u, 0u, 0u, 0u}};
                    }
                }
            } else {                                      // column pass only: back to Z for the other kernels
                uint32_t* zb = const_cast<uint32_t*>(a.Z) + t.off + c0;   // the plan's Z buffer
#pragma unroll
                for (int e = 0; e < FC_E; ++e) {
                    const int64_t o = REG01 ? ((int64_t)(fl0 + e * HB) << m2) + fcl
                                            : ((int64_t)((threadIdx.x + e * FC_THREADS) >> LOG_T) << m2) +
                                                  ((threadIdx.x + e * FC_THREADS) & (T - 1));
                    zb[o] = v0[e];
                    zb[a.N + o] = v1[e];
                }
            }
        }
    }
    };
    if (fast) run_steps(FcBool<true>{});
    else run_steps(FcBool<false>{});
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!fast) return;
    double yi[FC_E];
#pragma unroll
    for (int e = 0; e < FC_E; ++e) {
        if (nterms > s_pstart[1]) {
            acc192_shl(acc[e], s_fsh[1]);
            yi[e] = acc192_to_double(acc[e], -smax);
        } else {
            yi[e] = 0.0;
        }
    }
    const SigOut so = sig_out<SD>(a, b);
#pragma unroll
    for (int e = 0; e < FC_E; ++e) {
        const int idx = threadIdx.x + e * FC_THREADS;
        const int64_t j = REG01 ? ((int64_t)(fl0 + e * HB) << m2) + c0 + fcl
                                : ((int64_t)(idx >> LOG_T) << m2) + c0 + (idx & (T - 1));
        if (j < so.n) post_store(a, so, j, s_yr[e][threadIdx.x], yi[e]);
    }
}

constexpr int FC_TB = 2;

template <bool SD, int M1>
static cudaError_t launch_colcrt_m(const CrtArgs& a, int m2, const uint2* tw, cudaStream_t s)
{
    constexpr int LOG_T = 10 - M1;
    const size_t smem = (size_t)FC_STAGES * 2 * FC_TB * fc_words<LOG_T>() * sizeof(uint32_t);
    const int64_t grid = a.B * ((int64_t(1) << m2) >> LOG_T);
    // Garner without centering z0 (garner_u: every signal's values within the bound) or with it
    auto kern = a.garner_u ? colcrt_kernel<SD, M1, FC_TB, true> : colcrt_kernel<SD, M1, FC_TB, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, FC_THREADS, smem, s>>>(a, m2, tw);
    return cudaGetLastError();
}

bool colcrt_supported(int P, int m1, int m2, bool)
{
    return P == 2 && m1 >= 4 && m1 <= 8 && m2 >= 10 - m1;
}

cudaError_t launch_colcrt(const CrtArgs& a, int m1, int m2, const uint2* tw, cudaStream_t s)
{
    cudaError_t e = crt_init();
    if (e != cudaSuccess) return e;
    if (a.sd) {   // a length class of a plan over uneven lengths: per-signal lengths and outputs
        switch (m1) {
        case 4: return launch_colcrt_m<true, 4>(a, m2, tw, s);
        case 5: return launch_colcrt_m<true, 5>(a, m2, tw, s);
        case 6: return launch_colcrt_m<true, 6>(a, m2, tw, s);
        case 7: return launch_colcrt_m<true, 7>(a, m2, tw, s);
        case 8: return launch_colcrt_m<true, 8>(a, m2, tw, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (m1) {
    case 4: return launch_colcrt_m<false, 4>(a, m2, tw, s);
    case 5: return launch_colcrt_m<false, 5>(a, m2, tw, s);
    case 6: return launch_colcrt_m<false, 6>(a, m2, tw, s);
    case 7: return launch_colcrt_m<false, 7>(a, m2, tw, s);
    case 8: return launch_colcrt_m<false, 8>(a, m2, tw, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_crt_post(const CrtArgs& a, cudaStream_t s)
{
    cudaError_t e = crt_init();
    if (e != cudaSuccess) return e;
    const int64_t chunks = (a.n + CRT_CHUNK - 1) / CRT_CHUNK;
    const bool sd = a.sd != nullptr;
    if (a.P == 3) {
        if (sd) crt_fast3_kernel<true><<<(unsigned)(a.B * chunks), FAST_THREADS, 0, s>>>(a);
        else crt_fast3_kernel<false><<<(unsigned)(a.B * chunks), FAST_THREADS, 0, s>>>(a);
    } else {
        const unsigned grid = (unsigned)(a.B * chunks);
        if (a.garner_u) {
            if (sd) crt_fast_kernel<true, true><<<grid, FAST_THREADS, 0, s>>>(a);
            else crt_fast_kernel<false, true><<<grid, FAST_THREADS, 0, s>>>(a);
        } else {
            if (sd) crt_fast_kernel<true, false><<<grid, FAST_THREADS, 0, s>>>(a);
            else crt_fast_kernel<false, false><<<grid, FAST_THREADS, 0, s>>>(a);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // signals with three primes or a wide scale span: small blocks, limb columns in shared memory
    const size_t smem = sizeof(long long) * WIDE_LIMBS * WIDE_THREADS;
    const int64_t grid = a.B * chunks < 304 ? a.B * chunks : 304;
    if (sd) crt_wide_kernel<true><<<(unsigned)grid, WIDE_THREADS, smem, s>>>(a);
    else crt_wide_kernel<false><<<(unsigned)grid, WIDE_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// TS variant (Alg. 8 per real convolution, TS accumulation): for each output
// element, each convolution's groups in schedule order add z'/c = z' 2^-S to
// a TS accumulator with TSAdd; Re y' = TSSub(RR, II), Im y' = TSAdd(IR, RI);
// y = y' (.) w in TS (Alg. 4 step 4), then binary64 (the exact sum of the three
// words rounded once); the inverse and adjoint directions as in post_store.
__global__ void __launch_bounds__(FAST_THREADS) crt_ts_kernel(CrtArgs a)
{
    const int64_t chunks = (a.n + CRT_CHUNK - 1) / CRT_CHUNK;
    const int64_t b = blockIdx.x / chunks;
    const int64_t j0 = (blockIdx.x % chunks) * (int64_t)CRT_CHUNK;
    const int64_t j1 = min(a.n, j0 + CRT_CHUNK);
    const Sched* sc = a.sched + b * 4;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        ts3 acc[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[c] = ts3{0.0f, 0.0f, 0.0f};
            const Sched& S = sc[c];
            const uint32_t* zp = a.Z + ((b * 4 + c) * a.G) * 2 * a.N + j;
            for (int g = 0; g < S.ngroups; ++g) {
                const uint32_t z0 = __ldg(zp + (int64_t)g * 2 * a.N), z1 = __ldg(zp + (int64_t)g * 2 * a.N + a.N);
                acc[c] = ts_add(acc[c], ts_from_int_scaled(garner2(z0, z1), S.S[g]));
            }
        }
        const ts3 yr = ts_sub(acc[0], acc[1]), yi = ts_add(acc[2], acc[3]);
        const double2 wv = a.w[j];
        const ts3 wc = ts_from_double(wv.x), wd = ts_from_double(wv.y);
        const ts3 re = ts_sub(ts_mul(yr, wc), ts_mul(yi, wd));
        const ts3 im = ts_add(ts_mul(yr, wd), ts_mul(yi, wc));
        double x = ts_to_double(re), y = ts_to_double(im);
        if (a.direction > 0) y = -y;
        if (a.direction == 1 || a.direction == -2) {
            x = __ddiv_rn(x, (double)a.n);
            y = __ddiv_rn(y, (double)a.n);
        }
        a.out[b * a.n + j] = make_double2(x, y);
    }
}

cudaError_t launch_crt_ts(const CrtArgs& a, cudaStream_t s)
{
    cudaError_t e = crt_init();
    if (e != cudaSuccess) return e;
    const int64_t chunks = (a.n + CRT_CHUNK - 1) / CRT_CHUNK;
    crt_ts_kernel<<<(unsigned)(a.B * chunks), FAST_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace oz
