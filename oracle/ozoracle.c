/*
 * ozoracle.c -- CPU oracle for the Ozaki-scheme / 32-bit NTT double-precision FFT
 * of "Computing FFTs at Target Precision Using Lower-Precision FFTs"
 * (arXiv 2603.29129).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The GPU library never links,
 * includes or calls anything here, and nothing here includes or calls the GPU
 * library: the two implementations share no code.
 *
 * Everything is plain scalar C, written for obviousness rather than speed:
 *   - modular arithmetic through unsigned __int128 and the `%` operator;
 *   - the NTT by its definition (O(N^2), §3.3) and by the textbook iterative
 *     radix-2 Cooley-Tukey algorithm with a bit-reversal copy;
 *   - the split of Alg. 3 (§3.4) in binary64, u = 2^-53, with the split width
 *     alpha of §4.4 (two or three primes, accumulation bound L);
 *   - the flush schedule of Alg. 8 (§4.4), the four real convolutions of §4.5,
 *     Garner's algorithm with the symmetric remainder of Eq. (1) (§3.1, §3.3);
 *   - the exact sum of the rescaled CRT integers, rounded once to binary64
 *     (the quantity the TSAdd accumulation of Alg. 8 approximates);
 *   - the Bluestein wrapper of Alg. 1 (§3.2) with ZeroPad / ZeroPad+-;
 *   - a binary128 DFT (naive O(n^2), and radix-2 O(n log n) for large n) as
 *     the accuracy reference (the paper uses a 106-bit MPFR FFT, §5.1).
 *
 * Readings of points the paper leaves open (all repeated in the design notes):
 *   R1  precision: the FFT input, the chirp products and the split are binary64
 *       (u = 2^-53, rho = 53 - alpha); the paper's TS (3 x binary32) variant is
 *       the separate or_ozfft_ts at the end of this file (readings T1-T4).
 *   R2  chirp table: w(j) = exp(-i*pi*r/n), r = j^2 mod 2n, correctly rounded to
 *       binary64 (§4.2 assumes correctly rounded tables); evaluated in binary128
 *       after an exact octant reduction of r/n; components equal to zero are +0.
 *   R3  complex products: re = fma(a,c, -(b*d)), im = fma(a,d, b*c), with b*d
 *       and b*c rounded to binary64.
 *   R4  ceil(log2(mu)) is exact: mu = m*2^E, m in [1/2,1) gives E-1 when
 *       m == 1/2 and E otherwise.
 *   R5  alpha uses n (at most n non-zero products feed any output), not N.
 *   R6  NTT roots: w_N = g^((p-1)/N) with g the smallest primitive root of p.
 *   R7  accumulation: the rescaled CRT integers z'/c of all flush groups of
 *       RR and -II (real part), IR and RI (imaginary part) (§4.5) are summed
 *       exactly and the exact sum is rounded once to nearest binary64 (ties to
 *       even).  This is the plain definition of the sum that Alg. 8's TSAdd
 *       accumulation approximates; the oracle computes it with a two's-complement
 *       big integer in units of 2^-max(S).
 *   R8  inverse direction: conj -> forward -> conj -> round(v / n) (Eq. (4)).
 *       Two more directions serve reverse-mode differentiation: the adjoint of
 *       the forward transform, F^H g = conj(F conj g) (direction +2: R8 without
 *       the division), and the adjoint of the inverse, (1/n) F g (direction -2:
 *       the forward transform, then round(v / n)).
 *   R9  third prime (used only when three primes are requested): 15*2^27 + 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__aarch64__) && (__LDBL_MANT_DIG__ == 113)
typedef long double qreal; /* IEEE binary128 on AArch64 Linux */
#define QPI 3.141592653589793238462643383279502884L
#define QSIN sinl
#define QCOS cosl
#else
#include <quadmath.h>
typedef __float128 qreal;
#define QPI M_PIq
#define QSIN sinq
#define QCOS cosq
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_LENGTH 2
#define OR_ERR_ALLOC 3
#define OR_ERR_NONFINITE 5
#define OR_ERR_RANGE 6

#define OR_KMAX 64 /* level cap used when K = "infinity" (0) */

/* ------------------------------------------------------------------------- */
/* Moduli (§5.1 prints p0 and p1; p2 is reading R9).                          */
/* ------------------------------------------------------------------------- */
static const uint64_t OR_PRIMES[3] = {2130706433ull, 2113929217ull, 2013265921ull};

uint64_t or_prime(int i) { return (i >= 0 && i < 3) ? OR_PRIMES[i] : 0; }

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a * b) % m); }

uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime (Fermat) */
uint64_t or_invmod(uint64_t a, uint64_t p) { return or_powmod(a % p, p - 2, p); }

/* smallest primitive root of the prime p: g has order p-1 iff
   g^((p-1)/q) != 1 for every prime q dividing p-1 (R6). */
uint64_t or_generator(uint64_t p)
{
    uint64_t f[64];
    int nf = 0;
    uint64_t m = p - 1;
    for (uint64_t d = 2; d * d <= m; ++d) {
        if (m % d == 0) {
            f[nf++] = d;
            while (m % d == 0) m /= d;
        }
    }
    if (m > 1) f[nf++] = m;
    for (uint64_t g = 2; g < p; ++g) {
        int ok = 1;
        for (int i = 0; i < nf; ++i)
            if (or_powmod(g, (p - 1) / f[i], p) == 1) { ok = 0; break; }
        if (ok) return g;
    }
    return 0;
}

/* primitive N-th root of unity modulo p (R6); 0 when N does not divide p-1 */
uint64_t or_root(uint64_t p, uint64_t N)
{
    if (N == 0 || (p - 1) % N) return 0;
    return or_powmod(or_generator(p), (p - 1) / N, p);
}

/* ------------------------------------------------------------------------- */
/* NTT (§3.3).                                                                */
/* ------------------------------------------------------------------------- */

/* Definition of the NTT and its inverse: A(k) = sum_j a(j) w^(jk) mod p, and
   a(j) = N^-1 sum_k A(k) w^(-jk) mod p.  O(N^2). */
int or_ntt_naive(const uint32_t* a, uint32_t* A, int64_t N, uint64_t p, int inverse)
{
    uint64_t w = or_root(p, (uint64_t)N);
    if (!w) return OR_ERR_LENGTH;
    if (inverse) w = or_invmod(w, p);
    uint64_t* pw = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
    if (!pw) return OR_ERR_ALLOC;
    pw[0] = 1;
    for (int64_t i = 1; i < N; ++i) pw[i] = mulmod(pw[i - 1], w, p);
    uint64_t ninv = inverse ? or_invmod((uint64_t)N, p) : 1;
    for (int64_t k = 0; k < N; ++k) {
        uint64_t acc = 0;
        for (int64_t j = 0; j < N; ++j) {
            uint64_t e = (uint64_t)((u128)j * (u128)k % (u128)N);
            acc = (acc + mulmod(a[j] % p, pw[e], p)) % p;
        }
        A[k] = (uint32_t)mulmod(acc, ninv, p);
    }
    free(pw);
    return OR_OK;
}

/* Textbook iterative radix-2 Cooley-Tukey NTT (bit-reversal copy, then
   butterflies of growing span).  Natural order in and out. */
int or_ntt(const uint32_t* a, uint32_t* A, int64_t N, uint64_t p, int inverse)
{
    uint64_t w = or_root(p, (uint64_t)N);
    if (!w || (N & (N - 1))) return OR_ERR_LENGTH;
    if (inverse) w = or_invmod(w, p);
    int lg = 0;
    while (((int64_t)1 << lg) < N) ++lg;
    for (int64_t i = 0; i < N; ++i) {
        int64_t r = 0;
        for (int b = 0; b < lg; ++b)
            if (i >> b & 1) r |= (int64_t)1 << (lg - 1 - b);
        A[r] = (uint32_t)(a[i] % p);
    }
    for (int64_t len = 2; len <= N; len <<= 1) {
        uint64_t wl = or_powmod(w, (uint64_t)(N / len), p);
        for (int64_t i = 0; i < N; i += len) {
            uint64_t wj = 1;
            for (int64_t j = 0; j < len / 2; ++j) {
                uint64_t u = A[i + j];
                uint64_t v = mulmod(A[i + j + len / 2], wj, p);
                A[i + j] = (uint32_t)((u + v) % p);
                A[i + j + len / 2] = (uint32_t)((u + p - v) % p);
                wj = mulmod(wj, wl, p);
            }
        }
    }
    if (inverse) {
        uint64_t ninv = or_invmod((uint64_t)N, p);
        for (int64_t i = 0; i < N; ++i) A[i] = (uint32_t)mulmod(A[i], ninv, p);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Split width (§4.2 two-prime CRT alpha, §4.4 with the accumulation bound L).*/
/* alpha = max{a >= 0 : L * n * 2^(2a) < P / 2}, P the product of the primes. */
/* This is floor((log2(P/2) - log2(L n)) / 2) exactly (no tie: P is odd).     */
/* Returns -1 when no a >= 0 qualifies.  Capped at 52 so that rho >= 1.       */
/* ------------------------------------------------------------------------- */
int or_alpha(int64_t n, int64_t L, int nprimes)
{
    if (n < 1 || L < 1 || nprimes < 1 || nprimes > 3) return -1;
    u128 P = 1;
    for (int i = 0; i < nprimes; ++i) P *= OR_PRIMES[i];
    u128 base = (u128)2 * (u128)L * (u128)n; /* 2 L n */
    int bits = 0;
    while (((u128)1 << bits) <= base) ++bits; /* base < 2^bits */
    int a = -1;
    for (int t = 0; t <= 52; ++t) {
        if (bits + 2 * t >= 127) break;
        if ((base << (2 * t)) < P) a = t; else break;
    }
    return a;
}

/* ------------------------------------------------------------------------- */
/* Trigonometric values (reading R2): sin(pi*a/d), cos(pi*a/d) for a/d in    */
/* [0, 2), in binary128, after an exact octant reduction on the integers.    */
/* ------------------------------------------------------------------------- */
static void sincospi_q(uint64_t a, uint64_t d, qreal* s, qreal* c)
{
    int ss = 1, cs = 1, swap = 0;
    if (a >= d) { a -= d; ss = -ss; cs = -cs; }       /* pi*t + pi          */
    if (2 * a > d) { a = d - a; cs = -cs; }            /* pi - x             */
    if (4 * a > d) { a = d - 2 * a; d = 2 * d; swap = 1; } /* pi/2 - x       */
    qreal sv, cv;
    if (a == 0) { sv = 0; cv = 1; }
    else {
        qreal th = QPI * ((qreal)a / (qreal)d);
        sv = QSIN(th);
        cv = QCOS(th);
    }
    if (swap) { qreal t = sv; sv = cv; cv = t; }
    *s = ss > 0 ? sv : -sv;
    *c = cs > 0 ? cv : -cv;
}

/* Bluestein chirp w(j) = w_2n^(j^2) = exp(-i pi j^2 / n), j < n (§3.2),
   correctly rounded to binary64; interleaved (re, im). */
int or_chirp(int64_t n, double* w)
{
    if (n < 1) return OR_ERR_ARG;
    for (int64_t j = 0; j < n; ++j) {
        uint64_t r = (uint64_t)((u128)j * (u128)j % (u128)(2 * n));
        qreal s, c;
        sincospi_q(r, (uint64_t)n, &s, &c);
        double cd = (double)c, sd = (double)s;
        w[2 * j] = cd == 0.0 ? 0.0 : cd;       /* zero components are +0 (R2) */
        w[2 * j + 1] = sd == 0.0 ? 0.0 : -sd;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Binary64 helpers.                                                          */
/* ------------------------------------------------------------------------- */

/* complex product (reading R3) */
static void cmul(double a, double b, double c, double d, double* re, double* im)
{
    double bd = b * d;
    double bc = b * c;
    *re = fma(a, c, -bd);
    *im = fma(a, d, bc);
}

void or_cmul(const double* x, const double* y, double* z, int64_t cnt)
{
    for (int64_t i = 0; i < cnt; ++i)
        cmul(x[2 * i], x[2 * i + 1], y[2 * i], y[2 * i + 1], &z[2 * i], &z[2 * i + 1]);
}

/* ceil(log2(mu)) for finite mu > 0 (reading R4) */
static int ceil_log2(double mu)
{
    int E;
    double m = frexp(mu, &E);
    return m == 0.5 ? E - 1 : E;
}

/* ------------------------------------------------------------------------- */
/* Split (Alg. 3 with rho = 53 - alpha, §4.3-4.4 form of rho).                */
/* v: N doubles.  Produces up to Kcap levels (Kcap <= 0: until mu = 0, at most */
/* OR_KMAX).  For level k: the slice x^(k) (optional), its integer            */
/* q^(k) = c^(k) x^(k) with c^(k) = (u sigma^(k))^-1 = 2^sexp[k], and sexp[k]. */
/* Level arrays are laid out [k][N] for k < kdim; levels >= kdim are computed */
/* but not stored.                                                            */
/* ------------------------------------------------------------------------- */
int or_split(const double* v, int64_t N, int alpha, int Kcap, int kdim, double* slices,
             int64_t* q, int32_t* sexp, int32_t* kout)
{
    if (alpha < 1 || alpha > 52) return OR_ERR_ARG;
    int rho = 53 - alpha;
    double* r = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!r) return OR_ERR_ALLOC;
    for (int64_t j = 0; j < N; ++j) {
        if (!isfinite(v[j])) { free(r); return OR_ERR_NONFINITE; }
        r[j] = v[j];
    }
    int kmax = (Kcap <= 0 || Kcap > OR_KMAX) ? OR_KMAX : Kcap;
    int k = 0;
    int status = OR_OK;
    for (; k < kmax; ++k) {
        double mu = 0.0;
        for (int64_t j = 0; j < N; ++j) mu = fmax(mu, fabs(r[j]));
        if (mu == 0.0) break;
        int e = ceil_log2(mu);
        if (e + rho > 1023) { status = OR_ERR_RANGE; break; }
        double sigma = ldexp(1.0, e + rho);
        for (int64_t j = 0; j < N; ++j) {
            double s = (r[j] + sigma) - sigma;
            r[j] = r[j] - s;
            if (k < kdim) {
                if (slices) slices[(int64_t)k * N + j] = s;
                if (q) q[(int64_t)k * N + j] = (int64_t)ldexp(s, alpha - e);
            }
        }
        if (sexp && k < kdim) sexp[k] = alpha - e;
    }
    if (status == OR_OK && Kcap <= 0 && k == kmax) {
        double mu = 0.0;
        for (int64_t j = 0; j < N; ++j) mu = fmax(mu, fabs(r[j]));
        if (mu != 0.0) status = OR_ERR_RANGE; /* more than OR_KMAX levels */
    }
    free(r);
    *kout = k;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Symmetric remainder, Eq. (1): a mod m = a - m*floor(a/m + 1/2), odd m.     */
/* ------------------------------------------------------------------------- */
static i128 smod(i128 a, i128 m)
{
    i128 r = a % m;
    if (r < 0) r += m;            /* r in [0, m) */
    if (2 * r >= m) r -= m;       /* r in [-(m-1)/2, (m-1)/2] */
    return r;
}

/* Garner's algorithm (§3.3) with symmetric digits, for nprimes residues of
   one position (each in [0, p_i)).  Result in [-(P-1)/2, (P-1)/2]. */
static i128 garner(const uint32_t* z, int nprimes)
{
    i128 acc = smod((i128)z[0], (i128)OR_PRIMES[0]); /* z'_0 */
    i128 Pprev = (i128)OR_PRIMES[0];                   /* P'_0 */
    for (int j = 1; j < nprimes; ++j) {
        i128 pj = (i128)OR_PRIMES[j];
        uint64_t inv = or_invmod((uint64_t)(Pprev % pj), (uint64_t)pj);
        i128 d = smod(((i128)z[j] - acc) % pj * (i128)inv, pj);
        acc = acc + d * Pprev;
        Pprev *= pj;
    }
    return acc;
}

/* vector Garner: res[i*cnt + j] (prime i, position j) -> out[2j] = low 64 bits,
   out[2j+1] = high 64 bits (two's complement) */
void or_garner(const uint32_t* res, int64_t cnt, int nprimes, int64_t* out)
{
    uint32_t z[3];
    for (int64_t j = 0; j < cnt; ++j) {
        for (int i = 0; i < nprimes; ++i) z[i] = res[(int64_t)i * cnt + j];
        i128 v = garner(z, nprimes);
        out[2 * j] = (int64_t)(uint64_t)(u128)v;
        out[2 * j + 1] = (int64_t)(v >> 64);
    }
}

/* ------------------------------------------------------------------------- */
/* Exact accumulation (reading R7): a two's-complement big integer of nl      */
/* 32-bit digits, little-endian.                                              */
/* ------------------------------------------------------------------------- */

/* acc += z * 2^sh  (z an i128, sh >= 0); digits beyond nl are dropped, so the */
/* caller sizes nl to hold every partial sum. */
static void big_add_shifted(uint32_t* acc, int nl, i128 z, int sh)
{
    /* z as 4 sign-extended 32-bit digits (|z| < 2^127) */
    uint32_t d[4];
    u128 uz = (u128)z;
    for (int i = 0; i < 4; ++i) d[i] = (uint32_t)(uz >> (32 * i));
    uint32_t ext = z < 0 ? 0xffffffffu : 0u;
    int q = sh / 32, b = sh % 32;
    uint64_t carry = 0;
    for (int i = q; i < nl; ++i) {
        /* digit i-q of (z << b), built from z's digits k = i-q and k-1 */
        int k = i - q;
        uint32_t hi = k < 4 ? d[k] : ext;
        uint32_t lo = k == 0 ? 0u : (k - 1 < 4 ? d[k - 1] : ext);
        uint32_t v = b == 0 ? hi : (uint32_t)((hi << b) | (lo >> (32 - b)));
        uint64_t s = (uint64_t)acc[i] + v + carry;
        acc[i] = (uint32_t)s;
        carry = s >> 32;
    }
}

/* round the big integer acc * 2^unit to the nearest binary64 (ties to even) */
static double big_to_double(const uint32_t* acc_in, int nl, int unit)
{
    uint32_t* m = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nl);
    memcpy(m, acc_in, sizeof(uint32_t) * (size_t)nl);
    int neg = (m[nl - 1] >> 31) != 0;
    if (neg) { /* magnitude = two's complement negation */
        uint64_t c = 1;
        for (int i = 0; i < nl; ++i) {
            uint64_t s = (uint64_t)(uint32_t)~m[i] + c;
            m[i] = (uint32_t)s;
            c = s >> 32;
        }
    }
    int top = -1; /* index of the leading one bit */
    for (int i = nl - 1; i >= 0 && top < 0; --i)
        if (m[i])
            for (int bit = 31; bit >= 0; --bit)
                if (m[i] >> bit & 1) { top = 32 * i + bit; break; }
    double r = 0.0;
    if (top >= 0) {
        int lead = unit + top;                    /* exponent of the leading bit */
        int eulp = lead - 52 > -1074 ? lead - 52 : -1074;
        int drop = eulp - unit;                   /* low bits below the result's ulp */
        uint64_t qv = 0;
        if (drop <= 0) {
            for (int bit = top; bit >= 0; --bit) qv = qv << 1 | (m[bit / 32] >> (bit % 32) & 1);
            r = ldexp((double)qv, unit);
        } else {
            for (int bit = top; bit >= drop; --bit) qv = qv << 1 | (m[bit / 32] >> (bit % 32) & 1);
            int rbit = m[(drop - 1) / 32] >> ((drop - 1) % 32) & 1;
            int sticky = 0;
            for (int bit = drop - 2; bit >= 0 && !sticky; --bit) sticky = m[bit / 32] >> (bit % 32) & 1;
            if (rbit && (sticky || (qv & 1))) qv += 1;
            r = ldexp((double)qv, eulp);
        }
    }
    free(m);
    return neg ? -r : r;
}

void or_exact_sum(const int64_t* z2, const int32_t* S, const int32_t* sign, int64_t cnt, double* out)
{
    /* exposed for the tests: round(sum sign_i z_i 2^-S_i) */
    int smin = 0, smax = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (i == 0 || S[i] < smin) smin = S[i];
        if (i == 0 || S[i] > smax) smax = S[i];
    }
    int nl = (smax - smin + 128 + 16) / 32 + 2;
    uint32_t* acc = (uint32_t*)calloc((size_t)nl, sizeof(uint32_t));
    for (int64_t i = 0; i < cnt; ++i) {
        i128 z = (i128)(((u128)(uint64_t)z2[2 * i + 1] << 64) | (u128)(uint64_t)z2[2 * i]);
        big_add_shifted(acc, nl, sign[i] < 0 ? -z : z, smax - S[i]);
    }
    *out = big_to_double(acc, nl, -smax);
    free(acc);
}

/* ------------------------------------------------------------------------- */
/* Flush schedule of Alg. 8.  sx[kx], sy[ky]: scale exponents (c = 2^s, so   */
/* c_x c_y equality is equality of sx+sy).  Output: ngroups; for group g:    */
/* gS[g] = sx+sy, gsize[g], pairs gpairs[(g*pdim + m)*2 + {0,1}] = (s, t).     */
/* Returns the number of groups, or -1 if gdim/pdim is too small.             */
/* ------------------------------------------------------------------------- */
int or_schedule(int kx, const int32_t* sx, int ky, const int32_t* sy, int L, int gdim, int pdim,
                int32_t* gS, int32_t* gsize, int32_t* gpairs)
{
    if (kx <= 0 || ky <= 0) return 0;
    int g = 0;
    int l = 0;
    int32_t c = sx[kx - 1] + sy[ky - 1];
    for (int k = kx + ky - 2; k >= 0; --k) {
        int s0 = k - ky + 1 > 0 ? k - ky + 1 : 0;
        int s1 = kx - 1 < k ? kx - 1 : k;
        for (int s = s0; s <= s1; ++s) {
            int t = k - s;
            if (l >= L || c != sx[s] + sy[t]) { /* flush the current group */
                ++g;
                c = sx[s] + sy[t];
                l = 0;
            }
            if (g >= gdim || l >= pdim) return -1;
            gS[g] = c;
            gpairs[((int64_t)g * pdim + l) * 2 + 0] = s;
            gpairs[((int64_t)g * pdim + l) * 2 + 1] = t;
            ++l;
            gsize[g] = l;
        }
    }
    return g + 1;
}

/* ------------------------------------------------------------------------- */
/* The whole method (Alg. 1 around Alg. 8 x 4, §4.5) with optional trace.     */
/* ------------------------------------------------------------------------- */
typedef struct {
    /* outputs (always written) */
    int32_t alpha, rho;
    int32_t kcount[4];            /* levels of Re x~', Im x~', Re w~*, Im w~* */
    int32_t sexp[4][OR_KMAX];     /* scale exponents per level */
    int32_t ngroups[4];           /* flush groups of RR, II, IR, RI */
    int64_t n_fwd_runtime;        /* forward NTTs on the x~' slices */
    int64_t n_fwd_plan;           /* forward NTTs on the w~* slices */
    int64_t n_inv;                /* inverse NTTs */
    /* optional buffers (NULL = not wanted) */
    int32_t kdim, gdim;           /* level / group capacity of the buffers below */
    double* xprime;               /* [2][N] Re, Im of x~' */
    double* wstar;                /* [2][N] Re, Im of w~* */
    int64_t* q;                   /* [4][kdim][N] slice integers */
    uint32_t* spec;               /* [4][kdim][nprimes][N] forward NTT spectra */
    int32_t* gS;                  /* [4][gdim] */
    int32_t* gsize;               /* [4][gdim] */
    int32_t* gpairs;              /* [4][gdim][kdim][2] */
    uint32_t* zres;               /* [4][gdim][nprimes][N] inverse NTT residues */
    int64_t* zcrt;                /* [4][gdim][N][2] CRT integers (lo, hi) */
    double* yprime;               /* [n][2] y' before the post-multiply */
} or_trace;

/* transform directions (R8): -1 forward, +1 inverse, +2 / -2 their adjoints */
static int dir_ok(int d) { return d == -1 || d == 1 || d == 2 || d == -2; }
static int dir_conj(int d) { return d > 0; }              /* exponent sign + */
static int dir_scaled(int d) { return d == 1 || d == -2; } /* divide by n */

/* vector index pairs of the four real convolutions (§4.5): RR, II, IR, RI */
static const int CONV_X[4] = {0, 1, 1, 0};
static const int CONV_W[4] = {2, 3, 2, 3};
static const int CONV_OUT[4] = {0, 0, 1, 1};   /* 0: real part, 1: imaginary */
static const int CONV_NEG[4] = {0, 1, 0, 0};

int or_ozfft(int64_t n, int64_t N, int K, int L, int nprimes, int direction,
             const double* x, double* y, or_trace* tr)
{
    if (n < 1 || N < n || (N & (N - 1)) || L < 1 || K < 0 || nprimes < 2 || nprimes > 3 ||
        !dir_ok(direction))
        return OR_ERR_ARG;
    if (!(N == n || N >= 2 * n - 1)) return OR_ERR_LENGTH;
    for (int i = 0; i < nprimes; ++i)
        if ((OR_PRIMES[i] - 1) % (uint64_t)N) return OR_ERR_LENGTH;
    int alpha = or_alpha(n, L, nprimes);
    if (alpha < 1) return OR_ERR_LENGTH;

    int status = OR_OK;
    size_t szN = (size_t)N;
    int kcap = K == 0 ? OR_KMAX : (K > OR_KMAX ? OR_KMAX : K);
    int kq = 1; /* level capacity actually needed, known after the split counts */
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* vec = (double*)calloc(4 * szN, sizeof(double)); /* Re x', Im x', Re w*, Im w* */
    int64_t* q = NULL;
    uint32_t* spec = NULL;
    uint32_t* res = (uint32_t*)malloc(sizeof(uint32_t) * szN);
    uint32_t* Z = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nprimes * szN);
    uint32_t* zr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nprimes * szN);
    double* acc = (double*)calloc(2 * (size_t)n, sizeof(double)); /* y' [part][n] */
    uint32_t* bigacc = NULL;
    int nl = 0;
    int32_t* gS = NULL;
    int32_t* gsz = NULL;
    int32_t* gp = NULL;
    int32_t kcount[4] = {0, 0, 0, 0};
    int32_t sexp[4][OR_KMAX];
    int64_t nfr = 0, nfp = 0, ninv = 0;
    if (!w || !vec || !res || !Z || !zr || !acc) {
        status = OR_ERR_ALLOC;
        goto done;
    }

    /* Alg. 1 step 1: x' = x (.) w (inverse: conjugate the input, R8) */
    or_chirp(n, w);
    for (int64_t j = 0; j < n; ++j) {
        double a = x[2 * j], b = x[2 * j + 1];
        if (dir_conj(direction)) b = -b;
        cmul(a, b, w[2 * j], w[2 * j + 1], &vec[j], &vec[szN + j]);
    }
    /* ZeroPad (x~') is implicit in calloc; ZeroPad+- of w* (§3.2) */
    for (int64_t j = 0; j < N; ++j) {
        int64_t src = -1;
        if (j < n) src = j;
        else if (N != n && j >= N - n + 1) src = N - j;
        if (src >= 0) {
            vec[2 * szN + j] = w[2 * src];
            vec[3 * szN + j] = -w[2 * src + 1];
        }
    }

    /* split the four real vectors once each (split caching of §4.5): a first
       pass finds the level counts, the second stores the slice integers */
    for (int v = 0; v < 4 && status == OR_OK; ++v)
        status = or_split(&vec[(size_t)v * szN], N, alpha, kcap, OR_KMAX, NULL, NULL, sexp[v], &kcount[v]);
    if (status != OR_OK) goto done;
    for (int v = 0; v < 4; ++v) kq = kcount[v] > kq ? kcount[v] : kq;
    q = (int64_t*)malloc(sizeof(int64_t) * 4 * (size_t)kq * szN);
    spec = (uint32_t*)malloc(sizeof(uint32_t) * 4 * (size_t)kq * (size_t)nprimes * szN);
    gS = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)kq * (size_t)kq);
    gsz = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)kq * (size_t)kq);
    gp = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)kq * (size_t)kq * (size_t)kq * 2);
    if (!q || !spec || !gS || !gsz || !gp) { status = OR_ERR_ALLOC; goto done; }
    for (int v = 0; v < 4 && status == OR_OK; ++v) {
        int32_t kv;
        status = or_split(&vec[(size_t)v * szN], N, alpha, kcap, kq, NULL, &q[(size_t)v * kq * szN],
                          sexp[v], &kv);
    }
    if (status != OR_OK) goto done;

    /* residues and forward NTTs of every level for every prime (Alg. 6 tail) */
    for (int v = 0; v < 4; ++v)
        for (int k = 0; k < kcount[v]; ++k)
            for (int i = 0; i < nprimes; ++i) {
                int64_t p = (int64_t)OR_PRIMES[i];
                const int64_t* qk = &q[((size_t)v * kq + k) * szN];
                for (int64_t j = 0; j < N; ++j) {
                    int64_t a = qk[j] % p;
                    res[j] = (uint32_t)(a < 0 ? a + p : a);
                }
                or_ntt(res, &spec[(((size_t)v * kq + k) * nprimes + i) * szN], N, (uint64_t)p, 0);
                if (v < 2) ++nfr; else ++nfp;
            }

    /* Alg. 8 flush schedules of the four real convolutions */
    int ngs[4];
    const size_t gstride = (size_t)kq * (size_t)kq;
    int smin = 0, smax = 0, any = 0;
    for (int c = 0; c < 4; ++c) {
        int vx = CONV_X[c], vw = CONV_W[c];
        ngs[c] = or_schedule(kcount[vx], sexp[vx], kcount[vw], sexp[vw], L, kq * kq, kq, &gS[c * gstride],
                             &gsz[c * gstride], &gp[c * gstride * kq * 2]);
        if (ngs[c] < 0) { status = OR_ERR_ARG; goto done; }
        if (tr) tr->ngroups[c] = ngs[c];
        for (int g = 0; g < ngs[c]; ++g) {
            int S = gS[c * gstride + g];
            if (!any || S < smin) smin = S;
            if (!any || S > smax) smax = S;
            any = 1;
        }
    }
    /* exact accumulators (R7): per part and output, nl digits in units of 2^-smax */
    nl = (smax - smin + 128 + 16) / 32 + 2;
    bigacc = (uint32_t*)calloc(2 * (size_t)n * (size_t)nl, sizeof(uint32_t));
    if (!bigacc) { status = OR_ERR_ALLOC; goto done; }

    for (int c = 0; c < 4; ++c) {
        int vx = CONV_X[c], vw = CONV_W[c];
        int ng = ngs[c];
        const int32_t* cS = &gS[c * gstride];
        const int32_t* csz = &gsz[c * gstride];
        const int32_t* cp = &gp[c * gstride * kq * 2];
        for (int g = 0; g < ng; ++g) {
            /* NTT-domain accumulation: Z_i = sum X_s (.) Y_t mod p_i */
            for (int i = 0; i < nprimes; ++i) {
                uint64_t p = OR_PRIMES[i];
                uint32_t* Zi = &Z[(size_t)i * szN];
                memset(Zi, 0, sizeof(uint32_t) * szN);
                for (int m = 0; m < csz[g]; ++m) {
                    int s = cp[((size_t)g * kq + m) * 2], t = cp[((size_t)g * kq + m) * 2 + 1];
                    const uint32_t* X = &spec[(((size_t)vx * kq + s) * nprimes + i) * szN];
                    const uint32_t* Y = &spec[(((size_t)vw * kq + t) * nprimes + i) * szN];
                    for (int64_t j = 0; j < N; ++j) Zi[j] = (uint32_t)((Zi[j] + mulmod(X[j], Y[j], p)) % p);
                }
                or_ntt(Zi, &zr[(size_t)i * szN], N, p, 1);
                ++ninv;
            }
            /* Garner, then z' / c added exactly (R7) */
            uint32_t z3[3];
            int part = CONV_OUT[c];
            for (int64_t j = 0; j < N; ++j) {
                for (int i = 0; i < nprimes; ++i) z3[i] = zr[(size_t)i * szN + j];
                i128 zc = garner(z3, nprimes);
                if (tr && tr->zcrt && g < tr->gdim) {
                    int64_t* o = &tr->zcrt[(((size_t)c * tr->gdim + g) * szN + j) * 2];
                    o[0] = (int64_t)(uint64_t)(u128)zc;
                    o[1] = (int64_t)(zc >> 64);
                }
                if (j < n)
                    big_add_shifted(&bigacc[((size_t)part * n + j) * nl], nl, CONV_NEG[c] ? -zc : zc,
                                    smax - cS[g]);
            }
            if (tr && g < tr->gdim) {
                if (tr->gS) tr->gS[c * tr->gdim + g] = cS[g];
                if (tr->gsize) tr->gsize[c * tr->gdim + g] = csz[g];
                if (tr->gpairs)
                    for (int m = 0; m < csz[g] && m < tr->kdim; ++m) {
                        tr->gpairs[(((size_t)c * tr->gdim + g) * tr->kdim + m) * 2] = cp[((size_t)g * kq + m) * 2];
                        tr->gpairs[(((size_t)c * tr->gdim + g) * tr->kdim + m) * 2 + 1] =
                            cp[((size_t)g * kq + m) * 2 + 1];
                    }
                if (tr->zres)
                    memcpy(&tr->zres[((size_t)c * tr->gdim + g) * nprimes * szN], zr,
                           sizeof(uint32_t) * (size_t)nprimes * szN);
            }
        }
    }
    for (int part = 0; part < 2; ++part)
        for (int64_t j = 0; j < n; ++j)
            acc[(size_t)part * n + j] = any ? big_to_double(&bigacc[((size_t)part * n + j) * nl], nl, -smax) : 0.0;

    /* y' = rounded accumulators; Alg. 1 last step y = y' (.) w; inverse (R8) */
    for (int64_t j = 0; j < n; ++j) {
        double yr = acc[j];
        double yi = acc[(size_t)n + j];
        if (tr && tr->yprime) { tr->yprime[2 * j] = yr; tr->yprime[2 * j + 1] = yi; }
        double re, im;
        cmul(yr, yi, w[2 * j], w[2 * j + 1], &re, &im);
        if (dir_conj(direction)) im = -im;
        if (dir_scaled(direction)) {
            re = re / (double)n;
            im = im / (double)n;
        }
        y[2 * j] = re;
        y[2 * j + 1] = im;
    }

done:
    if (tr) {
        tr->alpha = alpha;
        tr->rho = 53 - alpha;
        for (int v = 0; v < 4; ++v) {
            tr->kcount[v] = kcount[v];
            for (int k = 0; k < kcount[v] && k < OR_KMAX; ++k) tr->sexp[v][k] = sexp[v][k];
        }
        tr->n_fwd_runtime = nfr;
        tr->n_fwd_plan = nfp;
        tr->n_inv = ninv;
        if (status == OR_OK) {
            if (tr->xprime) memcpy(tr->xprime, vec, sizeof(double) * 2 * szN);
            if (tr->wstar) memcpy(tr->wstar, &vec[2 * szN], sizeof(double) * 2 * szN);
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < kcount[v] && k < tr->kdim; ++k) {
                    if (tr->q)
                        memcpy(&tr->q[((size_t)v * tr->kdim + k) * szN], &q[((size_t)v * kq + k) * szN],
                               sizeof(int64_t) * szN);
                    if (tr->spec)
                        memcpy(&tr->spec[((size_t)v * tr->kdim + k) * nprimes * szN],
                               &spec[((size_t)v * kq + k) * nprimes * szN],
                               sizeof(uint32_t) * (size_t)nprimes * szN);
                }
        }
    }
    free(w); free(vec); free(q); free(spec); free(res); free(Z); free(zr); free(acc);
    free(gS); free(gsz); free(gp); free(bigacc);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Binary128 accuracy reference (the paper measures against a 106-bit MPFR   */
/* FFT, §5.1).  Outputs hi = RN64(v) and lo = RN64(v - hi) per component.     */
/* ------------------------------------------------------------------------- */

/* exp(sign * 2 pi i m / n) for m < n, binary128 */
static void unit_q(int64_t m, int64_t n, int sign, qreal* re, qreal* im)
{
    qreal s, c;
    sincospi_q((uint64_t)(2 * m), (uint64_t)n, &s, &c);
    *re = c;
    *im = sign < 0 ? -s : s;
}

static void store_q(qreal v, double* hi, double* lo)
{
    double h = (double)v;
    *hi = h;
    *lo = (double)(v - (qreal)h);
}

/* Naive DFT (Eq. (3)) / inverse DFT (Eq. (4)) / their adjoints (direction +2:
   exponent sign +, no division; -2: sign -, divided by n) at the requested bins (all when
   bins == NULL).  x interleaved (re, im); yhi, ylo interleaved per bin. */
int or_dft_q(int64_t n, const double* x, int direction, int64_t nbins, const int64_t* bins,
             double* yhi, double* ylo)
{
    if (n < 1 || !dir_ok(direction)) return OR_ERR_ARG;
    qreal* tw = (qreal*)malloc(sizeof(qreal) * 2 * (size_t)n);
    if (!tw) return OR_ERR_ALLOC;
    for (int64_t m = 0; m < n; ++m) unit_q(m, n, direction, &tw[2 * m], &tw[2 * m + 1]);
    int64_t nb = bins ? nbins : n;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t k = bins ? bins[b] : b;
        qreal ar = 0, ai = 0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t e = (int64_t)((u128)j * (u128)k % (u128)n);
            qreal xr = x[2 * j], xi = x[2 * j + 1];
            ar += xr * tw[2 * e] - xi * tw[2 * e + 1];
            ai += xr * tw[2 * e + 1] + xi * tw[2 * e];
        }
        if (dir_scaled(direction)) { ar /= (qreal)n; ai /= (qreal)n; }
        store_q(ar, &yhi[2 * b], &ylo[2 * b]);
        store_q(ai, &yhi[2 * b + 1], &ylo[2 * b + 1]);
    }
    free(tw);
    return OR_OK;
}

/* Radix-2 binary128 FFT for power-of-two n (textbook iterative Cooley-Tukey);
   checked against or_dft_q by the tests. */
int or_fft_q(int64_t n, const double* x, int direction, double* yhi, double* ylo)
{
    if (n < 1 || (n & (n - 1)) || !dir_ok(direction)) return OR_ERR_ARG;
    qreal* a = (qreal*)malloc(sizeof(qreal) * 2 * (size_t)n);
    qreal* tw = (qreal*)malloc(sizeof(qreal) * (size_t)n); /* (re, im) for m < n/2 */
    if (!a || !tw) { free(a); free(tw); return OR_ERR_ALLOC; }
    int lg = 0;
    while (((int64_t)1 << lg) < n) ++lg;
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = 0;
        for (int b = 0; b < lg; ++b)
            if (i >> b & 1) r |= (int64_t)1 << (lg - 1 - b);
        a[2 * r] = x[2 * i];
        a[2 * r + 1] = x[2 * i + 1];
    }
    for (int64_t m = 0; m < n / 2; ++m) unit_q(m, n, direction, &tw[2 * m], &tw[2 * m + 1]);
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t step = n / len;
        for (int64_t i = 0; i < n; i += len)
            for (int64_t j = 0; j < len / 2; ++j) {
                qreal wr = tw[2 * (j * step)], wi = tw[2 * (j * step) + 1];
                qreal* u = &a[2 * (i + j)];
                qreal* v = &a[2 * (i + j + len / 2)];
                qreal tr = v[0] * wr - v[1] * wi, ti = v[0] * wi + v[1] * wr;
                qreal ur = u[0], ui = u[1];
                u[0] = ur + tr; u[1] = ui + ti;
                v[0] = ur - tr; v[1] = ui - ti;
            }
    }
    for (int64_t i = 0; i < n; ++i) {
        qreal re = a[2 * i], im = a[2 * i + 1];
        if (dir_scaled(direction)) { re /= (qreal)n; im /= (qreal)n; }
        store_q(re, &yhi[2 * i], &ylo[2 * i]);
        store_q(im, &yhi[2 * i + 1], &ylo[2 * i + 1]);
    }
    free(a);
    free(tw);
    return OR_OK;
}

/* binary128 sin/cos of pi*a/d (exposed for the reduction tests) */
void or_sincospi_q(uint64_t a, uint64_t d, double* out /* s_hi, s_lo, c_hi, c_lo */)
{
    qreal s, c;
    sincospi_q(a, d, &s, &c);
    store_q(s, &out[0], &out[1]);
    store_q(c, &out[2], &out[3]);
}

/* ========================================================================= */
/* TS (triple-single) variant of the method (§4.1, Alg. 4, Alg. 6, Alg. 8).   */
/*                                                                           */
/* A TS number is a triple of binary32 values x0 + x1 + x2 (§4.1).  TSAdd and */
/* TSMul follow the triple-word arithmetic of Fabiano, Muller and Picot      */
/* (2019) in the form written here: exact transformations (2Sum, Fast2Sum,    */
/* 2Prod with an FMA) produce the partial terms, VecSum adds them without     */
/* error into a decreasing sequence, and the VecSumErrBranch renormalisation  */
/* keeps three words.  Readings for this variant:                            */
/*   T1  TS(x) of a binary64 x: x0 = RN32(x), x1 = RN32(x - x0),              */
/*       x2 = RN32(x - x0 - x1) (differences exact in binary64), so every      */
/*       binary64 in the binary32 exponent range converts exactly.           */
/*   T2  rho = 24 - alpha with alpha = min(alpha of R5, 23), so rho >= 1 and  */
/*       the split of Alg. 6 stays error free in binary32.                   */
/*   T3  z' / c of Alg. 8: the CRT integer (|z'| < p0 p1 / 2 < 2^62) is       */
/*       converted to TS exactly (three words of <= 24 bits) and each word   */
/*       scaled by 2^-S by binary32 multiplications by powers of two.         */
/*   T4  Alg. 8 runs once per real convolution (RR, II, IR, RI) with its own  */
/*       TS accumulator, groups in schedule order; Re y' = TSSub(RR, II),    */
/*       Im y' = TSAdd(IR, RI); y = y' (.) w in TS (Alg. 4); the binary64    */
/*       result is (double(y0) + double(y1)) + double(y2), i.e. the exact sum */
/*       rounded once; the inverse direction conjugates and divides by n in   */
/*       binary64 (R8).  Two primes only.                                    */
/* ========================================================================= */
typedef struct { float w[3]; } ts3;

static void f_two_sum(float a, float b, float* s, float* e)
{
    float ss = a + b;
    float bb = ss - a;
    float aa = ss - bb;
    *s = ss;
    *e = (a - aa) + (b - bb);
}

static void f_fast_two_sum(float a, float b, float* s, float* e)
{
    float ss = a + b;
    *s = ss;
    *e = b - (ss - a);
}

static void f_two_prod(float a, float b, float* p, float* e)
{
    float pp = a * b;
    *p = pp;
    *e = fmaf(a, b, -pp);
}

/* VecSum: x[0..n) -> x[0] = RN of the running sum from the last term up,
   x[1..n) the exact errors, x[0] + ... + x[n-1] unchanged */
static void f_vec_sum(float* x, int n)
{
    float s = x[n - 1];
    for (int i = n - 2; i >= 0; --i) {
        float e;
        f_two_sum(x[i], s, &s, &e);
        x[i + 1] = e;
    }
    x[0] = s;
}

/* VecSumErrBranch: renormalise e[0..n) into m words r (zeros where unused) */
static void f_vec_sum_err_branch(const float* e, int n, int m, float* r)
{
    for (int k = 0; k < m; ++k) r[k] = 0.0f;
    int j = 0;
    float eps = e[0];
    for (int i = 1; i < n; ++i) {
        float s, t;
        f_fast_two_sum(eps, e[i], &s, &t);
        if (t != 0.0f) {
            r[j] = s;
            if (j == m - 1) return;
            ++j;
            eps = t;
        } else {
            eps = s;
        }
    }
    r[j] = eps;
}

static ts3 ts_make(float a, float b, float c)
{
    ts3 t;
    t.w[0] = a;
    t.w[1] = b;
    t.w[2] = c;
    return t;
}

static ts3 ts_neg(ts3 a) { return ts_make(-a.w[0], -a.w[1], -a.w[2]); }

/* TSAdd: the six words merged by decreasing magnitude, VecSum, renormalised */
static ts3 ts_add(ts3 a, ts3 b)
{
    float z[6], r[3];
    int i = 0, j = 0;
    for (int k = 0; k < 6; ++k) {
        if (j >= 3 || (i < 3 && fabsf(a.w[i]) >= fabsf(b.w[j]))) z[k] = a.w[i++];
        else z[k] = b.w[j++];
    }
    f_vec_sum(z, 6);
    f_vec_sum_err_branch(z, 6, 3, r);
    return ts_make(r[0], r[1], r[2]);
}

static ts3 ts_sub(ts3 a, ts3 b) { return ts_add(a, ts_neg(b)); }

/* TSMul: the products of weight 1 and 2^-24 exactly (2Prod), those of weight
   2^-48 rounded, a1 b2 + a2 b1 + a2 b2 dropped; VecSum, renormalised */
static ts3 ts_mul(ts3 a, ts3 b)
{
    float z00, e00, z01, e01, z10, e10, r[3];
    f_two_prod(a.w[0], b.w[0], &z00, &e00);
    f_two_prod(a.w[0], b.w[1], &z01, &e01);
    f_two_prod(a.w[1], b.w[0], &z10, &e10);
    float t[9] = {z00, z01, z10, e00, a.w[0] * b.w[2], a.w[1] * b.w[1], a.w[2] * b.w[0], e01, e10};
    f_vec_sum(t, 9);
    f_vec_sum_err_branch(t, 9, 3, r);
    return ts_make(r[0], r[1], r[2]);
}

static ts3 ts_from_double(double x)    /* T1 */
{
    float a = (float)x;
    double r1 = x - (double)a;
    float b = (float)r1;
    float c = (float)(r1 - (double)b);
    return ts_make(a, b, c);
}

static double ts_to_double(ts3 a) { return ((double)a.w[0] + (double)a.w[1]) + (double)a.w[2]; }

/* exact x 2^e in binary32 steps (each a product by a normal power of two) */
static float f_scale_pow2(float x, int e)
{
    while (e > 127) { x *= 0x1p127f; e -= 127; }
    while (e < -126) { x *= 0x1p-126f; e += 126; }
    union { uint32_t u; float f; } p;
    p.u = (uint32_t)(e + 127) << 23;
    return x * p.f;
}

static ts3 ts_from_int_scaled(int64_t z, int S)   /* T3: z * 2^-S */
{
    float a = (float)z;
    int64_t r1 = z - (int64_t)a;
    float b = (float)r1;
    int64_t r2 = r1 - (int64_t)b;
    float c = (float)r2;
    return ts_make(f_scale_pow2(a, -S), f_scale_pow2(b, -S), f_scale_pow2(c, -S));
}

/* exact ceil(log2 m) of a positive binary32 (R4) */
static int ceil_log2_f(float m)
{
    int E;
    float f = frexpf(m, &E);
    return f == 0.5f ? E - 1 : E;
}

int or_alpha_ts(int64_t n, int L)    /* T2 */
{
    int a = or_alpha(n, L, 2);
    return a > 23 ? 23 : a;
}

/* vector helpers exposed for the tests: cnt TS numbers as [cnt][3] floats */
void or_ts_from_double(const double* x, int64_t cnt, float* out)
{
    for (int64_t i = 0; i < cnt; ++i) {
        ts3 t = ts_from_double(x[i]);
        memcpy(&out[3 * i], t.w, sizeof t.w);
    }
}

void or_ts_to_double(const float* a, int64_t cnt, double* out)
{
    for (int64_t i = 0; i < cnt; ++i) out[i] = ts_to_double(ts_make(a[3 * i], a[3 * i + 1], a[3 * i + 2]));
}

void or_ts_op(int op, const float* a, const float* b, int64_t cnt, float* out)   /* 0 add, 1 sub, 2 mul */
{
    for (int64_t i = 0; i < cnt; ++i) {
        ts3 x = ts_make(a[3 * i], a[3 * i + 1], a[3 * i + 2]);
        ts3 y = ts_make(b[3 * i], b[3 * i + 1], b[3 * i + 2]);
        ts3 r = op == 0 ? ts_add(x, y) : op == 1 ? ts_sub(x, y) : ts_mul(x, y);
        memcpy(&out[3 * i], r.w, sizeof r.w);
    }
}

/* Alg. 6 on one TS vector v[3][N] (planes of words 0, 1, 2): level k takes
   mu = ||r0||_inf, sigma = 2^(ceil(log2 mu) + rho), x^(k) = fl32((r0 + sigma)
   - sigma), then r0, r1 <- FastTwoSum(r0 - x^(k), r1) and r1, r2 <-
   FastTwoSum(r1, r2); the integer q^(k) = c^(k) x^(k) with c^(k) = (u32
   sigma)^-1 = 2^sexp[k].  Layout of q as or_split. */
int or_ts_split(const float* v, int64_t N, int alpha, int Kcap, int kdim, int64_t* q, int32_t* sexp, int32_t* kout)
{
    if (alpha < 1 || alpha > 23) return OR_ERR_ARG;
    const int rho = 24 - alpha;
    float* r = (float*)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    if (!r) return OR_ERR_ALLOC;
    for (int64_t j = 0; j < 3 * N; ++j) {
        if (!isfinite(v[j])) { free(r); return OR_ERR_NONFINITE; }
        r[j] = v[j];
    }
    float* r0 = r;
    float* r1 = r + N;
    float* r2 = r + 2 * N;
    int kmax = (Kcap <= 0 || Kcap > OR_KMAX) ? OR_KMAX : Kcap;
    int k = 0, status = OR_OK;
    for (; k < kmax; ++k) {
        float mu = 0.0f;
        for (int64_t j = 0; j < N; ++j) mu = fmaxf(mu, fabsf(r0[j]));
        if (mu == 0.0f) break;
        const int e = ceil_log2_f(mu);
        if (e + rho > 127 || e + rho < -126) { status = OR_ERR_RANGE; break; }
        const float sigma = f_scale_pow2(1.0f, e + rho);
        for (int64_t j = 0; j < N; ++j) {
            float s = (r0[j] + sigma) - sigma;
            float a, b, c, d;
            f_fast_two_sum(r0[j] - s, r1[j], &a, &b);
            f_fast_two_sum(b, r2[j], &c, &d);
            r0[j] = a;
            r1[j] = c;
            r2[j] = d;
            if (k < kdim && q) q[(int64_t)k * N + j] = (int64_t)f_scale_pow2(s, alpha - e);
        }
        if (sexp && k < kdim) sexp[k] = alpha - e;
    }
    free(r);
    *kout = k;
    return status;
}

/* The TS variant of the whole method (T1-T4): Alg. 4 around Alg. 8, two primes. */
int or_ozfft_ts(int64_t n, int64_t N, int K, int L, int direction, const double* x, double* y, or_trace* tr)
{
    const int nprimes = 2;
    if (n < 1 || N < n || (N & (N - 1)) || L < 1 || K < 0 || !dir_ok(direction)) return OR_ERR_ARG;
    if (!(N == n || N >= 2 * n - 1)) return OR_ERR_LENGTH;
    for (int i = 0; i < nprimes; ++i)
        if ((OR_PRIMES[i] - 1) % (uint64_t)N) return OR_ERR_LENGTH;
    const int alpha = or_alpha_ts(n, L);
    if (alpha < 1) return OR_ERR_LENGTH;
    const size_t szN = (size_t)N;
    const int kcap = K == 0 ? OR_KMAX : (K > OR_KMAX ? OR_KMAX : K);
    int status = OR_OK, kq = 1;
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    float* tv = (float*)calloc(4 * 3 * szN, sizeof(float));   /* [v][word][N]: Re x', Im x', Re w*, Im w* */
    ts3* wt = (ts3*)malloc(sizeof(ts3) * (size_t)n);             /* TS(w) */
    ts3* acc = (ts3*)calloc(4 * (size_t)n, sizeof(ts3));        /* Alg. 8 accumulators of RR, II, IR, RI */
    uint32_t* res = (uint32_t*)malloc(sizeof(uint32_t) * szN);
    uint32_t* Z = (uint32_t*)malloc(sizeof(uint32_t) * nprimes * szN);
    uint32_t* zr = (uint32_t*)malloc(sizeof(uint32_t) * nprimes * szN);
    int64_t* q = NULL;
    uint32_t* spec = NULL;
    int32_t *gS = NULL, *gsz = NULL, *gp = NULL;
    int32_t kcount[4] = {0, 0, 0, 0};
    int32_t sexp[4][OR_KMAX];
    int64_t nfr = 0, nfp = 0, ninv = 0;
    if (!w || !tv || !wt || !acc || !res || !Z || !zr) { status = OR_ERR_ALLOC; goto done; }

    /* Alg. 4 steps 1-2: TS conversion (T1) and x' = x (.) w in TS */
    or_chirp(n, w);
    for (int64_t j = 0; j < n; ++j) {
        double xr = x[2 * j], xi = x[2 * j + 1];
        if (!isfinite(xr) || !isfinite(xi)) { status = OR_ERR_NONFINITE; goto done; }
        if (dir_conj(direction)) xi = -xi;
        ts3 a = ts_from_double(xr), b = ts_from_double(xi);
        ts3 c = ts_from_double(w[2 * j]), d = ts_from_double(w[2 * j + 1]);
        wt[j] = c;   /* real part; the imaginary part is rebuilt from w below */
        ts3 re = ts_sub(ts_mul(a, c), ts_mul(b, d));
        ts3 im = ts_add(ts_mul(a, d), ts_mul(b, c));
        for (int k = 0; k < 3; ++k) {
            if (!isfinite(re.w[k]) || !isfinite(im.w[k])) { status = OR_ERR_RANGE; goto done; }
            tv[(0 * 3 + k) * szN + j] = re.w[k];
            tv[(1 * 3 + k) * szN + j] = im.w[k];
        }
    }
    /* w~* = ZeroPad+-(conj w) in TS (exact, T1) */
    for (int64_t j = 0; j < N; ++j) {
        int64_t src = -1;
        if (j < n) src = j;
        else if (N != n && j >= N - n + 1) src = N - j;
        if (src < 0) continue;
        ts3 a = ts_from_double(w[2 * src]), b = ts_from_double(-w[2 * src + 1]);
        for (int k = 0; k < 3; ++k) {
            tv[(2 * 3 + k) * szN + j] = a.w[k];
            tv[(3 * 3 + k) * szN + j] = b.w[k];
        }
    }
    if (tr && tr->xprime)   /* x~' rounded to binary64, for inspection */
        for (int v = 0; v < 2; ++v)
            for (int64_t j = 0; j < N; ++j)
                tr->xprime[(size_t)v * szN + j] = ts_to_double(ts_make(tv[(v * 3) * szN + j], tv[(v * 3 + 1) * szN + j],
                                                                      tv[(v * 3 + 2) * szN + j]));

    /* Alg. 6 on the four TS vectors: level counts first, then the integers */
    for (int v = 0; v < 4 && status == OR_OK; ++v)
        status = or_ts_split(&tv[(size_t)v * 3 * szN], N, alpha, kcap, OR_KMAX, NULL, sexp[v], &kcount[v]);
    if (status != OR_OK) goto done;
    for (int v = 0; v < 4; ++v) kq = kcount[v] > kq ? kcount[v] : kq;
    q = (int64_t*)malloc(sizeof(int64_t) * 4 * (size_t)kq * szN);
    spec = (uint32_t*)malloc(sizeof(uint32_t) * 4 * (size_t)kq * nprimes * szN);
    gS = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)kq * kq);
    gsz = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)kq * kq);
    gp = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)kq * kq * kq * 2);
    if (!q || !spec || !gS || !gsz || !gp) { status = OR_ERR_ALLOC; goto done; }
    for (int v = 0; v < 4 && status == OR_OK; ++v) {
        int32_t kv;
        status = or_ts_split(&tv[(size_t)v * 3 * szN], N, alpha, kcap, kq, &q[(size_t)v * kq * szN], sexp[v], &kv);
    }
    if (status != OR_OK) goto done;

    /* residues and forward NTTs (Alg. 6 tail), as in the binary64 variant */
    for (int v = 0; v < 4; ++v)
        for (int k = 0; k < kcount[v]; ++k)
            for (int i = 0; i < nprimes; ++i) {
                int64_t p = (int64_t)OR_PRIMES[i];
                const int64_t* qk = &q[((size_t)v * kq + k) * szN];
                for (int64_t j = 0; j < N; ++j) {
                    int64_t a = qk[j] % p;
                    res[j] = (uint32_t)(a < 0 ? a + p : a);
                }
                or_ntt(res, &spec[(((size_t)v * kq + k) * nprimes + i) * szN], N, (uint64_t)p, 0);
                if (v < 2) ++nfr; else ++nfp;
            }

    /* Alg. 8 per real convolution, accumulating z'/c with TSAdd (T3, T4) */
    const size_t gstride = (size_t)kq * kq;
    for (int c = 0; c < 4; ++c) {
        int vx = CONV_X[c], vw = CONV_W[c];
        int ng = or_schedule(kcount[vx], sexp[vx], kcount[vw], sexp[vw], L, kq * kq, kq, &gS[c * gstride],
                             &gsz[c * gstride], &gp[c * gstride * kq * 2]);
        if (ng < 0) { status = OR_ERR_ARG; goto done; }
        if (tr) tr->ngroups[c] = ng;
        const int32_t* cp = &gp[c * gstride * kq * 2];
        for (int g = 0; g < ng; ++g) {
            for (int i = 0; i < nprimes; ++i) {
                uint64_t p = OR_PRIMES[i];
                uint32_t* Zi = &Z[(size_t)i * szN];
                memset(Zi, 0, sizeof(uint32_t) * szN);
                for (int m = 0; m < gsz[c * gstride + g]; ++m) {
                    int s = cp[((size_t)g * kq + m) * 2], t = cp[((size_t)g * kq + m) * 2 + 1];
                    const uint32_t* X = &spec[(((size_t)vx * kq + s) * nprimes + i) * szN];
                    const uint32_t* Y = &spec[(((size_t)vw * kq + t) * nprimes + i) * szN];
                    for (int64_t j = 0; j < N; ++j) Zi[j] = (uint32_t)((Zi[j] + mulmod(X[j], Y[j], p)) % p);
                }
                or_ntt(Zi, &zr[(size_t)i * szN], N, p, 1);
                ++ninv;
            }
            const int S = gS[c * gstride + g];
            uint32_t z3[3] = {0, 0, 0};
            for (int64_t j = 0; j < n; ++j) {
                for (int i = 0; i < nprimes; ++i) z3[i] = zr[(size_t)i * szN + j];
                const i128 zc = garner(z3, nprimes);
                acc[(size_t)c * n + j] = ts_add(acc[(size_t)c * n + j], ts_from_int_scaled((int64_t)zc, S));
            }
            if (tr && g < tr->gdim) {
                if (tr->gS) tr->gS[c * tr->gdim + g] = S;
                if (tr->gsize) tr->gsize[c * tr->gdim + g] = gsz[c * gstride + g];
                if (tr->gpairs)
                    for (int m = 0; m < gsz[c * gstride + g] && m < tr->kdim; ++m) {
                        tr->gpairs[(((size_t)c * tr->gdim + g) * tr->kdim + m) * 2] = cp[((size_t)g * kq + m) * 2];
                        tr->gpairs[(((size_t)c * tr->gdim + g) * tr->kdim + m) * 2 + 1] =
                            cp[((size_t)g * kq + m) * 2 + 1];
                    }
                if (tr->zres)
                    memcpy(&tr->zres[((size_t)c * tr->gdim + g) * nprimes * szN], zr,
                           sizeof(uint32_t) * nprimes * szN);
            }
        }
    }

    /* y' = (RR - II) + i (IR + RI), y = y' (.) w in TS, then binary64 (T4) */
    for (int64_t j = 0; j < n; ++j) {
        ts3 yr = ts_sub(acc[j], acc[(size_t)n + j]);
        ts3 yi = ts_add(acc[2 * (size_t)n + j], acc[3 * (size_t)n + j]);
        if (tr && tr->yprime) { tr->yprime[2 * j] = ts_to_double(yr); tr->yprime[2 * j + 1] = ts_to_double(yi); }
        ts3 c = wt[j], d = ts_from_double(w[2 * j + 1]);
        ts3 re = ts_sub(ts_mul(yr, c), ts_mul(yi, d));
        ts3 im = ts_add(ts_mul(yr, d), ts_mul(yi, c));
        double a = ts_to_double(re), b = ts_to_double(im);
        if (dir_conj(direction)) b = -b;
        if (dir_scaled(direction)) { a = a / (double)n; b = b / (double)n; }
        y[2 * j] = a;
        y[2 * j + 1] = b;
    }

done:
    if (tr) {
        tr->alpha = alpha;
        tr->rho = 24 - alpha;
        for (int v = 0; v < 4; ++v) {
            tr->kcount[v] = kcount[v];
            for (int k = 0; k < kcount[v] && k < OR_KMAX; ++k) tr->sexp[v][k] = sexp[v][k];
        }
        tr->n_fwd_runtime = nfr;
        tr->n_fwd_plan = nfp;
        tr->n_inv = ninv;
        if (tr->q && q)
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < kcount[v] && k < tr->kdim; ++k)
                    memcpy(&tr->q[((size_t)v * tr->kdim + k) * szN], &q[((size_t)v * kq + k) * szN], sizeof(int64_t) * szN);
        if (tr->spec && spec)
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < kcount[v] && k < tr->kdim; ++k)
                    memcpy(&tr->spec[(((size_t)v * tr->kdim + k) * nprimes) * szN],
                           &spec[(((size_t)v * kq + k) * nprimes) * szN], sizeof(uint32_t) * nprimes * szN);
    }
    free(w); free(tv); free(wt); free(acc); free(res); free(Z); free(zr);
    free(q); free(spec); free(gS); free(gsz); free(gp);
    return status;
}
