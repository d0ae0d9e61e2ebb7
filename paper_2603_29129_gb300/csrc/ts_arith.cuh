// ts_arith.cuh -- TS (triple-single) arithmetic for the TS variant of the
// method (§4.1, Alg. 4, Alg. 6, Alg. 8).
//
// A TS number is a triple of binary32 words w0 + w1 + w2 (§4.1).  TSAdd and
// TSMul follow the triple-word arithmetic of Fabiano, Muller and Picot (2019):
// exact transformations (2Sum, Fast2Sum, 2Prod with an FMA) produce the
// partial terms, VecSum adds them without error into a decreasing sequence,
// and the VecSumErrBranch renormalisation keeps three words.
//   TSAdd: the six words merged by decreasing magnitude, VecSum, renormalised;
//   TSMul: the products of weight 1 and 2^-24 exactly, those of weight 2^-48
//          rounded, the rest dropped; VecSum, renormalised.
// Every operation is an explicitly rounded intrinsic, so nothing is contracted
// into an FMA behind the algorithm's back.  Conversions:
//   from binary64: w0 = RN32(x), w1 = RN32(x - w0), w2 = RN32(x - w0 - w1)
//                  (the differences are exact in binary64);
//   to binary64:   (w0 + w1) + w2 in binary64, the exact sum rounded once;
//   from an integer z (|z| < 2^62) times 2^-S: z split exactly into three
//                  words of at most 24 bits, each scaled by 2^-S.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace oz {

struct ts3 {
    float w0, w1, w2;
};

__device__ __forceinline__ void f_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float aa = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

__device__ __forceinline__ void f_fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void f_two_prod(float a, float b, float& p, float& e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// VecSum over M words: x[0] <- the running sum from the last word up, x[1..M)
// <- the exact errors (the total is unchanged)
template <int M>
__device__ __forceinline__ void f_vec_sum(float (&x)[M])
{
    float s = x[M - 1];
#pragma unroll
    for (int i = M - 2; i >= 0; --i) {
        float e;
        f_two_sum(x[i], s, s, e);
        x[i + 1] = e;
    }
    x[0] = s;
}

// VecSumErrBranch: renormalise e[0..M) into three words
template <int M>
__device__ __forceinline__ ts3 f_vec_sum_err_branch(const float (&e)[M])
{
    float r[3] = {0.0f, 0.0f, 0.0f};
    int j = 0;
    bool full = false;
    float eps = e[0];
#pragma unroll
    for (int i = 1; i < M; ++i) {
        if (!full) {
            float s, t;
            f_fast_two_sum(eps, e[i], s, t);
            if (t != 0.0f) {
                if (j == 0) r[0] = s; else if (j == 1) r[1] = s; else r[2] = s;
                if (j == 2) full = true;
                else { ++j; eps = t; }
            } else {
                eps = s;
            }
        }
    }
    if (!full) {
        if (j == 0) r[0] = eps; else if (j == 1) r[1] = eps; else r[2] = eps;
    }
    return {r[0], r[1], r[2]};
}

__device__ __forceinline__ ts3 ts_neg(ts3 a) { return {-a.w0, -a.w1, -a.w2}; }

__device__ __forceinline__ ts3 ts_add(ts3 a, ts3 b)
{
    const float av[3] = {a.w0, a.w1, a.w2}, bv[3] = {b.w0, b.w1, b.w2};
    float z[6];
    int i = 0, j = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        // merge by decreasing magnitude (ties take a's word first)
        const float ai = i == 0 ? av[0] : (i == 1 ? av[1] : av[2]);
        const float bj = j == 0 ? bv[0] : (j == 1 ? bv[1] : bv[2]);
        if (j >= 3 || (i < 3 && fabsf(ai) >= fabsf(bj))) { z[k] = ai; ++i; }
        else { z[k] = bj; ++j; }
    }
    f_vec_sum<6>(z);
    return f_vec_sum_err_branch<6>(z);
}

__device__ __forceinline__ ts3 ts_sub(ts3 a, ts3 b) { return ts_add(a, ts_neg(b)); }

__device__ __forceinline__ ts3 ts_mul(ts3 a, ts3 b)
{
    float z00, e00, z01, e01, z10, e10;
    f_two_prod(a.w0, b.w0, z00, e00);
    f_two_prod(a.w0, b.w1, z01, e01);
    f_two_prod(a.w1, b.w0, z10, e10);
    float t[9] = {z00, z01, z10, e00, __fmul_rn(a.w0, b.w2), __fmul_rn(a.w1, b.w1), __fmul_rn(a.w2, b.w0), e01, e10};
    f_vec_sum<9>(t);
    return f_vec_sum_err_branch<9>(t);
}

__device__ __forceinline__ ts3 ts_from_double(double x)
{
    const float a = __double2float_rn(x);
    const double r1 = __dsub_rn(x, (double)a);
    const float b = __double2float_rn(r1);
    const float c = __double2float_rn(__dsub_rn(r1, (double)b));
    return {a, b, c};
}

__device__ __forceinline__ double ts_to_double(ts3 a)
{
    return __dadd_rn(__dadd_rn((double)a.w0, (double)a.w1), (double)a.w2);
}

// x 2^e in binary32 steps, each a product by a normal power of two
__device__ __forceinline__ float f_scale_pow2(float x, int e)
{
    while (e > 127) { x = __fmul_rn(x, 0x1p127f); e -= 127; }
    while (e < -126) { x = __fmul_rn(x, 0x1p-126f); e += 126; }
    return __fmul_rn(x, __int_as_float((e + 127) << 23));
}

__device__ __forceinline__ ts3 ts_from_int_scaled(long long z, int S)
{
    const float a = __ll2float_rn(z);
    const long long r1 = z - __float2ll_rz(a);
    const float b = __ll2float_rn(r1);
    const long long r2 = r1 - __float2ll_rz(b);
    const float c = __ll2float_rn(r2);
    return {f_scale_pow2(a, -S), f_scale_pow2(b, -S), f_scale_pow2(c, -S)};
}

// exact ceil(log2 m) of a positive binary32
__device__ __forceinline__ int ceil_log2_f(float m)
{
    const unsigned u = __float_as_uint(m);
    const int E = (int)((u >> 23) & 0xff);
    unsigned mant = u & 0x7fffffu;
    if (E == 0) {   // subnormal: m = mant 2^-149
        const int lead = 31 - __clz((int)mant);
        return (mant & (mant - 1)) ? lead - 149 + 1 : lead - 149;
    }
    return mant == 0 ? E - 127 : E - 126;
}

}  // namespace oz
