// k_ts.cu -- the TS (triple-single) variant's pre-multiply and split for
// libozfft (§4.1, Alg. 4, Alg. 6).
//
//   ts_premul_kernel  x~' = x (.) w in TS (Alg. 4 step 2): TS(x), TS(w), then
//                     Re = TSSub(TSMul(Re x, Re w), TSMul(Im x, Im w)) and
//                     Im = TSAdd(TSMul(Re x, Im w), TSMul(Im x, Re w));
//   ts_wstar_kernel   w~* = ZeroPad+-(conj w, N) converted to TS (exact);
//   ts_split_kernel   one level of Alg. 6 on every TS vector: with
//                     mu = ||r0||_inf and sigma = 2^(ceil(log2 mu) + rho),
//                     x^(k) = fl32((r0 + sigma) - sigma), then
//                     (r0, r1) <- FastTwoSum(r0 - x^(k), r1) and
//                     (r1, r2) <- FastTwoSum(r1, r2); q = x^(k) 2^(alpha - e).
// A TS vector v (Re or Im of a signal) is three word planes r[v][0..2][N].
// The maxima mu[v][k] are kept as binary64 bit patterns of the binary32 value
// (exact), so the flush-schedule kernel reads them as in the binary64 variant.
#include "oz_common.cuh"
#include "oz_kernels.h"
#include "ts_arith.cuh"

namespace oz {

namespace {
constexpr int TS_THREADS = 256;
constexpr int TS_CHUNK = 4096;

__device__ __forceinline__ uint64_t umax64_ts(uint64_t a, uint64_t b) { return a > b ? a : b; }

__device__ __forceinline__ void block_umax_ts(uint64_t* dst, uint64_t v)
{
    __shared__ uint64_t redu[32];
    for (int o = 16; o > 0; o >>= 1) v = umax64_ts(v, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) redu[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? redu[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) v = umax64_ts(v, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o));
        if (lane == 0 && v) atomicMax((unsigned long long*)dst, (unsigned long long)v);
    }
}

// |w0| of a TS word as the bit pattern of the (exact) binary64 value
__device__ __forceinline__ uint64_t abs_bits(float w0)
{
    return (uint64_t)__double_as_longlong(fabs((double)w0));
}

__device__ __forceinline__ void store_ts(float* planes, int64_t N, int64_t j, ts3 t)
{
    planes[j] = t.w0;
    planes[N + j] = t.w1;
    planes[2 * N + j] = t.w2;
}

unsigned grid_ts(int64_t nvec, int64_t N) { return (unsigned)(nvec * ((N + TS_CHUNK - 1) / TS_CHUNK)); }
}  // namespace

__global__ void __launch_bounds__(TS_THREADS) ts_premul_kernel(const double2* __restrict__ x,
                                                               const double2* __restrict__ w, int64_t n, int64_t N,
                                                               int conj_in, float* __restrict__ r,
                                                               uint64_t* __restrict__ mu, int K, int* status)
{
    const int64_t chunks = (N + TS_CHUNK - 1) / TS_CHUNK;
    const int64_t b = blockIdx.x / chunks;
    const int64_t j0 = (blockIdx.x % chunks) * TS_CHUNK;
    const int64_t j1 = min(N, j0 + TS_CHUNK);
    float* rr = r + (2 * b) * 3 * N;
    float* ri = rr + 3 * N;
    uint64_t mr = 0, mi = 0;
    bool bad = false, range = false;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        ts3 re{0.0f, 0.0f, 0.0f}, im{0.0f, 0.0f, 0.0f};
        if (j < n) {
            const double2 xv = x[b * n + j];
            const double2 wv = w[j];
            if (!isfinite(xv.x) || !isfinite(xv.y)) bad = true;
            const ts3 a = ts_from_double(xv.x), bq = ts_from_double(conj_in ? -xv.y : xv.y);
            const ts3 c = ts_from_double(wv.x), d = ts_from_double(wv.y);
            re = ts_sub(ts_mul(a, c), ts_mul(bq, d));
            im = ts_add(ts_mul(a, d), ts_mul(bq, c));
            if (!isfinite(re.w0) || !isfinite(re.w1) || !isfinite(re.w2) || !isfinite(im.w0) || !isfinite(im.w1) ||
                !isfinite(im.w2))
                range = true;
        }
        store_ts(rr, N, j, re);
        store_ts(ri, N, j, im);
        mr = umax64_ts(mr, abs_bits(re.w0));
        mi = umax64_ts(mi, abs_bits(im.w0));
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    else if (range) atomicOr(status, ST_RANGE);
    block_umax_ts(&mu[(2 * b) * (K + 1)], mr);
    __syncthreads();
    block_umax_ts(&mu[(2 * b + 1) * (K + 1)], mi);
}

// w~* of the plan: vector 0 = Re, 1 = Im of ZeroPad+-(conj w, N), as TS
__global__ void __launch_bounds__(TS_THREADS) ts_wstar_kernel(const double2* __restrict__ w, int64_t n, int64_t N,
                                                              float* __restrict__ r, uint64_t* __restrict__ mu, int K)
{
    const int64_t chunks = (N + TS_CHUNK - 1) / TS_CHUNK;
    const int v = (int)(blockIdx.x / chunks);
    const int64_t j0 = (blockIdx.x % chunks) * TS_CHUNK;
    const int64_t j1 = min(N, j0 + TS_CHUNK);
    uint64_t m = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        int64_t src = -1;
        if (j < n) src = j;
        else if (N != n && j >= N - n + 1) src = N - j;
        double val = 0.0;
        if (src >= 0) {
            const double2 ws = w[src];
            val = v == 0 ? ws.x : -ws.y;   // conj(w)
        }
        const ts3 t = ts_from_double(val);
        store_ts(r + (int64_t)v * 3 * N, N, j, t);
        m = umax64_ts(m, abs_bits(t.w0));
    }
    block_umax_ts(&mu[(int64_t)v * (K + 1) + 0], m);
}

__global__ void __launch_bounds__(TS_THREADS) ts_split_kernel(int k, float* __restrict__ r, uint64_t* __restrict__ mu,
                                                              int64_t N, int K, int alpha, int P,
                                                              uint32_t* __restrict__ X, int write_r, int* status)
{
    const int64_t chunks = (N + TS_CHUNK - 1) / TS_CHUNK;
    const int64_t v = blockIdx.x / chunks;
    const int64_t j0 = (blockIdx.x % chunks) * TS_CHUNK;
    const int64_t j1 = min(N, j0 + TS_CHUNK);
    const uint64_t mub = mu[v * (K + 1) + k];
    if (mub == 0) return;                                 // level empty: mu^(k) = 0 ends the split
    const int e = ceil_log2_pos(__longlong_as_double((long long)mub));
    const int rho = 24 - alpha;
    if (e + rho > 127 || e + rho < -126) {
        if (threadIdx.x == 0) atomicOr(status, ST_RANGE);
        return;
    }
    const float sigma = __int_as_float((e + rho + 127) << 23);
    float* r0 = r + v * 3 * N;
    float* r1 = r0 + N;
    float* r2 = r1 + N;
    uint32_t* xk = X + ((v * K + k) * P) * N;
    uint64_t m = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const float a0 = r0[j];
        const float s = __fsub_rn(__fadd_rn(a0, sigma), sigma);
        float n0, t, n1, n2;
        f_fast_two_sum(__fsub_rn(a0, s), r1[j], n0, t);
        f_fast_two_sum(t, r2[j], n1, n2);
        const long long q = __float2ll_rz(f_scale_pow2(s, alpha - e));   // |q| <= 2^alpha < p
#pragma unroll
        for (int pi = 0; pi < MAX_PRIMES; ++pi) {
            if (pi >= P) break;
            const long long p = (long long)prime_of(pi);
            xk[pi * N + j] = (uint32_t)(q < 0 ? q + p : q);
        }
        if (write_r) {
            r0[j] = n0;
            r1[j] = n1;
            r2[j] = n2;
        }
        m = umax64_ts(m, abs_bits(n0));
    }
    if (k + 1 <= K) block_umax_ts(&mu[v * (K + 1) + k + 1], m);
}

cudaError_t launch_ts_premul(const double2* x, const double2* w, int64_t n, int64_t N, int64_t B, int conj_in,
                             float* r, uint64_t* mu, int K, int* status, cudaStream_t s)
{
    ts_premul_kernel<<<grid_ts(B, N), TS_THREADS, 0, s>>>(x, w, n, N, conj_in, r, mu, K, status);
    return cudaGetLastError();
}

cudaError_t launch_ts_wstar(const double2* w, int64_t n, int64_t N, float* r, uint64_t* mu, int K, cudaStream_t s)
{
    ts_wstar_kernel<<<grid_ts(2, N), TS_THREADS, 0, s>>>(w, n, N, r, mu, K);
    return cudaGetLastError();
}

cudaError_t launch_ts_split_level(int k, float* r, uint64_t* mu, int64_t N, int64_t nvec, int K, int alpha, int P,
                                  uint32_t* X, int write_r, int* status, cudaStream_t s)
{
    ts_split_kernel<<<grid_ts(nvec, N), TS_THREADS, 0, s>>>(k, r, mu, N, K, alpha, P, X, write_r, status);
    return cudaGetLastError();
}

}  // namespace oz
