// k_peak.cu -- the denominator of the integer roofline: the throughput of the
// NTT butterflies alone, with every operand in registers (no memory traffic).
//
// Each thread runs CHAINS independent butterfly chains (enough instruction-
// level parallelism to hide the multiply latency) for `iters` rounds; the CT
// form is the forward NTT's (a, b) -> (a + bW, a - bW), the GS form the
// inverse's (a, b) -> (a + b, (a - b)W), both with canonical residues and a
// Shoup product (ntt_impl.cuh).  One butterfly = one modular multiplication.
#include "ntt_impl.cuh"

namespace oz {

namespace {
constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 8;
}

template <bool INV>
__global__ void __launch_bounds__(PEAK_THREADS) butterfly_peak_kernel(uint32_t* out, int iters, uint2 w0, uint2 w1)
{
    const uint32_t p = PRIME0;
    uint32_t a[CHAINS], b[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
        a[c] = (threadIdx.x * 2654435761u + c * 40503u + blockIdx.x) % p;
        b[c] = (threadIdx.x * 2246822519u + c * 9973u + blockIdx.x * 7u) % p;
    }
    for (int it = 0; it < iters; ++it) {
        const uint2 w = (it & 1) ? w1 : w0;
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            if (INV) bfly_gs(a[c], b[c], w, p);
            else bfly_ct(a[c], b[c], w, p);
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc ^= a[c] ^ b[c];
    out[blockIdx.x * PEAK_THREADS + threadIdx.x] = acc;
}

// butterflies per second over `blocks` CTAs (a multiple of the SM count)
cudaError_t measure_butterfly_rate(int inverse, int blocks, int iters, uint32_t* scratch, double* rate,
                                   cudaStream_t s)
{
    const uint64_t wv = 1234567ull, wv2 = 7654321ull;
    const uint2 w0 = make_uint2((uint32_t)wv, (uint32_t)((wv << 32) / PRIME0));
    const uint2 w1 = make_uint2((uint32_t)wv2, (uint32_t)((wv2 << 32) / PRIME0));
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        if (inverse) butterfly_peak_kernel<true><<<blocks, PEAK_THREADS, 0, s>>>(scratch, iters, w0, w1);
        else butterfly_peak_kernel<false><<<blocks, PEAK_THREADS, 0, s>>>(scratch, iters, w0, w1);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;   // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess)
        *rate = (double)blocks * PEAK_THREADS * (double)iters * CHAINS / (best / 1e3);
    return e;
}

}  // namespace oz
