// k_ntt_col_tma.cu -- the NTT column pass (stages 0..m1-1, ntt_impl.cuh) with
// its tile moved by the tensor memory accelerator: one thread issues
// cp.async.bulk.tensor loads of the T-column x 2^m1-row tile into shared
// memory (completion counted on an mbarrier), the CTA runs the column rounds on
// the dense tile, and one thread stores it back with cp.async.bulk.tensor.
// With T >= 32 consecutive lanes work on consecutive columns, so the dense
// layout is free of bank conflicts without pad words.  Used for m1 >= 4
// (T <= 256 columns, the limit of one box dimension); boxes of at most 256
// rows are stacked along the rows.
//
// The wait on the mbarrier is bounded: after TMA_WAIT_LIMIT polls (with a
// short sleep between them) the CTA records ST_TIMEOUT in the status word,
// waits once more (bounded) for its copy, and returns without transforming.
#include "ntt_impl.cuh"

namespace oz {

namespace {
constexpr int TMA_WAIT_LIMIT = 1 << 20;   // polls of ~0.1-1 us: a copy of a few KB completes in microseconds

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t phase)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(phase) : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase)
{
    for (int i = 0; i < TMA_WAIT_LIMIT; ++i) {
        if (mbar_test(bar, phase)) return true;
        __nanosleep(64);
    }
    return false;
}
}  // namespace

template <bool INV, int M1>
__global__ void __launch_bounds__(NTT_THREADS, 8) ntt_col_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                     NttGeom g, const uint2* __restrict__ tw_all)
{
    extern __shared__ uint32_t sm_raw[];
    __shared__ alignas(8) uint64_t bar;
    constexpr int LOG_T = col_log_t(M1), T = 1 << LOG_T;
    constexpr int ROWS = 1 << M1, BOX_R = ROWS < 256 ? ROWS : 256, NBOX = ROWS / BOX_R;
    constexpr uint32_t BOX_WORDS = (uint32_t)T * BOX_R, BYTES = (uint32_t)T * ROWS * 4u;
    static_assert(T <= 256, "one box dimension holds at most 256 columns");
    // the tile at the first 128-byte boundary of the dynamic shared memory
    uint32_t* sm = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~uintptr_t(127));
    const int lg_tpv = g.m2 - LOG_T;                   // tiles per vector = N2 / T
    const unsigned vec = blockIdx.x >> lg_tpv;
    const int col0 = (int)(blockIdx.x & ((1u << lg_tpv) - 1)) << LOG_T;
    if (INV ? !inv_live(g, vec) : !fwd_live(g, vec)) return;
    const int pi = (int)(vec - udiv_small(vec, (unsigned)g.P) * (unsigned)g.P);
    const int zc = (int)(vec + g.vec0);
    const uint32_t sma = smem_addr(sm), bara = smem_addr(&bar);
    const uint64_t map = reinterpret_cast<uint64_t>(&tmap);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bara) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bara), "r"(BYTES + g.extra_tx)
                     : "memory");
#pragma unroll
        for (int b = 0; b < NBOX; ++b)
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                         " [%0], [%1, {%2, %3, %4}], [%5];"
                         ::"r"(sma + b * BOX_WORDS * 4u), "l"(map), "r"(col0), "r"(b * BOX_R), "r"(zc), "r"(bara)
                         : "memory");
    }
    __syncthreads();                                   // the barrier is initialised before anyone polls it
    if (!mbar_wait_bounded(bara, 0)) {
        if (threadIdx.x == 0) {
            atomicOr(g.status, ST_TIMEOUT);
            mbar_wait_bounded(bara, 0);                // let the copy land before the CTA leaves
        }
        return;
    }
    const PassArgs a{T, 1, 0, tw_all, g.N, pi, g.P, false};
    run_rounds<INV, true, M1, LOG_T, 0, false>(sm, a);   // ends with __syncthreads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the tile's writes, visible to the copy engine
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < NBOX; ++b)
            asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];"
                         ::"l"(map), "r"(sma + b * BOX_WORDS * 4u), "r"(col0), "r"(b * BOX_R), "r"(zc)
                         : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // the tile stays until it is read
    }
}

template <bool INV, int M1>
static cudaError_t launch_col_tma_m(const NttGeom& g, const uint2* tw, cudaStream_t s)
{
    constexpr int64_t tile = (int64_t(1) << col_log_t(M1)) << M1;
    const size_t smem = (size_t)tile * sizeof(uint32_t) + 128;
    cudaError_t e = ntt_prep(ntt_col_tma_kernel<INV, M1>, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = g.nvec * ((int64_t(1) << g.m2) >> col_log_t(M1));
    ntt_col_tma_kernel<INV, M1><<<(unsigned)grid, NTT_THREADS, smem, s>>>(*g.tmap, g, tw);
    return cudaGetLastError();
}

// the TMA column pass for m1 = 4..10; false: not handled here
bool launch_col_tma(bool inv, const NttGeom& g, const uint2* tw, cudaStream_t s, cudaError_t* err)
{
    if (!g.tmap || g.m1 < 4 || g.m1 > 10) return false;
    switch (g.m1) {
    case 4: *err = inv ? launch_col_tma_m<true, 4>(g, tw, s) : launch_col_tma_m<false, 4>(g, tw, s); break;
    case 5: *err = inv ? launch_col_tma_m<true, 5>(g, tw, s) : launch_col_tma_m<false, 5>(g, tw, s); break;
    case 6: *err = inv ? launch_col_tma_m<true, 6>(g, tw, s) : launch_col_tma_m<false, 6>(g, tw, s); break;
    case 7: *err = inv ? launch_col_tma_m<true, 7>(g, tw, s) : launch_col_tma_m<false, 7>(g, tw, s); break;
    case 8: *err = inv ? launch_col_tma_m<true, 8>(g, tw, s) : launch_col_tma_m<false, 8>(g, tw, s); break;
    case 9: *err = inv ? launch_col_tma_m<true, 9>(g, tw, s) : launch_col_tma_m<false, 9>(g, tw, s); break;
    default: *err = inv ? launch_col_tma_m<true, 10>(g, tw, s) : launch_col_tma_m<false, 10>(g, tw, s); break;
    }
    return true;
}

cudaError_t col_tma_timeout_selftest(int* status_host, cudaStream_t s)
{
    // one live vector of N = 2^16 (m1 = 4: 16 tiles of 256 columns x 16 rows) in fresh memory
    NttGeom g{};
    ntt_configure(g, int64_t(1) << 16);
    g.nvec = 1;
    g.P = 1;
    g.K = 1;
    g.G = 1;
    g.extra_tx = 4096;                                 // never delivered: the bounded wait must give up
    uint32_t* data = nullptr;
    uint2* tw = nullptr;
    int32_t* kcnt = nullptr;
    int* status = nullptr;
    CUtensorMap map;
    cudaError_t e = cudaMalloc((void**)&data, sizeof(uint32_t) << 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&tw, sizeof(uint2) << 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&kcnt, 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(data, 0, sizeof(uint32_t) << 16);
    if (e == cudaSuccess) e = cudaMemset(tw, 0, sizeof(uint2) << 16);
    const int32_t live[2] = {1, 1};
    if (e == cudaSuccess) e = cudaMemcpy(kcnt, live, sizeof live, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
    if (e == cudaSuccess && !ntt_make_tmap(&map, g, data, 1)) e = cudaErrorNotSupported;
    if (e == cudaSuccess) {
        g.kcnt = kcnt;
        g.tmap = &map;
        g.status = status;
        if (!launch_col_tma(false, g, tw, s, &e)) e = cudaErrorNotSupported;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(status_host, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(data);
    cudaFree(tw);
    cudaFree(kcnt);
    cudaFree(status);
    return e;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool ntt_make_tmap(CUtensorMap* map, const NttGeom& g, uint32_t* base, int64_t nvec)
{
    if (g.m1 < 4 || g.m1 > 10 || nvec < 1 || nvec > 0x7fffffff) return false;
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<EncodeTiled>(fn);
    }
    const int T = 1 << col_log_t(g.m1), rows = 1 << g.m1;
    const cuuint64_t dims[3] = {(cuuint64_t)1 << g.m2, (cuuint64_t)rows, (cuuint64_t)nvec};
    const cuuint64_t strides[2] = {((cuuint64_t)1 << g.m2) * 4u, (cuuint64_t)g.N * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)T, (cuuint32_t)(rows < 256 ? rows : 256), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace oz
