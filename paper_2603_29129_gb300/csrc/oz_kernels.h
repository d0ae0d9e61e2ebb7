// oz_kernels.h -- kernel launch interface between the plan (plan.cu) and the
// kernel translation units of libozfft.  Internal; not part of the C ABI.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "oz_common.cuh"

namespace oz {

// Per-signal layout of a plan over signals of uneven lengths.  Such a plan is
// cut into length classes (one convolution length N each); a class's kernels
// read its signals' descriptors.  Plans whose signals all have one length pass
// null and use the plan's n.
struct SigDesc {
    int64_t n;          // signal length
    int64_t io_off;     // first element of the signal in the packed input and output
    int64_t chirp_off;  // first entry of its chirp table w(0..n) in the class's chirp pool
    int32_t alpha;      // split width of this n (§4.4)
    int32_t pad;
};

// Input and output base pointers held in device memory, so that a captured
// CUDA graph reads the buffers of the current execution (null: use the
// pointers passed to the launch).
struct IoPtrs {
    const double2* in;
    double2* out;
};

// Geometry of one batched NTT launch (forward or inverse).
struct NttGeom {
    int64_t N;          // transform length 2^lgN
    int64_t nvec;       // vectors in the launch
    int lgN, m1, m2;    // column-pass stages m1 (0: single pass), row-pass stages m2
    int T;              // columns per CTA in the column pass
    int rows_per_cta;   // contiguous 2^m2 blocks per CTA in the row pass
    int P, K, G;        // primes, split cap, flush-group capacity
    const int32_t* kcnt;   // [B][2] live split levels of x~' (forward skip test)
    const Sched* sched;    // [B][4] flush schedules (inverse skip test and MAC)
    int merged;            // schedules merge the two convolutions of each output part
    int mac_reg;           // L = 1 or merged schedules: the inverse row pass forms the Alg. 8
                           // sums in registers instead of staging them in shared memory
    int inv_vecs_per_cta;  // inverse row pass with the MAC in registers: vectors of one prime
                           // per CTA (1, or 2 to share every twiddle load between two vectors)
    const CUtensorMap* tmap;   // column pass by tensor memory access: [vectors][2^m1][2^m2] map of the
                               // buffer (null: per-thread loads); host memory, passed by value
    int64_t vec0;          // index of the launch's first vector in that map
    int* status;           // status word for bounded waits that give up
    uint32_t extra_tx;     // self-test only: bytes the barrier expects beyond the tile (0)
    const int32_t* redo;   // forward column pass after the fused split: [B][2] nonzero for the real
                           // vectors split_fix_kernel redid (only those are transformed); null: all
};

// tensor map of a buffer of nvec vectors of 2^m1 x 2^m2 residues, box = one
// column tile of the column pass (false when the geometry has no TMA kernel)
bool ntt_make_tmap(CUtensorMap* map, const NttGeom& g, uint32_t* base, int64_t nvec);
// k_ntt_col_tma.cu: the column pass by tensor memory access when g.tmap is set
// and m1 >= 4; returns false (nothing launched) otherwise
bool launch_col_tma(bool inv, const NttGeom& g, const uint2* tw, cudaStream_t s, cudaError_t* err);
// self-test of the bounded wait: one forward column-pass tile (N = 2^16) whose
// barrier expects more bytes than its copy brings; *status receives the status bits
cudaError_t col_tma_timeout_selftest(int* status_host, cudaStream_t s);

// vectors per CTA of the inverse row pass with the MAC in registers when the plan
// does not choose (the autotuner times 1 and 2; with the schedules of real
// inputs the two are within a few percent at n = 2^18 x 64)
constexpr int INV_ROW_VECS = 1;

// Inputs of the multiply-accumulate fused into the inverse NTT's load.
struct MacSrc {
    const uint32_t* X;   // [B][2][K][P][N] forward spectra of x~' slices
    const uint32_t* Ym;  // [2][K][P][N]   w~* spectra * N^-1 * 2^32 mod p (per signal when ym_stride > 0)
    int64_t ym_stride;   // elements between consecutive signals' Ym (0: one Ym for the whole batch)
};

// k_ntt.cu
void ntt_configure(NttGeom& g, int64_t N);   // fills lgN, m1, m2, T, rows_per_cta
// the same with the row pass forced to 2^m2 residues (autotuning); false when
// no kernel instantiation covers that split
bool ntt_configure_split(NttGeom& g, int64_t N, int m2);
int64_t ntt_launches(const NttGeom& g);        // kernels per transform direction
// one pass each; a transform is col+row (forward) or row+col (inverse), the
// column pass only when g.m1 > 0
cudaError_t launch_ntt_fwd_col(const NttGeom& g, uint32_t* X, const uint2* tw, cudaStream_t s);
cudaError_t launch_ntt_fwd_row(const NttGeom& g, uint32_t* X, const uint2* tw, cudaStream_t s);
cudaError_t launch_ntt_inv_row(const NttGeom& g, uint32_t* Z, const uint2* twinv, MacSrc mac, cudaStream_t s);
cudaError_t launch_ntt_inv_col(const NttGeom& g, uint32_t* Z, const uint2* twinv, cudaStream_t s);
cudaError_t launch_ntt_forward(const NttGeom& g, uint32_t* X, const uint2* tw, cudaStream_t s);

// k_split.cu
// sd (optional, [B]): per-signal lengths, offsets and split widths; io
// (optional): device-held input/output pointers
cudaError_t launch_chirp(double2* w, int64_t n, cudaStream_t s);
cudaError_t launch_wstar(const double2* w, int64_t n, int64_t N, int64_t B, const SigDesc* sd, double* r,
                         uint64_t* mu, int K, int* status, cudaStream_t s);
cudaError_t launch_premul(const double2* x, const double2* w, int64_t n, int64_t N, int64_t B, int conj_in,
                          const SigDesc* sd, const IoPtrs* io, double* r, uint64_t* mu, int K, int* status,
                          cudaStream_t s);
cudaError_t launch_split_level(int k, double* r, const uint64_t* mu_in, uint64_t* mu_out, int64_t N,
                               int64_t nvec, int K, int alpha, const SigDesc* sd, int P, uint32_t* X, int write_r,
                               int* status, cudaStream_t s);
// every level at once with guessed exponents, then a per-vector check that
// redoes the vectors whose residual maxima contradict the guess (2 kernels)
cudaError_t launch_split_spec(double* r, uint64_t* mu, int64_t N, int64_t nvec, int K, int alpha, const SigDesc* sd,
                              int P, uint32_t* X, int* status, cudaStream_t s);
constexpr int SPLIT_SPEC_LAUNCHES = 2;
// the same split fused with the forward NTT's column pass (stages 0..m1-1, table
// tw): every level's residues are transformed on chip before they reach X.
// Vectors whose guessed level exponents fail are redone untransformed by the
// check kernel, which sets redo[v]; a column pass with NttGeom.redo = redo must
// follow (after the schedule).  split_col_supported tells where it applies.
bool split_col_supported(int K, int P, int m1, int m2);
cudaError_t launch_split_col(double* r, uint64_t* mu, int64_t N, int m1, int m2, int64_t nvec, int K, int alpha,
                             const SigDesc* sd, int P, uint32_t* X, const uint2* tw, int32_t* redo, int* status,
                             cudaStream_t s);
cudaError_t launch_set_io(IoPtrs* io, const void* in, void* out, cudaStream_t s);

// k_crt.cu
struct CrtArgs {
    const uint32_t* Z;     // [B][4][G][P][N] inverse NTT outputs (natural order)
    const Sched* sched;    // [B][4]
    const int32_t* span;   // [B][3] min S, max S, any group
    const double2* w;      // [n] chirp (a chirp pool with per-signal offsets when sd is set)
    double2* out;          // [B][n] (packed per-signal offsets when sd is set)
    int64_t n, N, B;       // n: the signals' length (their largest when sd is set)
    int P, G, direction;
    int* status;           // data-dependent status bits
    const SigDesc* sd;     // [B] per-signal lengths and offsets, or null
    const IoPtrs* io;      // device-held output pointer, or null
    int merged;            // merged schedules: the MAC already applied the sign of II
    int garner_u;          // |z| < p0 p1 / 2 - p0 for every value: two-prime CRT without centering z0
    int fused;             // colcrt_kernel already produced the Horner-path signals' outputs
};
int crt_launches();        // kernels per launch_crt_post
cudaError_t crt_init();    // uploads the Garner constants (once; call before any stream capture)
cudaError_t launch_crt_post(const CrtArgs& a, cudaStream_t s);
cudaError_t launch_crt_ts(const CrtArgs& a, cudaStream_t s);   // TS variant (two primes)
// the inverse NTT's column pass (stages 0..m1-1 of Z, table tw) fused with the
// CRT for the Horner-path signals; the others get the column pass only (plain
// plans: a.sd must be null)
bool colcrt_supported(int P, int m1, int m2, bool merged);
cudaError_t launch_colcrt(const CrtArgs& a, int m1, int m2, const uint2* tw, cudaStream_t s);

// k_peak.cu: butterflies per second with every operand in registers
cudaError_t measure_butterfly_rate(int inverse, int blocks, int iters, uint32_t* scratch, double* rate,
                                   cudaStream_t s);

// k_ts.cu: the TS variant's pre-multiply, w~* and split (TS vectors are three
// binary32 word planes r[v][0..2][N])
cudaError_t launch_ts_premul(const double2* x, const double2* w, int64_t n, int64_t N, int64_t B, int conj_in,
                             float* r, uint64_t* mu, int K, int* status, cudaStream_t s);
cudaError_t launch_ts_wstar(const double2* w, int64_t n, int64_t N, float* r, uint64_t* mu, int K, cudaStream_t s);
cudaError_t launch_ts_split_level(int k, float* r, uint64_t* mu, int64_t N, int64_t nvec, int K, int alpha, int P,
                                  uint32_t* X, int write_r, int* status, cudaStream_t s);

}  // namespace oz
