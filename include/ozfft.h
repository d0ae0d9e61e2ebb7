/*
 * ozfft.h -- C ABI of libozfft, a GB300 (sm_103a) implementation of the
 * double-precision FFT of "Computing FFTs at Target Precision Using
 * Lower-Precision FFTs" (arXiv 2603.29129).
 *
 * What one transform computes (forward direction), step by step:
 *   1. x'(j) = x(j) * w(j), w(j) = exp(-i pi j^2 / n)            Alg. 1, §3.2
 *   2. x~' = ZeroPad(x', N), w~* = ZeroPad+-(conj(w), N)           §3.2
 *   3. each of Re x~', Im x~', Re w~*, Im w~* is split into at most K integer
 *      slices q^(k) with |q^(k)| <= 2^alpha and scale c^(k) = 2^(s_k)      Alg. 3
 *      alpha = max{a : L n 2^(2a) < P/2}, P = product of the primes       §4.2, §4.4
 *   4. residues of every slice modulo each prime, forward 32-bit NTTs    §3.3, Alg. 6
 *   5. for each of the four real convolutions (RR, II, IR, RI, §4.5), the
 *      slice products with equal scale are summed in the NTT domain, at most
 *      L at a time (Alg. 8), and each sum is inverse-transformed           §4.4
 *   6. Garner CRT of the per-prime results (symmetric digits, Eq. (1))     §3.3
 *   7. rescale by 1/(c_x c_y) and accumulate: the exact integer sum of every
 *      group's term, rounded once to binary64 (the sum Alg. 8's TSAdd
 *      accumulation approximates)                                        Alg. 8
 *   8. y(k) = y'(k) * w(k)                                               Alg. 1
 * The inverse direction is conj -> forward -> conj -> divide by n (Eq. (4)).
 * Steps 1-8 all run in this library's CUDA kernels; w~*'s split and forward
 * NTTs (steps 2-4 for w~*) run once, when the plan is made (§4.5).
 *
 * Conventions for every function below:
 *   - complex data are interleaved binary64 pairs (re, im), i.e. the layout of
 *     a C `double _Complex` array or a contiguous torch.complex128 tensor;
 *     batched data are [batch][n], signal after signal;
 *   - "device pointer" means memory of the plan's CUDA device (cudaMalloc,
 *     torch CUDA tensors); "host pointer" means ordinary or pinned host memory;
 *   - the caller owns every buffer it passes; the plan owns its own tables and
 *     workspace and frees them in ozfft_destroy;
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that take a stream are asynchronous with respect to the
 *     host unless stated otherwise;
 *   - argument errors are returned synchronously as OZFFT_ERR_* codes; errors
 *     that depend on the data (non-finite input, exponent overflow) are
 *     recorded on the device and read with ozfft_get_status.
 */
#ifndef OZFFT_H
#define OZFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ozfft_plan_s* ozfft_plan_t;

/* Directions.  FORWARD: y = F x, F(k,j) = exp(-2 pi i jk/n) (Eq. (3)); INVERSE:
   y = (1/n) F^H x (Eq. (4)).  The two adjoints serve reverse-mode
   differentiation (the gradient of a real loss through a linear map A is A^H
   applied to the output gradient): ADJOINT: y = F^H x = conj(F conj x), the
   inverse without its division by n; INVERSE_ADJOINT: y = (1/n) F x, the forward
   transform with every component divided by n (one rounding). */
enum { OZFFT_FORWARD = -1, OZFFT_INVERSE = +1, OZFFT_ADJOINT = +2, OZFFT_INVERSE_ADJOINT = -2 };

enum {
    OZFFT_OK = 0,
    OZFFT_ERR_ARG = 1,       /* bad argument (null pointer, n < 1, batch < 1, K/L/nprimes out of range) */
    OZFFT_ERR_LENGTH = 2,    /* convolution length N is not a power of two, exceeds 2^24 (the 2-adic
                                order of p0 - 1), is shorter than 2n-1 without being n, or alpha < 1 */
    OZFFT_ERR_ALLOC = 3,     /* device or host allocation failed */
    OZFFT_ERR_CUDA = 4,      /* a CUDA runtime call failed (ozfft_last_error has the text) */
    OZFFT_ERR_NONFINITE = 5, /* device status: the input held a NaN or an infinity */
    OZFFT_ERR_RANGE = 6,     /* device status: 2^(ceil(log2 max|v|) + 53 - alpha) overflows binary64 */
    OZFFT_ERR_TIMEOUT = 7,   /* device status: a bounded device-side wait (the column pass's tile
                                barrier) gave up; the output of that execution is not valid */
    OZFFT_ERR_LEVELS = 8     /* device status (K = OZFFT_K_INF): a real vector still had a nonzero
                                residual after OZFFT_K_INF_CAP split levels; its result is that of
                                K = OZFFT_K_INF_CAP, not of K = infinity */
};

/* ozfft_options.K = OZFFT_K_INF selects K = infinity of §4.4 (Alg. 3 runs until the
   residual is zero, so the split is error free): every real vector gets as many
   levels as it needs, at most OZFFT_K_INF_CAP; the workspace is sized for the
   cap (G = 64 flush groups per convolution). */
enum { OZFFT_K_INF = -1, OZFFT_K_INF_CAP = 8 };

/* Plan options.  A zero field selects the default. */
typedef struct {
    int32_t K;        /* split cap K of §4.4 (default 3; 1..8, or OZFFT_K_INF for K = infinity) */
    int32_t L;        /* NTT-domain accumulation bound L of §4.4 (default 1 = none; 1..8) */
    int32_t nprimes;  /* 2 (default: p0 = 2130706433, p1 = 2113929217, §5.1) or 3 (adds 2013265921) */
    int64_t conv_len; /* cyclic length N (default: n if n is a power of two, else the least power of
                         two >= 2n-1; §3.2) */
    int32_t debug;    /* nonzero: keep the slice residues of each execution for ozfft_debug_dump
                         (costs one extra copy per execution; for tests) */
    int32_t chunk;    /* signals per inverse-stage chunk: the inverse NTTs and the CRT stage run
                         chunk by chunk, which bounds the inverse-NTT buffer to chunk signals
                         (default: the whole batch while that buffer fits in 16 GiB; debug plans
                         always use the whole batch) */
    int32_t autotune; /* nonzero: at plan time, time every supported split of each NTT length
                         into column and row passes (row tiles of 2^10 .. 2^14 residues) on the
                         plan's own buffers and keep the fastest; results are bit-identical */
    int32_t no_graph; /* plans over uneven lengths: nonzero runs the length classes on
                         concurrent streams without capturing them in a CUDA graph */
    int32_t merge;    /* nonzero: NTT-domain accumulation (§4.5) also across the two real
                         convolutions that feed one output part (RR with -II, IR with RI): their
                         equal-scale products share inverse NTTs, at most L per group.  With
                         L >= 2 this cuts the inverse NTTs and CRT reads (L = 2: 36 instead of 48
                         per transform and prime pair without gaps); the result is bit-identical
                         to merge = 0 with the same L, since y' is the exactly rounded sum of the
                         same products either way */
    int32_t row_log;  /* nonzero: stages of the NTT row pass (10..14, the rest in the column pass) for
                         both directions, instead of the default split or the autotuner's choice;
                         OZFFT_ERR_ARG if no kernel covers that split of N */
    int32_t ts;       /* nonzero: the TS (triple-single) variant of §4.1 (Alg. 4, Alg. 6, Alg. 8):
                         chirp products and the split in TS arithmetic (three binary32 words,
                         rho = 24 - alpha, alpha capped at 23), the rescaled CRT integers
                         accumulated per real convolution with TSAdd, the post-multiply in TS and
                         the result rounded to binary64.  Two primes, plain plans only; inputs
                         must stay inside the binary32 exponent range (else OZFFT_ERR_RANGE) */
    int32_t inv_vecs; /* inverse NTT row pass with the Alg. 8 sums formed in registers (L = 1 or
                         merged schedules, N >= 2^12, row tiles up to 2^12): vectors of one prime per
                         CTA (2: the same group of RR and RI, or of II and IR, sharing every twiddle
                         load).  0: 1 (or the autotuner's choice), 1 or 2 to force; results are
                         bit-identical */
    int32_t crt_fuse; /* inverse NTT column pass fused with Garner's CRT and the exact accumulation
                         (two primes, 4..8 column stages): 0 = default (fused for plain plans,
                         separate kernels for the length classes of uneven plans, or the
                         autotuner's choice per class), 1 = fused wherever supported, 2 = never
                         fused; results are bit-identical */
    int32_t split_fuse; /* the Ozaki split fused with the forward NTT's column pass (K <= 4, K P <= 9,
                         5..8 column stages): the slice residues are transformed on chip before they
                         reach device memory.  0 = apart (with autotune: the faster of fused and
                         apart, timed), 1 = wherever supported, 2 = never; never for debug or TS
                         plans; results are bit-identical */
} ozfft_options;

/* Create a plan for `batch` transforms of length n in `direction`, with default
   options, on the current CUDA device.  Returns NULL on error (see
   ozfft_last_error).  Synchronous: it computes the chirp table, the twiddle
   tables and the split + forward NTTs of w~* on the device and allocates the
   workspace for `batch` signals. */
ozfft_plan_t ozfft_plan(int64_t n, int64_t batch, int direction);

/* Same with explicit options (NULL = defaults). */
ozfft_plan_t ozfft_plan_ex(int64_t n, int64_t batch, int direction, const ozfft_options* opt);

/* A plan for `count` transforms of uneven lengths lengths[0..count) (each >= 1,
   any mix of powers of two and other lengths), computed exactly as ozfft_plan_ex
   would compute each signal alone (Alg. 1 around Alg. 8, §4.5; the arbitrary-
   length case of §5.6).  Input and output are packed: signal i occupies the
   complex128 elements [o_i, o_i + lengths[i]) with o_i = lengths[0] + ... +
   lengths[i-1].  The signals are grouped by convolution length N; every group
   runs batched (one launch per kernel and group, each signal's own chirp table,
   w~* spectra and split width alpha), the groups run as concurrent branches of
   one CUDA graph captured at plan time (or on concurrent streams with
   opt->no_graph), and the inverse-NTT buffers of all groups together are
   bounded by 16 GiB unless opt->chunk sets the signals per chunk.  opt->conv_len
   and opt->debug must be 0.  ozfft_execute, ozfft_execute_host, ozfft_get_status,
   ozfft_get_stats (n = total elements, N = the largest N, batch = count, alpha =
   the smallest alpha) and ozfft_destroy accept the plan; profiling and
   ozfft_debug_dump do not.  Returns NULL on error (see ozfft_last_error). */
ozfft_plan_t ozfft_plan_many(const int64_t* lengths, int64_t count, int direction, const ozfft_options* opt);

/* Transform `batch` signals: in and out are device pointers to [batch][n]
   complex128 (the packed signals of an ozfft_plan_many plan); in == out is
   allowed.  Enqueued on `stream`; nothing waits for the host.  A plan must not
   be executed on two streams at the same time. */
int ozfft_execute(ozfft_plan_t plan, const void* in, void* out, void* stream);

/* Same transform with HOST buffers: copies `in` to the device, transforms,
   copies the result to `out`, and returns after the stream has synchronized.
   Batches of 8 or more signals (plain plans) run as a pipeline of four parts:
   the copies in and out of neighbouring parts, on two streams of the plan,
   overlap the computation of a part on `stream`; from 28 signals on, the
   first and last parts are small (1/14 of the batch each), since only their
   copies are not hidden.  Pinned (page-locked) host memory gives the fastest
   copies and the overlap. */
int ozfft_execute_host(ozfft_plan_t plan, const void* in, void* out, void* stream);

/* Throughput form of ozfft_execute_host: enqueues the copy of `in` (host) to the
   plan's device staging buffer on an internal stream, the transform of the whole
   batch on `stream`, and the copy of the result to `out` (host) on a second
   internal stream, and returns without waiting.  Consecutive calls overlap: a
   call's copy in runs while the previous call computes (it waits only until
   that call's pre-multiply has read the staging buffer), and its copy out runs
   while the next call computes (whose CRT stage waits for it before writing
   the staging buffer).  `in` and `out` must stay valid and untouched until
   ozfft_execute_host_wait returns; with pinned host memory the copies are
   asynchronous.  A plan over uneven lengths, or a debug plan, runs
   ozfft_execute_host instead (synchronous). */
int ozfft_execute_host_async(ozfft_plan_t plan, const void* in, void* out, void* stream);

/* Wait until every ozfft_execute_host_async call of the plan has completed (its
   result is in its `out`), and until `stream` has synchronized. */
int ozfft_execute_host_wait(ozfft_plan_t plan, void* stream);

/* Synchronize `stream`, return the data-dependent status recorded by the
   executions since the previous call (OZFFT_OK, OZFFT_ERR_NONFINITE,
   OZFFT_ERR_RANGE, OZFFT_ERR_TIMEOUT or OZFFT_ERR_LEVELS, in that order of
   precedence when several were recorded), and clear it. */
int ozfft_get_status(ozfft_plan_t plan, void* stream);

/* Plan facts and the transform counts of the most recent execution.
   Synchronizes `stream` (the counts are computed on the device). */
typedef struct {
    int64_t n, N, batch;
    int32_t K, L, nprimes, alpha, direction;   /* K = OZFFT_K_INF for K = infinity */
    int32_t wstar_levels[2];      /* split levels of Re w~*, Im w~* */
    int64_t ntt_forward_runtime;  /* forward NTTs of x~' slices, summed over the batch */
    int64_t ntt_forward_plan;     /* forward NTTs of w~* slices (once per plan) */
    int64_t ntt_inverse;          /* inverse NTTs, summed over the batch */
    int64_t kernel_launches;      /* kernels enqueued by one ozfft_execute */
    int64_t workspace_bytes;      /* device memory held by the plan */
    int32_t row_log_fwd;          /* forward NTT: stages in the row pass (the rest in the column pass) */
    int32_t row_log_inv;          /* inverse NTT: stages in the row pass (uneven plans: of the largest N) */
    int32_t inv_vecs;             /* vectors per CTA of the inverse row pass (uneven plans: of the largest
                                     N; 1 where the two-vector kernel does not apply) */
    int32_t crt_fused_classes;    /* length classes (1 for a plain plan) whose inverse column pass runs
                                     fused with the CRT */
    int32_t classes;              /* length classes (1 for a plain plan) */
    int32_t split_fused_classes;  /* length classes (1 for a plain plan) whose Ozaki split runs fused
                                     with the forward NTT's column pass */
} ozfft_stats;
int ozfft_get_stats(ozfft_plan_t plan, void* stream, ozfft_stats* out);

/* Per-kernel device time of executions (the time breakdown of §5.5).  With
   profiling enabled, ozfft_execute records a CUDA event on its stream before
   and after every kernel it launches.  ozfft_get_profile synchronizes `stream`,
   returns the device time summed per kernel slot over the executions since the
   previous call, and restarts the sums.  Slots: */
enum {
    OZFFT_PROF_PREMUL = 0,      /* x~' = x (.) w and level-0 maxima */
    OZFFT_PROF_SPLIT = 1,       /* the K split levels (two launches; K for the TS variant) */
    OZFFT_PROF_SCHEDULE = 2,    /* Alg. 8 flush schedule */
    OZFFT_PROF_NTT_FWD_COL = 3, /* forward NTT, column pass (two-pass lengths only) */
    OZFFT_PROF_NTT_FWD_ROW = 4, /* forward NTT, row pass */
    OZFFT_PROF_NTT_INV_ROW = 5, /* NTT-domain multiply-accumulate + inverse NTT row pass */
    OZFFT_PROF_NTT_INV_COL = 6, /* inverse NTT, column pass (two-pass lengths whose column pass
                                   is not fused with the CRT) */
    OZFFT_PROF_CRT = 7,         /* Garner, rescale, accumulation, post-multiply; with two primes
                                   and m1 = 4..8 column stages also the inverse column pass, fused */
    OZFFT_PROF_SLOTS = 8
};
typedef struct {
    int64_t executions;                  /* executions summed */
    int64_t launches[OZFFT_PROF_SLOTS];  /* kernel launches per slot, summed */
    double ms[OZFFT_PROF_SLOTS];         /* device milliseconds per slot, summed */
} ozfft_profile;
int ozfft_set_profiling(ozfft_plan_t plan, int enable);
int ozfft_get_profile(ozfft_plan_t plan, void* stream, ozfft_profile* out);

/* The denominator of the integer roofline of the NTT kernels (the paper has no
   counterpart: it measures on CPUs): radix-2 butterflies per second on the
   current device with every operand in registers and no memory traffic, for
   the forward (inverse = 0: Cooley-Tukey, (a, b) -> (a + bW, a - bW)) or the
   inverse (inverse = 1: Gentleman-Sande, (a, b) -> (a + b, (a - b)W)) form the
   NTT kernels use, canonical residues and Shoup products, i.e. the rate of
   modular multiplications inside that instruction mix.  Runs a few milliseconds
   of kernels on `stream` and synchronizes it; allocates and frees 1.2 MiB of
   device memory.  *rate receives butterflies per second. */
int ozfft_measure_butterfly_rate(int inverse, double* rate, void* stream);

/* Self-test of failure detection (the paper has no counterpart): the device
   waits of libozfft are bounded (the column pass polls its tile's mbarrier at
   most 2^20 times, then records OZFFT_ERR_TIMEOUT in the plan's status word and
   skips the tile).  This call runs one column-pass tile whose barrier expects
   4 KiB more than its copy delivers, so the wait must give up; no address is
   invalid and nothing spins without a limit.  It allocates and frees about
   0.8 MiB, synchronizes `stream`, and returns OZFFT_ERR_TIMEOUT when the
   timeout path reported the stall (the expected result), OZFFT_OK if the wait
   completed, or an error code. */
int ozfft_selftest_wait_timeout(void* stream);

/* Transform without any allocation (the paper has no counterpart): for
   callers that cannot call cudaMalloc, such as code inside an application that
   owns the whole device memory pool (a stray cudaMalloc fails or fragments it)
   or a latency-critical path that must not enter the allocator.  Transforms
   one signal of length n in `direction` with the default options, exactly as
   ozfft_execute on a plan from ozfft_plan(n, 1, direction) would (bit-identical
   output).  `in`/`out` are device pointers to n complex128 (caller-owned).
   Every table and work buffer lives in one static device array of 4 MiB that
   each GPU loading the library holds until the process exits; N (the
   convolution length) must be <= 8192, i.e. n <= 8192 for powers of two and
   n <= 4096 otherwise, else OZFFT_ERR_LENGTH.  The first call on a device, and
   the first call after a call with another n, builds the tables of n in the
   array and synchronizes the device: make that call before any stream capture.
   Later calls only enqueue kernels on `stream`.  All calls share the array and
   it keeps the last call's contents; a call for another n first waits for the
   device to finish earlier work, so calls in a row (on one stream) are safe,
   but calls that overlap on the GPU (two streams at once) race on it.  The
   call runs on the current CUDA device, which must hold `in` and `out`.
   Data-dependent status is recorded in the array and not reported. */
int ozfft_execute_noalloc(int64_t n, int direction, const void* in, void* out, void* stream);

/* Host-side fault hook for tests of failure handling (the paper has no
   counterpart; nothing it does faults or stalls a GPU).  The environment
   variable OZFFT_FAULT, read at every plan creation and execution, makes the
   library take its own error paths:
     "alloc"     every device allocation of libozfft fails as a failed
                 cudaMalloc would: plan creation returns NULL (ozfft_last_error
                 names the injection) and a first host-buffer execution returns
                 OZFFT_ERR_ALLOC; the plan and the CUDA context stay usable;
     "alloc:N"   only the N-th allocation (N >= 1) of each plan creation, or of a
                 host-buffer execution's staging buffers, fails (the cleanup of a
                 partly built plan);
     "status:C"  every execution records the device status of code C (one of
                 OZFFT_ERR_NONFINITE, _RANGE, _TIMEOUT, _LEVELS) after its
                 kernels, as its kernels would on such data; ozfft_get_status
                 then returns C once.
   Unset or empty: no injection.  Any other value makes plan creation and
   executions fail with OZFFT_ERR_ARG.  ozfft_fault_config parses the current
   value without touching a GPU: *kind = 0 (none), 1 (alloc) or 2 (status),
   *arg = N (0 for plain "alloc") or C; returns OZFFT_OK or OZFFT_ERR_ARG. */
enum { OZFFT_FAULT_NONE = 0, OZFFT_FAULT_ALLOC = 1, OZFFT_FAULT_STATUS = 2 };
int ozfft_fault_config(int32_t* kind, int64_t* arg);

/* Release every resource of the plan (synchronizes its device first). */
void ozfft_destroy(ozfft_plan_t plan);

/* Text of an error code, and the detailed message of the last failure in the
   calling thread. */
const char* ozfft_error_string(int code);
const char* ozfft_last_error(void);

/* Test hook: copy one intermediate of the most recent execution (or of the
   plan) to host memory in the oracle's natural layout.  Synchronizes
   `stream`.  `index` selects the signal b (or is ignored).  Stages:
     OZFFT_DUMP_CHIRP     n complex128                 chirp table w
     OZFFT_DUMP_XPRIME    [2][N] binary64              Re/Im of x~' of signal b
     OZFFT_DUMP_MU        [2][K+1] binary64            per-level maxima of signal b: entry 0 is
                                                       max |x~'|; entry k >= 1 is 2^ceil(log2 max
                                                       |r^(k)|) (Alg. 3 uses mu only through
                                                       ceil(log2 mu)), 0 for an empty level
     OZFFT_DUMP_XRES      [2][K][P][N] uint32          slice residues of signal b before the NTT
                                                       (plans made with options.debug only)
     OZFFT_DUMP_XSPEC     [2][K][P][N] uint32          forward spectra of signal b, natural order
     OZFFT_DUMP_YSPEC     [2][K][P][N] uint32          w~* spectra, natural order, times N^-1 * 2^32 mod p
     OZFFT_DUMP_SCHED     [4][641] int32               per convolution RR, II, IR, RI of signal b:
                                                       ngroups, S[64], size[64], pair[64][8] where
                                                       S = s_x + s_y (c_x c_y = 2^S) and each pair
                                                       is s*16 + t, in Alg. 8's flush order
     OZFFT_DUMP_ZRES      [4][G][P][N] uint32          inverse-NTT outputs of signal b, G = K*K
                                                       (groups beyond ngroups hold no data;
                                                       kept for every signal by debug plans only)
   Returns the number of bytes written (or a negative OZFFT_ERR_* code); a
   NULL `dst` just returns the size.  Valid only after one ozfft_execute. */
enum {
    OZFFT_DUMP_CHIRP = 0, OZFFT_DUMP_XPRIME = 1, OZFFT_DUMP_MU = 2, OZFFT_DUMP_XRES = 3,
    OZFFT_DUMP_XSPEC = 4, OZFFT_DUMP_YSPEC = 5, OZFFT_DUMP_SCHED = 6, OZFFT_DUMP_ZRES = 7
};
int64_t ozfft_debug_dump(ozfft_plan_t plan, int stage, int64_t index, void* dst, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OZFFT_H */
