// plan.cu -- plans, the C ABI of include/ozfft.h, and the two small kernels
// that run between the big stages: the Alg. 8 flush schedule and the
// conversion of the w~* spectra to Montgomery form.
//
// Device memory of a plan (B = batch, K = split cap, P = primes, G = K*K):
//   chirp  [n] double2                         w(j) = exp(-i pi j^2/n)
//   tw     [P][N] uint2, twinv likewise        per-block twiddles in bit-reversed order with
//                                              Shoup quotients (k_ntt.cu)
//   Ym     [2][K][P][N] uint32                 w~* spectra * N^-1 * 2^32 mod p (bit-reversed order)
//   r      [B][2][N] binary64                  x~' then the split residuals
//   mu     [B][2][K+1] uint64                  bit patterns of ||r^(k)||_inf
//   X      [B][2][K][P][N] uint32              slice residues, then spectra (bit-reversed)
//   kcnt   [B][2] int32, sched [B][4] Sched    live levels, flush schedules
//   span   [B][3] int32                        min S, max S, any group (per signal)
//   Z      [chunk][4][G][P][N] uint32          inverse NTT outputs of one chunk of signals
//                                              (natural order); the inverse NTTs and the CRT
//                                              stage run chunk by chunk (default: the whole
//                                              batch while Z fits in 16 GiB)
// Every array is allocated once per plan; an execution allocates nothing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ozfft.h"
#include "oz_common.cuh"
#include "oz_kernels.h"

using namespace oz;

static thread_local std::string g_last_error;

static int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

// NVTX range around one stage of an execution (or plan creation), so that a
// timeline tool (Nsight Systems) labels the kernels by stage; with no tool
// attached a range costs a few nanoseconds.
struct StageRange {
    explicit StageRange(const char* name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange&) = delete;
    StageRange& operator=(const StageRange&) = delete;
};

// ------------------------------------------------------- host-side fault hook
// OZFFT_FAULT (read at every plan creation and execution) makes libozfft take
// its own error paths without any GPU fault:
//   alloc       every device allocation of libozfft fails as a failed
//               cudaMalloc would (OZFFT_ERR_ALLOC);
//   alloc:N     the N-th device allocation (N >= 1) of each plan creation, or
//               of a host-buffer execution's staging, fails;
//   status:C    every execution records the device status of error code C
//               (OZFFT_ERR_NONFINITE, _RANGE, _TIMEOUT or _LEVELS) after its
//               kernels, as the kernels would on such data.
// Anything else (set and not empty) is an argument error of the call.
enum { FAULT_NONE = 0, FAULT_ALLOC = 1, FAULT_STATUS = 2 };
static thread_local int64_t g_alloc_seq = 0;   // allocations since the current plan creation / staging began

static int fault_read(int32_t* kind, int64_t* arg)
{
    *kind = FAULT_NONE;
    *arg = 0;
    const char* v = std::getenv("OZFFT_FAULT");
    if (!v || !*v) return OZFFT_OK;
    const std::string s(v);
    auto number = [](const std::string& t, int64_t* out) {
        if (t.empty() || t.size() > 18) return false;
        int64_t x = 0;
        for (char c : t) {
            if (c < '0' || c > '9') return false;
            x = x * 10 + (c - '0');
        }
        *out = x;
        return true;
    };
    if (s == "alloc") { *kind = FAULT_ALLOC; return OZFFT_OK; }
    if (s.rfind("alloc:", 0) == 0 && number(s.substr(6), arg) && *arg >= 1) { *kind = FAULT_ALLOC; return OZFFT_OK; }
    if (s.rfind("status:", 0) == 0 && number(s.substr(7), arg) && *arg >= OZFFT_ERR_NONFINITE &&
        *arg <= OZFFT_ERR_LEVELS) {
        *kind = FAULT_STATUS;
        return OZFFT_OK;
    }
    *arg = 0;
    return fail(OZFFT_ERR_ARG, "OZFFT_FAULT: unknown setting '" + s + "' (alloc, alloc:N, status:C)");
}

static int fault_status_bit(int64_t code)
{
    switch (code) {
    case OZFFT_ERR_NONFINITE: return ST_NONFINITE;
    case OZFFT_ERR_RANGE: return ST_RANGE;
    case OZFFT_ERR_TIMEOUT: return ST_TIMEOUT;
    case OZFFT_ERR_LEVELS: return ST_LEVELS;
    default: return 0;
    }
}

__global__ void fault_status_kernel(int* status, int bit) { atomicOr(status, bit); }

// after an execution's kernels: the status that OZFFT_FAULT=status:C asks for
static int fault_after_execution(int* status, cudaStream_t s)
{
    int32_t kind;
    int64_t arg;
    const int rc = fault_read(&kind, &arg);
    if (rc) return rc;
    if (kind == FAULT_STATUS) {
        fault_status_kernel<<<1, 1, 0, s>>>(status, fault_status_bit(arg));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(OZFFT_ERR_CUDA, std::string("fault hook: ") + cudaGetErrorString(e));
    }
    return OZFFT_OK;
}

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(OZFFT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

struct ozfft_plan_s {
    int64_t n = 0, N = 0, B = 0;
    int direction = -1, K = 3, L = 1, P = 2, alpha = 0, G = 9, debug = 0, merge = 0, ts = 0;
    int kinf = 0;                // K = infinity: K holds the level cap MAX_K
    int crt_fused = 1;           // inverse column pass fused with the CRT where colcrt_supported
    int split_fused = 0;         // the split fused with the forward column pass where split_col_supported
    int tune_vecs = 1;           // the autotuner may choose the inverse row pass's vectors per CTA
    int tune_fuse = 1;           // ... and whether the inverse column pass is fused with the CRT
    int tune_sfuse = 1;          // ... and whether the split is fused with the forward column pass
    int garner_u = 0;            // every convolution value |z| < p0 p1 / 2 - p0 (CRT without centering z0)
    int64_t chunk = 1;           // signals per inverse-stage chunk (Z holds one chunk)
    int device = 0;
    NttGeom geom_fwd{}, geom_inv{};
    CUtensorMap tmap_x{}, tmap_z{};   // column-pass tensor maps of X and Z (when the geometry has them)
    int64_t launches = 0, bytes = 0;
    int32_t wk_host[2] = {0, 0};
    // device
    double2* chirp = nullptr;
    uint2* tw = nullptr;
    uint2* twinv = nullptr;
    uint32_t* Ym = nullptr;
    int32_t* wk = nullptr;       // [2]
    int32_t* wsexp = nullptr;    // [2][K]
    double* r = nullptr;
    uint64_t* mu = nullptr;
    uint32_t* X = nullptr;
    int32_t* kcnt = nullptr;
    Sched* sched = nullptr;
    int32_t* span = nullptr;     // [B][3] scale span of each signal's flush groups
    int32_t* redo = nullptr;     // [B][2] vectors the split's check redid (fused split + column pass)
    uint32_t* Z = nullptr;
    int* status = nullptr;
    double* dbg_r = nullptr;     // [B][2][N] (debug plans)
    uint32_t* dbg_X = nullptr;   // [B][2][K][P][N] (debug plans)
    double2* stage_in = nullptr; // host-buffer execution staging [B][n]
    double2* stage_out = nullptr;
    // host-buffer execution pipeline: copy streams and per-part events
    static constexpr int HOST_PARTS = 4;
    cudaStream_t cs_in = nullptr, cs_out = nullptr;
    cudaEvent_t ev_go = nullptr, ev_in[HOST_PARTS] = {}, ev_done[HOST_PARTS] = {};
    // asynchronous host-buffer executions (ozfft_execute_host_async): the previous call's
    // premultiply (done reading stage_in) and copy out (done reading stage_out)
    cudaEvent_t ev_a_premul = nullptr, ev_a_in = nullptr, ev_a_done = nullptr, ev_a_out = nullptr;
    bool async_pending = false;      // an asynchronous call may still be copying out
    cudaEvent_t rec_after_premul = nullptr;   // run_plan_range: record after the premultiply
    cudaEvent_t wait_before_out = nullptr;    // run_plan_range: wait before the first kernel writing out
    bool executed = false;
    int64_t total = 0;           // complex elements per execution (B n, or the packed lengths)
    int64_t fwd_plan = 0;        // forward NTTs of the w~* slices
    // one length class of a plan over uneven lengths: per-signal layout
    std::vector<SigDesc> sd_host;
    SigDesc* sd = nullptr;       // [B] device
    int64_t ym_stride = 0;       // Ym per signal (elements), 0: one Ym for the batch
    const IoPtrs* io_ref = nullptr;  // the parent's device-held in/out pointers
    // a plan over uneven lengths: its length classes and their execution
    std::vector<ozfft_plan_s*> classes;
    IoPtrs* io = nullptr;        // device
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // per-kernel timing: each execution leaves a start event and one event per kernel
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec {
        cudaEvent_t start;
        std::vector<std::pair<int, cudaEvent_t>> marks;
    };
    std::vector<Rec> pending;
    Rec* cur = nullptr;
};

static cudaEvent_t take_event(ozfft_plan_s* p)
{
    cudaEvent_t e = nullptr;
    if (!p->ev_pool.empty()) {
        e = p->ev_pool.back();
        p->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

// record the end of a kernel of `slot` on the execution stream (profiling only)
static void mark(ozfft_plan_s* p, int slot, cudaStream_t s)
{
    if (!p->cur) return;
    cudaEvent_t e = take_event(p);
    if (!e) return;
    cudaEventRecord(e, s);
    p->cur->marks.emplace_back(slot, e);
}

// ------------------------------------------------------------ host modular math
static uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }
static uint64_t powmod_h(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = mulmod_h(r, b, m);
        b = mulmod_h(b, b, m);
    }
    return r;
}
// smallest g whose order modulo the prime p is p - 1
static uint64_t primitive_root_h(uint64_t p)
{
    std::vector<uint64_t> f;
    uint64_t m = p - 1;
    for (uint64_t d = 2; d * d <= m; ++d)
        if (m % d == 0) {
            f.push_back(d);
            while (m % d == 0) m /= d;
        }
    if (m > 1) f.push_back(m);
    for (uint64_t g = 2;; ++g) {
        bool ok = true;
        for (uint64_t q : f) ok = ok && powmod_h(g, (p - 1) / q, p) != 1;
        if (ok) return g;
    }
}

// alpha = max{a : 2 L n 4^a < P} (§4.4), capped at 52; -1 if none
static int alpha_h(int64_t n, int L, int P)
{
    unsigned __int128 prod = 1;
    for (int i = 0; i < P; ++i) prod *= prime_of(i);
    const unsigned __int128 base = (unsigned __int128)2 * (unsigned)L * (uint64_t)n;
    int a = -1;
    for (int t = 0; t <= 52; ++t) {
        int bits = 0;
        while (bits < 128 && ((unsigned __int128)1 << bits) <= base) ++bits;
        if (bits + 2 * t >= 127) break;
        if ((base << (2 * t)) < prod) a = t; else break;
    }
    return a;
}

// |z| <= L n 4^alpha for every convolution value of a signal (|q| <= 2^alpha
// for every slice); the two-prime CRT may skip centering z0 when that stays
// below p0 p1 / 2 - p0
static bool garner_u_ok(int64_t n, int L, int alpha)
{
    if (alpha < 0 || alpha > 40) return false;
    const unsigned __int128 P01 = (unsigned __int128)prime_of(0) * prime_of(1);
    const unsigned __int128 zmax = (unsigned __int128)((uint64_t)L * (uint64_t)n) << (2 * alpha);
    return 2 * (zmax + prime_of(0)) < P01;
}

static int ceil_log2_h(double mu)
{
    int E;
    double m = std::frexp(mu, &E);
    return m == 0.5 ? E - 1 : E;
}

// ------------------------------------------------------------ small kernels
// Alg. 8 flush schedules of every signal's four real convolutions: the x~'
// split levels and scales come from mu, those of w~* from the plan (per
// signal in a length class of a plan over uneven lengths, where sd gives each
// signal's alpha).  One thread per signal; it also records the signal's scale
// span over all groups for the exact accumulation: span[b] = {min S, max S,
// flags}, flags bit 0 = any group, bit 1 = the scales of every convolution are
// non-increasing in group order (always, unless split levels have gaps).
//
// Merged schedules (merge != 0) extend Alg. 8's accumulation across the two
// convolutions that feed one output part (RR and II into the real part, IR and
// RI into the imaginary part): the identity that lets products of equal scale
// share an inverse NTT holds for any products whose results are summed, so the
// products of both convolutions are ordered by scale (anti-diagonal order
// within a scale) and cut into groups of at most L equal-scale products, II
// products carrying a minus sign.  Part q keeps its groups in the slots of
// convolutions 2q (first G groups) and 2q + 1 (the rest).
__global__ void schedule_kernel(const uint64_t* __restrict__ mu, int64_t B, int K, int L, int alpha,
                                const SigDesc* __restrict__ sd, const int32_t* __restrict__ wk,
                                const int32_t* __restrict__ wsexp, Sched* __restrict__ sched,
                                int32_t* __restrict__ kcnt, int32_t* __restrict__ span, int merge, int kinf,
                                int* __restrict__ status)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (sd) {
        alpha = sd[b].alpha;
        wk += 2 * b;
        wsexp += 2 * K * b;
    }
    int sx[2][MAX_K];
    int kxv[2];
    for (int v = 0; v < 2; ++v) {
        int kx = 0;
        for (int k = 0; k < K; ++k) {
            const double m = __longlong_as_double((long long)mu[(b * 2 + v) * (K + 1) + k]);
            if (!(m > 0.0)) break;
            sx[v][kx++] = alpha - ceil_log2_pos(m);
        }
        kxv[v] = kx;
        kcnt[b * 2 + v] = kx;
        // K = infinity (Alg. 3 until the residual is zero) under the level cap: a
        // residual left after the last level means the split was not error free
        if (kinf && mu[(b * 2 + v) * (K + 1) + K] != 0) atomicOr(status, ST_LEVELS);
    }
    int smin = 0, smax = 0, any = 0, mono = 1;   // mono: every convolution's scales non-increasing
    if (merge) {
        const int G = K * K;
        for (int part = 0; part < 2; ++part) {
            int ps[2 * MAX_K * MAX_K], pp[2 * MAX_K * MAX_K];
            int np = 0;
            for (int k = 2 * K - 2; k >= 0; --k)
                for (int c = 2 * part; c < 2 * part + 2; ++c) {
                    const int vx = (c == 0 || c == 3) ? 0 : 1;
                    const int vw = (c == 0 || c == 2) ? 0 : 1;
                    const int kx = kxv[vx], ky = wk[vw];
                    const int s0 = max(0, k - ky + 1), s1 = min(kx - 1, k);
                    for (int s = s0; s <= s1; ++s) {
                        const int t = k - s;
                        const int sc = sx[vx][s] + wsexp[vw * K + t];
                        int i = np++;   // stable insertion by descending scale
                        while (i > 0 && ps[i - 1] < sc) {
                            ps[i] = ps[i - 1];
                            pp[i] = pp[i - 1];
                            --i;
                        }
                        ps[i] = sc;
                        pp[i] = c * 256 + s * 16 + t;
                    }
                }
            int g = 0, l = 0;
            for (int i = 0; i < np; ++i) {
                if (i > 0 && (l >= L || ps[i] != ps[i - 1])) {
                    ++g;
                    l = 0;
                }
                Sched& S = sched[b * 4 + 2 * part + g / G];
                S.S[g % G] = ps[i];
                S.pair[g % G][l] = pp[i];
                ++l;
                S.size[g % G] = l;
                smin = any ? min(smin, ps[i]) : ps[i];
                smax = any ? max(smax, ps[i]) : ps[i];
                any = 1;
            }
            const int ng = np > 0 ? g + 1 : 0;
            sched[b * 4 + 2 * part].ngroups = min(ng, G);
            sched[b * 4 + 2 * part + 1].ngroups = max(ng - G, 0);
        }
        span[b * 3 + 0] = smin;
        span[b * 3 + 1] = smax;
        span[b * 3 + 2] = any | 2;   // sorted by scale: non-increasing in group order
        return;
    }
    for (int c = 0; c < 4; ++c) {
        const int vx = (c == 0 || c == 3) ? 0 : 1;
        const int vw = (c == 0 || c == 2) ? 0 : 1;
        const int kx = kxv[vx], ky = wk[vw];
        Sched& S = sched[b * 4 + c];
        int g = 0, l = 0;
        if (kx > 0 && ky > 0) {
            int cur = sx[vx][kx - 1] + wsexp[vw * K + ky - 1];
            for (int k = kx + ky - 2; k >= 0; --k) {
                const int s0 = max(0, k - ky + 1), s1 = min(kx - 1, k);
                for (int s = s0; s <= s1; ++s) {
                    const int t = k - s;
                    const int sc = sx[vx][s] + wsexp[vw * K + t];
                    if (l >= L || sc != cur) {   // flush: start a new group
                        if (sc > cur) mono = 0;
                        ++g;
                        cur = sc;
                        l = 0;
                    }
                    S.S[g] = cur;
                    S.pair[g][l] = s * 16 + t;
                    ++l;
                    S.size[g] = l;
                    smin = any ? min(smin, cur) : cur;
                    smax = any ? max(smax, cur) : cur;
                    any = 1;
                }
            }
            ++g;
        }
        S.ngroups = g;
    }
    span[b * 3 + 0] = smin;
    span[b * 3 + 1] = smax;
    span[b * 3 + 2] = any | (mono << 1);
}

// Y -> Y * N^-1 * 2^32 mod p, via Montgomery with the constant N^-1 2^64 mod p
__global__ void ymont_kernel(uint32_t* Y, int64_t N, int64_t total, int P, uint32_t c0, uint32_t c1, uint32_t c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int pi = (int)((i / N) % P);
        const uint32_t c = pi == 0 ? c0 : (pi == 1 ? c1 : c2);
        Y[i] = mont_mul(Y[i], c, prime_of(pi), pneg_inv_of(pi));
    }
}

// autotuner input of the split: r uniform in (-1, 1) from a counter hash, every
// vector's mu[v][0] = 1 (e_0 = 0) and the level maxima cleared
__global__ void tune_fill_kernel(double* r, uint64_t* mu, int64_t N, int64_t nvec, int K)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec * N; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull;
        z = (z ^ (z >> 29)) * 0xbf58476d1ce4e5b9ull;
        z ^= z >> 32;
        r[i] = ((double)(z >> 11) * 0x1.0p-53) * 2.0 - 1.0;
        if (i < nvec * (K + 1)) mu[i] = i % (K + 1) == 0 ? 0x3ff0000000000000ull : 0ull;
    }
}

// ------------------------------------------------------------ plan lifetime
static void plan_free(ozfft_plan_s* p)
{
    void* ptrs[] = {p->chirp, p->tw, p->twinv, p->Ym, p->wk, p->wsexp, p->r, p->mu, p->X, p->kcnt, p->sched,
                    p->span, p->Z, p->status, p->dbg_r, p->dbg_X, p->stage_in, p->stage_out, p->sd, p->io, p->redo};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (ozfft_plan_s* c : p->classes) plan_free(c);
    if (p->cs_in) cudaStreamDestroy(p->cs_in);
    if (p->cs_out) cudaStreamDestroy(p->cs_out);
    if (p->ev_go) cudaEventDestroy(p->ev_go);
    for (cudaEvent_t e : {p->ev_a_premul, p->ev_a_in, p->ev_a_done, p->ev_a_out})
        if (e) cudaEventDestroy(e);
    for (int i = 0; i < ozfft_plan_s::HOST_PARTS; ++i) {
        if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
        if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
    }
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (cudaStream_t st : p->streams) cudaStreamDestroy(st);
    for (cudaEvent_t e : p->joins) cudaEventDestroy(e);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->capture) cudaStreamDestroy(p->capture);
    for (auto& r : p->pending) {
        p->ev_pool.push_back(r.start);
        for (auto& m : r.marks) p->ev_pool.push_back(m.second);
    }
    for (cudaEvent_t e : p->ev_pool)
        if (e) cudaEventDestroy(e);
    delete p;
}

template <typename T>
static int dalloc(ozfft_plan_s* p, T** ptr, size_t count)
{
    const size_t bytes = sizeof(T) * (count ? count : 1);
    int32_t fk;
    int64_t fa;
    const int frc = fault_read(&fk, &fa);
    ++g_alloc_seq;
    if (frc) {
        *ptr = nullptr;
        return frc;
    }
    if (fk == FAULT_ALLOC && (fa == 0 || fa == g_alloc_seq)) {
        *ptr = nullptr;
        return fail(OZFFT_ERR_ALLOC, std::string("cudaMalloc of ") + std::to_string(bytes) +
                                         " bytes: failure injected by OZFFT_FAULT");
    }
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return fail(OZFFT_ERR_ALLOC, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " +
                                         cudaGetErrorString(e));
    }
    p->bytes += (int64_t)bytes;
    return OZFFT_OK;
}

static void attach_tmaps(ozfft_plan_s* p);

// twiddle tables, one per prime and direction: w_N = g^((p-1)/N) (inverse:
// w_N^-1); entry 2^s + i = w^((N/2^(s+1)) bitrev_s(i)) with its Shoup
// quotient, for the block-i butterflies of stage s (k_ntt.cu)
static int build_twiddles(ozfft_plan_s* p)
{
    const int64_t N = p->N;
    const int P = p->P;
    std::vector<uint2> t((size_t)P * N), ti((size_t)P * N);
    std::vector<uint64_t> pw(N > 1 ? N / 2 : 1), pwi(N > 1 ? N / 2 : 1);
    int lg = 0;
    while ((int64_t(1) << lg) < N) ++lg;
    for (int i = 0; i < P; ++i) {
        const uint64_t pr = prime_of(i);
        const uint64_t w = powmod_h(primitive_root_h(pr), (pr - 1) / (uint64_t)N, pr);
        const uint64_t wi = powmod_h(w, pr - 2, pr);
        pw[0] = pwi[0] = 1;
        for (int64_t e = 1; e < N / 2; ++e) {
            pw[e] = mulmod_h(pw[e - 1], w, pr);
            pwi[e] = mulmod_h(pwi[e - 1], wi, pr);
        }
        auto entry = [&](uint64_t a) { return make_uint2((uint32_t)a, (uint32_t)((a << 32) / pr)); };
        uint2* ti_ = &ti[(size_t)i * N];
        uint2* t_ = &t[(size_t)i * N];
        t_[0] = ti_[0] = entry(1);
        for (int s = 0; s < lg; ++s) {
            const int64_t m = int64_t(1) << s;
            for (int64_t b = 0; b < m; ++b) {
                int64_t r = 0;
                for (int k = 0; k < s; ++k)
                    if (b >> k & 1) r |= int64_t(1) << (s - 1 - k);
                const int64_t e = (N / (2 * m)) * r;
                t_[m + b] = entry(pw[e]);
                ti_[m + b] = entry(pwi[e]);
            }
        }
    }
    CUDA_TRY(cudaMemcpy(p->tw, t.data(), sizeof(uint2) * t.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->twinv, ti.data(), sizeof(uint2) * ti.size(), cudaMemcpyHostToDevice));
    return OZFFT_OK;
}

// Tables and workspace of a plan.  A length class of a plan over uneven
// lengths (sd_host set) has one chirp table, w~* split and w~* spectra per
// signal; a plain plan has one of each for the batch.
static int plan_build(ozfft_plan_s* p)
{
    p->garner_u = p->P == 2;
    if (p->sd_host.empty()) p->garner_u = p->garner_u && garner_u_ok(p->n, p->L, p->alpha);
    for (const SigDesc& d : p->sd_host) p->garner_u = p->garner_u && garner_u_ok(d.n, p->L, d.alpha);
    const int64_t N = p->N, B = p->B;
    const int K = p->K, P = p->P;
    const bool uneven = !p->sd_host.empty();
    const int64_t BW = uneven ? B : 1;           // signals with their own w~*
    int rc;
    CUDA_TRY(cudaGetDevice(&p->device));
    for (int i = 0; i < P; ++i)
        if ((uint32_t)(prime_of(i) * pneg_inv_of(i)) != 0xffffffffu) return fail(OZFFT_ERR_ARG, "Montgomery constant");
    int64_t nchirp = p->n;
    if (uneven) {
        nchirp = 0;
        for (const SigDesc& d : p->sd_host) nchirp += d.n;
        if ((rc = dalloc(p, &p->sd, (size_t)B))) return rc;
        CUDA_TRY(cudaMemcpy(p->sd, p->sd_host.data(), sizeof(SigDesc) * B, cudaMemcpyHostToDevice));
        p->ym_stride = (int64_t)2 * K * P * N;
    }
    if ((rc = dalloc(p, &p->chirp, nchirp))) return rc;
    if ((rc = dalloc(p, &p->tw, (size_t)P * N))) return rc;
    if ((rc = dalloc(p, &p->twinv, (size_t)P * N))) return rc;
    if ((rc = dalloc(p, &p->Ym, (size_t)BW * 2 * K * P * N))) return rc;
    if ((rc = dalloc(p, &p->wk, (size_t)BW * 2))) return rc;
    if ((rc = dalloc(p, &p->wsexp, (size_t)BW * 2 * K))) return rc;
    // r: binary64 residuals [B][2][N], or (TS) three binary32 word planes per vector [B][2][3][N]
    if ((rc = dalloc(p, &p->r, (size_t)B * (p->ts ? 3 : 2) * N))) return rc;
    if ((rc = dalloc(p, &p->mu, (size_t)B * 2 * (K + 1)))) return rc;
    if ((rc = dalloc(p, &p->X, (size_t)B * 2 * K * P * N))) return rc;
    if ((rc = dalloc(p, &p->kcnt, (size_t)B * 2))) return rc;
    if ((rc = dalloc(p, &p->sched, (size_t)B * 4))) return rc;
    if ((rc = dalloc(p, &p->span, (size_t)B * 3))) return rc;
    if ((rc = dalloc(p, &p->Z, (size_t)p->chunk * 4 * p->G * P * N))) return rc;
    if ((rc = dalloc(p, &p->status, 1))) return rc;
    if ((rc = dalloc(p, &p->redo, (size_t)B * 2))) return rc;
    if (p->debug) {
        if ((rc = dalloc(p, &p->dbg_r, (size_t)B * 2 * N))) return rc;
        if ((rc = dalloc(p, &p->dbg_X, (size_t)B * 2 * K * P * N))) return rc;
    }
    CUDA_TRY(cudaMemset(p->status, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(p->sched, 0, sizeof(Sched) * B * 4));
    CUDA_TRY(cudaMemset(p->kcnt, 0, sizeof(int32_t) * B * 2));
    if ((rc = build_twiddles(p))) return rc;

    ntt_configure(p->geom_fwd, N);
    p->geom_fwd.P = P;
    p->geom_fwd.K = K;
    p->geom_fwd.G = p->G;
    p->geom_fwd.merged = p->merge;
    p->geom_fwd.mac_reg = p->L == 1 || p->merge;   // measured: staged loads win only for unmerged L > 1
    p->geom_fwd.inv_vecs_per_cta = INV_ROW_VECS;
    p->geom_inv = p->geom_fwd;

    // chirp tables, then w~* split + forward NTTs (§4.5: precomputed once); the
    // split runs in r and mu, which executions overwrite
    cudaStream_t s = 0;
    if (uneven) {
        for (const SigDesc& d : p->sd_host) CUDA_TRY(launch_chirp(p->chirp + d.chirp_off, d.n, s));
    } else {
        CUDA_TRY(launch_chirp(p->chirp, p->n, s));
    }
    {
        CUDA_TRY(cudaMemset(p->mu, 0, sizeof(uint64_t) * BW * 2 * (K + 1)));
        if (p->ts) {
            CUDA_TRY(launch_ts_wstar(p->chirp, p->n, N, (float*)p->r, p->mu, K, s));
            for (int k = 0; k < K; ++k)
                CUDA_TRY(launch_ts_split_level(k, (float*)p->r, p->mu, N, 2, K, p->alpha, P, p->Ym, k + 1 < K,
                                               p->status, s));
        } else {
            CUDA_TRY(launch_wstar(p->chirp, p->n, N, BW, p->sd, p->r, p->mu, K, p->status, s));
            for (int k = 0; k < K; ++k)
                CUDA_TRY(launch_split_level(k, p->r, p->mu, p->mu, N, BW * 2, K, p->alpha, p->sd, P, p->Ym,
                                            k + 1 < K, p->status, s));
        }
        std::vector<uint64_t> hmu((size_t)BW * 2 * (K + 1));
        CUDA_TRY(cudaMemcpy(hmu.data(), p->mu, sizeof(uint64_t) * hmu.size(), cudaMemcpyDeviceToHost));
        std::vector<int32_t> sexp((size_t)BW * 2 * K, 0), wk((size_t)BW * 2, 0);
        p->fwd_plan = 0;
        for (int64_t b = 0; b < BW; ++b) {
            const int alpha = uneven ? p->sd_host[b].alpha : p->alpha;
            for (int v = 0; v < 2; ++v) {
                int k = 0;
                for (; k < K; ++k) {
                    double m;
                    std::memcpy(&m, &hmu[(b * 2 + v) * (K + 1) + k], sizeof m);
                    if (!(m > 0.0)) break;
                    if (p->ts ? ceil_log2_h(m) + 24 - alpha > 127 : ceil_log2_h(m) + 53 - alpha > 1023)
                        return fail(OZFFT_ERR_RANGE, "w* scale");
                    sexp[(b * 2 + v) * K + k] = alpha - ceil_log2_h(m);
                }
                wk[b * 2 + v] = k;
                p->fwd_plan += (int64_t)k * P;
                if (p->kinf && hmu[(b * 2 + v) * (K + 1) + K] != 0)
                    return fail(OZFFT_ERR_LEVELS, "w* needs more than " + std::to_string(K) + " split levels");
            }
        }
        p->wk_host[0] = wk[0];
        p->wk_host[1] = wk[1];
        CUDA_TRY(cudaMemcpy(p->wk, wk.data(), sizeof(int32_t) * wk.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(p->wsexp, sexp.data(), sizeof(int32_t) * sexp.size(), cudaMemcpyHostToDevice));
        NttGeom gw = p->geom_fwd;
        gw.nvec = BW * 2 * K * P;
        gw.kcnt = p->wk;
        CUDA_TRY(launch_ntt_forward(gw, p->Ym, p->tw, s));
        uint32_t c[3] = {0, 0, 0};
        for (int i = 0; i < P; ++i) {
            const uint64_t pr = prime_of(i);
            const uint64_t ninv = powmod_h((uint64_t)N % pr, pr - 2, pr);
            c[i] = (uint32_t)mulmod_h(ninv, mulmod_h(1ull << 32, 1ull << 32, pr), pr);
        }
        const int64_t total = BW * 2 * K * P * N;
        ymont_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 65535), 256, 0, s>>>(p->Ym, N, total, P, c[0],
                                                                                           c[1], c[2]);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaDeviceSynchronize());
        int st = 0;
        CUDA_TRY(cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st) return fail(OZFFT_ERR_RANGE, "w* split status");
    }
    p->geom_fwd.nvec = B * 2 * K * P;
    p->geom_fwd.kcnt = p->kcnt;
    p->geom_fwd.sched = p->sched;
    p->geom_inv.nvec = p->chunk * 4 * p->G * P;
    p->geom_inv.kcnt = p->kcnt;
    p->geom_inv.sched = p->sched;
    const int64_t nchunks = (B + p->chunk - 1) / p->chunk;
    p->launches = 1 /*premul*/ + (p->ts ? K : SPLIT_SPEC_LAUNCHES) /*split*/ + 1 /*schedule*/ + ntt_launches(p->geom_fwd) +
                  nchunks * (ntt_launches(p->geom_inv) + (p->ts ? 1 : crt_launches()));
    attach_tmaps(p);
    CUDA_TRY(crt_init());
    return OZFFT_OK;
}

// the column-pass tensor maps of X (forward) and Z (inverse) for the plan's
// current geometry; without them the column pass uses per-thread loads
static void attach_tmaps(ozfft_plan_s* p)
{
    p->geom_fwd.status = p->geom_inv.status = p->status;
    p->geom_fwd.vec0 = p->geom_inv.vec0 = 0;
    p->geom_fwd.tmap = ntt_make_tmap(&p->tmap_x, p->geom_fwd, p->X, p->B * 2 * p->K * p->P) ? &p->tmap_x : nullptr;
    p->geom_inv.tmap = ntt_make_tmap(&p->tmap_z, p->geom_inv, p->Z, p->chunk * 4 * p->G * p->P) ? &p->tmap_z : nullptr;
}

// ozfft_options.row_log: the row pass of both directions forced to 2^m2 residues
static int force_split(ozfft_plan_s* p, int m2)
{
    NttGeom gf = p->geom_fwd, gi = p->geom_inv;
    if (!ntt_configure_split(p->geom_fwd, p->N, m2) || !ntt_configure_split(p->geom_inv, p->N, m2))
        return fail(OZFFT_ERR_ARG, "ozfft_plan: no kernel for a row pass of 2^" + std::to_string(m2) + " residues");
    p->geom_fwd.nvec = gf.nvec; p->geom_fwd.kcnt = gf.kcnt; p->geom_fwd.sched = gf.sched;
    p->geom_inv.nvec = gi.nvec; p->geom_inv.kcnt = gi.kcnt; p->geom_inv.sched = gi.sched;
    p->geom_inv.inv_vecs_per_cta = gi.inv_vecs_per_cta;
    const int64_t nchunks = (p->B + p->chunk - 1) / p->chunk;
    p->launches = 1 + (p->ts ? p->K : SPLIT_SPEC_LAUNCHES) + 1 + ntt_launches(p->geom_fwd) +
                  nchunks * (ntt_launches(p->geom_inv) + (p->ts ? 1 : crt_launches()));
    attach_tmaps(p);
    return OZFFT_OK;
}

// Autotuning (ozfft_options.autotune): time every supported split of the
// plan's NTT length into column and row passes, forward and inverse, on the
// plan's own buffers with every vector live, and keep the fastest of each.
// The inverse side is timed with what follows it: the inverse column pass
// fused with the CRT or the column pass and the CRT apart (each where allowed),
// so the split and the fusion are chosen together; then, at that choice, one
// or two vectors per CTA in the inverse row pass.  The forward side is timed
// with the Ozaki split before it (on uniform synthetic input), fused with the
// column pass or apart, so its split and fusion are chosen together too.  Each choice changes only
// the order in which the same operations run, so results are bit-identical.
static int autotune_ntt(ozfft_plan_s* p)
{
    StageRange range("ozfft_autotune");
    const int lg = p->geom_fwd.lgN;
    std::vector<int> cands;
    for (int m2 = 10; m2 <= 14; ++m2) {
        NttGeom g{};
        if (ntt_configure_split(g, p->N, m2)) cands.push_back(m2);
    }
    if (lg <= 14) {
        NttGeom g{};
        if (ntt_configure_split(g, p->N, lg) && std::find(cands.begin(), cands.end(), lg) == cands.end())
            cands.push_back(lg);
    }
    if (std::find(cands.begin(), cands.end(), p->geom_inv.m2) == cands.end()) cands.push_back(p->geom_inv.m2);
    const int64_t B = p->B, K = p->K, G = p->G;
    // every vector live: K levels, G groups of one product (s, t) each, all
    // scales equal (every signal on the Horner path of the CRT)
    std::vector<int32_t> kc((size_t)B * 2, (int32_t)K), sp((size_t)B * 3, 0);
    for (int64_t b = 0; b < B; ++b) sp[b * 3 + 2] = 3;
    std::vector<Sched> sc((size_t)B * 4);
    for (Sched& S : sc) {
        std::memset(&S, 0, sizeof S);
        S.ngroups = (int32_t)G;
        for (int g = 0; g < G; ++g) {
            S.size[g] = 1;
            S.pair[g][0] = (g / (int)K) * 16 + g % (int)K;
        }
    }
    CUDA_TRY(cudaMemcpy(p->kcnt, kc.data(), sizeof(int32_t) * kc.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->sched, sc.data(), sizeof(Sched) * sc.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->span, sp.data(), sizeof(int32_t) * sp.size(), cudaMemcpyHostToDevice));
    // the CRT's output while timing: the signals' packed range (length classes) or chunk x n
    const bool with_crt = !p->ts && !p->debug;
    double2* tout = nullptr;
    if (with_crt) {
        int64_t out_elems = p->chunk * p->n;
        for (const SigDesc& d : p->sd_host) out_elems = std::max(out_elems, d.io_off + d.n);
        int rc = dalloc(p, &tout, (size_t)out_elems);
        if (rc) return rc;
        p->bytes -= (int64_t)sizeof(double2) * out_elems;   // temporary
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    auto time_ms = [&](auto&& launch) {
        float best = 1e30f;
        for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
            float ms = 0.f;
            err = cudaEventRecord(e0, 0);
            if (err == cudaSuccess) err = launch();
            if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);
        }
        return best;
    };
    // the forward side with its split: synthetic split input in r and mu
    const bool with_split = !p->ts && !p->debug;
    if (with_split && err == cudaSuccess) {
        const int64_t nv = B * 2;
        tune_fill_kernel<<<(unsigned)std::min<int64_t>((nv * p->N + 255) / 256, 65535), 256>>>(p->r, p->mu, p->N, nv,
                                                                                             (int)K);
        err = cudaGetLastError();
    }
    const MacSrc mac{p->X, p->Ym, p->ym_stride};
    const CrtArgs ca0{p->Z, p->sched, p->span, p->chirp, tout, p->n, p->N, p->chunk, p->P, p->G, p->direction,
                      p->status, p->sd, nullptr, p->merge, p->garner_u, 0};
    float best_f = 1e30f, best_i = 1e30f;
    int m2f = p->geom_fwd.m2, m2i = p->geom_inv.m2, fused = p->crt_fused, sfused = p->split_fused;
    // OZFFT_TUNE_LOG=path: every candidate's time is appended to that file (one line per
    // candidate: N, batch, what, row-pass stages, option, ms), for tuning reports
    FILE* tlog = nullptr;
    if (const char* path = std::getenv("OZFFT_TUNE_LOG"))
        if (*path) tlog = std::fopen(path, "a");
    auto logt = [&](const char* what, int m2, int opt, float ms) {
        if (tlog) std::fprintf(tlog, "%lld %lld %s %d %d %.4f\n", (long long)p->N, (long long)p->B, what, m2, opt, ms);
    };
    for (int m2 : cands) {
        if (err != cudaSuccess) break;
        NttGeom gf = p->geom_fwd, gi = p->geom_inv;
        ntt_configure_split(gf, p->N, m2);
        ntt_configure_split(gi, p->N, m2);
        gf.nvec = p->geom_fwd.nvec; gf.P = p->P; gf.K = p->K; gf.G = p->G; gf.kcnt = p->kcnt; gf.sched = p->sched;
        gi.nvec = p->geom_inv.nvec; gi.P = p->P; gi.K = p->K; gi.G = p->G; gi.kcnt = p->kcnt; gi.sched = p->sched;
        CUtensorMap tx{}, tz{};   // this split's tensor maps, so the candidates run the kernels they would use
        gf.tmap = ntt_make_tmap(&tx, gf, p->X, gf.nvec) ? &tx : nullptr;
        gi.tmap = ntt_make_tmap(&tz, gi, p->Z, gi.nvec) ? &tz : nullptr;
        const bool can_sfuse = with_split && gf.m1 > 0 && split_col_supported((int)K, p->P, gf.m1, gf.m2);
        for (int f = 0; f <= 1; ++f) {
            if (f && !(can_sfuse && (p->tune_sfuse || p->split_fused))) continue;
            if (!f && !p->tune_sfuse && p->split_fused && can_sfuse) continue;   // fusion forced where it applies
            const float tf = time_ms([&] {
                if (!with_split) return launch_ntt_forward(gf, p->X, p->tw, 0);
                cudaError_t e;
                NttGeom gc = gf;
                if (f) {
                    e = launch_split_col(p->r, p->mu, p->N, gf.m1, gf.m2, B * 2, (int)K, p->alpha, p->sd, p->P, p->X,
                                         p->tw, p->redo, p->status, 0);
                    gc.redo = p->redo;
                } else {
                    e = launch_split_spec(p->r, p->mu, p->N, B * 2, (int)K, p->alpha, p->sd, p->P, p->X, p->status, 0);
                }
                if (e == cudaSuccess && gc.m1 > 0) e = launch_ntt_fwd_col(gc, p->X, p->tw, 0);
                return e != cudaSuccess ? e : launch_ntt_fwd_row(gf, p->X, p->tw, 0);
            });
            logt(with_split ? (f ? "split+forward_fused" : "split+forward_apart") : "forward", m2, f, tf);
            if (tf < best_f) { best_f = tf; m2f = m2; sfused = f; }
        }
        const bool can_fuse = with_crt && gi.m1 > 0 && colcrt_supported(p->P, gi.m1, gi.m2, p->merge);
        for (int f = 0; f <= 1; ++f) {
            if (f && !(can_fuse && (p->tune_fuse || p->crt_fused))) continue;
            if (!f && !p->tune_fuse && p->crt_fused && can_fuse) continue;   // fusion forced where it applies
            const float ti = time_ms([&] {
                cudaError_t e = launch_ntt_inv_row(gi, p->Z, p->twinv, mac, 0);
                if (e != cudaSuccess || !with_crt) {
                    if (e == cudaSuccess && gi.m1 > 0) e = launch_ntt_inv_col(gi, p->Z, p->twinv, 0);
                    return e;
                }
                CrtArgs c = ca0;
                if (f) {
                    e = launch_colcrt(c, gi.m1, gi.m2, p->twinv, 0);
                    c.fused = 1;
                } else if (gi.m1 > 0) {
                    e = launch_ntt_inv_col(gi, p->Z, p->twinv, 0);
                }
                return e != cudaSuccess ? e : launch_crt_post(c, 0);
            });
            logt(with_crt ? (f ? "inverse+crt_fused" : "inverse+crt_apart") : "inverse", m2, f, ti);
            if (ti < best_i) { best_i = ti; m2i = m2; fused = f; }
        }
    }
    NttGeom gf = p->geom_fwd, gi = p->geom_inv;
    if (err == cudaSuccess) {
        ntt_configure_split(p->geom_fwd, p->N, m2f);
        ntt_configure_split(p->geom_inv, p->N, m2i);
        if (p->tune_fuse && with_crt) p->crt_fused = fused;
        if (p->tune_sfuse && with_split) p->split_fused = sfused;
    }
    // at the chosen split and fusion: one or two vectors per CTA in the inverse row pass
    if (err == cudaSuccess && p->tune_vecs) {
        NttGeom g2 = p->geom_inv;
        g2.nvec = gi.nvec; g2.P = p->P; g2.K = p->K; g2.G = p->G; g2.kcnt = p->kcnt; g2.sched = p->sched;
        if (g2.mac_reg && g2.lgN >= 12 && g2.m2 >= 5 && g2.m2 <= 12 && g2.nvec % (4 * p->G * p->P) == 0) {
            float t[3] = {0.f, 0.f, 0.f};
            for (int v = 1; v <= 2; ++v) {
                g2.inv_vecs_per_cta = v;
                t[v] = time_ms([&] { return launch_ntt_inv_row(g2, p->Z, p->twinv, mac, 0); });
                logt("inverse_row_vecs", g2.m2, v, t[v]);
            }
            if (err == cudaSuccess) gi.inv_vecs_per_cta = t[1] < t[2] ? 1 : 2;
        }
    }
    if (tlog) {
        std::fprintf(tlog, "%lld %lld chosen %d %d %d\n", (long long)p->N, (long long)p->B, m2f, m2i,
                     (p->split_fused ? 1 : 0) * 100 + (p->crt_fused ? 1 : 0) * 10 + gi.inv_vecs_per_cta);
        std::fclose(tlog);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (tout) cudaFree(tout);
    if (err != cudaSuccess) return fail(OZFFT_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(err));
    CUDA_TRY(cudaMemset(p->kcnt, 0, sizeof(int32_t) * B * 2));
    CUDA_TRY(cudaMemset(p->sched, 0, sizeof(Sched) * B * 4));
    CUDA_TRY(cudaMemset(p->span, 0, sizeof(int32_t) * B * 3));
    CUDA_TRY(cudaMemset(p->status, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(p->redo, 0, sizeof(int32_t) * B * 2));
    p->geom_fwd.nvec = gf.nvec; p->geom_fwd.P = gf.P; p->geom_fwd.K = gf.K; p->geom_fwd.G = gf.G;
    p->geom_fwd.kcnt = gf.kcnt; p->geom_fwd.sched = gf.sched;
    p->geom_inv.nvec = gi.nvec; p->geom_inv.P = gi.P; p->geom_inv.K = gi.K; p->geom_inv.G = gi.G;
    p->geom_inv.kcnt = gi.kcnt; p->geom_inv.sched = gi.sched; p->geom_inv.inv_vecs_per_cta = gi.inv_vecs_per_cta;
    const int64_t nchunks = (B + p->chunk - 1) / p->chunk;
    p->launches = 1 + (p->ts ? K : SPLIT_SPEC_LAUNCHES) + 1 + ntt_launches(p->geom_fwd) +
                  nchunks * (ntt_launches(p->geom_inv) + (p->ts ? 1 : crt_launches()));
    attach_tmaps(p);
    return OZFFT_OK;
}

// One execution of the signals [sb0, sb0 + B) of a plan (all of them, or one
// length class of a plan over uneven lengths, whose input and output pointers
// come from io_ref): every kernel is enqueued on s.
static int run_plan_range(ozfft_plan_s* p, const void* in, void* out, cudaStream_t s, int64_t sb0, int64_t B)
{
    const int64_t N = p->N;
    const int K = p->K, P = p->P;
    // the signals [sb0, sb0 + B) of the plan's per-signal buffers; in and out point at signal sb0
    uint64_t* mu = p->mu + sb0 * 2 * (K + 1);
    double* r = p->r + sb0 * (p->ts ? 3 : 2) * N;
    uint32_t* X = p->X + sb0 * 2 * K * P * N;
    int32_t* kcnt = p->kcnt + sb0 * 2;
    Sched* sched = p->sched + sb0 * 4;
    int32_t* span = p->span + sb0 * 3;
    const SigDesc* sd = p->sd ? p->sd + sb0 : nullptr;
    const uint32_t* Ym = p->Ym + sb0 * p->ym_stride;
    const bool whole = sb0 == 0 && B == p->B;
    int32_t* redo = p->redo + sb0 * 2;
    // the split fused with the forward column pass (the residues are transformed on
    // chip), unless the stage dumps need the untransformed residues or the plan is TS
    const bool fuse_fwd = !p->ts && !p->debug && p->split_fused && p->redo && p->geom_fwd.m1 > 0 &&
                          split_col_supported(K, P, p->geom_fwd.m1, p->geom_fwd.m2);
    CUDA_TRY(cudaMemsetAsync(mu, 0, sizeof(uint64_t) * B * 2 * (K + 1), s));
    p->cur = nullptr;
    if (p->profiling) {
        cudaEvent_t e0 = take_event(p);
        if (e0) {
            cudaEventRecord(e0, s);
            p->pending.push_back({e0, {}});
            p->cur = &p->pending.back();
        }
    }
    {
        StageRange range("premultiply (chirp, Alg. 1)");
        if (p->ts)
            CUDA_TRY(launch_ts_premul((const double2*)in, p->chirp, p->n, N, B, p->direction > 0, (float*)r, mu, K,
                                      p->status, s));
        else
            CUDA_TRY(launch_premul((const double2*)in, p->chirp, p->n, N, B, p->direction > 0, sd, p->io_ref, r, mu,
                                   K, p->status, s));
        mark(p, OZFFT_PROF_PREMUL, s);
        if (p->rec_after_premul) CUDA_TRY(cudaEventRecord(p->rec_after_premul, s));
    }
    if (p->debug && whole && !p->ts)
        CUDA_TRY(cudaMemcpyAsync(p->dbg_r, p->r, sizeof(double) * B * 2 * N, cudaMemcpyDeviceToDevice, s));
    {
        StageRange range("split (Alg. 3) and residues");
        if (p->ts) {
            for (int k = 0; k < K; ++k) {
                CUDA_TRY(launch_ts_split_level(k, (float*)r, mu, N, B * 2, K, p->alpha, P, X, k + 1 < K, p->status, s));
                mark(p, OZFFT_PROF_SPLIT, s);
            }
        } else if (fuse_fwd) {
            CUDA_TRY(launch_split_col(r, mu, N, p->geom_fwd.m1, p->geom_fwd.m2, B * 2, K, p->alpha, sd, P, X, p->tw,
                                      redo, p->status, s));
            mark(p, OZFFT_PROF_SPLIT, s);
        } else {
            CUDA_TRY(launch_split_spec(r, mu, N, B * 2, K, p->alpha, sd, P, X, p->status, s));
            mark(p, OZFFT_PROF_SPLIT, s);
        }
    }
    if (p->debug && whole)
        CUDA_TRY(cudaMemcpyAsync(p->dbg_X, p->X, sizeof(uint32_t) * B * 2 * K * P * N, cudaMemcpyDeviceToDevice, s));
    schedule_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(mu, B, K, p->L, p->alpha, sd, p->wk, p->wsexp, sched,
                                                                 kcnt, span, p->merge, p->kinf, p->status);
    CUDA_TRY(cudaGetLastError());
    mark(p, OZFFT_PROF_SCHEDULE, s);
    NttGeom gf = p->geom_fwd;
    gf.nvec = B * 2 * K * P;
    gf.kcnt = kcnt;
    gf.sched = sched;
    gf.vec0 = sb0 * 2 * K * P;   // the launch's first vector in the tensor map of X
    StageRange range_fwd("forward NTTs");
    if (gf.m1 > 0) {
        NttGeom gc = gf;
        if (fuse_fwd) gc.redo = redo;   // only the vectors the split's check redid
        CUDA_TRY(launch_ntt_fwd_col(gc, X, p->tw, s));
        mark(p, OZFFT_PROF_NTT_FWD_COL, s);
    }
    CUDA_TRY(launch_ntt_fwd_row(gf, X, p->tw, s));
    mark(p, OZFFT_PROF_NTT_FWD_ROW, s);
    // inverse stages chunk by chunk: Z of one chunk stays in L2 between the passes
    for (int64_t b0 = 0; b0 < B; b0 += p->chunk) {
        StageRange range_inv("Alg. 8 MAC, inverse NTTs, Garner CRT, accumulation, post-multiply");
        const int64_t nb = std::min<int64_t>(p->chunk, B - b0);
        NttGeom gi = p->geom_inv;
        gi.nvec = nb * 4 * p->G * P;
        gi.kcnt = kcnt;
        gi.sched = sched + b0 * 4;
        const MacSrc mac{X + b0 * 2 * K * P * N, Ym + b0 * p->ym_stride, p->ym_stride};
        CUDA_TRY(launch_ntt_inv_row(gi, p->Z, p->twinv, mac, s));
        mark(p, OZFFT_PROF_NTT_INV_ROW, s);
        CrtArgs ca{p->Z, sched + b0 * 4, span + b0 * 3, p->chirp,
                   sd ? (double2*)out : (double2*)out + b0 * p->n, p->n, N, nb,
                   P, p->G, p->direction, p->status, sd ? sd + b0 : nullptr, p->io_ref, p->merge,
                   p->garner_u, 0};
        // the column pass fused with the CRT (Z stays on chip), unless the
        // stage dumps need Z, the schedule is one the fused kernel does not take,
        // or the plan (a length class) runs them apart (crt_fused: the default
        // for uneven plans, measured faster there overall, or the autotuner's choice)
        const bool fuse = !p->ts && !p->debug && p->crt_fused && gi.m1 > 0 && colcrt_supported(P, gi.m1, gi.m2, p->merge);
        if (b0 == 0 && p->wait_before_out) CUDA_TRY(cudaStreamWaitEvent(s, p->wait_before_out, 0));
        if (fuse) {
            CUDA_TRY(launch_colcrt(ca, gi.m1, gi.m2, p->twinv, s));
            ca.fused = 1;
        } else if (gi.m1 > 0) {
            CUDA_TRY(launch_ntt_inv_col(gi, p->Z, p->twinv, s));
            mark(p, OZFFT_PROF_NTT_INV_COL, s);
        }
        if (p->ts) CUDA_TRY(launch_crt_ts(ca, s));
        else CUDA_TRY(launch_crt_post(ca, s));
        if (b0 + p->chunk < B) mark(p, OZFFT_PROF_CRT, s);
    }
    mark(p, OZFFT_PROF_CRT, s);
    p->cur = nullptr;
    p->executed = true;
    return OZFFT_OK;
}

// One execution of a plan (or of one length class of a plan over uneven
// lengths, whose input and output pointers come from io_ref): every kernel is
// enqueued on s.
static int run_plan(ozfft_plan_s* p, const void* in, void* out, cudaStream_t s)
{
    return run_plan_range(p, in, out, s, 0, p->B);
}

// The length classes of a plan over uneven lengths, forked from s onto their
// own streams and joined back (captured once into the plan's graph, or run
// directly with no_graph).
static int run_classes(ozfft_plan_s* p, cudaStream_t s)
{
    CUDA_TRY(cudaEventRecord(p->fork, s));
    for (size_t c = 0; c < p->classes.size(); ++c) {
        CUDA_TRY(cudaStreamWaitEvent(p->streams[c], p->fork, 0));
        const int rc = run_plan(p->classes[c], nullptr, nullptr, p->streams[c]);
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(p->joins[c], p->streams[c]));
        CUDA_TRY(cudaStreamWaitEvent(s, p->joins[c], 0));
    }
    return OZFFT_OK;
}

static int run_many(ozfft_plan_s* p, const void* in, void* out, cudaStream_t s)
{
    CUDA_TRY(launch_set_io(p->io, in, out, s));
    if (p->gexec) {
        CUDA_TRY(cudaGraphLaunch(p->gexec, s));
    } else {
        const int rc = run_classes(p, s);
        if (rc) return rc;
    }
    for (ozfft_plan_s* c : p->classes) c->executed = true;
    p->executed = true;
    return OZFFT_OK;
}

extern "C" {

ozfft_plan_t ozfft_plan_ex(int64_t n, int64_t batch, int direction, const ozfft_options* opt)
{
    ozfft_options o{};
    if (opt) o = *opt;
    const int kinf = o.K == OZFFT_K_INF;
    const int K = kinf ? MAX_K : (o.K ? o.K : 3), L = o.L ? o.L : 1, P = o.nprimes ? o.nprimes : 2;
    if (n < 1 || batch < 1 || (direction != OZFFT_FORWARD && direction != OZFFT_INVERSE && direction != OZFFT_ADJOINT &&
                               direction != OZFFT_INVERSE_ADJOINT) || K < 1 || K > MAX_K ||
        L < 1 || L > MAX_L || P < 2 || P > 3) {
        fail(OZFFT_ERR_ARG, "ozfft_plan: argument out of range");
        return nullptr;
    }
    int64_t N = o.conv_len;
    if (N == 0) {
        if ((n & (n - 1)) == 0) N = n;
        else { N = 1; while (N < 2 * n - 1) N <<= 1; }
    }
    if (N < n || (N & (N - 1)) || N > (int64_t(1) << 24) || !(N == n || N >= 2 * n - 1)) {
        fail(OZFFT_ERR_LENGTH, "ozfft_plan: convolution length must be a power of two <= 2^24, equal to n or >= 2n-1");
        return nullptr;
    }
    if (o.inv_vecs < 0 || o.inv_vecs > 2 || o.crt_fuse < 0 || o.crt_fuse > 2 || o.split_fuse < 0 ||
        o.split_fuse > 2) {
        fail(OZFFT_ERR_ARG, "ozfft_plan: inv_vecs, crt_fuse and split_fuse must be 0..2");
        return nullptr;
    }
    if (o.ts && (P != 2 || o.merge || kinf)) {
        fail(OZFFT_ERR_ARG, "ozfft_plan: the TS variant takes two primes, no merged schedules and a finite K");
        return nullptr;
    }
    int alpha = alpha_h(n, L, P);
    if (o.ts && alpha > 23) alpha = 23;   // rho = 24 - alpha >= 1 in binary32
    if (alpha < 1) {
        fail(OZFFT_ERR_LENGTH, "ozfft_plan: no split width alpha >= 1 for this n, L and prime count");
        return nullptr;
    }
    StageRange range("ozfft_plan");
    g_alloc_seq = 0;
    {
        int32_t fk;
        int64_t fa;
        if (fault_read(&fk, &fa)) return nullptr;   // a malformed OZFFT_FAULT
    }
    ozfft_plan_s* p = new ozfft_plan_s;
    p->n = n;
    p->N = N;
    p->B = batch;
    p->direction = direction;
    p->K = K;
    p->kinf = kinf;
    p->L = L;
    p->P = P;
    p->G = K * K;
    p->alpha = alpha;
    p->debug = o.debug;
    p->merge = o.merge != 0;
    p->ts = o.ts != 0;
    {
        const int64_t zbytes = (int64_t)4 * p->G * P * N * 4;   // Z of one signal
        int64_t c = o.chunk > 0 ? o.chunk : std::max<int64_t>(1, (int64_t(16) << 30) / zbytes);
        if (p->debug) c = batch;                              // dumps read Z of any signal
        p->chunk = std::min<int64_t>(c, batch);
    }
    p->total = n * batch;
    p->crt_fused = o.crt_fuse != 2;
    p->split_fused = o.split_fuse == 1;   // apart unless forced or tuned (apart measured faster at N = 2^17 .. 2^20)
    p->tune_sfuse = o.split_fuse == 0;
    p->tune_fuse = o.crt_fuse == 0;
    p->tune_vecs = o.inv_vecs == 0;
    if (plan_build(p) != OZFFT_OK) {
        plan_free(p);
        return nullptr;
    }
    if (o.inv_vecs) p->geom_inv.inv_vecs_per_cta = o.inv_vecs;
    if ((o.autotune && !o.row_log && autotune_ntt(p) != OZFFT_OK) ||
        (o.row_log && force_split(p, o.row_log) != OZFFT_OK)) {
        plan_free(p);
        return nullptr;
    }
    return p;
}

ozfft_plan_t ozfft_plan(int64_t n, int64_t batch, int direction) { return ozfft_plan_ex(n, batch, direction, nullptr); }

static int64_t default_conv_len(int64_t n)
{
    if ((n & (n - 1)) == 0) return n;
    int64_t N = 1;
    while (N < 2 * n - 1) N <<= 1;
    return N;
}

ozfft_plan_t ozfft_plan_many(const int64_t* lengths, int64_t count, int direction, const ozfft_options* opt)
{
    ozfft_options o{};
    if (opt) o = *opt;
    const int kinf = o.K == OZFFT_K_INF;
    const int K = kinf ? MAX_K : (o.K ? o.K : 3), L = o.L ? o.L : 1, P = o.nprimes ? o.nprimes : 2;
    if (!lengths || count < 1 || (direction != OZFFT_FORWARD && direction != OZFFT_INVERSE &&
                                  direction != OZFFT_ADJOINT && direction != OZFFT_INVERSE_ADJOINT) ||
        K < 1 || K > MAX_K || L < 1 || L > MAX_L || P < 2 || P > 3 || o.conv_len != 0 || o.debug != 0 || o.chunk < 0 ||
        o.ts != 0 || o.inv_vecs < 0 || o.inv_vecs > 2 || o.crt_fuse < 0 || o.crt_fuse > 2 || o.split_fuse < 0 ||
        o.split_fuse > 2) {
        fail(OZFFT_ERR_ARG, "ozfft_plan_many: argument out of range");
        return nullptr;
    }
    // length classes by convolution length, largest first (their work dominates)
    std::vector<std::pair<int64_t, std::vector<int64_t>>> cls;
    {
        std::vector<int64_t> Ns(count);
        for (int64_t i = 0; i < count; ++i) {
            const int64_t n = lengths[i];
            if (n < 1 || n > (int64_t(1) << 24)) {
                fail(OZFFT_ERR_LENGTH, "ozfft_plan_many: length " + std::to_string(n) + " out of range");
                return nullptr;
            }
            Ns[i] = default_conv_len(n);
            if (Ns[i] > (int64_t(1) << 24) || alpha_h(n, L, P) < 1) {
                fail(OZFFT_ERR_LENGTH, "ozfft_plan_many: length " + std::to_string(n) + " unsupported");
                return nullptr;
            }
        }
        std::vector<int64_t> order(count);
        for (int64_t i = 0; i < count; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return Ns[a] > Ns[b]; });
        for (int64_t i : order) {
            if (cls.empty() || cls.back().first != Ns[i]) cls.push_back({Ns[i], {}});
            cls.back().second.push_back(i);
        }
    }
    std::vector<int64_t> off(count + 1, 0);
    for (int64_t i = 0; i < count; ++i) off[i + 1] = off[i] + lengths[i];
    // inverse-NTT buffers: the same fraction of every class's signals per chunk,
    // all classes together within 16 GiB (or opt->chunk signals per chunk)
    const int G = K * K;
    double zdemand = 0;
    for (auto& c : cls) zdemand += (double)c.second.size() * 4.0 * G * P * c.first * 4.0;
    const double frac = std::min(1.0, (double)(int64_t(16) << 30) / zdemand);

    StageRange range("ozfft_plan_many");
    g_alloc_seq = 0;
    {
        int32_t fk;
        int64_t fa;
        if (fault_read(&fk, &fa)) return nullptr;   // a malformed OZFFT_FAULT
    }
    ozfft_plan_s* p = new ozfft_plan_s;
    p->B = count;
    p->n = off[count];
    p->total = off[count];
    p->N = cls.front().first;
    p->direction = direction;
    p->K = K;
    p->kinf = kinf;
    p->L = L;
    p->P = P;
    p->G = G;
    p->alpha = 64;
    p->chunk = 0;
    auto bail = [&](int code, const std::string& msg) {
        if (code) fail(code, msg);
        plan_free(p);
        return (ozfft_plan_t) nullptr;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: no device");
    if (dalloc(p, &p->io, 1)) return bail(0, "");
    for (auto& c : cls) {
        ozfft_plan_s* q = new ozfft_plan_s;
        p->classes.push_back(q);
        q->N = c.first;
        q->B = (int64_t)c.second.size();
        q->direction = direction;
        q->K = K;
        q->kinf = kinf;
        q->L = L;
        q->P = P;
        q->G = G;
        q->merge = o.merge != 0;
        q->io_ref = p->io;
        int64_t chirp_off = 0;
        for (int64_t i : c.second) {
            SigDesc d{};
            d.n = lengths[i];
            d.io_off = off[i];
            d.chirp_off = chirp_off;
            d.alpha = alpha_h(lengths[i], L, P);
            chirp_off += d.n;
            q->sd_host.push_back(d);
            q->n = std::max(q->n, d.n);
            q->alpha = std::max(q->alpha, d.alpha);
            p->alpha = std::min(p->alpha, d.alpha);
        }
        q->total = chirp_off;
        q->chunk = o.chunk > 0 ? std::min<int64_t>(o.chunk, q->B)
                               : std::max<int64_t>(1, std::min<int64_t>(q->B, (int64_t)(q->B * frac)));
        q->crt_fused = o.crt_fuse == 1;   // length classes keep the CRT apart unless forced or tuned
        q->split_fused = o.split_fuse == 1;
        q->tune_sfuse = o.split_fuse == 0;
        q->tune_fuse = o.crt_fuse == 0;
        q->tune_vecs = o.inv_vecs == 0;
        if (plan_build(q) != OZFFT_OK) return bail(0, "");
        if (o.inv_vecs) q->geom_inv.inv_vecs_per_cta = o.inv_vecs;
        if (o.autotune && !o.row_log && autotune_ntt(q) != OZFFT_OK) return bail(0, "");
        if (o.row_log) {   // the forced split, for every class whose N admits it
            NttGeom t{};
            if (ntt_configure_split(t, q->N, o.row_log) && force_split(q, o.row_log) != OZFFT_OK) return bail(0, "");
        }
        p->bytes += q->bytes;
        p->launches += q->launches;
        p->fwd_plan += q->fwd_plan;
        p->chunk = std::max(p->chunk, q->chunk);
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: stream");
        p->streams.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: event");
        p->joins.push_back(ev);
    }
    p->launches += 1;   // the in/out pointer update
    if (cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: event");
    if (dalloc(p, &p->status, 1)) return bail(0, "");
    if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess)
        return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: status word");
    if (!o.no_graph) {
        // capture every class's kernels once; executions replay the graph
        if (cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking) != cudaSuccess)
            return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: stream");
        if (cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: begin capture");
        const int rc = run_classes(p, p->capture);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(p->capture, &g);
        p->graph = g;
        if (rc || ce != cudaSuccess)
            return bail(rc ? 0 : OZFFT_ERR_CUDA,
                        std::string("ozfft_plan_many: capture: ") + cudaGetErrorString(ce));
        if (cudaGraphInstantiate(&p->gexec, p->graph, 0) != cudaSuccess)
            return bail(OZFFT_ERR_CUDA, "ozfft_plan_many: graph instantiation");
    }
    for (ozfft_plan_s* q : p->classes) q->executed = false;
    return p;
}

int ozfft_execute(ozfft_plan_t p, const void* in, void* out, void* stream)
{
    if (!p || !in || !out) return fail(OZFFT_ERR_ARG, "ozfft_execute: null argument");
    StageRange range("ozfft_execute");
    const int rc = p->classes.empty() ? run_plan(p, in, out, (cudaStream_t)stream)
                                      : run_many(p, in, out, (cudaStream_t)stream);
    if (rc) return rc;
    return fault_after_execution(p->status, (cudaStream_t)stream);
}

int ozfft_set_profiling(ozfft_plan_t p, int enable)
{
    if (!p) return fail(OZFFT_ERR_ARG, "ozfft_set_profiling: null plan");
    if (!p->classes.empty()) return fail(OZFFT_ERR_ARG, "ozfft_set_profiling: not available for uneven-length plans");
    p->profiling = enable != 0;
    return OZFFT_OK;
}

int ozfft_get_profile(ozfft_plan_t p, void* stream, ozfft_profile* out)
{
    if (!p || !out) return fail(OZFFT_ERR_ARG, "ozfft_get_profile: null argument");
    if (!p->classes.empty()) return fail(OZFFT_ERR_ARG, "ozfft_get_profile: not available for uneven-length plans");
    std::memset(out, 0, sizeof(*out));
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    for (auto& r : p->pending) {
        cudaEvent_t prev = r.start;
        for (auto& m : r.marks) {
            float ms = 0.f;
            CUDA_TRY(cudaEventSynchronize(m.second));
            CUDA_TRY(cudaEventElapsedTime(&ms, prev, m.second));
            out->ms[m.first] += ms;
            out->launches[m.first] += 1;
            prev = m.second;
        }
        out->executions += 1;
        p->ev_pool.push_back(r.start);
        for (auto& m : r.marks) p->ev_pool.push_back(m.second);
    }
    p->pending.clear();
    return OZFFT_OK;
}

int ozfft_measure_butterfly_rate(int inverse, double* rate, void* stream)
{
    if (!rate) return fail(OZFFT_ERR_ARG, "ozfft_measure_butterfly_rate: null argument");
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;                    // eight 256-thread CTAs per SM
    uint32_t* scratch = nullptr;
    CUDA_TRY(cudaMalloc((void**)&scratch, sizeof(uint32_t) * 256 * (size_t)blocks));
    const cudaError_t e = measure_butterfly_rate(inverse, blocks, 4096, scratch, rate, (cudaStream_t)stream);
    cudaFree(scratch);
    if (e != cudaSuccess) return fail(OZFFT_ERR_CUDA, std::string("butterfly rate: ") + cudaGetErrorString(e));
    return OZFFT_OK;
}

int ozfft_selftest_wait_timeout(void* stream)
{
    int st = 0;
    const cudaError_t e = col_tma_timeout_selftest(&st, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(OZFFT_ERR_CUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
    return (st & ST_TIMEOUT) ? OZFFT_ERR_TIMEOUT : OZFFT_OK;
}

// the device staging buffers of host-buffer executions (both, or neither)
static int ensure_staging(ozfft_plan_s* p)
{
    if (!p->stage_in || !p->stage_out) {
        g_alloc_seq = 0;
        int rc = OZFFT_OK;
        if (!p->stage_in) rc = dalloc(p, &p->stage_in, p->total);
        if (!rc && !p->stage_out) rc = dalloc(p, &p->stage_out, p->total);
        if (rc) {   // keep neither half: the next call allocates both again
            const int64_t bytes_each = (int64_t)sizeof(double2) * p->total;
            if (p->stage_in) { cudaFree(p->stage_in); p->bytes -= bytes_each; }
            if (p->stage_out) { cudaFree(p->stage_out); p->bytes -= bytes_each; }
            p->stage_in = p->stage_out = nullptr;
            return rc;
        }
    }
    return OZFFT_OK;
}

int ozfft_execute_host(ozfft_plan_t p, const void* in, void* out, void* stream)
{
    if (!p || !in || !out) return fail(OZFFT_ERR_ARG, "ozfft_execute_host: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double2) * p->total;
    StageRange range("ozfft_execute_host");
    {
        const int rc = ensure_staging(p);
        if (rc) return rc;
    }
    if (p->async_pending) {   // an asynchronous call's copy out may still read stage_out
        CUDA_TRY(cudaEventSynchronize(p->ev_a_out));
        p->async_pending = false;
    }
    const int parts = (p->classes.empty() && !p->debug && p->B >= 8) ? ozfft_plan_s::HOST_PARTS : 1;
    if (parts == 1) {
        CUDA_TRY(cudaMemcpyAsync(p->stage_in, in, bytes, cudaMemcpyHostToDevice, s));
        int rc = ozfft_execute(p, p->stage_in, p->stage_out, stream);
        if (rc) return rc;
        CUDA_TRY(cudaMemcpyAsync(out, p->stage_out, bytes, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return OZFFT_OK;
    }
    // a pipeline over parts of the batch: the copy in of part i + 1 and the copy
    // out of part i - 1 run on their own streams while part i computes on s
    if (!p->cs_in) {
        CUDA_TRY(cudaStreamCreateWithFlags(&p->cs_in, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamCreateWithFlags(&p->cs_out, cudaStreamNonBlocking));
    }
    if (!p->ev_go) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_go, cudaEventDisableTiming));
    for (int i = 0; i < parts; ++i) {
        if (!p->ev_in[i]) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming));
        if (!p->ev_done[i]) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_done[i], cudaEventDisableTiming));
    }
    CUDA_TRY(cudaEventRecord(p->ev_go, s));             // earlier work on s may still use the staging
    CUDA_TRY(cudaStreamWaitEvent(p->cs_in, p->ev_go, 0));
    // only the first part's copy in and the last part's copy out are not hidden
    // behind computation, so those parts are small (weights 1, 6, 6, 1 of the
    // batch; equal parts for small batches)
    static constexpr int W[ozfft_plan_s::HOST_PARTS] = {1, 6, 6, 1};
    int64_t cut[ozfft_plan_s::HOST_PARTS + 1] = {0};
    const int wsum = W[0] + W[1] + W[2] + W[3];
    for (int i = 0, acc = 0; i < parts; ++i) {
        acc += W[i];
        cut[i + 1] = p->B >= 2 * wsum ? p->B * acc / wsum : std::min<int64_t>(p->B, (i + 1) * ((p->B + parts - 1) / parts));
    }
    for (int i = 0; i < parts; ++i) {
        const int64_t b0 = cut[i], nb = cut[i + 1] - cut[i];
        if (nb <= 0) continue;
        const size_t off = (size_t)(b0 * p->n), cnt = (size_t)(nb * p->n);
        CUDA_TRY(cudaMemcpyAsync(p->stage_in + off, (const double2*)in + off, sizeof(double2) * cnt,
                                 cudaMemcpyHostToDevice, p->cs_in));
        CUDA_TRY(cudaEventRecord(p->ev_in[i], p->cs_in));
        CUDA_TRY(cudaStreamWaitEvent(s, p->ev_in[i], 0));
        const int rc = run_plan_range(p, p->stage_in + off, p->stage_out + off, s, b0, nb);
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(p->ev_done[i], s));
        CUDA_TRY(cudaStreamWaitEvent(p->cs_out, p->ev_done[i], 0));
        CUDA_TRY(cudaMemcpyAsync((double2*)out + off, p->stage_out + off, sizeof(double2) * cnt,
                                 cudaMemcpyDeviceToHost, p->cs_out));
    }
    const int frc = fault_after_execution(p->status, s);
    CUDA_TRY(cudaStreamSynchronize(p->cs_out));
    CUDA_TRY(cudaStreamSynchronize(s));
    return frc;
}

int ozfft_execute_host_async(ozfft_plan_t p, const void* in, void* out, void* stream)
{
    if (!p || !in || !out) return fail(OZFFT_ERR_ARG, "ozfft_execute_host_async: null argument");
    if (!p->classes.empty() || p->debug) return ozfft_execute_host(p, in, out, stream);
    StageRange range("ozfft_execute_host_async");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double2) * p->total;
    {
        const int rc = ensure_staging(p);
        if (rc) return rc;
    }
    if (!p->ev_a_out) {
        if (!p->cs_in) {
            CUDA_TRY(cudaStreamCreateWithFlags(&p->cs_in, cudaStreamNonBlocking));
            CUDA_TRY(cudaStreamCreateWithFlags(&p->cs_out, cudaStreamNonBlocking));
        }
        if (!p->ev_go) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_go, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&p->ev_a_premul, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&p->ev_a_in, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&p->ev_a_done, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&p->ev_a_out, cudaEventDisableTiming));
    }
    // copy in once the previous call's premultiply has read stage_in (the first
    // asynchronous call: once earlier work on the stream is done with it)
    if (p->async_pending) {
        CUDA_TRY(cudaStreamWaitEvent(p->cs_in, p->ev_a_premul, 0));
    } else {
        CUDA_TRY(cudaEventRecord(p->ev_go, s));
        CUDA_TRY(cudaStreamWaitEvent(p->cs_in, p->ev_go, 0));
    }
    CUDA_TRY(cudaMemcpyAsync(p->stage_in, in, bytes, cudaMemcpyHostToDevice, p->cs_in));
    CUDA_TRY(cudaEventRecord(p->ev_a_in, p->cs_in));
    CUDA_TRY(cudaStreamWaitEvent(s, p->ev_a_in, 0));
    // the transform on the caller's stream; its CRT stage, which writes stage_out,
    // waits for the previous call's copy out (long done when the CRT starts)
    p->rec_after_premul = p->ev_a_premul;
    p->wait_before_out = p->async_pending ? p->ev_a_out : nullptr;
    int rc = run_plan(p, p->stage_in, p->stage_out, s);
    p->rec_after_premul = p->wait_before_out = nullptr;
    if (!rc) rc = fault_after_execution(p->status, s);
    if (rc) return rc;
    CUDA_TRY(cudaEventRecord(p->ev_a_done, s));
    CUDA_TRY(cudaStreamWaitEvent(p->cs_out, p->ev_a_done, 0));
    CUDA_TRY(cudaMemcpyAsync(out, p->stage_out, bytes, cudaMemcpyDeviceToHost, p->cs_out));
    CUDA_TRY(cudaEventRecord(p->ev_a_out, p->cs_out));
    p->async_pending = true;
    return OZFFT_OK;
}

int ozfft_execute_host_wait(ozfft_plan_t p, void* stream)
{
    if (!p) return fail(OZFFT_ERR_ARG, "ozfft_execute_host_wait: null plan");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (p->async_pending) CUDA_TRY(cudaEventSynchronize(p->ev_a_out));
    p->async_pending = false;
    return OZFFT_OK;
}

int ozfft_get_status(ozfft_plan_t p, void* stream)
{
    if (!p) return fail(OZFFT_ERR_ARG, "ozfft_get_status: null plan");
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(p->status, 0, sizeof(int)));
    for (ozfft_plan_s* c : p->classes) {   // a plan over uneven lengths: every class's word
        int sc = 0;
        CUDA_TRY(cudaMemcpy(&sc, c->status, sizeof(int), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemset(c->status, 0, sizeof(int)));
        st |= sc;
    }
    if (st & ST_NONFINITE) return OZFFT_ERR_NONFINITE;
    if (st & ST_RANGE) return OZFFT_ERR_RANGE;
    if (st & ST_TIMEOUT) return OZFFT_ERR_TIMEOUT;
    if (st & ST_LEVELS) return OZFFT_ERR_LEVELS;
    return OZFFT_OK;
}

int ozfft_get_stats(ozfft_plan_t p, void* stream, ozfft_stats* out)
{
    if (!p || !out) return fail(OZFFT_ERR_ARG, "ozfft_get_stats: null argument");
    std::memset(out, 0, sizeof(*out));
    out->n = p->n;
    out->N = p->N;
    out->batch = p->B;
    out->K = p->kinf ? OZFFT_K_INF : p->K;
    out->L = p->L;
    out->nprimes = p->P;
    out->alpha = p->alpha;
    out->direction = p->direction;
    out->wstar_levels[0] = p->wk_host[0];
    out->wstar_levels[1] = p->wk_host[1];
    out->ntt_forward_plan = p->fwd_plan;
    out->kernel_launches = p->launches;
    out->workspace_bytes = p->bytes;
    const ozfft_plan_s* g0 = p->classes.empty() ? p : p->classes.front();
    out->row_log_fwd = g0->geom_fwd.m2;
    out->row_log_inv = g0->geom_inv.m2;
    {
        const NttGeom& gi = g0->geom_inv;
        const bool vk = gi.mac_reg && gi.lgN >= 12 && gi.m2 >= 5 && gi.m2 <= 12 &&
                        (g0->chunk * 4 * g0->G * g0->P) % (4 * g0->G * g0->P) == 0;
        out->inv_vecs = vk ? gi.inv_vecs_per_cta : 1;
    }
    out->classes = p->classes.empty() ? 1 : (int32_t)p->classes.size();
    for (const ozfft_plan_s* q : (p->classes.empty() ? std::vector<ozfft_plan_s*>{p} : p->classes)) {
        const NttGeom& gi = q->geom_inv;
        out->crt_fused_classes += !q->ts && !q->debug && q->crt_fused && gi.m1 > 0 &&
                                  colcrt_supported(q->P, gi.m1, gi.m2, q->merge);
        const NttGeom& gf = q->geom_fwd;
        out->split_fused_classes += !q->ts && !q->debug && q->split_fused && gf.m1 > 0 &&
                                    split_col_supported(q->K, q->P, gf.m1, gf.m2);
    }
    std::vector<ozfft_plan_s*> parts = p->classes;
    if (parts.empty()) parts.push_back(p);
    if (p->executed) CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    for (ozfft_plan_s* q : parts) {
        if (!q->executed) continue;
        std::vector<int32_t> kc(q->B * 2);
        std::vector<Sched> sc(q->B * 4);
        CUDA_TRY(cudaMemcpy(kc.data(), q->kcnt, sizeof(int32_t) * kc.size(), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(sc.data(), q->sched, sizeof(Sched) * sc.size(), cudaMemcpyDeviceToHost));
        for (int32_t k : kc) out->ntt_forward_runtime += (int64_t)k * q->P;
        for (const Sched& s : sc) out->ntt_inverse += (int64_t)s.ngroups * q->P;
    }
    return OZFFT_OK;
}

void ozfft_destroy(ozfft_plan_t p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    plan_free(p);
}

const char* ozfft_error_string(int code)
{
    switch (code) {
    case OZFFT_OK: return "ok";
    case OZFFT_ERR_ARG: return "invalid argument";
    case OZFFT_ERR_LENGTH: return "unsupported length";
    case OZFFT_ERR_ALLOC: return "allocation failed";
    case OZFFT_ERR_CUDA: return "CUDA runtime error";
    case OZFFT_ERR_NONFINITE: return "non-finite input";
    case OZFFT_ERR_RANGE: return "input magnitude out of range";
    case OZFFT_ERR_TIMEOUT: return "device wait timed out";
    case OZFFT_ERR_LEVELS: return "K = infinity: a vector needs more split levels than the cap";
    default: return "unknown error";
    }
}

const char* ozfft_last_error(void) { return g_last_error.c_str(); }

int ozfft_fault_config(int32_t* kind, int64_t* arg)
{
    if (!kind || !arg) return fail(OZFFT_ERR_ARG, "ozfft_fault_config: null argument");
    return fault_read(kind, arg);
}

// bit reversal of the low lg bits
static int64_t bitrev(int64_t v, int lg)
{
    int64_t r = 0;
    for (int b = 0; b < lg; ++b)
        if (v >> b & 1) r |= int64_t(1) << (lg - 1 - b);
    return r;
}

int64_t ozfft_debug_dump(ozfft_plan_t p, int stage, int64_t index, void* dst, void* stream)
{
    if (!p) return -fail(OZFFT_ERR_ARG, "ozfft_debug_dump: null plan");
    if (!p->classes.empty()) return -fail(OZFFT_ERR_ARG, "ozfft_debug_dump: not available for uneven-length plans");
    const int64_t N = p->N, K = p->K, P = p->P, G = p->G;
    const int64_t b = index;
    const bool per_signal = stage != OZFFT_DUMP_CHIRP && stage != OZFFT_DUMP_YSPEC;
    if (per_signal && (b < 0 || b >= p->B)) return -fail(OZFFT_ERR_ARG, "ozfft_debug_dump: signal index");
    const void* src = nullptr;
    int64_t bytes = 0;
    bool bitrev_vectors = false;
    switch (stage) {
    case OZFFT_DUMP_CHIRP: src = p->chirp; bytes = 16 * p->n; break;
    case OZFFT_DUMP_XPRIME: src = p->dbg_r ? p->dbg_r + b * 2 * N : nullptr; bytes = 8 * 2 * N; break;
    case OZFFT_DUMP_MU: src = p->mu + b * 2 * (K + 1); bytes = 8 * 2 * (K + 1); break;
    case OZFFT_DUMP_XRES: src = p->dbg_X ? p->dbg_X + b * 2 * K * P * N : nullptr; bytes = 4 * 2 * K * P * N; break;
    case OZFFT_DUMP_XSPEC: src = p->X + b * 2 * K * P * N; bytes = 4 * 2 * K * P * N; bitrev_vectors = true; break;
    case OZFFT_DUMP_YSPEC: src = p->Ym; bytes = 4 * 2 * K * P * N; bitrev_vectors = true; break;
    case OZFFT_DUMP_SCHED: src = p->sched + b * 4; bytes = sizeof(Sched) * 4; break;
    case OZFFT_DUMP_ZRES:
        src = (p->chunk == p->B) ? p->Z + b * 4 * G * P * N : nullptr;
        bytes = 4 * 4 * G * P * N;
        break;
    default: return -fail(OZFFT_ERR_ARG, "ozfft_debug_dump: unknown stage");
    }
    if (!src) return -fail(OZFFT_ERR_ARG, "ozfft_debug_dump: stage kept only by debug plans");
    if (!dst) return bytes;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -fail(OZFFT_ERR_CUDA, "ozfft_debug_dump: copy failed");
    if (bitrev_vectors) {
        int lg = 0;
        while ((int64_t(1) << lg) < N) ++lg;
        uint32_t* d = (uint32_t*)dst;
        std::vector<uint32_t> tmp(N);
        for (int64_t v = 0; v < bytes / 4 / N; ++v) {
            uint32_t* vec = d + v * N;
            for (int64_t k = 0; k < N; ++k) tmp[k] = vec[bitrev(k, lg)];
            std::memcpy(vec, tmp.data(), 4 * N);
        }
    }
    return bytes;
}

}  // extern "C"

// ============================================================================
// Transform without allocation: ozfft_execute_noalloc.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// application which owns the device memory pool (an extra cudaMalloc there
// fails or fragments the pool), and latency-critical paths that must not
// block in the allocator or fail on it.  For them, this entry point runs the
// kernels of ozfft_execute on one signal of length n with the default options
// (K = 3, L = 1, two primes, N as ozfft_plan picks it), with every table and
// work buffer carved out of g_noalloc_scratch, a file-scope device array of
// NOALLOC_BYTES that each GPU which loads the library holds until the process
// exits.  The convolution length N is limited to NOALLOC_MAX_N.
//
// The array's name in host code is only a host-side stand-in, never a device
// address: the first call on a device, with that device current, asks
// cudaGetSymbolAddress for the real address and passes that to every kernel.
// The first call for a length n (and the first call on a device) also builds
// the length's tables in the array and synchronizes the device, so it should
// come before any stream capture; later calls with the same n only enqueue
// kernels on `stream`.  All calls share the array, which keeps the last call's
// contents: each call clears what must start at zero.  A call for another n
// first waits for the device to finish earlier work, so calls in a row stay
// safe; calls that overlap on the GPU (two streams at once) race on it.
// ============================================================================
#include <mutex>

namespace {
constexpr int64_t NOALLOC_MAX_N = 8192;
constexpr size_t NOALLOC_BYTES = size_t(4) << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoallocState {
    bool have_base = false;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
    int64_t n = 0;                   // length the tables in the array belong to (0: none)
    ozfft_plan_s plan;               // views into the array, never freed
};
NoallocState g_noalloc[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mutex;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// the NTT twiddle table of one prime (same entries as plan_build's host table):
// tw[2^s + i] = w^((N/2^(s+1)) bitrev_s(i)) with its Shoup quotient, tw[0] = 1
__global__ void noalloc_twiddle_kernel(uint2* tw, int64_t N, uint32_t p, uint32_t w)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t e = 0;
        if (k > 0) {
            const int s = 63 - __clzll((long long)k);
            const int64_t i = k - (int64_t(1) << s);
            int64_t r = 0;
            for (int b = 0; b < s; ++b)
                if (i >> b & 1) r |= int64_t(1) << (s - 1 - b);
            e = (uint64_t)((N >> (s + 1)) * r);
        }
        uint64_t a = 1, x = w;
        for (; e; e >>= 1) {
            if (e & 1) a = a * x % p;
            x = x * x % p;
        }
        tw[k] = make_uint2((uint32_t)a, (uint32_t)((a << 32) / p));
    }
}

static unsigned char* noalloc_take(unsigned char*& cur, size_t bytes)
{
    unsigned char* q = cur;
    cur += (bytes + 255) & ~size_t(255);
    return q;
}

// lay the plan's buffers out in the array and build the tables for length n
static int noalloc_setup(NoallocState& st, int dev, int64_t n, int64_t N, int alpha)
{
    if (!st.have_base) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(OZFFT_ERR_CUDA, std::string("ozfft_execute_noalloc: cudaGetSymbolAddress: ") +
                                            cudaGetErrorString(e));
        st.base = (unsigned char*)ptr;
        st.have_base = true;
    }
    // a previous call's kernels (on any stream) may still read the tables that
    // are about to be rewritten: wait for them, so that calls in a row on one
    // stream stay safe when n changes
    CUDA_TRY(cudaDeviceSynchronize());
    st.n = 0;
    ozfft_plan_s& p = st.plan;
    const int K = 3, P = 2, NM = (int)NOALLOC_MAX_N;
    p.n = n; p.N = N; p.B = 1; p.K = K; p.L = 1; p.P = P; p.G = K * K; p.alpha = alpha; p.debug = 0; p.chunk = 1;
    p.garner_u = garner_u_ok(n, 1, alpha);
    p.device = dev; p.profiling = false; p.bytes = 0;
    p.split_fused = 0;   // no redo flags in the static workspace (and N <= 2^13: one column stage at most)
    unsigned char* cur = st.base;
    p.chirp = (double2*)noalloc_take(cur, sizeof(double2) * NM);
    p.tw = (uint2*)noalloc_take(cur, sizeof(uint2) * P * NM);
    p.twinv = (uint2*)noalloc_take(cur, sizeof(uint2) * P * NM);
    p.Ym = (uint32_t*)noalloc_take(cur, sizeof(uint32_t) * 2 * K * P * NM);
    p.wk = (int32_t*)noalloc_take(cur, sizeof(int32_t) * 2);
    p.wsexp = (int32_t*)noalloc_take(cur, sizeof(int32_t) * 2 * K);
    p.r = (double*)noalloc_take(cur, sizeof(double) * 2 * NM);
    p.mu = (uint64_t*)noalloc_take(cur, sizeof(uint64_t) * 2 * (K + 1));
    p.X = (uint32_t*)noalloc_take(cur, sizeof(uint32_t) * 2 * K * P * NM);
    p.kcnt = (int32_t*)noalloc_take(cur, sizeof(int32_t) * 2);
    p.sched = (Sched*)noalloc_take(cur, sizeof(Sched) * 4);
    p.span = (int32_t*)noalloc_take(cur, sizeof(int32_t) * 3);
    p.Z = (uint32_t*)noalloc_take(cur, sizeof(uint32_t) * 4 * K * K * P * NM);
    p.status = (int*)noalloc_take(cur, sizeof(int));
    if ((size_t)(cur - st.base) > NOALLOC_BYTES)
        return fail(OZFFT_ERR_ALLOC, "ozfft_execute_noalloc: static workspace layout exceeds its array");

    // tables: twiddles, chirp, then w~*'s split and forward NTTs (as plan_build)
    for (int i = 0; i < P; ++i) {
        const uint64_t pr = prime_of(i);
        const uint64_t w = powmod_h(primitive_root_h(pr), (pr - 1) / (uint64_t)N, pr);
        noalloc_twiddle_kernel<<<(unsigned)((N + 255) / 256), 256>>>(p.tw + (int64_t)i * N, N, (uint32_t)pr, (uint32_t)w);
        noalloc_twiddle_kernel<<<(unsigned)((N + 255) / 256), 256>>>(p.twinv + (int64_t)i * N, N, (uint32_t)pr,
                                                                    (uint32_t)powmod_h(w, pr - 2, pr));
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(launch_chirp(p.chirp, n, 0));
    CUDA_TRY(cudaMemset(p.status, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(p.mu, 0, sizeof(uint64_t) * 2 * (K + 1)));
    CUDA_TRY(launch_wstar(p.chirp, n, N, 1, nullptr, p.r, p.mu, K, p.status, 0));
    for (int k = 0; k < K; ++k)
        CUDA_TRY(launch_split_level(k, p.r, p.mu, p.mu, N, 2, K, alpha, nullptr, P, p.Ym, k + 1 < K, p.status, 0));
    uint64_t hmu[2 * (MAX_K + 1)];
    CUDA_TRY(cudaMemcpy(hmu, p.mu, sizeof(uint64_t) * 2 * (K + 1), cudaMemcpyDeviceToHost));
    int32_t sexp[2 * MAX_K] = {0};
    for (int v = 0; v < 2; ++v) {
        int k = 0;
        for (; k < K; ++k) {
            double m;
            std::memcpy(&m, &hmu[v * (K + 1) + k], sizeof m);
            if (!(m > 0.0)) break;
            sexp[v * K + k] = alpha - ceil_log2_h(m);
        }
        p.wk_host[v] = k;
    }
    CUDA_TRY(cudaMemcpy(p.wk, p.wk_host, sizeof(int32_t) * 2, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p.wsexp, sexp, sizeof(int32_t) * 2 * K, cudaMemcpyHostToDevice));
    ntt_configure(p.geom_fwd, N);
    p.geom_fwd.P = P;
    p.geom_fwd.K = K;
    p.geom_fwd.G = p.G;
    p.geom_fwd.mac_reg = 1;   // L = 1
    p.geom_fwd.inv_vecs_per_cta = INV_ROW_VECS;
    p.geom_inv = p.geom_fwd;
    NttGeom gw = p.geom_fwd;
    gw.nvec = (int64_t)2 * K * P;
    gw.kcnt = p.wk;
    CUDA_TRY(launch_ntt_forward(gw, p.Ym, p.tw, 0));
    uint32_t c[3] = {0, 0, 0};
    for (int i = 0; i < P; ++i) {
        const uint64_t pr = prime_of(i);
        c[i] = (uint32_t)mulmod_h(powmod_h((uint64_t)N % pr, pr - 2, pr), mulmod_h(1ull << 32, 1ull << 32, pr), pr);
    }
    const int64_t total = (int64_t)2 * K * P * N;
    ymont_kernel<<<(unsigned)((total + 255) / 256), 256>>>(p.Ym, N, total, P, c[0], c[1], c[2]);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemset(p.sched, 0, sizeof(Sched) * 4));
    CUDA_TRY(cudaMemset(p.kcnt, 0, sizeof(int32_t) * 2));
    CUDA_TRY(cudaDeviceSynchronize());
    int stv = 0;
    CUDA_TRY(cudaMemcpy(&stv, p.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (stv) return fail(OZFFT_ERR_RANGE, "ozfft_execute_noalloc: w* split status");
    p.geom_fwd.nvec = 2 * K * P;
    p.geom_fwd.kcnt = p.kcnt;
    p.geom_fwd.sched = p.sched;
    p.geom_inv.nvec = 4 * p.G * P;
    p.geom_inv.kcnt = p.kcnt;
    p.geom_inv.sched = p.sched;
    CUDA_TRY(crt_init());   // Garner constants of this device (per device, once)
    st.n = n;
    return OZFFT_OK;
}

extern "C" int ozfft_execute_noalloc(int64_t n, int direction, const void* in, void* out, void* stream)
{
    if (!in || !out || n < 1 || (direction != OZFFT_FORWARD && direction != OZFFT_INVERSE))
        return fail(OZFFT_ERR_ARG, "ozfft_execute_noalloc: bad argument");
    int64_t N = n;
    if (n & (n - 1)) { N = 1; while (N < 2 * n - 1) N <<= 1; }
    if (N > NOALLOC_MAX_N)
        return fail(OZFFT_ERR_LENGTH, "ozfft_execute_noalloc: convolution length " + std::to_string(N) +
                                          " exceeds the static workspace limit " + std::to_string(NOALLOC_MAX_N) +
                                          " (n <= 8192 for powers of two, n <= 4096 otherwise)");
    const int alpha = alpha_h(n, 1, 2);
    if (alpha < 1) return fail(OZFFT_ERR_LENGTH, "ozfft_execute_noalloc: no split width for this n");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(OZFFT_ERR_ARG, "ozfft_execute_noalloc: device index");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocState& st = g_noalloc[dev];
    if (st.n != n) {
        const int rc = noalloc_setup(st, dev, n, N, alpha);
        if (rc != OZFFT_OK) return rc;
    }
    st.plan.direction = direction;
    CUDA_TRY(cudaMemsetAsync(st.plan.status, 0, sizeof(int), (cudaStream_t)stream));
    return ozfft_execute(&st.plan, in, out, stream);
}
