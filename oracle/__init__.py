"""CPU oracle for the Ozaki-scheme / 32-bit NTT double-precision FFT.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The GPU product path never imports this
package.  The arithmetic lives in ``ozoracle.c`` (plain scalar C, one thread);
this module only compiles it and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ozoracle.c")
LIB = os.path.join(HERE, "liboracle.so")

KMAX = 64
OK, ERR_ARG, ERR_LENGTH, ERR_ALLOC, ERR_NONFINITE, ERR_RANGE = 0, 1, 2, 3, 5, 6
FORWARD, INVERSE = -1, 1
ADJOINT, INVERSE_ADJOINT = 2, -2   # F^H x and (1/n) F x (reverse-mode adjoints)


def build_command():
    # -O3 without -march=native (the library must build and agree on x86-64 and
    # aarch64 hosts); -ffp-contract=off and -fno-fast-math keep every binary64
    # operation as written, so the optimisation level cannot change a result
    cmd = ["gcc", "-O3", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", SRC, "-o", LIB, "-lm"]
    if platform.machine() not in ("aarch64", "arm64"):
        cmd.insert(-1, "-lquadmath")
    return cmd


def build(force: bool = False) -> str:
    """Compile ozoracle.c into liboracle.so (idempotent)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(__file__)):
        subprocess.run(build_command(), check=True)
    return LIB


_lib = None
_lock = threading.Lock()


class Trace(C.Structure):
    _fields_ = [
        ("alpha", C.c_int32), ("rho", C.c_int32),
        ("kcount", C.c_int32 * 4),
        ("sexp", (C.c_int32 * KMAX) * 4),
        ("ngroups", C.c_int32 * 4),
        ("n_fwd_runtime", C.c_int64), ("n_fwd_plan", C.c_int64), ("n_inv", C.c_int64),
        ("kdim", C.c_int32), ("gdim", C.c_int32),
        ("xprime", C.c_void_p), ("wstar", C.c_void_p), ("q", C.c_void_p),
        ("spec", C.c_void_p), ("gS", C.c_void_p), ("gsize", C.c_void_p),
        ("gpairs", C.c_void_p), ("zres", C.c_void_p), ("zcrt", C.c_void_p),
        ("yprime", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.c_void_p
            i64, u64, i32 = C.c_int64, C.c_uint64, C.c_int32
            L.or_prime.restype = u64; L.or_prime.argtypes = [C.c_int]
            L.or_powmod.restype = u64; L.or_powmod.argtypes = [u64, u64, u64]
            L.or_invmod.restype = u64; L.or_invmod.argtypes = [u64, u64]
            L.or_generator.restype = u64; L.or_generator.argtypes = [u64]
            L.or_root.restype = u64; L.or_root.argtypes = [u64, u64]
            L.or_ntt_naive.restype = C.c_int; L.or_ntt_naive.argtypes = [P, P, i64, u64, C.c_int]
            L.or_ntt.restype = C.c_int; L.or_ntt.argtypes = [P, P, i64, u64, C.c_int]
            L.or_alpha.restype = C.c_int; L.or_alpha.argtypes = [i64, i64, C.c_int]
            L.or_chirp.restype = C.c_int; L.or_chirp.argtypes = [i64, P]
            L.or_cmul.restype = None; L.or_cmul.argtypes = [P, P, P, i64]
            L.or_split.restype = C.c_int
            L.or_split.argtypes = [P, i64, C.c_int, C.c_int, C.c_int, P, P, P, P]
            L.or_garner.restype = None; L.or_garner.argtypes = [P, i64, C.c_int, P]
            L.or_exact_sum.restype = None; L.or_exact_sum.argtypes = [P, P, P, i64, P]
            L.or_schedule.restype = C.c_int
            L.or_schedule.argtypes = [C.c_int, P, C.c_int, P, C.c_int, C.c_int, C.c_int, P, P, P]
            L.or_ozfft.restype = C.c_int
            L.or_ozfft.argtypes = [i64, i64, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P]
            L.or_dft_q.restype = C.c_int; L.or_dft_q.argtypes = [i64, P, C.c_int, i64, P, P, P]
            L.or_fft_q.restype = C.c_int; L.or_fft_q.argtypes = [i64, P, C.c_int, P, P]
            L.or_sincospi_q.restype = None; L.or_sincospi_q.argtypes = [u64, u64, P]
            L.or_alpha_ts.restype = C.c_int; L.or_alpha_ts.argtypes = [i64, C.c_int]
            L.or_ts_from_double.restype = None; L.or_ts_from_double.argtypes = [P, i64, P]
            L.or_ts_to_double.restype = None; L.or_ts_to_double.argtypes = [P, i64, P]
            L.or_ts_op.restype = None; L.or_ts_op.argtypes = [C.c_int, P, P, i64, P]
            L.or_ts_split.restype = C.c_int
            L.or_ts_split.argtypes = [P, i64, C.c_int, C.c_int, C.c_int, P, P, P]
            L.or_ozfft_ts.restype = C.c_int
            L.or_ozfft_ts.argtypes = [i64, i64, C.c_int, C.c_int, C.c_int, P, P, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


# --- modular arithmetic ------------------------------------------------------
def prime(i: int) -> int:
    return int(lib().or_prime(i))


def powmod(b, e, m):
    return int(lib().or_powmod(b, e, m))


def invmod(a, p):
    return int(lib().or_invmod(a, p))


def generator(p):
    return int(lib().or_generator(p))


def root(p, N):
    return int(lib().or_root(p, N))


def ntt(a, p, inverse=False, naive=False):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    out = np.empty_like(a)
    f = lib().or_ntt_naive if naive else lib().or_ntt
    st = f(_p(a), _p(out), a.size, p, int(inverse))
    if st:
        raise OracleError(st, "ntt")
    return out


def alpha(n, L, nprimes):
    return int(lib().or_alpha(n, L, nprimes))


def chirp(n):
    w = np.empty(2 * n, dtype=np.float64)
    st = lib().or_chirp(n, _p(w))
    if st:
        raise OracleError(st, "chirp")
    return w[0::2] + 1j * w[1::2]


def cmul(x, y):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.ascontiguousarray(y, dtype=np.complex128)
    z = np.empty_like(x)
    lib().or_cmul(_p(x), _p(y), _p(z), x.size)
    return z


def split(v, alpha_, K, kdim=None, want_slices=True):
    """Alg. 3: returns (slices [k][N] float64, q [k][N] int64, sexp [k], status)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    kdim = kdim or (K if K > 0 else KMAX)
    N = v.size
    sl = np.zeros((kdim, N)) if want_slices else None
    q = np.zeros((kdim, N), dtype=np.int64)
    se = np.zeros(kdim, dtype=np.int32)
    kout = C.c_int32(0)
    st = lib().or_split(_p(v), N, alpha_, K, kdim, _p(sl), _p(q), _p(se), C.byref(kout))
    k = kout.value
    return (sl[:k] if sl is not None else None), q[:k], se[:k].copy(), st


def garner(res, nprimes):
    """res: [nprimes][cnt] uint32 -> list of Python ints (symmetric representatives)."""
    res = np.ascontiguousarray(res, dtype=np.uint32)
    cnt = res.shape[1]
    out = np.empty(2 * cnt, dtype=np.int64)
    lib().or_garner(_p(res), cnt, nprimes, _p(out))
    return [int(np.uint64(out[2 * j])) + (int(out[2 * j + 1]) << 64) for j in range(cnt)]


def int128_to_pairs(vals):
    out = np.empty(2 * len(vals), dtype=np.int64)
    for j, v in enumerate(vals):
        out[2 * j] = np.int64(np.uint64(v & ((1 << 64) - 1)).view(np.int64))
        out[2 * j + 1] = v >> 64
    return out


def exact_sum(zs, Ss, signs=None):
    """round(sum sign_i z_i 2^-S_i) to binary64 (reading R7 of the oracle)."""
    z2 = int128_to_pairs(list(zs))
    S = np.ascontiguousarray(Ss, dtype=np.int32)
    sg = np.ascontiguousarray(signs if signs is not None else np.ones(len(S)), dtype=np.int32)
    out = np.empty(1)
    lib().or_exact_sum(_p(z2), _p(S), _p(sg), len(S), _p(out))
    return float(out[0])


def schedule(sx, sy, L):
    sx = np.ascontiguousarray(sx, dtype=np.int32)
    sy = np.ascontiguousarray(sy, dtype=np.int32)
    kx, ky = sx.size, sy.size
    gdim, pdim = max(1, kx * ky), max(1, min(kx, ky))
    gS = np.zeros(gdim, dtype=np.int32)
    gs = np.zeros(gdim, dtype=np.int32)
    gp = np.zeros((gdim, pdim, 2), dtype=np.int32)
    ng = lib().or_schedule(kx, _p(sx), ky, _p(sy), L, gdim, pdim, _p(gS), _p(gs), _p(gp))
    if ng < 0:
        raise OracleError(ng, "schedule")
    return [(int(gS[g]), [tuple(int(v) for v in gp[g, m]) for m in range(gs[g])]) for g in range(ng)]


def ozfft(x, N=None, K=3, L=1, nprimes=2, direction=FORWARD, trace=None):
    """Alg. 1 around Alg. 8 x 4 (§4.5).  x: complex128 [n].  Returns (y, info).

    trace: optional set of names among {"xprime","wstar","q","spec","groups",
    "zres","zcrt","yprime"} to capture (sized from kdim/gdim below)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    n = x.size
    if N is None:
        N = n if (n & (n - 1)) == 0 else 1 << (2 * n - 2).bit_length()
    y = np.empty(n, dtype=np.complex128)
    tr = Trace()
    keep = {}
    trace = set(trace or ())
    kdim = K if K > 0 else KMAX
    gdim = kdim * kdim
    tr.kdim, tr.gdim = kdim, gdim
    if "xprime" in trace:
        keep["xprime"] = np.zeros((2, N)); tr.xprime = keep["xprime"].ctypes.data
    if "wstar" in trace:
        keep["wstar"] = np.zeros((2, N)); tr.wstar = keep["wstar"].ctypes.data
    if "q" in trace:
        keep["q"] = np.zeros((4, kdim, N), dtype=np.int64); tr.q = keep["q"].ctypes.data
    if "spec" in trace:
        keep["spec"] = np.zeros((4, kdim, nprimes, N), dtype=np.uint32); tr.spec = keep["spec"].ctypes.data
    if "groups" in trace:
        keep["gS"] = np.zeros((4, gdim), dtype=np.int32); tr.gS = keep["gS"].ctypes.data
        keep["gsize"] = np.zeros((4, gdim), dtype=np.int32); tr.gsize = keep["gsize"].ctypes.data
        keep["gpairs"] = np.zeros((4, gdim, kdim, 2), dtype=np.int32); tr.gpairs = keep["gpairs"].ctypes.data
    if "zres" in trace:
        keep["zres"] = np.zeros((4, gdim, nprimes, N), dtype=np.uint32); tr.zres = keep["zres"].ctypes.data
    if "zcrt" in trace:
        keep["zcrt"] = np.zeros((4, gdim, N, 2), dtype=np.int64); tr.zcrt = keep["zcrt"].ctypes.data
    if "yprime" in trace:
        keep["yprime"] = np.zeros(n, dtype=np.complex128); tr.yprime = keep["yprime"].ctypes.data
    st = lib().or_ozfft(n, N, K, L, nprimes, direction, _p(x), _p(y), C.byref(tr))
    info = {
        "status": st, "alpha": tr.alpha, "rho": tr.rho, "N": N,
        "kcount": list(tr.kcount),
        "sexp": [list(tr.sexp[v])[: tr.kcount[v]] for v in range(4)],
        "ngroups": list(tr.ngroups),
        "n_fwd_runtime": tr.n_fwd_runtime, "n_fwd_plan": tr.n_fwd_plan, "n_inv": tr.n_inv,
    }
    info["ntt_runtime"] = info["n_fwd_runtime"] + info["n_inv"]
    info["ntt_total"] = info["ntt_runtime"] + info["n_fwd_plan"]
    info.update(keep)
    if st:
        raise OracleError(st, "ozfft")
    return y, info


# --- TS (triple-single) variant ----------------------------------------------
def alpha_ts(n, L):
    return int(lib().or_alpha_ts(n, L))


def ts_from_double(x):
    """binary64 values -> [cnt, 3] float32 TS words (reading T1)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.empty((x.size, 3), dtype=np.float32)
    lib().or_ts_from_double(_p(x), x.size, _p(out))
    return out


def ts_to_double(t):
    t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.float64)
    lib().or_ts_to_double(_p(t), t.shape[0], _p(out))
    return out


def ts_op(op, a, b):
    """TSAdd ('add'), TSSub ('sub') or TSMul ('mul') of [cnt, 3] float32 arrays."""
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 3)
    b = np.ascontiguousarray(b, dtype=np.float32).reshape(-1, 3)
    out = np.empty_like(a)
    lib().or_ts_op({"add": 0, "sub": 1, "mul": 2}[op], _p(a), _p(b), a.shape[0], _p(out))
    return out


def ts_split(v, alpha, K=0):
    """Alg. 6 on a TS vector v [3, N] (word planes).  Returns (q [k, N] int64, sexp)."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    N = v.shape[1]
    kdim = K if K > 0 else KMAX
    q = np.zeros((kdim, N), dtype=np.int64)
    sexp = np.zeros(KMAX, dtype=np.int32)
    k = C.c_int32(0)
    st = lib().or_ts_split(_p(v), N, alpha, K, kdim, _p(q), _p(sexp), C.byref(k))
    if st:
        raise OracleError(st, "ts_split")
    return q[:k.value], [int(e) for e in sexp[:k.value]]


def ozfft_ts(x, N=None, K=3, L=1, direction=FORWARD, trace=None):
    """The TS variant (Alg. 4 around Alg. 8, readings T1-T4), two primes.
    Returns (y, info) like ozfft."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    n = x.size
    if N is None:
        N = n if (n & (n - 1)) == 0 else 1 << (2 * n - 2).bit_length()
    y = np.empty(n, dtype=np.complex128)
    tr = Trace()
    keep = {}
    trace = set(trace or ())
    kdim = K if K > 0 else KMAX
    gdim = kdim * kdim
    tr.kdim, tr.gdim = kdim, gdim
    if "xprime" in trace:
        keep["xprime"] = np.zeros((2, N)); tr.xprime = keep["xprime"].ctypes.data
    if "q" in trace:
        keep["q"] = np.zeros((4, kdim, N), dtype=np.int64); tr.q = keep["q"].ctypes.data
    if "spec" in trace:
        keep["spec"] = np.zeros((4, kdim, 2, N), dtype=np.uint32); tr.spec = keep["spec"].ctypes.data
    if "groups" in trace:
        keep["gS"] = np.zeros((4, gdim), dtype=np.int32); tr.gS = keep["gS"].ctypes.data
        keep["gsize"] = np.zeros((4, gdim), dtype=np.int32); tr.gsize = keep["gsize"].ctypes.data
        keep["gpairs"] = np.zeros((4, gdim, kdim, 2), dtype=np.int32); tr.gpairs = keep["gpairs"].ctypes.data
    if "zres" in trace:
        keep["zres"] = np.zeros((4, gdim, 2, N), dtype=np.uint32); tr.zres = keep["zres"].ctypes.data
    if "yprime" in trace:
        keep["yprime"] = np.zeros(n, dtype=np.complex128); tr.yprime = keep["yprime"].ctypes.data
    st = lib().or_ozfft_ts(n, N, K, L, direction, _p(x), _p(y), C.byref(tr))
    info = {"status": st, "alpha": tr.alpha, "rho": tr.rho, "N": N, "kcount": list(tr.kcount),
            "sexp": [list(tr.sexp[v])[: tr.kcount[v]] for v in range(4)], "ngroups": list(tr.ngroups),
            "n_fwd_runtime": tr.n_fwd_runtime, "n_fwd_plan": tr.n_fwd_plan, "n_inv": tr.n_inv}
    info.update(keep)
    if st:
        raise OracleError(st, "ozfft_ts")
    return y, info


# --- binary128 reference -------------------------------------------------------
def dft_q(x, direction=FORWARD, bins=None):
    """binary128 naive DFT at `bins` (all if None).  Returns (hi, lo) complex128."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    n = x.size
    b = None if bins is None else np.ascontiguousarray(bins, dtype=np.int64)
    nb = n if b is None else b.size
    hi = np.empty(nb, dtype=np.complex128)
    lo = np.empty(nb, dtype=np.complex128)
    st = lib().or_dft_q(n, _p(x), direction, nb, _p(b), _p(hi), _p(lo))
    if st:
        raise OracleError(st, "dft_q")
    return hi, lo


def fft_q(x, direction=FORWARD):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    hi = np.empty_like(x)
    lo = np.empty_like(x)
    st = lib().or_fft_q(x.size, _p(x), direction, _p(hi), _p(lo))
    if st:
        raise OracleError(st, "fft_q")
    return hi, lo


def sincospi_q(a, d):
    out = np.empty(4)
    lib().or_sincospi_q(a, d, _p(out))
    return out


def rel_l2_error(y, ref_hi, ref_lo):
    """||y - ref|| / ||ref|| with ref = hi + lo kept in two parts (§5.1)."""
    d = (y - ref_hi) - ref_lo
    return float(np.sqrt(np.sum(np.abs(d) ** 2)) / np.sqrt(np.sum(np.abs(ref_hi) ** 2)))
