"""ctypes binding of libozfft (include/ozfft.h).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  There is
no CPU fallback: if libozfft.so is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libozfft.so")

FORWARD, INVERSE = -1, 1
ADJOINT, INVERSE_ADJOINT = 2, -2   # F^H x and (1/n) F x: the adjoints of FORWARD and INVERSE
OK, ERR_ARG, ERR_LENGTH, ERR_ALLOC, ERR_CUDA, ERR_NONFINITE, ERR_RANGE, ERR_TIMEOUT, ERR_LEVELS = range(9)
K_INF, K_INF_CAP = -1, 8   # K = infinity of the paper (split until the residual is zero), level cap
DUMP_CHIRP, DUMP_XPRIME, DUMP_MU, DUMP_XRES, DUMP_XSPEC, DUMP_YSPEC, DUMP_SCHED, DUMP_ZRES = range(8)
MAX_GROUPS, MAX_L = 64, 8

# every symbol include/ozfft.h declares
EXPORTS = ("ozfft_plan", "ozfft_plan_ex", "ozfft_execute", "ozfft_execute_host", "ozfft_get_status",
           "ozfft_get_stats", "ozfft_set_profiling", "ozfft_get_profile", "ozfft_destroy", "ozfft_error_string",
           "ozfft_last_error", "ozfft_debug_dump", "ozfft_execute_noalloc", "ozfft_plan_many",
           "ozfft_measure_butterfly_rate", "ozfft_selftest_wait_timeout", "ozfft_fault_config",
           "ozfft_execute_host_async", "ozfft_execute_host_wait")
PROF_SLOTS = ("premul", "split", "schedule", "ntt_fwd_col", "ntt_fwd_row", "ntt_inv_row", "ntt_inv_col", "crt")


class Options(C.Structure):
    _fields_ = [("K", C.c_int32), ("L", C.c_int32), ("nprimes", C.c_int32), ("conv_len", C.c_int64),
                ("debug", C.c_int32), ("chunk", C.c_int32), ("autotune", C.c_int32), ("no_graph", C.c_int32),
                ("merge", C.c_int32), ("row_log", C.c_int32), ("ts", C.c_int32), ("inv_vecs", C.c_int32),
                ("crt_fuse", C.c_int32), ("split_fuse", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("N", C.c_int64), ("batch", C.c_int64),
                ("K", C.c_int32), ("L", C.c_int32), ("nprimes", C.c_int32), ("alpha", C.c_int32),
                ("direction", C.c_int32), ("wstar_levels", C.c_int32 * 2),
                ("ntt_forward_runtime", C.c_int64), ("ntt_forward_plan", C.c_int64), ("ntt_inverse", C.c_int64),
                ("kernel_launches", C.c_int64), ("workspace_bytes", C.c_int64),
                ("row_log_fwd", C.c_int32), ("row_log_inv", C.c_int32), ("inv_vecs", C.c_int32),
                ("crt_fused_classes", C.c_int32), ("classes", C.c_int32), ("split_fused_classes", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("executions", C.c_int64), ("launches", C.c_int64 * 8), ("ms", C.c_double * 8)]


class OzfftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ozfft error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libozfft.so (raises if it is missing: build it with build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise OzfftError(ERR_ARG, f"{path} not found; run paper_2603_29129_gb300.build.build()")
            L = C.CDLL(path)
            P, i64 = C.c_void_p, C.c_int64
            L.ozfft_plan.restype = P; L.ozfft_plan.argtypes = [i64, i64, C.c_int]
            L.ozfft_plan_ex.restype = P; L.ozfft_plan_ex.argtypes = [i64, i64, C.c_int, C.POINTER(Options)]
            L.ozfft_execute.restype = C.c_int; L.ozfft_execute.argtypes = [P, P, P, P]
            L.ozfft_execute_host.restype = C.c_int; L.ozfft_execute_host.argtypes = [P, P, P, P]
            L.ozfft_execute_host_async.restype = C.c_int; L.ozfft_execute_host_async.argtypes = [P, P, P, P]
            L.ozfft_execute_host_wait.restype = C.c_int; L.ozfft_execute_host_wait.argtypes = [P, P]
            L.ozfft_get_status.restype = C.c_int; L.ozfft_get_status.argtypes = [P, P]
            L.ozfft_get_stats.restype = C.c_int; L.ozfft_get_stats.argtypes = [P, P, C.POINTER(Stats)]
            L.ozfft_set_profiling.restype = C.c_int; L.ozfft_set_profiling.argtypes = [P, C.c_int]
            L.ozfft_get_profile.restype = C.c_int; L.ozfft_get_profile.argtypes = [P, P, C.POINTER(Profile)]
            L.ozfft_destroy.restype = None; L.ozfft_destroy.argtypes = [P]
            L.ozfft_error_string.restype = C.c_char_p; L.ozfft_error_string.argtypes = [C.c_int]
            L.ozfft_last_error.restype = C.c_char_p; L.ozfft_last_error.argtypes = []
            L.ozfft_debug_dump.restype = i64; L.ozfft_debug_dump.argtypes = [P, C.c_int, i64, P, P]
            L.ozfft_execute_noalloc.restype = C.c_int
            L.ozfft_execute_noalloc.argtypes = [i64, C.c_int, P, P, P]
            L.ozfft_measure_butterfly_rate.restype = C.c_int
            L.ozfft_measure_butterfly_rate.argtypes = [C.c_int, C.POINTER(C.c_double), P]
            L.ozfft_selftest_wait_timeout.restype = C.c_int
            L.ozfft_selftest_wait_timeout.argtypes = [P]
            L.ozfft_fault_config.restype = C.c_int
            L.ozfft_fault_config.argtypes = [C.POINTER(C.c_int32), C.POINTER(i64)]
            L.ozfft_plan_many.restype = P
            L.ozfft_plan_many.argtypes = [C.POINTER(i64), i64, C.c_int, C.POINTER(Options)]
            _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        L = load()
        raise OzfftError(rc, f"{L.ozfft_error_string(rc).decode()} ({L.ozfft_last_error().decode()})")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Plan:
    """A plan for `batch` transforms of length n (see ozfft_plan_ex)."""

    def __init__(self, n, batch=1, direction=FORWARD, K=3, L=1, nprimes=2, conv_len=0, debug=False, chunk=0,
                 autotune=False, merge=False, ts=False, row_log=0, inv_vecs=0, crt_fuse=0, split_fuse=0):
        lib = load()
        self.n, self.batch, self.direction = int(n), int(batch), int(direction)
        self.K, self.L, self.nprimes, self.merge, self.ts = int(K), int(L), int(nprimes), bool(merge), bool(ts)
        self.levels = K_INF_CAP if self.K == K_INF else self.K   # level dimension of the buffers
        opt = Options(self.K, self.L, self.nprimes, int(conv_len), int(bool(debug)), int(chunk), int(bool(autotune)), 0,
                      int(self.merge), int(row_log), int(self.ts), int(inv_vecs), int(crt_fuse), int(split_fuse))
        self._h = lib.ozfft_plan_ex(self.n, self.batch, self.direction, C.byref(opt))
        if not self._h:
            raise OzfftError(-1, lib.ozfft_last_error().decode())
        st = self.stats()
        self.N, self.alpha = st["N"], st["alpha"]
        self.total = self.n * self.batch

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ozfft_destroy(h)
            self._h = None

    close = __del__

    # -- execution -------------------------------------------------------------
    def execute(self, x, out=None, stream=None):
        """x: contiguous CUDA complex128 tensor [batch, n] (or [n] for batch 1)."""
        import torch
        if x.dtype != torch.complex128 or not x.is_cuda or not x.is_contiguous():
            raise OzfftError(ERR_ARG, "input must be a contiguous CUDA complex128 tensor")
        if x.numel() != self.total:
            raise OzfftError(ERR_ARG, f"input has {x.numel()} elements, plan wants {self.total}")
        if out is None:
            out = torch.empty_like(x)
        elif out.numel() != self.total or out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous():
            raise OzfftError(ERR_ARG, "output must be a contiguous CUDA complex128 tensor of the input's size")
        _check(load().ozfft_execute(self._h, x.data_ptr(), out.data_ptr(), _stream_ptr(stream)))
        return out

    def execute_ptr(self, in_ptr, out_ptr, stream_ptr):
        _check(load().ozfft_execute(self._h, in_ptr, out_ptr, stream_ptr))

    def _host_ptrs(self, x, out):
        ptrs = []
        for a in (x, out):
            if isinstance(a, np.ndarray):
                ok = a.dtype == np.complex128 and a.flags.c_contiguous and a.size == self.total
                ptrs.append(a.ctypes.data)
            else:
                import torch
                ok = a.dtype == torch.complex128 and a.is_contiguous() and not a.is_cuda and a.numel() == self.total
                ptrs.append(a.data_ptr())
            if not ok:
                raise OzfftError(ERR_ARG, f"host buffers must be contiguous complex128 with {self.total} elements")
        return ptrs

    def execute_host(self, x, out, stream=None):
        """x, out: host buffers (numpy complex128 arrays or pinned CPU tensors) of `total` elements."""
        xp, op = self._host_ptrs(x, out)
        _check(load().ozfft_execute_host(self._h, xp, op, _stream_ptr(stream)))
        return out

    def execute_host_async(self, x, out, stream=None):
        """Enqueue a host-buffer transform (ozfft_execute_host_async); x and out
        are kept alive here and must not be touched until host_wait()."""
        xp, op = self._host_ptrs(x, out)
        _check(load().ozfft_execute_host_async(self._h, xp, op, _stream_ptr(stream)))
        self.__dict__.setdefault("_pending", []).append((x, out))
        return out

    def host_wait(self, stream=None):
        """Wait for every execute_host_async call (ozfft_execute_host_wait)."""
        _check(load().ozfft_execute_host_wait(self._h, _stream_ptr(stream)))
        self.__dict__["_pending"] = []

    def status(self, stream=None):
        return load().ozfft_get_status(self._h, _stream_ptr(stream))

    def stats(self, stream=0):
        s = Stats()
        _check(load().ozfft_get_stats(self._h, _stream_ptr(stream), C.byref(s)))
        d = {name: getattr(s, name) for name, _ in Stats._fields_}
        d["wstar_levels"] = list(s.wstar_levels)
        return d

    def set_profiling(self, enable=True):
        _check(load().ozfft_set_profiling(self._h, int(bool(enable))))

    def profile(self, stream=None):
        """Per-kernel-slot device time summed over the executions since the last call."""
        pr = Profile()
        _check(load().ozfft_get_profile(self._h, _stream_ptr(stream), C.byref(pr)))
        return {"executions": pr.executions,
                "slots": {name: {"launches": pr.launches[i], "ms": pr.ms[i]} for i, name in enumerate(PROF_SLOTS)}}

    # -- test hook -------------------------------------------------------------
    def dump(self, stage, index=0, stream=None):
        lib = load()
        sp = _stream_ptr(stream)
        nbytes = lib.ozfft_debug_dump(self._h, stage, index, None, sp)
        if nbytes < 0:
            _check(-nbytes)
        buf = np.empty(nbytes, dtype=np.uint8)
        got = lib.ozfft_debug_dump(self._h, stage, index, buf.ctypes.data, sp)
        if got < 0:
            _check(-got)
        N, P = self.N, self.nprimes
        K = self.levels
        G = K * K
        if stage == DUMP_CHIRP:
            return buf.view(np.complex128)
        if stage == DUMP_XPRIME:
            return buf.view(np.float64).reshape(2, N)
        if stage == DUMP_MU:
            return buf.view(np.float64).reshape(2, K + 1)
        if stage in (DUMP_XRES, DUMP_XSPEC, DUMP_YSPEC):
            return buf.view(np.uint32).reshape(2, K, P, N)
        if stage == DUMP_SCHED:
            raw = buf.view(np.int32).reshape(4, 1 + 2 * MAX_GROUPS + MAX_GROUPS * MAX_L)
            out = []
            for c in range(4):
                ng = int(raw[c, 0])
                S = raw[c, 1:1 + MAX_GROUPS]
                sz = raw[c, 1 + MAX_GROUPS:1 + 2 * MAX_GROUPS]
                pr = raw[c, 1 + 2 * MAX_GROUPS:].reshape(MAX_GROUPS, MAX_L)
                out.append([(int(S[g]), [(int(v) >> 4, int(v) & 15) for v in pr[g, :sz[g]]]) for g in range(ng)])
            return out
        if stage == DUMP_ZRES:
            return buf.view(np.uint32).reshape(4, G, P, N)
        return buf


class PlanMany(Plan):
    """A plan over signals of uneven lengths (ozfft_plan_many): the input and
    output are packed, signal i at elements [offsets[i], offsets[i+1])."""

    def __init__(self, lengths, direction=FORWARD, K=3, L=1, nprimes=2, chunk=0, autotune=False, graph=True,
                 merge=False, row_log=0, inv_vecs=0, crt_fuse=0, split_fuse=0):
        lib = load()
        lens = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
        self.lengths = lens
        self.offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        self.direction, self.K, self.L, self.nprimes = int(direction), int(K), int(L), int(nprimes)
        self.levels = K_INF_CAP if self.K == K_INF else self.K
        self.merge = bool(merge)
        opt = Options(self.K, self.L, self.nprimes, 0, 0, int(chunk), int(bool(autotune)), int(not graph),
                      int(self.merge), int(row_log), 0, int(inv_vecs), int(crt_fuse), int(split_fuse))
        self._h = lib.ozfft_plan_many(lens.ctypes.data_as(C.POINTER(C.c_int64)), lens.size, self.direction,
                                      C.byref(opt))
        if not self._h:
            raise OzfftError(-1, lib.ozfft_last_error().decode())
        st = self.stats()
        self.n, self.batch, self.N, self.alpha = int(self.offsets[-1]), lens.size, st["N"], st["alpha"]
        self.total = self.n

    def split(self, y):
        """The packed output as a list of per-signal views."""
        return [y[self.offsets[i]:self.offsets[i + 1]] for i in range(self.batch)]


def butterfly_rate(inverse=False, stream=None):
    """Radix-2 NTT butterflies per second with operands in registers (the
    integer roofline's denominator, ozfft_measure_butterfly_rate)."""
    r = C.c_double(0.0)
    _check(load().ozfft_measure_butterfly_rate(int(bool(inverse)), C.byref(r), _stream_ptr(stream)))
    return r.value


def fault_config():
    """(rc, kind, arg) of the host-side fault hook that OZFFT_FAULT selects now
    (ozfft_fault_config; kind 0 none, 1 alloc, 2 status)."""
    k, a = C.c_int32(0), C.c_int64(0)
    rc = load().ozfft_fault_config(C.byref(k), C.byref(a))
    return rc, k.value, a.value


def selftest_wait_timeout(stream=None):
    """Status code of ozfft_selftest_wait_timeout (ERR_TIMEOUT when the bounded
    device wait gave up as it must)."""
    return load().ozfft_selftest_wait_timeout(_stream_ptr(stream))


def execute_noalloc(x, out, direction=FORWARD, stream=None):
    """One transform of a CUDA complex128 vector through ozfft_execute_noalloc,
    which allocates no device memory (its workspace is a static device array;
    n <= 8192 for powers of two, n <= 4096 otherwise)."""
    import torch
    for t in (x, out):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise OzfftError(ERR_ARG, "input and output must be contiguous CUDA complex128 tensors")
    if out.shape != x.shape or out.device != x.device:
        raise OzfftError(ERR_ARG, "input and output must have one shape and one device")
    # the C call runs on the current device: make it the tensors' device
    with torch.cuda.device(x.device):
        _check(load().ozfft_execute_noalloc(x.numel(), int(direction), x.data_ptr(), out.data_ptr(),
                                            _stream_ptr(stream)))
    return out


_plans = {}
_plans_lock = threading.Lock()


def transform(x, direction=FORWARD, K=3, L=1, nprimes=2, stream=None):
    """The transform of the last axis of a CUDA complex128 tensor in `direction`
    (FORWARD, INVERSE, ADJOINT or INVERSE_ADJOINT), with plans cached per
    (length, batch, direction, options, device)."""
    shape = x.shape
    n = shape[-1]
    batch = x.numel() // n
    key = (n, batch, int(direction), K, L, nprimes, x.device.index)
    with _plans_lock:
        p = _plans.get(key)
        if p is None:
            p = _plans[key] = Plan(n, batch, direction, K, L, nprimes)
    return p.execute(x.contiguous().reshape(batch, n), stream=stream).reshape(shape)


def fft(x, K=3, L=1, nprimes=2, stream=None):
    """FP64-accurate DFT (Eq. (3)) of the last axis of a CUDA complex128 tensor.
    Differentiable: with autograd recording and x requiring grad, the backward
    pass runs the adjoint transform through the same kernels."""
    if x.requires_grad:
        import torch
        if torch.is_grad_enabled():
            from .autograd import OzFFTFunction
            return OzFFTFunction.apply(x, FORWARD, K, L, nprimes)
    return transform(x, FORWARD, K, L, nprimes, stream)


def ifft(x, K=3, L=1, nprimes=2, stream=None):
    """FP64-accurate inverse DFT (Eq. (4)); differentiable like fft."""
    if x.requires_grad:
        import torch
        if torch.is_grad_enabled():
            from .autograd import OzFFTFunction
            return OzFFTFunction.apply(x, INVERSE, K, L, nprimes)
    return transform(x, INVERSE, K, L, nprimes, stream)
