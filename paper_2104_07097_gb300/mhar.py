"""Thin ctypes binding of libmhar (include/mhar.h): argument marshalling only.

Every step of the sampler runs in the library's CUDA kernels.  If the shared
library is missing or cannot be loaded this module raises; there is no CPU
fallback.  The same names as the C ABI are exported (``mhar_create``,
``mhar_run``, ...), plus a small ``Sampler`` convenience class.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FP64 = 0
FP32 = 1
MIXED_F16X3 = 2
MIXED_RECOMPUTE = 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed": MIXED_F16X3, "f16x3": MIXED_F16X3,
              "mixed_rs": MIXED_RECOMPUTE}

OK = 0
E_ARG = -1
E_X0_INFEASIBLE = -2
E_UNBOUNDED = -3
E_NONFINITE = -4
E_CUDA = -5
E_RANK = -6
E_UNSUPPORTED = -7
E_TIMEOUT = -8
E_INFEASIBLE_DRIFT = -9

ST_UNBOUNDED = 1
ST_STALL = 2
ST_NONFINITE = 4
ST_DRIFT = 8

# Every symbol include/mhar.h declares.
EXPORTS = ("mhar_default_opts", "mhar_create", "mhar_run", "mhar_get_state", "mhar_set_state",
           "mhar_get_chord", "mhar_check", "mhar_get_stats", "mhar_time_kernels",
           "mhar_chord_noalloc", "mhar_set_preconditioner", "mhar_get_preconditioner",
           "mhar_fit_preconditioner", "mhar_fit_moments", "mhar_fit_from_moments",
           "mhar_batch_create", "mhar_batch_tune", "mhar_batch_set_shape", "mhar_batch_run",
           "mhar_batch_set_bucket_shape", "mhar_batch_get_shapes",
           "mhar_batch_get_state", "mhar_batch_check", "mhar_batch_last_error",
           "mhar_batch_destroy", "mhar_kernel_name", "mhar_last_error", "mhar_strerror",
           "mhar_status_code", "mhar_set_audit", "mhar_batch_set_audit", "mhar_destroy")


class MharOpts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("refresh_k", ctypes.c_int32), ("out_on_device", ctypes.c_int32),
                ("walker0", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("graph_chunk", ctypes.c_int32), ("refresh_fp64", ctypes.c_int32),
                ("smem_operands", ctypes.c_int32), ("emit_walkers", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("audit_every", ctypes.c_int32),
                ("audit_walkers", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class MharStats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_uint64), ("walker_steps", ctypes.c_int64),
                ("stalls", ctypes.c_int64), ("unbounded", ctypes.c_int64),
                ("status_bits", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("refresh_drift", ctypes.c_double), ("max_violation", ctypes.c_double),
                ("eq_residual", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("run_max_violation", ctypes.c_double), ("run_eq_residual", ctypes.c_double),
                ("audits", ctypes.c_int64)]


class MharProblem(ctypes.Structure):
    _fields_ = [("A", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.POINTER(ctypes.c_double)),
                ("m", ctypes.c_int32), ("n", ctypes.c_int32),
                ("x0", ctypes.POINTER(ctypes.c_double))]


class MharError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} ({code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads libmhar.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmhar.so not built ({path}); run paper_2104_07097_gb300.build.build()")
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    lib.mhar_default_opts.argtypes = [ctypes.POINTER(MharOpts)]
    lib.mhar_default_opts.restype = None
    lib.mhar_create.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp,
                                ctypes.c_int, ctypes.POINTER(MharOpts), ctypes.POINTER(vp)]
    lib.mhar_create.restype = ctypes.c_int
    lib.mhar_run.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, vp]
    lib.mhar_run.restype = ctypes.c_int
    lib.mhar_get_state.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_uint64)]
    lib.mhar_get_state.restype = ctypes.c_int
    lib.mhar_set_state.argtypes = [vp, dp, ctypes.c_uint64]
    lib.mhar_set_state.restype = ctypes.c_int
    lib.mhar_get_chord.argtypes = [vp, dp, dp, dp]
    lib.mhar_get_chord.restype = ctypes.c_int
    lib.mhar_check.argtypes = [vp, ctypes.POINTER(MharStats)]
    lib.mhar_check.restype = ctypes.c_int
    lib.mhar_get_stats.argtypes = [vp, ctypes.POINTER(MharStats)]
    lib.mhar_get_stats.restype = ctypes.c_int
    lib.mhar_time_kernels.argtypes = [vp, ctypes.c_int, dp]
    lib.mhar_time_kernels.restype = ctypes.c_int
    lib.mhar_chord_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int,
                                       vp, vp, vp]
    lib.mhar_chord_noalloc.restype = ctypes.c_int
    lib.mhar_set_preconditioner.argtypes = [vp, dp, dp, ctypes.c_int32]
    lib.mhar_set_preconditioner.restype = ctypes.c_int
    lib.mhar_get_preconditioner.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int32)]
    lib.mhar_get_preconditioner.restype = ctypes.c_int
    lib.mhar_fit_preconditioner.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32]
    lib.mhar_fit_preconditioner.restype = ctypes.c_int
    lib.mhar_fit_moments.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, dp, dp, dp,
                                     ctypes.POINTER(ctypes.c_int64)]
    lib.mhar_fit_moments.restype = ctypes.c_int
    lib.mhar_fit_from_moments.argtypes = [vp, dp, dp, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_int32]
    lib.mhar_fit_from_moments.restype = ctypes.c_int
    lib.mhar_batch_create.argtypes = [ctypes.POINTER(MharProblem), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(MharOpts), ctypes.POINTER(vp)]
    lib.mhar_batch_create.restype = ctypes.c_int
    lib.mhar_batch_tune.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    lib.mhar_batch_tune.restype = ctypes.c_int
    lib.mhar_batch_set_shape.argtypes = [vp, ctypes.c_int32]
    lib.mhar_batch_set_shape.restype = ctypes.c_int
    lib.mhar_batch_set_bucket_shape.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    lib.mhar_batch_set_bucket_shape.restype = ctypes.c_int
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.mhar_batch_get_shapes.argtypes = [vp, i32p, i32p, i32p]
    lib.mhar_batch_get_shapes.restype = ctypes.c_int
    lib.mhar_batch_run.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(vp)]
    lib.mhar_batch_run.restype = ctypes.c_int
    lib.mhar_batch_get_state.argtypes = [vp, ctypes.c_int32, dp, ctypes.POINTER(ctypes.c_uint64)]
    lib.mhar_batch_get_state.restype = ctypes.c_int
    lib.mhar_batch_check.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(MharStats)]
    lib.mhar_batch_check.restype = ctypes.c_int
    lib.mhar_batch_last_error.argtypes = [vp]
    lib.mhar_batch_last_error.restype = ctypes.c_char_p
    lib.mhar_batch_destroy.argtypes = [vp]
    lib.mhar_batch_destroy.restype = None
    lib.mhar_kernel_name.argtypes = [vp]
    lib.mhar_kernel_name.restype = ctypes.c_char_p
    lib.mhar_last_error.argtypes = [vp]
    lib.mhar_last_error.restype = ctypes.c_char_p
    lib.mhar_strerror.argtypes = [ctypes.c_int]
    lib.mhar_strerror.restype = ctypes.c_char_p
    lib.mhar_status_code.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.mhar_status_code.restype = ctypes.c_int
    lib.mhar_set_audit.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    lib.mhar_set_audit.restype = ctypes.c_int
    lib.mhar_batch_set_audit.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    lib.mhar_batch_set_audit.restype = ctypes.c_int
    lib.mhar_destroy.argtypes = [vp]
    lib.mhar_destroy.restype = None
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def mhar_default_opts() -> MharOpts:
    o = MharOpts()
    load().mhar_default_opts(ctypes.byref(o))
    return o


def mhar_strerror(code: int) -> str:
    return load().mhar_strerror(code).decode()


def mhar_last_error(ctx) -> str:
    return load().mhar_last_error(ctx).decode()


def mhar_status_code(status_bits: int, wait_expired: int) -> int:
    return load().mhar_status_code(int(status_bits), int(wait_expired))


def mhar_create(A, b, AE, bE, x0, z: int, opts: MharOpts):
    A, b, x0 = _f64(A), _f64(b), _f64(x0)
    m, n = A.shape
    AE = None if AE is None or np.size(AE) == 0 else _f64(np.atleast_2d(AE))
    bE = None if AE is None else _f64(np.atleast_1d(bE))
    mE = 0 if AE is None else AE.shape[0]
    ctx = ctypes.c_void_p()
    rc = load().mhar_create(_dp(A), _dp(b), m, n, _dp(AE), _dp(bE), mE, _dp(x0), int(z),
                            ctypes.byref(opts), ctypes.byref(ctx))
    if rc != OK:
        raise MharError(rc, f"mhar_create failed: {mhar_strerror(rc)}: {mhar_last_error(None)}")
    return ctx


def mhar_run(ctx, steps: int, thin: int, out_ptr) -> int:
    return load().mhar_run(ctx, int(steps), int(thin), out_ptr)


def mhar_destroy(ctx) -> None:
    if ctx:
        load().mhar_destroy(ctx)


def mhar_get_state(ctx, z: int, n: int):
    X = np.zeros((z, n))
    step = ctypes.c_uint64()
    rc = load().mhar_get_state(ctx, _dp(X), ctypes.byref(step))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    return X, int(step.value)


def mhar_set_state(ctx, X, step: int) -> None:
    X = _f64(X)
    rc = load().mhar_set_state(ctx, _dp(X), int(step))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))


def mhar_get_chord(ctx, z: int):
    lo, hi, t = np.zeros(z), np.zeros(z), np.zeros(z)
    rc = load().mhar_get_chord(ctx, _dp(lo), _dp(hi), _dp(t))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    return lo, hi, t


def mhar_check(ctx) -> MharStats:
    s = MharStats()
    rc = load().mhar_check(ctx, ctypes.byref(s))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    return s


def mhar_get_stats(ctx) -> MharStats:
    s = MharStats()
    rc = load().mhar_get_stats(ctx, ctypes.byref(s))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    return s


def mhar_time_kernels(ctx, iters: int):
    ms = np.zeros(3)
    rc = load().mhar_time_kernels(ctx, int(iters), _dp(ms))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    return ms


def mhar_set_preconditioner(ctx, n: int, delta, U=None) -> None:
    """delta None removes the preconditioner; U is n x r (r <= 32) or None."""
    if delta is None:
        rc = load().mhar_set_preconditioner(ctx, None, None, 0)
    else:
        delta = _f64(delta).reshape(n)
        r = 0
        if U is not None and np.size(U) > 0:
            U = _f64(U).reshape(n, -1)
            r = U.shape[1]
        else:
            U = None
        rc = load().mhar_set_preconditioner(ctx, _dp(delta), _dp(U), r)
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))


def mhar_get_preconditioner(ctx, n: int):
    """(delta, U) or None when directions are isotropic."""
    r = ctypes.c_int32()
    rc = load().mhar_get_preconditioner(ctx, None, None, ctypes.byref(r))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    if r.value < 0:
        return None
    delta = np.zeros(n)
    U = np.zeros((n, r.value))
    rc = load().mhar_get_preconditioner(ctx, _dp(delta), _dp(U) if r.value > 0 else None,
                                        ctypes.byref(r))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    return delta, U


def mhar_fit_preconditioner(ctx, warmup: int, snapshots: int, rank: int, power_iters: int) -> None:
    rc = load().mhar_fit_preconditioner(ctx, int(warmup), int(snapshots), int(rank),
                                        int(power_iters))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))


def mhar_fit_moments(ctx, n: int, warmup: int, snapshots: int, shift=None):
    """(s1, s2, count) of the warm-up points about `shift` (see mhar.h)."""
    s1 = np.zeros(n)
    s2 = np.zeros((n, n))
    count = ctypes.c_int64()
    sh = None if shift is None else _f64(shift)
    rc = load().mhar_fit_moments(ctx, int(warmup), int(snapshots), _dp(sh), _dp(s1), _dp(s2),
                                 ctypes.byref(count))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))
    return s1, s2, int(count.value)


def mhar_fit_from_moments(ctx, s1, s2, count: int, rank: int, power_iters: int) -> None:
    s1, s2 = _f64(s1), _f64(s2)
    rc = load().mhar_fit_from_moments(ctx, _dp(s1), _dp(s2), int(count), int(rank),
                                      int(power_iters))
    if rc != OK:
        raise MharError(rc, mhar_last_error(ctx))


def mhar_chord_noalloc(A_ptr, b_ptr, m: int, n: int, X_ptr, D_ptr, z: int, lmin_ptr, lmax_ptr,
                       stream=None) -> int:
    """Allocation-free chord of every walker; all array arguments are device
    pointers (ints) to FP64 row-major buffers.  Returns the C return code."""
    vp = ctypes.c_void_p
    s = None if stream is None else vp(int(getattr(stream, "cuda_stream", stream)))
    return load().mhar_chord_noalloc(vp(A_ptr), vp(b_ptr), int(m), int(n), vp(X_ptr), vp(D_ptr),
                                     int(z), vp(lmin_ptr), vp(lmax_ptr), s)


class Sampler:
    """z MHAR walkers on {A x <= b, AE x = bE} (Algorithm 2), all starting at x0.

    ``precision``: "fp64" | "fp32" | "mixed" (stored slack) | "mixed_rs"
    (slack recomputed on the tensor cores every iteration).  ``stream``: a torch.cuda.Stream,
    a raw cudaStream_t (int) or None.
    """

    def __init__(self, A, b, x0, z: int, AE=None, bE=None, precision: str | int = "fp64",
                 seed: int = 0, refresh_k: int = 64, walker0: int = 0, stream=None,
                 graph_chunk: int = 16, out_on_device: bool = False, refresh_fp64: bool = False,
                 smem_operands: bool = False, emit_walkers: int = 0, schedule: int = 0,
                 audit_every: int = 0, audit_walkers: int = 0):
        o = mhar_default_opts()
        o.seed = int(seed)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.refresh_k = int(refresh_k)
        o.walker0 = int(walker0)
        o.graph_chunk = int(graph_chunk)
        o.out_on_device = 1 if out_on_device else 0
        o.refresh_fp64 = 1 if refresh_fp64 else 0
        o.smem_operands = 1 if smem_operands else 0
        o.emit_walkers = int(emit_walkers)
        o.schedule = int(schedule)
        o.audit_every = int(audit_every)
        o.audit_walkers = int(audit_walkers)
        if stream is not None:
            o.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        A = _f64(A)
        self.m, self.n = A.shape
        self.z = int(z) if z > 0 else max(self.m, self.n) + 1
        self.out_on_device = out_on_device
        self.emit_walkers = int(emit_walkers) if emit_walkers > 0 else self.z
        self._ctx = mhar_create(A, b, AE, bE, x0, self.z, o)

    def run(self, steps: int, thin: int = 0, out=None):
        """Advances `steps` iterations; with thin > 0 returns (or fills) the
        floor(steps/thin) x W x n samples (W = emit_walkers, default z).
        `out` may be a numpy array (host)
        or, for out_on_device samplers, a CUDA tensor / raw device pointer."""
        nsamp = steps // thin if thin > 0 else 0
        ptr = None
        if nsamp > 0:
            if out is None:
                if self.out_on_device:
                    raise ValueError("out_on_device sampler needs a device `out`")
                out = np.zeros((nsamp, self.emit_walkers, self.n))
            if isinstance(out, np.ndarray):
                if (out.dtype != np.float64 or not out.flags.c_contiguous
                        or out.size < nsamp * self.emit_walkers * self.n):
                    raise ValueError("out must be a C-contiguous float64 array of the sample shape")
                ptr = ctypes.c_void_p(out.ctypes.data)
            elif hasattr(out, "data_ptr"):
                ptr = ctypes.c_void_p(out.data_ptr())
            else:
                ptr = ctypes.c_void_p(int(out))
        rc = mhar_run(self._ctx, steps, thin, ptr)
        if rc != OK:
            raise MharError(rc, mhar_last_error(self._ctx))
        return out

    def state(self):
        return mhar_get_state(self._ctx, self.z, self.n)

    def set_state(self, X, step: int) -> None:
        mhar_set_state(self._ctx, X, step)

    def chord(self):
        return mhar_get_chord(self._ctx, self.z)

    def check(self) -> MharStats:
        return mhar_check(self._ctx)

    def stats(self) -> MharStats:
        return mhar_get_stats(self._ctx)

    def set_audit(self, every: int, walkers: int = 0) -> None:
        """FP64 feasibility audit after every `every` iterations (0: off)."""
        rc = load().mhar_set_audit(self._ctx, int(every), int(walkers))
        if rc != OK:
            raise MharError(rc, mhar_last_error(self._ctx))

    def set_preconditioner(self, delta, U=None) -> None:
        """Directions d = P (delta * h + U g); delta None restores isotropic ones."""
        mhar_set_preconditioner(self._ctx, self.n, delta, U)

    def preconditioner(self):
        return mhar_get_preconditioner(self._ctx, self.n)

    def fit_preconditioner(self, warmup: int, snapshots: int = 10, rank: int = 32,
                           power_iters: int = 4) -> None:
        """Learns (delta, U) from `warmup` iterations of the chain and freezes it."""
        mhar_fit_preconditioner(self._ctx, warmup, snapshots, min(rank, self.n), power_iters)

    def fit_moments(self, warmup: int, snapshots: int = 10, shift=None):
        """The warm-up half of the fit: (s1, s2, count) about `shift`, to be
        summed over the shards of one ensemble and passed to fit_from_moments."""
        return mhar_fit_moments(self._ctx, self.n, warmup, snapshots, shift)

    def fit_from_moments(self, s1, s2, count: int, rank: int = 32, power_iters: int = 4) -> None:
        """The factor half of the fit, from (pooled) moments; then frozen."""
        mhar_fit_from_moments(self._ctx, s1, s2, count, min(rank, self.n), power_iters)

    def kernel_name(self) -> str:
        """The kernel that runs each iteration's chord on this sampler."""
        return load().mhar_kernel_name(self._ctx).decode()

    def time_kernels(self, iters: int):
        """Average device ms of (directions, chord+update, refresh)."""
        return mhar_time_kernels(self._ctx, iters)

    def close(self) -> None:
        if getattr(self, "_ctx", None):
            mhar_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many polytopes advanced together, a chord launch and a walker-update
    launch per iteration (``mhar_batch_*``).  ``problems``: list of (A, b, x0); problem p uses
    Philox key seed + p; every problem has z walkers; recompute tensor-core mode."""

    def __init__(self, problems, z: int, seed: int = 0, stream=None, out_on_device: bool = False,
                 emit_walkers: int = 0, audit_every: int = 0, audit_walkers: int = 0):
        o = mhar_default_opts()
        o.seed = int(seed)
        o.precision = MIXED_RECOMPUTE
        o.out_on_device = 1 if out_on_device else 0
        o.emit_walkers = int(emit_walkers)
        o.audit_every = int(audit_every)
        o.audit_walkers = int(audit_walkers)
        if stream is not None:
            o.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        self._keep = []
        arr = (MharProblem * len(problems))()
        self.shapes = []
        for q, (A, b, x0) in enumerate(problems):
            A, b, x0 = _f64(A), _f64(b), _f64(x0)
            self._keep += [A, b, x0]
            m, n = A.shape
            arr[q] = MharProblem(_dp(A), _dp(b), m, n, _dp(x0))
            self.shapes.append((m, n))
        self.z = int(z)
        self.emit_walkers = int(emit_walkers) if emit_walkers > 0 else self.z
        self.out_on_device = out_on_device
        ctx = ctypes.c_void_p()
        rc = load().mhar_batch_create(arr, len(problems), self.z, ctypes.byref(o), ctypes.byref(ctx))
        if rc != OK:
            raise MharError(rc, f"mhar_batch_create failed: {mhar_strerror(rc)}: "
                                f"{mhar_last_error(None)}")
        self._b = ctx

    def _err(self, rc):
        raise MharError(rc, load().mhar_batch_last_error(self._b).decode())

    def tune(self, iters: int = 8) -> int:
        """The autotuner: returns the single shape kept (0, 1, 2, 4, 8) or -1
        for per-bucket shapes (see ``get_shapes``)."""
        c = ctypes.c_int32()
        rc = load().mhar_batch_tune(self._b, int(iters), ctypes.byref(c))
        if rc != OK:
            self._err(rc)
        return int(c.value)

    def set_shape(self, shape: int) -> None:
        """0: the persistent launch (CTAs pull units from a device queue); 1, 2,
        4, 8: clusters of that many CTAs per unit."""
        rc = load().mhar_batch_set_shape(self._b, int(shape))
        if rc != OK:
            self._err(rc)

    def set_bucket_shape(self, bucket: int, shape: int) -> None:
        """Per-bucket mode; bucket 0..4 by the 64-column K chunks of n (1, 2,
        3-4, 5-8, more) gets launch shape ``shape``."""
        rc = load().mhar_batch_set_bucket_shape(self._b, int(bucket), int(shape))
        if rc != OK:
            self._err(rc)

    def get_shapes(self):
        """(per_bucket, shape of each of the 5 buckets (-1: empty), bucket of
        every problem)."""
        per = ctypes.c_int32()
        shapes = (ctypes.c_int32 * 5)()
        of = (ctypes.c_int32 * len(self.shapes))()
        rc = load().mhar_batch_get_shapes(self._b, ctypes.byref(per), shapes, of)
        if rc != OK:
            self._err(rc)
        return bool(per.value), list(shapes), list(of)

    def run(self, steps: int, thin: int = 0, outs=None):
        """Advances every problem; with thin > 0 returns (or fills) one
        floor(steps/thin) x W x n array per problem (host numpy, or device
        tensors / pointers for out_on_device batches)."""
        nsamp = steps // thin if thin > 0 else 0
        ptrs = (ctypes.c_void_p * len(self.shapes))()
        if nsamp > 0:
            if outs is None:
                if self.out_on_device:
                    raise ValueError("out_on_device batch needs device outputs")
                outs = [np.zeros((nsamp, self.emit_walkers, n)) for (_, n) in self.shapes]
            for q, o in enumerate(outs):
                if o is None:
                    ptrs[q] = None
                elif isinstance(o, np.ndarray):
                    ptrs[q] = o.ctypes.data
                elif hasattr(o, "data_ptr"):
                    ptrs[q] = o.data_ptr()
                else:
                    ptrs[q] = int(o)
        rc = load().mhar_batch_run(self._b, int(steps), int(thin), ptrs if nsamp > 0 else None)
        if rc != OK:
            self._err(rc)
        return outs

    def state(self, q: int):
        m, n = self.shapes[q]
        X = np.zeros((self.z, n))
        step = ctypes.c_uint64()
        rc = load().mhar_batch_get_state(self._b, int(q), _dp(X), ctypes.byref(step))
        if rc != OK:
            self._err(rc)
        return X, int(step.value)

    def check(self, q: int) -> MharStats:
        st = MharStats()
        rc = load().mhar_batch_check(self._b, int(q), ctypes.byref(st))
        if rc != OK:
            self._err(rc)
        return st

    def set_audit(self, every: int, walkers: int = 0) -> None:
        rc = load().mhar_batch_set_audit(self._b, int(every), int(walkers))
        if rc != OK:
            self._err(rc)

    def close(self) -> None:
        if getattr(self, "_b", None):
            load().mhar_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
