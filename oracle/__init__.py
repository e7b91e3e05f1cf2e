"""FP64 CPU oracle for Matrix Hit-and-Run (arXiv 2104.07097), as a ctypes module.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never loads it; the two share no code (this package compiles its
own C source, ``mhar_oracle.c``, with gcc).

Functions follow the paper:
  * ``philox``            -- Philox4x32-10 block function (Salmon et al. 2011),
  * ``direction_normals`` -- Section 4.3, Box-Muller N(0,1) direction entries,
  * ``chord_uniform``     -- the uniform that places theta on the chord,
  * ``projector``         -- Section 3.2, P = I - A_E^T (A_E A_E^T)^{-1} A_E,
  * ``chord``             -- Section 4.4, (lambda_min, lambda_max),
  * ``mhar_run``          -- Algorithm 2 (z walks, thinning),
  * ``stream_normals``    -- the same Box-Muller normals on any Philox stream,
  * ``mhar_run_pre``      -- Algorithm 2 with preconditioned directions
                             d = P (delta * h + U g) (``oracle.precond`` fits them).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhar_oracle.c")
_HDR = os.path.join(_HERE, "mhar_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmhar_oracle.so")

UNBOUNDED = 1
STALL = 2
NONFINITE = 4

STREAM_DIRECTION = 0
STREAM_CHORD = 1
STREAM_LOWRANK = 2
STREAM_FIT = 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest_src:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.orc_philox4x32_10.restype = None
        lib.orc_direction_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_int, dp]
        lib.orc_direction_normals.restype = None
        lib.orc_chord_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        lib.orc_chord_uniform.restype = ctypes.c_double
        lib.orc_projector.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        lib.orc_projector.restype = ctypes.c_int
        lib.orc_chord.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        lib.orc_chord.restype = ctypes.c_int
        lib.orc_mhar_run.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp]
        lib.orc_mhar_run.restype = ctypes.c_int
        lib.orc_stream_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_int, dp]
        lib.orc_stream_normals.restype = None
        lib.orc_mhar_run_pre.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                         ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_int64, ctypes.c_int64, dp, dp, ctypes.c_int,
                                         dp, dp, dp, dp]
        lib.orc_mhar_run_pre.restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox(ctr, key) -> np.ndarray:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def direction_normals(seed: int, step: int, walker: int, n: int) -> np.ndarray:
    lib = _load()
    h = np.zeros(n, dtype=np.float64)
    lib.orc_direction_normals(seed, step, walker, n, _ptr(h))
    return h


def stream_normals(seed: int, step: int, walker: int, stream: int, count: int) -> np.ndarray:
    """``count`` N(0,1) values of Philox stream ``stream`` for (step, walker)."""
    lib = _load()
    h = np.zeros(max(count, 1), dtype=np.float64)
    lib.orc_stream_normals(seed, step, walker, stream, count, _ptr(h))
    return h[:count]


def chord_uniform(seed: int, step: int, walker: int) -> float:
    return float(_load().orc_chord_uniform(seed, step, walker))


def projector(AE) -> np.ndarray:
    AE = _f64(np.atleast_2d(AE))
    mE, n = AE.shape
    P = np.zeros((n, n), dtype=np.float64)
    rc = _load().orc_projector(_ptr(AE), mE, n, _ptr(P))
    if rc != 0:
        raise ValueError("A_E A_E^T is not positive definite")
    return P


def chord(A, b, x, d):
    A = _f64(A)
    b = _f64(b)
    x = _f64(x)
    d = _f64(d)
    m, n = A.shape
    lo = ctypes.c_double()
    hi = ctypes.c_double()
    st = _load().orc_chord(_ptr(A), _ptr(b), m, n, _ptr(x), _ptr(d), ctypes.byref(lo),
                           ctypes.byref(hi))
    return lo.value, hi.value, st


def mhar_run(A, b, X0, steps: int, thin: int = 1, seed: int = 0, step0: int = 0,
             AE=None, walker0: int = 0, P=None, trace: bool = False):
    """Algorithm 2 from per-walker starts X0 (z x n).

    Returns a dict with ``X`` (final z x n), ``samples`` (floor(steps/thin) x z x n),
    ``status`` and, when ``trace``, ``t``, ``lmin``, ``lmax`` (steps x z).
    ``P`` may be passed to reuse a projector; otherwise it is built from ``AE``.
    """
    return mhar_run_pre(A, b, X0, steps, None, None, thin=thin, seed=seed, step0=step0, AE=AE,
                        walker0=walker0, P=P, trace=trace)


def mhar_run_pre(A, b, X0, steps: int, delta, U, thin: int = 1, seed: int = 0, step0: int = 0,
                 AE=None, walker0: int = 0, P=None, trace: bool = False):
    """Algorithm 2 with directions d = P (delta * h + U g); ``delta`` None = isotropic.

    ``U`` is n x r (r <= 32) or None (diagonal preconditioner only).
    """
    A = _f64(A)
    b = _f64(b)
    m, n = A.shape
    X = _f64(X0).copy()
    if X.ndim == 1:
        raise ValueError("X0 must be z x n")
    z = X.shape[0]
    if P is None and AE is not None and np.size(AE) > 0:
        P = projector(AE)
    P = None if P is None else _f64(P)
    r = 0
    if delta is not None:
        delta = _f64(delta).reshape(n)
        if U is not None:
            U = _f64(U).reshape(n, -1)
            r = U.shape[1]
            if r > 32:
                raise ValueError("rank must be <= 32")
    elif U is not None:
        raise ValueError("U needs delta")
    nsamp = steps // thin if thin > 0 else 0
    out = np.zeros((nsamp, z, n), dtype=np.float64)
    t_tr = lmin_tr = lmax_tr = None
    if trace:
        t_tr = np.zeros((steps, z))
        lmin_tr = np.zeros((steps, z))
        lmax_tr = np.zeros((steps, z))
    st = _load().orc_mhar_run_pre(_ptr(A), _ptr(b), m, n, _ptr(P), _ptr(X), z, walker0, seed,
                                  step0, steps, thin, _ptr(delta), _ptr(U if r > 0 else None), r,
                                  _ptr(out) if nsamp > 0 else None, _ptr(t_tr), _ptr(lmin_tr),
                                  _ptr(lmax_tr))
    if st < 0:
        raise MemoryError("oracle allocation failed")
    res = {"X": X, "samples": out, "status": st}
    if trace:
        res.update(t=t_tr, lmin=lmin_tr, lmax=lmax_tr)
    return res
