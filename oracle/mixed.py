"""The reduced-precision readings of Algorithm 2, in FP64 (TEST INFRASTRUCTURE ONLY).

Only ``tests/`` and ``bench.py``'s CPU legs may import this module; the CUDA
library never loads it and shares no code with it.

The pure oracle (``oracle.mhar_run``) is Algorithm 2 in exact-as-possible
FP64.  The library's FP32 and tensor-core modes run the same algorithm on
rounded operands and, to keep every point inside the body despite their
rounding, find each chord end from a slack lowered by a bound on its error
and an a_i . d pushed away from zero by its own bound (include/mhar.h,
"Feasibility in every mode").  That changes the chord by up to about the
bound, far more than the kernels' own rounding, so they are held to this
module instead, which computes -- in FP64 -- exactly the quantities the
library documents:

  * directions quantised as the library quantises them: the FP64 normals of
    Section 4.3 (``oracle.direction_normals``) rounded to FP32 (and, with a
    preconditioner, delta * h + U g rounded to FP32); in the tensor-core modes
    divided by the coordinate scale sigma_i and split into an FP16 pair
    (round to nearest even); the walk moves along sigma (d_hi + d_lo), or, with
    equalities, along its exact projection (Section 3.2);
  * the chord of Section 4.4 with the documented error margins, from the
    same row quantities (the FP16 pair of each scaled row, its exact
    representation error, its nonzero 16-column blocks) and walker norms
    (2-norms and max-norms of the FP16 hi parts of the scaled point and
    direction);
  * theta = lambda_min + u (lambda_max - lambda_min) rounded to FP32
    (Section 4.5), u the chord uniform of the pure oracle.

Everything else is the pure oracle's arithmetic in FP64.  ``margins=False``
and ``quantise=False`` turn the two departures off; with both off the walk is
the pure oracle's up to FP64 rounding order (pinned in tests/test_oracle_mixed.py).

Mode names follow the library: "fp32" (CUDA cores, FP32), "mixed_rs"
(tensor cores, slack recomputed every iteration), "mixed" (tensor cores,
slack stored and refreshed every ``refresh_k`` iterations).
"""
from __future__ import annotations

import numpy as np

from . import chord_uniform, direction_normals, stream_normals

_U32 = 2.0 ** -24


def f32(v):
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def fp16_pair(v32):
    """FP16 hi + lo of FP32 values (round to nearest even, as __float2half_rn)."""
    v32 = np.asarray(v32, dtype=np.float32)
    hi = v32.astype(np.float16)
    lo = (v32 - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float64), lo.astype(np.float64)


def _up32(v):
    """FP32 value >= v (v >= 0)."""
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    bump = f.astype(np.float64) < v
    return np.where(bump, np.nextafter(f, np.float32(np.inf)), f).astype(np.float64)


def column_scales(A):
    """sigma_j = 2^-e_j with max_i |a_ij| = f 2^e_j, f in [0.5, 1), divided by
    the largest, kept >= 2^-13 (1 for all-zero columns)."""
    cm = np.abs(A).max(axis=0)
    e = np.frexp(cm)[1]
    sig = np.where(cm > 0, np.ldexp(1.0, -e), 1.0)
    return np.maximum(sig / sig.max(), 2.0 ** -13)


def precond_scales(sig_a, delta, U, tensor: bool):
    """Coordinate scales with a preconditioner (the library's rule)."""
    if not tensor:
        return sig_a.copy()
    var = delta ** 2 + ((U ** 2).sum(axis=1) if U is not None else 0.0)
    sd = np.sqrt(var)
    l1 = delta + (np.abs(U).sum(axis=1) if U is not None else 0.0)
    rmax = float((sd / sig_a).max())
    ec = np.frexp(rmax)[1] if rmax > 0 and np.isfinite(rmax) else 0
    v = np.ldexp(sig_a, ec)
    e_hi = np.frexp(sd * 256.0)[1]
    v = np.where(sd > 0, np.minimum(v, np.ldexp(1.0, e_hi - 1)), v)
    lo = 6.8 * l1 / 65504.0
    e_lo = np.frexp(lo)[1]
    v = np.where(lo > 0, np.maximum(v, np.ldexp(1.0, e_lo)), v)
    return v


class _Rows:
    """Per-row quantities of the tensor-core modes (the library's
    prepare_tc_kernel and row_blocks_kernel, restated)."""

    def __init__(self, A, b, sig, per_step: int, d2: float, dinf: float):
        m, n = A.shape
        As = A * sig[None, :]
        mx = np.abs(As).max(axis=1)
        e = np.frexp(mx)[1]
        self.scale = np.where(mx > 0, np.ldexp(1.0, e), 1.0)
        ah = As / self.scale[:, None]
        hi, lo = fp16_pair(ah.astype(np.float32))
        rep = ah - hi - lo
        nz = ah != 0.0
        nblk = np.array([len({j // 16 for j in np.nonzero(nz[i])[0]}) for i in range(m)])
        g = (per_step * nblk + 1) * 2.0 ** -22 * (1 + 2.0 ** -9)
        up = 1 + 1e-12
        na2, na1 = np.sqrt((ah ** 2).sum(1)) * up, np.abs(ah).sum(1) * up
        rp2, rp1 = np.sqrt((rep ** 2).sum(1)) * up, np.abs(rep).sum(1) * up
        lo2, lo1 = np.sqrt((lo ** 2).sum(1)) * up, np.abs(lo).sum(1) * up
        nnz = nz.sum(1)
        kg2 = rp2 + 2.0 ** -11 * lo2 * (1 + 2.0 ** -11) + g * na2
        ks2 = kg2 + na2 * (2.0 ** -21 + 2.0 ** -24 * np.sqrt(nnz)) + 2.0 ** -22 * na2
        kg1 = rp1 + 2.0 ** -11 * lo1 * (1 + 2.0 ** -11) + g * na1
        ks1 = kg1 + na1 * (2.0 ** -21 + 2.0 ** -24) + 2.0 ** -22 * na1
        self.ks2, self.kg2, self.ks1, self.kg1 = (_up32(v) for v in (ks2, kg2, ks1, kg1))
        bs = b / self.scale
        bf = bs.astype(np.float32)
        bf = bf - np.float32(2.0 ** -21) * np.abs(bf)
        bf = np.where(bf.astype(np.float64) > bs, np.nextafter(bf, np.float32(-np.inf)), bf)
        self.bS = bf.astype(np.float64)
        # Block forms over groups of 32 rows (rows past m count as zero).
        mpad = -(-m // 128) * 128
        pad = lambda v: np.concatenate([v, np.zeros(mpad - m)])
        s2 = pad(self.kg2).reshape(-1, 32).sum(1)
        s1 = pad(self.kg1).reshape(-1, 32).sum(1)
        d2f, dif = float(np.float32(d2)), float(np.float32(dinf))
        inf_blk = s1 * dif < s2 * d2f
        form = np.repeat(inf_blk, 32)[:m]
        self.inf = form
        self.ks = np.where(form, self.ks1, self.ks2)
        self.kg = np.where(form, self.kg1, self.kg2)


def _dir_norms(sig, var):
    r = np.sqrt(var) / sig
    return max(float(np.sqrt((r ** 2).sum())), 1e-30), max(3.0 * float(r.max()), 1e-30)


def _chord(s, g):
    """(lambda_min, lambda_max) per walker from slacks s >= 0 and g (z x m)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        r = s / g
    lmax = np.where(g > 0, r, np.inf).min(axis=1)
    lmin = np.where(g < 0, r, -np.inf).max(axis=1)
    return lmin, lmax


def _simt_rows(A, b, sig):
    As = A * sig[None, :]
    nnz = (As != 0).sum(1)
    k = nnz + 4
    gamma = k * _U32 / (1 - k * _U32) * (1 + 1e-6)
    k2 = _up32(gamma * np.sqrt((As ** 2).sum(1)))
    k1 = _up32(gamma * np.abs(As).sum(1))
    n2 = _up32(np.sqrt((As ** 2).sum(1)) * (1 + 1e-6))
    lb = b - 3 * _U32 * np.abs(b)
    bt = lb.astype(np.float32)
    bt = np.where(bt.astype(np.float64) > lb, np.nextafter(bt, np.float32(-np.inf)), bt)
    return bt.astype(np.float64), k2, k1, n2


def mixed_run(A, b, X0, steps: int, mode: str, thin: int = 1, seed: int = 0, step0: int = 0,
              AE=None, delta=None, U=None, refresh_k: int = 64, walker0: int = 0,
              trace: bool = False, margins: bool = True, quantise: bool = True):
    """Algorithm 2 as the library's FP32 / tensor-core modes compute it (module
    docstring).  X0: z x n starts.  Returns ``X``, ``samples`` and, with
    ``trace``, ``t``, ``lmin``, ``lmax`` (steps x z), like ``oracle.mhar_run``,
    and ``D`` (steps x z x n), the quantised directions the chords are found on.
    "mixed" counts refreshes from step0 (a fresh context or a new state)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m, n = A.shape
    X = np.array(X0, dtype=np.float64, copy=True)
    z = X.shape[0]
    tensor = mode in ("mixed", "mixed_rs")
    q = (lambda v: f32(v)) if quantise else (lambda v: np.asarray(v, dtype=np.float64))
    sig_a = column_scales(A)
    if delta is not None:
        delta = np.asarray(delta, dtype=np.float64)
        U = None if U is None or np.size(U) == 0 else np.asarray(U, dtype=np.float64).reshape(n, -1)
        sig = precond_scales(sig_a, delta, U, tensor)
        var = delta ** 2 + ((U ** 2).sum(1) if U is not None else 0.0)
    else:
        sig, var = sig_a, np.ones(n)
    if AE is not None and np.size(AE) > 0:
        AE = np.atleast_2d(np.asarray(AE, dtype=np.float64))
        G = AE @ AE.T
    else:
        AE = None
    kdim = -(-n // 16) * 16
    if tensor:
        per_step = 4 if mode == "mixed" else 3
        d2, dinf = _dir_norms(sig, var)
        rows = _Rows(A, b, sig, per_step, d2, dinf)
        growth = 1.0 / (4 * per_step * (kdim // 16) + 4)
    else:
        bm, k2, k1, an2 = _simt_rows(A, b, sig)
    nsamp = steps // thin if thin > 0 else 0
    out = np.zeros((nsamp, z, n))
    tr = {k: np.zeros((steps, z)) for k in ("t", "lmin", "lmax")} if trace else None
    if trace:
        tr["D"] = np.zeros((steps, z, n))
    nx_ref = theta_acc = None
    since = 0
    for j in range(steps):
        step = step0 + j
        ks = np.arange(z) + walker0
        # Directions (Section 4.3), quantised.
        H = np.array([direction_normals(seed, step, int(k), n) for k in ks])
        if delta is not None:
            r = 0 if U is None else U.shape[1]
            Dd = delta[None, :] * q(H)
            if r:
                Gn = np.array([stream_normals(seed, step, int(k), 2, r) for k in ks])
                Dd = Dd + q(Gn) @ U.T
            D = q(Dd)
        else:
            D = q(H)
        if AE is not None:   # Section 3.2: d = P h, the FP32 result
            D = q(D - (np.linalg.solve(G, AE @ D.T)).T @ AE)
        if tensor and quantise:
            dh, dl = fp16_pair((D / sig[None, :]).astype(np.float32))
            D = sig[None, :] * (dh + dl)
        elif tensor:
            dh = D / sig[None, :]
        Dmove = D
        corrn = np.zeros(z)
        if AE is not None:   # exact null-space correction of the rounded direction
            cp = np.linalg.solve(G, AE @ D.T).T
            Dmove = D - cp @ AE
            corrn = np.sqrt((((cp @ AE) / sig[None, :]) ** 2).sum(1)) * (1 + 2.0 ** -10)
        # Chord (Section 4.4) with the margins.
        if tensor:
            if mode == "mixed" and (nx_ref is None or since >= refresh_k > 0):
                nx_ref = np.sqrt(((q(X) / sig[None, :]) ** 2).sum(1)) * (1 + 2.0 ** -8)
                theta_acc = np.zeros(z)
                since = 0
            S = (rows.bS if margins else b / rows.scale)[None, :] - (X @ A.T) / rows.scale[None, :]
            Gm = (D @ A.T) / rows.scale[None, :]
            nd2 = np.sqrt((dh ** 2).sum(1)) * (1 + 2.0 ** -8) + 2.0 ** 22 * corrn
            ndi = np.abs(dh).max(1) * (1 + 2.0 ** -8) + 2.0 ** 22 * corrn
            if margins and mode == "mixed_rs":
                xs = q(X)
                mxw = (np.abs(xs) / sig[None, :]).max(1)
                ws = np.where(mxw > 0, np.ldexp(1.0, np.frexp(mxw)[1]), 1.0)
                xh, _ = fp16_pair((xs / ws[:, None] / sig[None, :]).astype(np.float32))
                nxw2 = ws * np.sqrt((xh ** 2).sum(1)) * (1 + 2.0 ** -8)
                fx = np.where(rows.inf[None, :], ws[:, None], nxw2[:, None])
                fd = np.where(rows.inf[None, :], ndi[:, None], nd2[:, None])
                S = S - rows.ks[None, :] * fx
                Gm = Gm + np.where(Gm >= 0, 1.0, -1.0) * rows.kg[None, :] * fd
            elif margins:   # stored slack: its tracked error since the refresh
                E = (nx_ref + theta_acc) * (1 + since * (growth + 2.0 ** -22)) * 1.0001
                jk = since * _U32 * np.abs(rows.bS) * 1.0001
                S = S - (rows.ks2[None, :] * E[:, None] + jk[None, :])
                Gm = Gm + np.where(Gm >= 0, 1.0, -1.0) * rows.kg2[None, :] * nd2[:, None]
        else:
            xs = q(X)
            S = (bm if margins else b)[None, :] - X @ A.T
            Gm = D @ A.T
            if margins:
                n2x = np.sqrt(((xs / sig) ** 2).sum(1)) * (1 + 2.0 ** -10)
                nix = np.abs(xs / sig).max(1)
                n2d = np.sqrt(((D / sig) ** 2).sum(1)) * (1 + 2.0 ** -10)
                nid = np.abs(D / sig).max(1)
                S = S - np.minimum(k2[None, :] * n2x[:, None], k1[None, :] * nix[:, None])
                eg = np.minimum(k2[None, :] * n2d[:, None], k1[None, :] * nid[:, None])
                eg = eg + an2[None, :] * corrn[:, None]
                Gm = Gm + np.where(Gm >= 0, 1.0, -1.0) * eg
        S = np.maximum(S, 0.0)
        lmin, lmax = _chord(S, Gm)
        # Theta (Section 4.5), rounded to FP32; stalls and open sides keep 0.
        u = np.array([chord_uniform(seed, step, int(k)) for k in ks])
        ok = np.isfinite(lmin) & np.isfinite(lmax) & (lmin <= lmax)
        with np.errstate(invalid="ignore"):
            t = np.where(ok, lmin + u * (lmax - lmin), 0.0)
        t = np.where(ok, f32(t) if quantise else t, 0.0)
        X = X + t[:, None] * Dmove
        if tensor and mode == "mixed" and margins:
            theta_acc = theta_acc + np.abs(t) * nd2
            since += 1
        if trace:
            tr["t"][j], tr["lmin"][j], tr["lmax"][j] = t, lmin, lmax
            tr["D"][j] = D
        if thin > 0 and (j + 1) % thin == 0 and (j + 1) // thin <= nsamp:
            out[(j + 1) // thin - 1] = X
    res = {"X": X, "samples": out}
    if trace:
        res.update(tr)
    return res
