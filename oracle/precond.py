"""FP64 oracle for the learned direction preconditioner (numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the CUDA library never
imports it.

The paper samples with isotropic Gaussian directions and assumes the body has
been brought to near-isotropic position beforehand (Section 1.2, "The
blueprint", and Section 3.1, where elongated bodies are noted to mix slowly).
The preconditioner makes that pre-processing part of the sampler: the
direction of every walker becomes

    d = P (delta * h + U g),   h ~ N(0, I_n),  g ~ N(0, I_r),

so d ~ N(0, P C P) with C = diag(delta^2) + U U^T.  The law of d does not depend
on the walker's position and is centrally symmetric, so hit-and-run with it is
still reversible for the uniform distribution on the body (the argument of
Section 4.5 for theta uniform on the chord holds for any such direction law).
C is learned from warm-up samples of the chain itself and then frozen:

  1. covariance  Sigma = sum_k (x_k - mu)(x_k - mu)^T / (N - 1) over the N
     warm-up points x_k (every walker at every snapshot);
  2. randomized subspace iteration for the leading rank-r subspace of Sigma:
     Y = Sigma Omega, Omega n x r with N(0,1) entries (Philox stream 3, column c
     drawn as walker c at step 0); then `power_iters` times Q = orth(Y),
     Y = Sigma Q; finally Q = orth(Y).  orth(Y) is the Q factor of the thin QR
     factorisation of Y with a non-negative diagonal in R;
  3. Rayleigh-Ritz: T = Q^T Sigma Q = V Lambda V^T, U = Q V Lambda_+^{1/2}
     (eigenvalues clipped at 0, largest first);
  4. diagonal: delta_i^2 = max(Sigma_ii - (U U^T)_ii, eps_rel Sigma_ii,
     eps_abs trace(Sigma) / n), so every coordinate keeps a share of its own
     variance and the directions span the whole space (irreducibility).
"""
from __future__ import annotations

import numpy as np

from . import STREAM_FIT, stream_normals

EPS_REL = 1e-2
EPS_ABS = 1e-9


def covariance(snapshots) -> np.ndarray:
    """Sample covariance of the rows of all snapshots (each z x n), divisor N - 1."""
    Xs = np.concatenate([np.asarray(s, dtype=np.float64).reshape(-1, np.shape(s)[-1])
                         for s in snapshots], axis=0)
    N = Xs.shape[0]
    if N < 2:
        raise ValueError("need at least two points")
    mu = Xs.sum(axis=0) / N
    Zc = Xs - mu
    return Zc.T @ Zc / (N - 1)


def omega(n: int, r: int, seed: int) -> np.ndarray:
    """The starting block: column c is stream 3's normals for walker c at step 0."""
    Om = np.zeros((n, r))
    for c in range(r):
        Om[:, c] = stream_normals(seed, 0, c, STREAM_FIT, n)
    return Om


def orth(Y: np.ndarray) -> np.ndarray:
    """Q of the thin QR factorisation of Y, signs chosen so that diag(R) >= 0."""
    Q, R = np.linalg.qr(Y)
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * s


def fit(Sigma, rank: int, power_iters: int, seed: int, eps_rel: float = EPS_REL,
        eps_abs: float = EPS_ABS):
    """(delta, U) of the rank-`rank` plus diagonal model of Sigma (steps 2-4 above)."""
    Sigma = np.asarray(Sigma, dtype=np.float64)
    n = Sigma.shape[0]
    r = min(rank, n)
    diag = np.diag(Sigma).copy()
    floor = np.maximum(eps_rel * diag, eps_abs * diag.sum() / n)
    if r == 0:
        return np.sqrt(np.maximum(diag, floor)), np.zeros((n, 0))
    Y = Sigma @ omega(n, r, seed)
    for _ in range(power_iters):
        Q = orth(Y)
        Y = Sigma @ Q
    Q = orth(Y)
    T = Q.T @ Sigma @ Q
    T = 0.5 * (T + T.T)
    lam, V = np.linalg.eigh(T)
    order = np.argsort(lam)[::-1]
    lam = np.maximum(lam[order], 0.0)
    V = V[:, order]
    U = (Q @ V) * np.sqrt(lam)
    delta2 = np.maximum(diag - (U * U).sum(axis=1), floor)
    return np.sqrt(delta2), U


def direction_covariance(delta, U) -> np.ndarray:
    """C = diag(delta^2) + U U^T, the covariance of delta * h + U g."""
    C = np.diag(np.asarray(delta, dtype=np.float64) ** 2)
    if U is not None and np.size(U):
        C = C + U @ U.T
    return C
