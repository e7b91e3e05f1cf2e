"""Effective sample size of MHAR traces (host-side numpy).

The paper judges mixing with the Friedman-Rafsky test (Section 6.4) and does
not define an effective sample size.  The reading used here is the standard
multi-chain one:

* the trace of W walkers over T iterations is centred by its pooled mean;
* the autocovariance of every walker's series is taken with an FFT (the biased
  estimator, divisor T) and averaged over the W walkers, then normalised by its
  lag-0 value to give rho_t;
* the integrated autocorrelation time follows Geyer's initial monotone
  sequence estimator (Geyer 1992, "Practical Markov chain Monte Carlo",
  Statistical Science 7(4)): Gamma_k = rho_{2k} + rho_{2k+1} is summed while it
  stays positive, each term capped by the one before it, and
  tau = -1 + 2 sum_k Gamma_k;
* ESS = W T / tau per coordinate; min-ESS is the minimum over coordinates.

Walkers are independent chains (Section 4.1), so the ESS of all z walkers is
the ESS of a traced subset of W walkers scaled by z / W.

An ESS is only meaningful once the chains have left their transient.  The
check used with it is the split potential scale reduction (Gelman et al.,
Bayesian Data Analysis, 3rd ed., Section 11.4): every walker's series is
cut into halves, and for the 2W half-chains of length N
  B = N var(half-chain means),  Wv = mean(half-chain variances),
  R_hat = sqrt(((N - 1) / N Wv + B / N) / Wv);
a drifting (still transient) chain has halves with different means and an
R_hat well above 1.  The maximum over coordinates is reported.
"""
from __future__ import annotations

import numpy as np


def autocorrelation(chains: np.ndarray) -> np.ndarray:
    """rho_t, t = 0..T-1, of a (W, T) array of W series of one coordinate."""
    x = np.asarray(chains, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    W, T = x.shape
    x = x - x.mean()
    nfft = 1
    while nfft < 2 * T:
        nfft <<= 1
    f = np.fft.rfft(x, nfft, axis=1)
    acov = np.fft.irfft(f * np.conj(f), nfft, axis=1)[:, :T] / T
    acov = acov.mean(axis=0)
    if acov[0] <= 0.0:
        return np.zeros(T)
    return acov / acov[0]


def integrated_time(rho: np.ndarray) -> float:
    """Geyer's initial monotone sequence estimate of tau from rho_0..rho_{T-1}."""
    T = len(rho)
    if T < 2 or rho[0] == 0.0:
        return float("inf")
    total = 0.0
    prev = np.inf
    for k in range(T // 2):
        g = rho[2 * k] + rho[2 * k + 1]
        if g <= 0.0:
            break
        g = min(g, prev)
        total += g
        prev = g
    return -1.0 + 2.0 * total


def ess_per_coordinate(trace: np.ndarray) -> np.ndarray:
    """ESS of every coordinate of a (T, W, n) trace (iterations, walkers, coordinates)."""
    tr = np.asarray(trace, dtype=np.float64)
    T, W, n = tr.shape
    out = np.empty(n)
    for i in range(n):
        tau = integrated_time(autocorrelation(tr[:, :, i].T))
        out[i] = W * T / tau if np.isfinite(tau) and tau > 0 else 0.0
    return out


def min_ess(trace: np.ndarray, z_total: int | None = None) -> float:
    """Minimum over coordinates of the ESS, scaled to z_total walkers when given."""
    tr = np.asarray(trace)
    e = float(ess_per_coordinate(tr).min())
    if z_total is not None:
        e *= z_total / tr.shape[1]
    return e


def split_rhat(trace: np.ndarray) -> np.ndarray:
    """Split R_hat of every coordinate of a (T, W, n) trace."""
    tr = np.asarray(trace, dtype=np.float64)
    T, W, n = tr.shape
    N = T // 2
    halves = np.concatenate([tr[:N], tr[T - N:]], axis=1)   # (N, 2W, n)
    means = halves.mean(axis=0)                             # (2W, n)
    var = halves.var(axis=0, ddof=1)                        # (2W, n)
    B = N * means.var(axis=0, ddof=1)
    Wv = var.mean(axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.sqrt(((N - 1) / N * Wv + B / N) / Wv)
    return np.where(Wv > 0, r, np.inf)
