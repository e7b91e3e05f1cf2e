"""Pins of the reduced-precision oracle (oracle/mixed.py), CPU only.

It must reduce to the pure FP64 oracle when its two departures (quantised
operands, error margins) are off, round FP16 pairs to nearest even, compute
the documented column scales, and its margined chords must lie inside the
exact chords of the same (quantised) directions with both ends feasible in
FP64 -- the property the margins exist for.
"""
import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_2104_07097_gb300 import workloads as wl


@pytest.mark.parametrize("mode", ["fp32", "mixed_rs", "mixed"])
@pytest.mark.parametrize("body", ["rand", "simplex", "pre"])
def test_reduces_to_pure_oracle(mode, body):
    if body == "simplex":
        p = wl.simplex_cuts(9, 20, seed=2)
    else:
        p = wl.random_polytope(7, 40, seed=3)
    z, steps = 6, 12
    X0 = np.tile(p.x0, (z, 1))
    delta = U = None
    if body == "pre":
        rng = np.random.default_rng(0)
        delta, U = rng.uniform(0.5, 1.5, p.n), 0.3 * rng.standard_normal((p.n, 3))
    ref = oracle.mhar_run_pre(p.A, p.b, X0, steps, delta, U, thin=1, seed=4, AE=p.AE, trace=True)
    got = mixed.mixed_run(p.A, p.b, X0, steps, mode, seed=4, AE=p.AE, delta=delta, U=U,
                          trace=True, margins=False, quantise=False)
    np.testing.assert_allclose(got["samples"], ref["samples"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(got["lmax"], ref["lmax"], rtol=1e-10)
    np.testing.assert_allclose(got["lmin"], ref["lmin"], rtol=1e-10)


def test_fp16_pair_rounds_to_nearest_even():
    v = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 1 + 2.0 ** -12, 65504.0, 2.0 ** -25],
                 dtype=np.float32)
    hi, lo = mixed.fp16_pair(v)
    # ties go to the even significand; the low part carries the rest exactly
    np.testing.assert_array_equal(hi, [1.0, 1 + 2.0 ** -9, 1.0, 65504.0, 0.0])
    np.testing.assert_array_equal(lo, [2.0 ** -11, -2.0 ** -11, 2.0 ** -12, 0.0, 0.0])
    # 2^-25 lies halfway between 0 and the smallest FP16 subnormal 2^-24: even is 0
    assert mixed.fp16_pair(np.float32(3 * 2.0 ** -26))[0] == 2.0 ** -24


def test_column_scales_closed_form():
    A = np.array([[3.0, 0.0, 0.01], [-1.0, 0.0, 0.0], [0.5, 0.0, -0.02]])
    # column maxima 3 = 0.75 2^2, (zero column), 0.02 = 0.64 2^-5
    sig = mixed.column_scales(A)
    np.testing.assert_array_equal(sig, [2.0 ** -2 / 2.0 ** 5, 1.0 / 2.0 ** 5, 1.0])
    # every nonzero column of A sigma has its largest entry in [0.5, 1) times
    # one common power of two
    cm = np.abs(A * sig).max(axis=0)
    assert np.frexp(cm[0])[1] == np.frexp(cm[2])[1]


@pytest.mark.parametrize("mode", ["fp32", "mixed_rs", "mixed"])
@pytest.mark.parametrize("body", ["illcond", "simplex", "far"])
def test_margined_chord_inside_and_feasible(mode, body):
    """The guarantee: every margined chord is inside the exact chord of its own
    direction, and x + lambda d at both ends satisfies A x <= b in FP64."""
    if body == "illcond":
        p = wl.ill_conditioned(12, 80, seed=4, smin=1e-3)
    elif body == "simplex":
        p = wl.simplex_cuts(15, 40, seed=5)
    else:
        p = wl.random_polytope(8, 17, seed=6)   # m near 2n: long axes
    z, steps = 16, 30
    X0 = np.tile(p.x0, (z, 1))
    res = mixed.mixed_run(p.A, p.b, X0, steps, mode, seed=7, AE=p.AE, trace=True, refresh_k=8)
    X = X0.copy()
    for j in range(steps):
        D = res["D"][j]
        for k in range(z):
            lo, hi, _ = oracle.chord(p.A, p.b, X[k], D[k])
            assert res["lmin"][j, k] >= lo - 1e-15 * abs(lo)
            assert res["lmax"][j, k] <= hi + 1e-15 * abs(hi)
            for lam in (res["lmin"][j, k], res["lmax"][j, k]):
                viol = p.A @ (X[k] + lam * D[k]) - p.b
                assert viol.max() <= 1e-13 * max(1.0, np.abs(p.A @ X[k]).max())
        X = res["samples"][j] if j + 1 < steps else res["X"]
        if p.mE:
            assert np.abs(X @ p.AE.T - p.bE).max() <= 1e-12


def test_margins_are_small_on_a_well_conditioned_body():
    # The chord shrinks by the bounds only: about 1.5e-5 of its length (median)
    # for a dense 30-dimensional body, mostly the accumulation term of a . d
    # times the distance to the chord end; more where the binding row is
    # nearly parallel to the direction (small a . d, large relative bound).
    p = wl.random_polytope(30, 200, seed=8)
    z, steps = 20, 10
    X0 = np.tile(p.x0, (z, 1))
    a = mixed.mixed_run(p.A, p.b, X0, steps, "mixed_rs", seed=2, trace=True)
    shrink = []
    X = X0
    for j in range(steps):
        for k in range(z):
            lo, hi, _ = oracle.chord(p.A, p.b, X[k], a["D"][j, k])
            shrink.append(max(hi - a["lmax"][j, k], a["lmin"][j, k] - lo) / (hi - lo))
        X = a["samples"][j]
    shrink = np.array(shrink)
    assert shrink.min() >= 0.0
    assert np.median(shrink) < 4e-5
    assert np.percentile(shrink, 90) < 2e-4
