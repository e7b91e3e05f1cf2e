"""Pins of the preconditioner oracle (oracle.precond, oracle.mhar_run_pre) and of
the ESS estimator, against closed forms, constructed spectra, invariances of
hit-and-run and distribution laws.  All CPU.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.precond as pc
from paper_2104_07097_gb300 import diagnostics
from paper_2104_07097_gb300 import workloads as wl


def _bm_pair(w0, w1):
    # Box-Muller on two 32-bit words mapped to (w + 1/2) 2^-32.
    ua = (w0 + 0.5) / 2.0 ** 32
    ub = (w1 + 0.5) / 2.0 ** 32
    r = math.sqrt(-2.0 * math.log(ua))
    return r * math.cos(2 * math.pi * ub), r * math.sin(2 * math.pi * ub)


# ----------------------------------------------------------------------------
# Streams 2 and 3: counter layout
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("stream", [oracle.STREAM_LOWRANK, oracle.STREAM_FIT])
def test_stream_normals_counter_layout(stream):
    seed, step, walker = 0x1234_5678_9ABC, (7 << 32) | 11, 5
    got = oracle.stream_normals(seed, step, walker, stream, 8)
    for q in range(2):
        ctr = [q, walker, step & 0xFFFFFFFF, ((step >> 32) << 8) | stream]
        w = oracle.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        want = _bm_pair(int(w[0]), int(w[1])) + _bm_pair(int(w[2]), int(w[3]))
        np.testing.assert_allclose(got[4 * q:4 * q + 4], want, rtol=1e-14, atol=1e-14)
    # a different stream gives different numbers
    assert not np.allclose(got, oracle.direction_normals(seed, step, walker, 8))


def test_omega_columns_are_stream3_walkers():
    Om = pc.omega(9, 4, seed=3)
    for c in range(4):
        np.testing.assert_array_equal(Om[:, c], oracle.stream_normals(3, 0, c, oracle.STREAM_FIT, 9))


# ----------------------------------------------------------------------------
# Covariance (step 1)
# ----------------------------------------------------------------------------
def test_covariance_hand_example():
    # Four points symmetric about 0: sum x^2 = 2, sum y^2 = 8, sum xy = 0; divisor N-1 = 3.
    pts = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 2.0], [0.0, -2.0]])
    S = pc.covariance([pts[:2], pts[2:]])
    np.testing.assert_allclose(S, [[2 / 3, 0.0], [0.0, 8 / 3]], atol=1e-15)
    # shifting every point leaves it unchanged
    np.testing.assert_allclose(pc.covariance([pts + 1e3]), S, atol=1e-9)


def test_covariance_of_cube_samples():
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, size=(200000, 3))
    np.testing.assert_allclose(pc.covariance([X]), np.eye(3) / 3, atol=5e-3)


# ----------------------------------------------------------------------------
# Fit (steps 2-4) on constructed spectra
# ----------------------------------------------------------------------------
def test_fit_recovers_leading_eigenspace():
    rng = np.random.default_rng(1)
    n, r = 40, 4
    Q0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([[100.0, 60.0, 30.0, 20.0], np.linspace(1.0, 0.1, n - r)])
    S = (Q0 * lam) @ Q0.T
    delta, U = pc.fit(S, r, power_iters=12, seed=0)
    lead = (Q0[:, :r] * lam[:r]) @ Q0[:, :r].T
    np.testing.assert_allclose(U @ U.T, lead, atol=1e-9 * lam[0])
    rest = np.diag(S) - np.diag(lead)
    floor = np.maximum(pc.EPS_REL * np.diag(S), pc.EPS_ABS * np.trace(S) / n)
    np.testing.assert_allclose(delta ** 2, np.maximum(rest, floor), rtol=1e-8)
    # the model keeps the diagonal of S wherever the floor is not active
    C = pc.direction_covariance(delta, U)
    keep = rest > floor
    np.testing.assert_allclose(np.diag(C)[keep], np.diag(S)[keep], rtol=1e-8)


def test_fit_diagonal_covariance_picks_largest_coordinates():
    v = np.array([1e-6, 3.0, 1e4, 0.5, 1e3, 2.0])
    delta, U = pc.fit(np.diag(v), 2, power_iters=8, seed=5)
    top = np.zeros(6)
    top[[2, 4]] = v[[2, 4]]
    np.testing.assert_allclose(U @ U.T, np.diag(top), atol=1e-9 * v.max())
    floor = np.maximum(pc.EPS_REL * v, pc.EPS_ABS * v.sum() / 6)
    want = np.where(top > 0, floor, v)
    want = np.maximum(want, floor)
    np.testing.assert_allclose(delta ** 2, want, rtol=1e-6)


def test_fit_rank_zero_is_diagonal():
    v = np.array([4.0, 1.0, 0.25])
    delta, U = pc.fit(np.diag(v), 0, power_iters=3, seed=0)
    assert U.shape == (3, 0)
    np.testing.assert_allclose(delta, np.sqrt(v))


def test_orth_signs_and_orthonormality():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((30, 5))
    Q = pc.orth(Y)
    np.testing.assert_allclose(Q.T @ Q, np.eye(5), atol=1e-13)
    R = Q.T @ Y
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(np.triu(R), R, atol=1e-12)  # Y = Q R, R upper triangular


# ----------------------------------------------------------------------------
# Preconditioned Algorithm 2: reductions and invariances
# ----------------------------------------------------------------------------
def _box(s):
    n = len(s)
    A = np.vstack([np.eye(n), -np.eye(n)])
    b = np.concatenate([s, s])
    return A, b


def test_identity_preconditioner_is_plain_mhar():
    p = wl.random_polytope(6, 30, seed=4)
    X0 = np.tile(p.x0, (7, 1))
    a = oracle.mhar_run(p.A, p.b, X0, 25, seed=9, trace=True)
    c = oracle.mhar_run_pre(p.A, p.b, X0, 25, np.ones(6), np.zeros((6, 3)), seed=9, trace=True)
    np.testing.assert_array_equal(a["X"], c["X"])
    np.testing.assert_array_equal(a["t"], c["t"])


def test_scalar_preconditioner_leaves_the_walk_unchanged():
    # x + theta d with theta uniform on the chord does not depend on |d|:
    # scaling d by 2.5 scales the chord by 1/2.5 and lands on the same point.
    p = wl.random_polytope(5, 25, seed=6)
    X0 = np.tile(p.x0, (4, 1))
    a = oracle.mhar_run(p.A, p.b, X0, 30, seed=2)
    c = oracle.mhar_run_pre(p.A, p.b, X0, 30, np.full(5, 2.5), None, seed=2)
    np.testing.assert_allclose(c["X"], a["X"], rtol=0, atol=1e-12)


def test_lowrank_term_on_the_interval_closed_form():
    # n = 1, delta = 0, U = [[0.7]]: d = 0.7 g with g the stream-2 normal, and the
    # new point is -1 + 2u when d > 0, 1 - 2u when d < 0 (the chord is [-1, 1]).
    A = np.array([[1.0], [-1.0]])
    b = np.array([1.0, 1.0])
    seed = 77
    for walker in range(6):
        X0 = np.array([[0.3]])
        res = oracle.mhar_run_pre(A, b, X0, 1, np.zeros(1), np.array([[0.7]]), seed=seed,
                                  walker0=walker)
        w = oracle.philox([0, walker, 0, oracle.STREAM_LOWRANK], [seed, 0])
        g, _ = _bm_pair(int(w[0]), int(w[1]))
        wu = oracle.philox([0, walker, 0, oracle.STREAM_CHORD], [seed, 0])
        u = (int(wu[0]) + 0.5) / 2.0 ** 32
        want = -1 + 2 * u if g > 0 else 1 - 2 * u
        assert abs(res["X"][0, 0] - want) < 1e-15


def test_preconditioned_projection_keeps_equalities():
    p = wl.simplex(12)
    rng = np.random.default_rng(3)
    delta = rng.uniform(0.1, 2.0, 12)
    U = rng.standard_normal((12, 3))
    X0 = np.tile(p.x0, (5, 1))
    res = oracle.mhar_run_pre(p.A, p.b, X0, 40, delta, U, seed=1, AE=p.AE)
    np.testing.assert_allclose(res["X"] @ p.AE.T, np.tile(p.bE, (5, 1)), atol=1e-13)
    assert np.all(res["X"] @ p.A.T <= p.b + 1e-12)


def test_preconditioned_uniform_on_stretched_box():
    # Box [-s_i, s_i]: marginals x_i / s_i are Uniform[-1, 1] whatever the
    # (fixed, symmetric) direction law; a correlated U does not bias them.
    s = np.array([1.0, 0.02, 0.3])
    A, b = _box(s)
    rng = np.random.default_rng(8)
    U = rng.standard_normal((3, 2)) * s[:, None]
    z = 3000
    res = oracle.mhar_run_pre(A, b, np.zeros((z, 3)), 60, s, U, seed=4)
    for i in range(3):
        p = stats.kstest(res["X"][:, i] / s[i], stats.uniform(loc=-1, scale=2).cdf).pvalue
        assert p > 1e-3


def test_preconditioned_step_is_stationary():
    s = np.array([2.0, 0.05])
    A, b = _box(s)
    rng = np.random.default_rng(11)
    X0 = rng.uniform(-1, 1, size=(20000, 2)) * s
    res = oracle.mhar_run_pre(A, b, X0, 1, np.array([0.3, 1.0]), np.array([[1.0], [0.5]]), seed=6)
    for i in range(2):
        p = stats.kstest(res["X"][:, i] / s[i], stats.uniform(loc=-1, scale=2).cdf).pvalue
        assert p > 1e-3


def test_learned_preconditioner_speeds_mixing_on_stretched_box():
    # Power check: on a box with side ratio 100 a fitted preconditioner gives a
    # far larger min-ESS than isotropic directions for the same iterations.
    s = np.array([1.0, 0.01, 0.1, 0.5])
    A, b = _box(s)
    z, T = 64, 400
    warm = oracle.mhar_run(A, b, np.zeros((z, 4)), 200, thin=20, seed=1)
    delta, U = pc.fit(pc.covariance(warm["samples"][5:]), 2, 4, seed=1)
    iso = oracle.mhar_run(A, b, warm["X"], T, thin=1, seed=2)
    pre = oracle.mhar_run_pre(A, b, warm["X"], T, delta, U, thin=1, seed=2)
    e_iso = diagnostics.min_ess(iso["samples"])
    e_pre = diagnostics.min_ess(pre["samples"])
    assert e_pre > 5 * e_iso


# ----------------------------------------------------------------------------
# ESS estimator (Geyer initial monotone sequence)
# ----------------------------------------------------------------------------
def _ar1(rho, W, T, seed):
    rng = np.random.default_rng(seed)
    x = np.empty((W, T))
    x[:, 0] = rng.standard_normal(W)
    e = rng.standard_normal((W, T)) * math.sqrt(1 - rho * rho)
    for t in range(1, T):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_integrated_time_of_ar1(rho):
    # AR(1) with coefficient rho: tau = (1 + rho) / (1 - rho).
    x = _ar1(rho, 64, 4000, seed=int(rho * 10))
    tau = diagnostics.integrated_time(diagnostics.autocorrelation(x))
    want = (1 + rho) / (1 - rho)
    assert abs(tau - want) < 0.08 * want


def test_autocorrelation_of_alternating_series():
    # x_t = (-1)^t: rho_t = (-1)^t (T - t) / T for the biased estimator.
    T = 64
    x = np.array([(-1.0) ** t for t in range(T)])
    rho = diagnostics.autocorrelation(x)
    want = np.array([(-1.0) ** t * (T - t) / T for t in range(T)])
    np.testing.assert_allclose(rho, want, atol=1e-12)


def test_min_ess_scales_with_walkers():
    x = _ar1(0.5, 32, 2000, seed=5)
    trace = np.stack([x.T, x.T * 2 + 1], axis=2)  # (T, W, 2)
    e = diagnostics.ess_per_coordinate(trace)
    np.testing.assert_allclose(e[0], e[1], rtol=1e-10)  # affine maps do not change ESS
    assert diagnostics.min_ess(trace, z_total=320) == pytest.approx(10 * e.min())
