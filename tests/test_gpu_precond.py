"""GPU parity of the learned direction preconditioner: preconditioned walks
d = P (delta * h + U g) against oracle.mhar_run_pre, the on-device fit against
oracle.precond on the same warm-up points, and the sampler's law with a
fitted preconditioner (uniform marginals, faster mixing).
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.precond as opc
from oracle import mixed
from paper_2104_07097_gb300 import diagnostics
from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4, "mixed": 1e-4, "mixed_rs": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()


def stretched(n, m, seed, s):
    """The random polytope mapped by diag(s): {x : A diag(1/s) x <= 1}."""
    p = wl.random_polytope(n, m, seed=seed)
    return wl.Polytope(A=p.A / s[None, :], b=p.b, x0=np.zeros(n), name=f"stretched{n}x{m}")


def box(s):
    n = len(s)
    return wl.Polytope(A=np.vstack([np.eye(n), -np.eye(n)]), b=np.concatenate([s, s]),
                       x0=np.zeros(n), name=f"box{n}")


def scaled_err(got, ref, s):
    """Normwise error in the whitened coordinates x / s."""
    g, r = got / s, ref / s
    return float(np.abs(g - r).max() / max(1.0, np.abs(r).max()))


def case(name):
    if name == "rand37x300":
        p = wl.random_polytope(37, 300, seed=11)
        s = np.ones(37)
    elif name == "simplex23+60":
        p = wl.simplex_cuts(23, 60, seed=13)
        s = np.ones(23)
    elif name == "illcond40x400":
        s = np.exp(np.random.default_rng(7).uniform(np.log(1e-3), 0.0, 40))
        p = stretched(40, 400, 17, s)
    else:
        raise KeyError(name)
    rng = np.random.default_rng(3)
    delta = rng.uniform(0.5, 1.5, p.n) * s
    U = rng.standard_normal((p.n, 5)) * 0.4 * s[:, None]
    return p, s, delta, U


CASES = [("rand37x300", 200), ("simplex23+60", 150), ("illcond40x400", 160)]


@pytest.mark.parametrize("name,z", CASES)
def test_preconditioned_fp64_free_running_50(name, z):
    p, s, delta, U = case(name)
    X0 = np.tile(p.x0, (z, 1))
    ref = oracle.mhar_run_pre(p.A, p.b, X0, 50, delta, U, thin=1, seed=5, AE=p.AE, trace=True)
    with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision="fp64", seed=5) as smp:
        smp.set_preconditioner(delta, U)
        got = smp.run(50, thin=1)
        lo, hi, t = smp.chord()
        st = smp.check()
    err = max(scaled_err(got[j], ref["samples"][j], s) for j in range(50))
    assert err <= TOL["fp64"], err
    np.testing.assert_allclose(lo, ref["lmin"][-1], rtol=1e-9)
    np.testing.assert_allclose(hi, ref["lmax"][-1], rtol=1e-9)
    assert st.max_violation <= 1e-6 * np.abs(p.b).max()
    if p.mE:
        assert st.eq_residual <= 1e-8


@pytest.mark.parametrize("prec", ["fp32", "mixed", "mixed_rs", "mixed_rs_smem"])
@pytest.mark.parametrize("name,z", CASES)
def test_preconditioned_step_for_step_50(name, z, prec):
    """Each iteration restarted from the pure oracle's state X_j and compared
    with the reduced-precision oracle's step from it (oracle.mixed: quantised
    directions, error-bounded chords); the ill-conditioned body (axes from
    1e-3 to 1) is measured in its whitened coordinates."""
    p, s, delta, U = case(name)
    X0 = np.tile(p.x0, (z, 1))
    pure = oracle.mhar_run_pre(p.A, p.b, X0, 50, delta, U, thin=1, seed=5, AE=p.AE, trace=True)
    kw = {}
    if prec == "mixed_rs_smem":
        prec, kw = "mixed_rs", {"smem_operands": True}
    worst = worst_pure = 0.0
    with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision=prec, seed=5, **kw) as smp:
        smp.set_preconditioner(delta, U)
        for j in range(50):
            start = X0 if j == 0 else pure["samples"][j - 1]
            ref = mixed.mixed_run(p.A, p.b, start, 1, prec, seed=5, step0=j, AE=p.AE,
                                  delta=delta, U=U, trace=True)
            smp.set_state(start, j)
            got = smp.run(1, thin=1)[0]
            worst = max(worst, scaled_err(got, ref["samples"][0], s))
            worst_pure = max(worst_pure, scaled_err(got, pure["samples"][j], s))
            lo, hi, t = smp.chord()
            span = np.maximum(1.0, ref["lmax"][0] - ref["lmin"][0])
            assert np.all(np.abs(lo - ref["lmin"][0]) <= TOL[prec] * span)
            assert np.all(np.abs(hi - ref["lmax"][0]) <= TOL[prec] * span)
            viol = (got @ p.A.T - p.b).max()
            assert viol <= 1e-6 * np.abs(p.b).max()
    assert worst <= TOL[prec], worst
    assert worst_pure <= 3e-3, worst_pure


def _snapshot_steps(warmup, snapshots):
    gap = max(1, warmup // (2 * snapshots))
    first = warmup - (snapshots - 1) * gap
    return [first + k * gap for k in range(snapshots)]


def _fit_body():
    s = np.array([6.0, 5.0, 4.0, 3.0] + [1.0] * 12)
    return stretched(16, 120, 23, s)


def _compare_fit(got, want):
    (dg, Ug), (dw, Uw) = got, want
    np.testing.assert_allclose(dg, dw, rtol=1e-6)
    Cg, Cw = opc.direction_covariance(dg, Ug), opc.direction_covariance(dw, Uw)
    assert np.linalg.norm(Cg - Cw) <= 1e-6 * np.linalg.norm(Cw)
    np.testing.assert_allclose(Ug @ Ug.T, Uw @ Uw.T, atol=1e-6 * np.abs(Uw @ Uw.T).max())


def test_fit_parity_fp64():
    p = _fit_body()
    z, W, S, r, q = 512, 120, 6, 4, 8
    with mhar.Sampler(p.A, p.b, p.x0, z, precision="fp64", seed=9) as smp:
        smp.fit_preconditioner(W, S, r, q)
        got = smp.preconditioner()
    ref = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (z, 1)), W, thin=1, seed=9)
    snaps = [ref["samples"][t - 1] for t in _snapshot_steps(W, S)]
    want = opc.fit(opc.covariance(snaps), r, q, seed=9)
    _compare_fit(got, want)


@pytest.mark.parametrize("prec", ["fp32", "mixed", "mixed_rs"])
def test_fit_parity_on_the_same_points(prec):
    # A twin sampler replays the same chain and hands its snapshots to the oracle fit.
    p = _fit_body()
    z, W, S, r, q = 384, 90, 5, 4, 8
    with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=4) as smp:
        smp.fit_preconditioner(W, S, r, q)
        got = smp.preconditioner()
    snaps, done = [], 0
    with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=4) as twin:
        for t in _snapshot_steps(W, S):
            twin.run(t - done)
            done = t
            snaps.append(twin.state()[0])
    want = opc.fit(opc.covariance(snaps), r, q, seed=4)
    _compare_fit(got, want)


@pytest.mark.parametrize("prec", ["fp64", "mixed_rs"])
def test_fit_pooled_over_shards(prec):
    # Two shards of one ensemble (walker0 = 0 and z) pool their warm-up moments
    # about a common shift (x0) and both adopt the fit of the pooled moments:
    # the same moments, the same fit as one context holding all 2 z walkers,
    # and the oracle's fit of the pooled covariance.
    p = _fit_body()
    z, W, S, r, q = 256, 90, 5, 4, 8
    parts = []
    for w0 in (0, z):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=7, walker0=w0) as smp:
            parts.append(smp.fit_moments(W, S, shift=p.x0))
    s1 = parts[0][0] + parts[1][0]
    s2 = parts[0][1] + parts[1][1]
    count = parts[0][2] + parts[1][2]
    assert count == 2 * z * S
    np.testing.assert_allclose(s2, s2.T, rtol=0, atol=0)
    with mhar.Sampler(p.A, p.b, p.x0, 2 * z, precision=prec, seed=7) as whole:
        w1, w2, wc = whole.fit_moments(W, S, shift=p.x0)
        whole.fit_from_moments(w1, w2, wc, r, q)
        want_whole = whole.preconditioner()
        X_whole = whole.run(6, thin=6)[0]
    assert wc == count
    scale = np.abs(w2).max()
    np.testing.assert_allclose(s1, w1, rtol=0, atol=1e-12 * max(1.0, np.abs(w1).max()))
    np.testing.assert_allclose(s2, w2, rtol=0, atol=1e-12 * scale)
    got, walks = [], []
    for w0 in (0, z):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=7, walker0=w0) as smp:
            smp.run(W)   # the same warm-up the moments came from
            smp.fit_from_moments(s1, s2, count, r, q)
            got.append(smp.preconditioner())
            walks.append(smp.run(6, thin=6)[0])
    _compare_fit(got[0], want_whole)
    np.testing.assert_array_equal(got[0][0], got[1][0])
    np.testing.assert_array_equal(got[0][1], got[1][1])
    Sigma = (s2 - np.outer(s1, s1) / count) / (count - 1)
    _compare_fit(got[0], opc.fit(Sigma, r, q, seed=7))
    if prec == "fp64":
        # The shards then walk as the whole ensemble does, walker for walker.
        err = np.abs(np.vstack(walks) - X_whole).max() / max(1.0, np.abs(X_whole).max())
        assert err <= 1e-9, err


def test_fit_moments_errors():
    p = _fit_body()
    with mhar.Sampler(p.A, p.b, p.x0, 64, precision="fp64") as smp:
        with pytest.raises(mhar.MharError) as e:
            smp.fit_moments(10, 11)
        assert e.value.code == mhar.E_ARG
        with pytest.raises(mhar.MharError) as e:
            smp.fit_moments(10, 2, shift=np.full(p.n, np.nan))
        assert e.value.code == mhar.E_NONFINITE
        s1, s2, c = smp.fit_moments(10, 2)
        with pytest.raises(mhar.MharError) as e:
            smp.fit_from_moments(s1, s2, 1, 4, 2)
        assert e.value.code == mhar.E_ARG
        bad = s2.copy()
        bad[0, 0] = np.inf
        with pytest.raises(mhar.MharError) as e:
            smp.fit_from_moments(s1, bad, c, 4, 2)
        assert e.value.code == mhar.E_NONFINITE
        smp.fit_from_moments(s1, s2, c, 4, 2)
        assert smp.preconditioner() is not None
        smp.run(3)


def test_fit_rank_zero_and_full_rank():
    p = _fit_body()
    with mhar.Sampler(p.A, p.b, p.x0, 256, precision="fp64", seed=1) as smp:
        smp.fit_preconditioner(40, 4, 0, 0)
        d0, U0 = smp.preconditioner()
        assert U0.shape == (16, 0) and np.all(d0 > 0)
    with mhar.Sampler(p.A, p.b, p.x0, 256, precision="fp64", seed=1) as smp:
        smp.fit_preconditioner(40, 4, 16, 3)
        d, U = smp.preconditioner()
        ref = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (256, 1)), 40, thin=1, seed=1)
        snaps = [ref["samples"][t - 1] for t in _snapshot_steps(40, 4)]
        Sig = opc.covariance(snaps)
        # rank n: U U^T is Sigma itself and delta sits on its floor
        np.testing.assert_allclose(U @ U.T, Sig, atol=1e-8 * np.abs(Sig).max())
        floor = np.maximum(opc.EPS_REL * np.diag(Sig), opc.EPS_ABS * np.trace(Sig) / 16)
        np.testing.assert_allclose(d ** 2, floor, rtol=1e-6)


def test_set_get_clear_roundtrip():
    p = wl.random_polytope(20, 120, seed=2)
    rng = np.random.default_rng(0)
    delta, U = rng.uniform(0.1, 1, 20), rng.standard_normal((20, 3))
    for prec in ("fp64", "mixed_rs", "mixed"):
        with mhar.Sampler(p.A, p.b, p.x0, 64, precision=prec, seed=3) as a, \
                mhar.Sampler(p.A, p.b, p.x0, 64, precision=prec, seed=3) as b:
            assert a.preconditioner() is None
            a.set_preconditioner(delta, U)
            dg, Ug = a.preconditioner()
            np.testing.assert_array_equal(dg, delta)
            np.testing.assert_array_equal(Ug, U)
            a.set_preconditioner(None)
            assert a.preconditioner() is None
            # Removing it restores exactly the isotropic walk.
            np.testing.assert_array_equal(a.run(7, thin=7), b.run(7, thin=7))


def test_emit_walkers_subset():
    p = wl.random_polytope(12, 60, seed=5)
    with mhar.Sampler(p.A, p.b, p.x0, 200, precision="mixed_rs", seed=6) as full, \
            mhar.Sampler(p.A, p.b, p.x0, 200, precision="mixed_rs", seed=6, emit_walkers=17) as sub:
        a = full.run(9, thin=3)
        b = sub.run(9, thin=3)
    assert b.shape == (3, 17, 12)
    np.testing.assert_array_equal(a[:, :17], b)


def test_errors():
    p = wl.random_polytope(10, 50, seed=1)
    with mhar.Sampler(p.A, p.b, p.x0, 32, precision="mixed_rs") as smp:
        with pytest.raises(mhar.MharError) as e:
            smp.set_preconditioner(np.ones(10), np.ones((10, 33)))
        assert e.value.code == mhar.E_ARG
        with pytest.raises(mhar.MharError) as e:
            smp.set_preconditioner(np.full(10, np.nan))
        assert e.value.code == mhar.E_NONFINITE
        with pytest.raises(mhar.MharError) as e:
            smp.set_preconditioner(-np.ones(10))
        assert e.value.code == mhar.E_ARG
        for args in [(0, 1, 2, 1), (10, 11, 2, 1), (10, 2, 11, 1), (10, 2, 2, 65)]:
            with pytest.raises(mhar.MharError) as e:
                mhar.mhar_fit_preconditioner(smp._ctx, *args)
            assert e.value.code == mhar.E_ARG
        assert smp.preconditioner() is None
        smp.run(3)  # still usable


@pytest.mark.parametrize("prec", ["fp32", "mixed_rs"])
def test_fitted_walk_is_uniform_and_mixes_faster(prec):
    # Box with axes 1 .. 1e-3: marginals x_i / s_i are Uniform[-1, 1] with the
    # learned directions too, and the learned walk's min-ESS is far larger.
    # A fit only sees the spread the warm-up has reached, so it is repeated:
    # each round warms up with the previous round's directions.
    s = np.array([1.0, 0.3, 0.05, 0.01, 0.003, 0.001])
    p = box(s)
    z, T = 1024, 300
    ess = {}
    for learned in (False, True):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=11, emit_walkers=128) as smp:
            if learned:
                for _ in range(3):
                    smp.fit_preconditioner(100, 5, 4, 4)
            else:
                smp.run(300)
            tr = smp.run(T, thin=1)
            X = smp.state()[0]
            st = smp.check()
        assert st.max_violation <= 1e-6 * s.max()
        ess[learned] = diagnostics.min_ess(tr)
        if learned:
            for i in range(6):
                pv = stats.kstest(X[:, i] / s[i], stats.uniform(loc=-1, scale=2).cdf).pvalue
                assert pv > 1e-3 / 6, (i, pv)
    assert ess[True] > 8 * ess[False], ess
