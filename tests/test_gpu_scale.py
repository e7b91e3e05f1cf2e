"""Parity and invariants at the benchmark's full size (random polytope
n = 100, m = 2000, z = 4096, mixed tensor-core mode, the launch configuration
bench.py times), on sampled walkers the oracle computes one by one, plus the
simplex-with-cuts body (n = 1000, m_E = 1) at reduced walker count."""
import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()


@pytest.fixture(scope="module")
def rand100():
    return wl.random_polytope(100, 2000, seed=2)


@pytest.mark.parametrize("prec", ["mixed", "mixed_rs"])
def test_full_size_sampled_parity(rand100, prec):
    p, z, steps = rand100, 4096, 10
    with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=0) as s:
        got = s.run(steps, thin=1)
    for w0, cnt in ((0, 12), (2048, 12), (4084, 12)):
        ref = mixed.mixed_run(p.A, p.b, np.tile(p.x0, (cnt, 1)), steps, prec, thin=1, seed=0,
                              walker0=w0)
        for j in range(steps):
            want = ref["samples"][j]
            err = np.abs(got[j, w0:w0 + cnt] - want).max() / max(1.0, np.abs(want).max())
            assert err <= 1e-4, (w0, j, err)


def test_full_size_feasibility_recompute(rand100):
    # Recomputed slack: every iteration's step is taken from b - A x formed
    # afresh, so there is no drift to bound; check points every 16 iterations.
    p, z = rand100, 4096
    with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", seed=3) as s:
        samples = s.run(640, thin=16)
        st = s.check()
    worst = max(float((X @ p.A.T - p.b).max()) for X in samples)
    assert worst <= 1e-6, worst
    assert st.max_violation <= 1e-6 and st.stalls == 0 and st.unbounded == 0


@pytest.mark.parametrize("refresh_fp64", [False, True])
def test_full_size_feasibility_and_drift(rand100, refresh_fp64):
    p, z = rand100, 4096
    with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed", seed=3,
                      refresh_fp64=refresh_fp64) as s:
        samples = s.run(640, thin=64)
        st = s.check()
    worst = max(float((X @ p.A.T - p.b).max()) for X in samples)
    assert worst <= 1e-6, worst
    assert st.max_violation <= 1e-6
    assert st.refresh_drift <= 1e-5, st.refresh_drift
    assert st.stalls == 0 and st.unbounded == 0


@pytest.mark.parametrize("prec", ["mixed", "mixed_rs"])
def test_simplex_cuts_equalities_hold(prec):
    p = wl.simplex_cuts(1000, 4000, seed=3)
    z = 1024
    with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision=prec, seed=1) as s:
        samples = s.run(200, thin=50)
        st = s.check()
    for X in samples:
        assert np.abs(X.sum(axis=1) - 1.0).max() <= 1e-8
        assert (X @ p.A.T - p.b).max() <= 1e-6
    assert st.eq_residual <= 1e-8 and st.max_violation <= 1e-6
    # The walkers moved away from the start.
    assert np.abs(samples[-1] - p.x0).max() > 1e-3


@pytest.mark.parametrize("prec", ["mixed", "mixed_rs"])
def test_time_kernels_reports_device_times(rand100, prec):
    p = rand100
    with mhar.Sampler(p.A, p.b, p.x0, 4096, precision=prec, seed=0) as s:
        ms = s.time_kernels(32)
        X, step = s.state()
    assert step == 32
    # In the recompute mode the chord kernel draws the next directions itself,
    # so the separate direction time is 0.
    assert (0 < ms[0] < 1.0 if prec == "mixed" else ms[0] == 0.0)
    assert 0 < ms[1] < 5.0 and 0 <= ms[2] < 5.0
    assert (X @ p.A.T - p.b).max() <= 1e-6
