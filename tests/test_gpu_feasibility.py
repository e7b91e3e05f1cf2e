"""Feasibility at every iteration on the bodies where rounding is hardest.

Every chord end is computed from a slack lowered by a bound on its rounding
error and from an a_i . d pushed away from zero by its own bound (include/mhar.h,
"Feasibility in every mode"), so a point on the computed chord satisfies
A x <= b exactly under the error model.  These tests audit that in FP64 after
every iteration (opts.audit_every = 1, every walker) on
  * an ill-conditioned body (axes from 1e-3 to 1, the benchmark's mixing
    workload at a smaller size): large row norms, coordinates of very
    different size;
  * random bodies with m close to 2n: nearly unbounded, with long axes, so
    the points and chords are long and sum |a_ij x_j| is large;
  * the simplex with cuts (one equality, checked to 1e-8);
in every arithmetic mode and launch schedule.  The required bound is
max(A x - b) <= 1e-6 |b|_inf at every step; the construction aims at <= 0 up
to the FP64 rounding of the audit itself, which is asserted too.
"""
import numpy as np
import pytest

from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _audited(s, steps):
    before = s.stats().audits
    s.run(steps)
    st = s.stats()
    assert st.audits - before == steps
    return st


@pytest.fixture(scope="module")
def illcond():
    return wl.ill_conditioned(200, 4000, seed=7, smin=1e-3)


@pytest.mark.parametrize("prec,kw", [
    ("mixed_rs", {"schedule": 1}),
    ("mixed_rs", {"schedule": 2}),
    ("mixed", {"refresh_k": 16}),
    ("fp32", {}),
    ("fp64", {}),
])
def test_ill_conditioned_every_iteration(illcond, prec, kw):
    p = illcond
    with mhar.Sampler(p.A, p.b, p.x0, 1024, precision=prec, seed=3, audit_every=1, **kw) as s:
        st = _audited(s, 200 if prec == "fp64" else 400)
        assert st.stalls <= 1e-3 * 1024 * 400
    bmax = np.abs(p.b).max()
    assert st.run_max_violation <= TOL * bmax, st.run_max_violation
    # The margins make the exact slack non-negative; the audit's own FP64
    # rounding is far below this.
    assert st.run_max_violation <= 1e-10 * bmax, st.run_max_violation


def test_ill_conditioned_preconditioned_every_iteration(illcond):
    # The axes' own scales as the preconditioner (a perfect diagonal fit), and
    # a fitted one: both change the coordinate scales of the FP16 operands.
    p = illcond
    s_axes = 1.0 / np.abs(p.A).max(axis=0)
    with mhar.Sampler(p.A, p.b, p.x0, 1024, precision="mixed_rs", seed=4, audit_every=1) as s:
        s.set_preconditioner(s_axes / s_axes.max())
        st = _audited(s, 300)
    assert st.run_max_violation <= 1e-10
    with mhar.Sampler(p.A, p.b, p.x0, 1024, precision="mixed_rs", seed=5, audit_every=1) as s:
        s.fit_preconditioner(60, snapshots=4, rank=16)
        st = _audited(s, 300)
    assert st.run_max_violation <= 1e-10


@pytest.mark.parametrize("n,m,smem", [(100, 215, False), (100, 215, True), (300, 620, False)])
def test_nearly_unbounded_every_iteration(n, m, smem):
    p = wl.random_polytope(n, m, seed=17)
    with mhar.Sampler(p.A, p.b, p.x0, 512, precision="mixed_rs", seed=2, audit_every=1,
                      smem_operands=smem) as s:
        st = _audited(s, 600)
        X, _ = s.state()
    # The walk did reach far out (long axes): the margins were exercised.
    assert np.abs(X).max() > 1.5
    assert st.run_max_violation <= 1e-10


def test_batch_of_nearly_unbounded_bodies_every_iteration():
    bodies = wl.batch(6, seed=11, nmin=20, nmax=160, mfac=(2, 3))
    with mhar.Batch([(p.A, p.b, p.x0) for p in bodies], 256, seed=5, audit_every=1) as bt:
        bt.tune(2)
        bt.run(400)
        for q in range(len(bodies)):
            st = bt.check(q)
            assert st.audits == 400    # the tuner's iterations are not audited
            assert st.run_max_violation <= 1e-10, (q, st.run_max_violation)
            assert st.max_violation <= 1e-10


@pytest.mark.parametrize("prec", ["mixed_rs", "mixed", "fp32"])
def test_simplex_cuts_every_iteration(prec):
    p = wl.simplex_cuts(300, 1200, seed=9)
    with mhar.Sampler(p.A, p.b, p.x0, 512, AE=p.AE, bE=p.bE, precision=prec, seed=6,
                      audit_every=1, refresh_k=16) as s:
        st = _audited(s, 300)
    assert st.run_max_violation <= 1e-10
    assert st.run_eq_residual <= 1e-8


def test_audit_of_a_subset_and_a_period():
    p = wl.random_polytope(40, 300, seed=3)
    with mhar.Sampler(p.A, p.b, p.x0, 300, precision="mixed_rs", seed=1, audit_every=7,
                      audit_walkers=50) as s:
        s.run(30, thin=10)
        st = s.stats()
    assert st.audits == 4          # after iterations 7, 14, 21, 28
    assert st.run_max_violation <= 1e-10
