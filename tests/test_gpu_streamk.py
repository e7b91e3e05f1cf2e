"""GPU tests of the stream-K schedule of the recompute kernel (shared-memory
operands, n > 128).

Clusters along the rows and stream-K cut the (walker strip, row tile) work
differently, but the chord is a max / min over rows (exact in any order) and
every other step is per walker, so the two schedules must agree bit for bit;
the oracle checks the walk itself.  The shapes cover strips split over many
SMs, SMs that take several whole strips, and ranges that cross strips.
"""
import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# (n, m, z): row tiles x strips = 8 x 2 (each strip cut into 8 segments),
# 40 x 32 (ranges of ~8.4 tiles crossing strips), 3 x 200 (whole strips and
# split ones), 3 x 5.
SHAPES = [(150, 900, 256), (300, 5000, 4096), (140, 300, 25600), (130, 300, 640)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()


@pytest.mark.parametrize("n,m,z", SHAPES)
def test_stream_k_equals_clusters(n, m, z):
    p = wl.random_polytope(n, m, seed=n + m, check_bounded="auto")
    outs = {}
    for sched in (1, 2):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", seed=11, schedule=sched) as s:
            X = s.run(20, thin=5)
            lo, hi, t = s.chord()
            st = s.check()
        assert st.max_violation <= 1e-6
        outs[sched] = (X, lo, hi, t)
    for a, b in zip(outs[1], outs[2]):
        np.testing.assert_array_equal(a, b)


def test_stream_k_against_oracle():
    p = wl.random_polytope(150, 900, seed=5)
    z, steps = 200, 10
    ref = mixed.mixed_run(p.A, p.b, np.tile(p.x0, (z, 1)), steps, "mixed_rs", thin=1, seed=3,
                          trace=True)
    with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", seed=3, schedule=2) as s:
        got = s.run(steps, thin=1)
        lo, hi, t = s.chord()
    err = np.abs(got - ref["samples"]).max() / max(1.0, np.abs(ref["samples"]).max())
    assert err <= 1e-4, err
    span = np.maximum(1.0, ref["lmax"][-1] - ref["lmin"][-1])
    assert np.all(np.abs(lo - ref["lmin"][-1]) <= 1e-4 * span)


def test_stream_k_with_equalities_and_preconditioner():
    p = wl.simplex_cuts(150, 400, seed=9)
    rng = np.random.default_rng(1)
    delta, U = rng.uniform(0.5, 1.5, 150), 0.2 * rng.standard_normal((150, 3))
    outs = []
    for sched in (1, 2):
        with mhar.Sampler(p.A, p.b, p.x0, 384, AE=p.AE, bE=p.bE, precision="mixed_rs", seed=2,
                          schedule=sched) as s:
            s.run(5)
            s.set_preconditioner(delta, U)
            outs.append(s.run(12, thin=4))
            st = s.check()
        assert st.max_violation <= 1e-6 and st.eq_residual <= 1e-8
    np.testing.assert_array_equal(outs[0], outs[1])


def test_schedule_option_rejected_out_of_range():
    p = wl.random_polytope(150, 400, seed=2)
    with pytest.raises(mhar.MharError) as e:
        mhar.Sampler(p.A, p.b, p.x0, 128, precision="mixed_rs", schedule=3)
    assert e.value.code == mhar.E_ARG


def test_tall_body_goes_to_stream_k():
    # m = 40000 rows exceeds clusters of 8 CTAs x 32 row tiles; the automatic
    # schedule takes stream-K, which has no such limit.
    p = wl.random_polytope(20, 40000, seed=3, check_bounded="auto")
    z, steps = 128, 5
    with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", seed=6, smem_operands=True) as s:
        assert s.kernel_name() == "recompute_sk_kernel"
        got = s.run(steps, thin=1)
    ref = mixed.mixed_run(p.A, p.b, np.tile(p.x0, (z, 1)), steps, "mixed_rs", thin=1, seed=6)
    err = np.abs(got - ref["samples"]).max() / max(1.0, np.abs(ref["samples"]).max())
    assert err <= 1e-4, err
    with pytest.raises(mhar.MharError) as e:
        mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", smem_operands=True, schedule=1)
    assert e.value.code == mhar.E_UNSUPPORTED


def test_contexts_of_different_sizes_side_by_side():
    """Dynamic shared memory limits are set per kernel function, not per
    context: a small context created after a large one must leave the large
    one launchable (the stream-K walker update stages 4 walkers of n = 1000
    but 8 of n = 200; the projection keeps h of either length)."""
    big = wl.simplex_cuts(1000, 600, seed=2)
    small = wl.simplex_cuts(200, 300, seed=3)
    opts = dict(precision="mixed_rs", smem_operands=True, schedule=2)
    with mhar.Sampler(big.A, big.b, big.x0, 256, AE=big.AE, bE=big.bE, seed=1, **opts) as a:
        with mhar.Sampler(small.A, small.b, small.x0, 256, AE=small.AE, bE=small.bE, seed=2,
                          **opts) as b:
            assert a.kernel_name() == b.kernel_name() == "recompute_sk_kernel"
            a.run(2)
            b.run(2)
            a.run(2)
            for s in (a, b):
                st = s.check()
                assert st.max_violation <= 1e-10 and st.eq_residual <= 1e-8
