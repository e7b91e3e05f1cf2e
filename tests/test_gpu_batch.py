"""GPU tests of the batched launch (mhar_batch_*): many polytopes of different
sizes advanced by one kernel launch per iteration.

Each problem p of a batch is the recompute-mode sampler with Philox key
seed + p, so it must equal, bit for bit, a single context with that key and
the same (shared-memory operand) kernel; the chord's min / max reductions are
exact, so the cluster size the autotuner picks cannot change a result.  The
oracle checks the walks themselves.
"""
import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SHAPES = [(12, 40, 1), (37, 300, 2), (100, 700, 3), (150, 900, 4), (20, 45, 5), (64, 2100, 6)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()


@pytest.fixture(scope="module")
def bodies():
    return [wl.random_polytope(n, m, seed=s) for (n, m, s) in SHAPES]


def _tuned_iterations(bodies, iters):
    """Iterations the tuner runs: 1 + iters per candidate shape (the persistent
    launch and the cluster sizes)."""
    max_tiles = max((p.m + 127) // 128 for p in bodies)
    return sum(1 + iters for c in (0, 1, 2, 4, 8) if c <= max_tiles)


def _problems(bodies):
    return [(p.A, p.b, p.x0) for p in bodies]


def test_batch_equals_single_contexts(bodies):
    z, seed = 256, 40
    with mhar.Batch(_problems(bodies), z, seed=seed) as bt:
        got = bt.run(20, thin=5)
        C = bt.tune(4)
        assert C in (0, 1, 2, 4, 8)
        got2 = bt.run(12, thin=12)
    for q, p in enumerate(bodies):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", seed=seed + q,
                          smem_operands=True) as s:
            want = s.run(20, thin=5)
            s.run(_tuned_iterations(bodies, 4))
            want2 = s.run(12, thin=12)
        np.testing.assert_array_equal(got[q], want, err_msg=f"problem {q}")
        np.testing.assert_array_equal(got2[q], want2, err_msg=f"problem {q} after tuning")


def test_batch_against_oracle(bodies):
    z, seed, steps = 130, 7, 10
    with mhar.Batch(_problems(bodies), z, seed=seed) as bt:
        got = bt.run(steps, thin=1)
        stats = [bt.check(q) for q in range(len(bodies))]
    for q, p in enumerate(bodies):
        ref = mixed.mixed_run(p.A, p.b, np.tile(p.x0, (z, 1)), steps, "mixed_rs", thin=1,
                              seed=seed + q)
        err = np.abs(got[q] - ref["samples"]).max() / max(1.0, np.abs(ref["samples"]).max())
        assert err <= 1e-4, (q, err)
        assert stats[q].max_violation <= 1e-6


@pytest.mark.parametrize("z", [256, 4096])
def test_batch_shapes_bit_equal(bodies, z):
    # z = 256: 12 units, fewer than the SMs (one unit per CTA of the
    # persistent launch); z = 4096: 192 units of n from 12 to 150 on 152
    # SMs, so CTAs pull several units and the shared-memory rings and the
    # unit ring wrap, switching between resident (n <= 128) and streamed
    # walker operands.
    out = {}
    for shape in (0, 1, 2, 4):
        with mhar.Batch(_problems(bodies), z, seed=11) as bt:
            bt.set_shape(shape)
            out[shape] = bt.run(15, thin=5)
            stats = [bt.check(q) for q in range(len(bodies))]
        assert all(st.max_violation <= 1e-10 for st in stats), shape
    for shape in (0, 2, 4):
        for q in range(len(bodies)):
            np.testing.assert_array_equal(out[shape][q], out[1][q], err_msg=f"shape {shape} problem {q}")


def test_batch_persistent_against_oracle(bodies):
    z, seed, steps = 200, 9, 8
    with mhar.Batch(_problems(bodies), z, seed=seed) as bt:
        bt.set_shape(0)
        got = bt.run(steps, thin=1)
    for q, p in enumerate(bodies):
        ref = mixed.mixed_run(p.A, p.b, np.tile(p.x0, (z, 1)), steps, "mixed_rs", thin=1,
                              seed=seed + q)
        err = np.abs(got[q] - ref["samples"]).max() / max(1.0, np.abs(ref["samples"]).max())
        assert err <= 1e-4, (q, err)


def test_batch_shape_rejected(bodies):
    with mhar.Batch(_problems(bodies[:1]), 64) as bt:    # one row tile
        for bad in (3, -1, 2, 16):
            with pytest.raises(mhar.MharError) as e:
                bt.set_shape(bad)
            assert e.value.code == mhar.E_ARG


def test_batch_feasible_over_many_iterations(bodies):
    with mhar.Batch(_problems(bodies), 384, seed=3) as bt:
        bt.tune(2)
        bt.run(300)
        for q, p in enumerate(bodies):
            X, step = bt.state(q)
            assert step == 300 + _tuned_iterations(bodies, 2)
            assert (X @ p.A.T - p.b).max() <= 1e-6
            assert bt.check(q).max_violation <= 1e-6


def test_batch_trace_subset(bodies):
    with mhar.Batch(_problems(bodies[:3]), 256, seed=2) as full, \
            mhar.Batch(_problems(bodies[:3]), 256, seed=2, emit_walkers=17) as sub:
        a = full.run(6, thin=3)
        b = sub.run(6, thin=3)
    for q in range(3):
        assert b[q].shape == (2, 17, bodies[q].n)
        np.testing.assert_array_equal(a[q][:, :17], b[q])


def test_batch_errors(bodies):
    p = bodies[0]
    with pytest.raises(mhar.MharError) as e:
        mhar.Batch([(p.A, p.b, p.x0), (p.A, p.b, p.x0 + 100.0)], 64)
    assert e.value.code == mhar.E_X0_INFEASIBLE
    with pytest.raises(mhar.MharError):
        mhar.Batch([], 64)
