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


def _problems(bodies):
    return [(p.A, p.b, p.x0) for p in bodies]


def test_batch_equals_single_contexts(bodies):
    z, seed = 256, 40
    with mhar.Batch(_problems(bodies), z, seed=seed) as bt:
        got = bt.run(20, thin=5)
        C = bt.tune(4)
        assert C in (-1, 0, 1, 2, 4, 8)
        # The tuner's timed iterations are real ones and advance every problem
        # alike, whatever shapes it tries.
        steps = [bt.state(q)[1] for q in range(len(bodies))]
        assert len(set(steps)) == 1 and steps[0] > 20
        tuned = steps[0] - 20
        got2 = bt.run(12, thin=12)
    for q, p in enumerate(bodies):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", seed=seed + q,
                          smem_operands=True) as s:
            want = s.run(20, thin=5)
            s.run(tuned)
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


def test_batch_per_bucket_shapes_bit_equal(bodies):
    # Buckets by the 64-column K chunks of n: n = 12, 37, 20, 64 -> bucket 0;
    # n = 100 -> bucket 1; n = 150 -> bucket 2.  Each bucket on its own
    # stream with its own shape gives the bits of one shape for the batch.
    z = 256
    with mhar.Batch(_problems(bodies), z, seed=21) as bt:
        bt.set_shape(1)
        ref = bt.run(15, thin=5)
        per, shapes, of = bt.get_shapes()
        assert not per and shapes == [1, 1, 1, -1, -1] and of == [0, 0, 1, 2, 0, 0]
    for mix in ((2, 0, 4), (0, 1, 0), (4, 2, 1)):
        with mhar.Batch(_problems(bodies), z, seed=21) as bt:
            for k, c in enumerate(mix):
                bt.set_bucket_shape(k, c)
            per, shapes, _ = bt.get_shapes()
            assert per and shapes == list(mix) + [-1, -1]
            got = bt.run(15, thin=5)
            stats = [bt.check(q) for q in range(len(bodies))]
            steps = {bt.state(q)[1] for q in range(len(bodies))}
        assert steps == {15}
        assert all(st.max_violation <= 1e-10 for st in stats), mix
        for q in range(len(bodies)):
            np.testing.assert_array_equal(got[q], ref[q], err_msg=f"shapes {mix} problem {q}")
    # Back to one shape after per-bucket mode.
    with mhar.Batch(_problems(bodies), z, seed=21) as bt:
        bt.set_bucket_shape(2, 0)
        bt.run(5)
        bt.set_shape(1)
        got = bt.run(10, thin=5)
        assert not bt.get_shapes()[0]
    for q in range(len(bodies)):
        np.testing.assert_array_equal(got[q], ref[q][1:], err_msg=f"problem {q}")


def test_batch_bucket_shape_rejected(bodies):
    with mhar.Batch(_problems(bodies), 64) as bt:
        for bucket, shape in ((3, 1), (4, 0), (-1, 1), (5, 1), (1, 3), (1, 16), (2, -1)):
            with pytest.raises(mhar.MharError) as e:
                bt.set_bucket_shape(bucket, shape)
            assert e.value.code == mhar.E_ARG, (bucket, shape)


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
        tuned = bt.state(0)[1]
        bt.run(300)
        for q, p in enumerate(bodies):
            X, step = bt.state(q)
            assert step == 300 + tuned
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
