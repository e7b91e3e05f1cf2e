"""Parity where the configurations run: the simplex with 4000 cuts (n = 1000,
16 K chunks, one equality) and the ill-conditioned body (n = 500, stream-K,
with a fitted preconditioner) at their full walker counts, on sampled
walkers the oracles compute one by one (walker0 offsets); and equality
systems from 2 to 96 rows (random full-rank ones and transportation
polytopes'), in FP64 against the pure oracle (1e-10) and in the FP32 and
tensor-core modes against the reduced-precision oracle (1e-4); and the
rejection of an A_E too ill-conditioned for the projector; and a body past
the length the projection keeps in shared memory (n = 1700).

Section 3.2 (the projector, Lemma 3.1), Section 4.4 (line sets).
"""
import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SAMPLES = ((0, 6), (4093, 6))


def _rel(got, want, scale):
    return float(np.abs(got - want).max() / scale)


@pytest.mark.parametrize("prec", ["mixed_rs", "mixed"])
def test_simplex1000_cuts4000_sampled_parity(prec):
    p = wl.simplex_cuts(1000, 4000, seed=3)
    z, steps = 8192, 4
    with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision=prec, seed=0) as s:
        assert prec != "mixed_rs" or s.kernel_name() == "recompute_sk_kernel"
        got = s.run(steps, thin=1)
        st = s.check()
    assert st.eq_residual <= 1e-8
    for w0, cnt in SAMPLES + ((z - 6, 6),):
        ref = mixed.mixed_run(p.A, p.b, np.tile(p.x0, (cnt, 1)), steps, prec, seed=0, AE=p.AE,
                              walker0=w0)
        for j in range(steps):
            want = ref["samples"][j]
            # coordinates are about 1/n: relative to the largest one, not to 1
            err = _rel(got[j, w0:w0 + cnt], want, np.abs(want).max())
            assert err <= 1e-4, (w0, j, err)


@pytest.mark.parametrize("prec", ["fp32", "mixed_rs"])
def test_equalities_past_kept_length(prec):
    """n = 1700, one equality: past the 1536 coordinates the projection keeps
    in shared memory, so its second pass draws h again (Section 3.2, 4.3)."""
    p = wl.simplex_cuts(1700, 600, seed=9)
    z, steps = 64, 3
    with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision=prec, seed=4) as s:
        got = s.run(steps, thin=1)
        st = s.check()
    assert st.eq_residual <= 1e-8
    ref = mixed.mixed_run(p.A, p.b, np.tile(p.x0, (z, 1)), steps, prec, seed=4, AE=p.AE)
    for j in range(steps):
        want = ref["samples"][j]
        err = _rel(got[j], want, np.abs(want).max())
        assert err <= 1e-4, (j, err)


def test_illcond500_fitted_stream_k_sampled_parity():
    p = wl.ill_conditioned(500, 10000, seed=5, smin=1e-3)
    s_axes = 1.0 / np.abs(p.A).max(axis=0)
    z = 16384
    with mhar.Sampler(p.A, p.b, p.x0, z, precision="mixed_rs", seed=0) as s:
        assert s.kernel_name() == "recompute_sk_kernel"
        s.set_preconditioner(s_axes / s_axes.max())
        s.fit_preconditioner(60, 3, 32, 2)
        delta, U = s.preconditioner()
        X0, step0 = s.state()
        got = s.run(3, thin=1)
    for w0, cnt in SAMPLES + ((z - 6, 6),):
        ref = mixed.mixed_run(p.A, p.b, X0[w0:w0 + cnt], 3, "mixed_rs", seed=0, step0=step0,
                              delta=delta, U=U, walker0=w0)
        for j in range(3):
            # whitened coordinates x_i / s_i: every axis on the same scale
            err = _rel(got[j, w0:w0 + cnt] / s_axes, ref["samples"][j] / s_axes,
                       max(1.0, np.abs(ref["samples"][j] / s_axes).max()))
            assert err <= 1e-4, (w0, j, err)


def _subspace_body(n, m, mE, seed):
    """Random cuts a.x <= 1 (unit rows) intersected with A_E x = 0, A_E a random
    full-rank mE x n matrix; x0 = 0 is interior."""
    p = wl.random_polytope(n, m, seed=seed)
    rng = np.random.default_rng(seed + 1)
    AE = rng.standard_normal((mE, n))
    return wl.Polytope(A=p.A, b=p.b, x0=np.zeros(n), AE=AE, bE=np.zeros(mE),
                       name=f"rand{n}x{m}+{mE}eq")


def _transportation(rows, cols, seed):
    """{X >= 0 (rows x cols), row sums r, column sums c}: the equalities are
    every row sum and all column sums but the last (rows + cols - 1 independent
    rows); x0 = r_i c_j / total is interior."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(1.0, 2.0, rows)
    c = rng.uniform(1.0, 2.0, cols)
    c *= r.sum() / c.sum()
    n = rows * cols
    AE, bE = [], []
    for i in range(rows):
        e = np.zeros((rows, cols)); e[i, :] = 1.0
        AE.append(e.ravel()); bE.append(r[i])
    for j in range(cols - 1):
        e = np.zeros((rows, cols)); e[:, j] = 1.0
        AE.append(e.ravel()); bE.append(c[j])
    x0 = (np.outer(r, c) / r.sum()).ravel()
    return wl.Polytope(A=-np.eye(n), b=np.zeros(n), x0=x0, AE=np.array(AE), bE=np.array(bE),
                       name=f"transport{rows}x{cols}")


BODIES = {
    "rand60x300+5eq": lambda: _subspace_body(60, 300, 5, seed=31),
    "rand80x400+32eq": lambda: _subspace_body(80, 400, 32, seed=32),
    "rand160x500+96eq": lambda: _subspace_body(160, 500, 96, seed=34),
    "transport5x7": lambda: _transportation(5, 7, seed=33),
    "transport12x16": lambda: _transportation(12, 16, seed=35),
}


@pytest.mark.parametrize("name", sorted(BODIES))
def test_equalities_fp64_free_running_50(name):
    p = BODIES[name]()
    z = 96
    X0 = np.tile(p.x0, (z, 1))
    ref = oracle.mhar_run(p.A, p.b, X0, steps=50, thin=1, seed=7, AE=p.AE, trace=True)
    with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision="fp64", seed=7) as s:
        got = s.run(50, thin=1)
        st = s.check()
    scale = max(1.0, np.abs(ref["samples"]).max())
    assert _rel(got, ref["samples"], scale) <= 1e-10
    assert st.eq_residual <= 1e-8 and st.max_violation <= 1e-6 * max(1.0, np.abs(p.b).max())


@pytest.mark.parametrize("prec", ["fp32", "mixed", "mixed_rs"])
@pytest.mark.parametrize("name", sorted(BODIES))
def test_equalities_step_for_step_50(name, prec):
    p = BODIES[name]()
    z = 96
    X0 = np.tile(p.x0, (z, 1))
    pure = oracle.mhar_run(p.A, p.b, X0, steps=50, thin=1, seed=7, AE=p.AE)
    with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision=prec, seed=7,
                      audit_every=1) as s:
        worst = 0.0
        for j in range(50):
            start = X0 if j == 0 else pure["samples"][j - 1]
            ref = mixed.mixed_run(p.A, p.b, start, 1, prec, seed=7, step0=j, AE=p.AE, trace=True)
            s.set_state(start, j)
            got = s.run(1, thin=1)[0]
            scale = max(1.0, np.abs(ref["samples"][0]).max())
            worst = max(worst, _rel(got, ref["samples"][0], scale))
            lo, hi, t = s.chord()
            span = np.maximum(1.0, ref["lmax"][0] - ref["lmin"][0])
            assert np.all(np.abs(lo - ref["lmin"][0]) <= 1e-4 * span)
            assert np.all(np.abs(hi - ref["lmax"][0]) <= 1e-4 * span)
        st = s.stats()
    assert worst <= 1e-4, worst
    assert st.run_max_violation <= 1e-10 and st.run_eq_residual <= 1e-8


def test_ill_conditioned_equalities_rejected():
    # Two rows 1e-9 apart in direction: cond(A_E) ~ 1e9, past what the FP64
    # CholeskyQR2 factor resolves.
    p = wl.random_polytope(20, 60, seed=2)
    AE = np.zeros((2, 20))
    AE[0, 0] = AE[1, 0] = 1.0
    AE[1, 1] = 1e-9
    with pytest.raises(mhar.MharError) as e:
        mhar.Sampler(p.A, p.b, np.zeros(20), 8, AE=AE, bE=np.zeros(2))
    assert e.value.code == mhar.E_RANK
