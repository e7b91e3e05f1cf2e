"""Parity at the edges of the kernels' tiling, through the C ABI.

The tensor-core kernels cut n into 64-column K chunks of 16-column K steps
(n <= 128 keeps the walker operands in tensor memory, larger n streams them),
m into 128-row tiles and z into strips of 128 walkers; the CUDA-core kernels
use 64 x 64 tiles or a warp per walker.  These cases sit on and next to each
boundary -- n = 1, 2, 15, 16, 17, 63, 64, 65, 127, 128, 129, 192, 193; m with
a ragged last tile; a single walker and a ragged last strip (z = 1, 131) --
in every mode: the FP64 mode against the pure oracle at 1e-10 over 8
iterations, the FP32 and tensor-core modes step for step against the
reduced-precision oracle at 1e-4, with an FP64 audit after every iteration.
Algorithm 2; Sections 4.3-4.5.
"""
import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NS = [1, 2, 15, 16, 17, 63, 64, 65, 127, 128, 129, 192, 193]
ZS = [1, 131]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()


def _body(n):
    # m = 3n + 5 rows: for every n here a ragged last 128-row tile.
    return wl.random_polytope(n, 3 * n + 5, seed=1000 + n, check_bounded="auto")


def _nw(a, b):
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


@pytest.mark.parametrize("z", ZS)
@pytest.mark.parametrize("n", NS)
def test_fp64_edges(n, z):
    p = _body(n)
    ref = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (z, 1)), steps=8, thin=1, seed=3)
    with mhar.Sampler(p.A, p.b, p.x0, z, precision="fp64", seed=3, audit_every=1) as s:
        got = s.run(8, thin=1)
        st = s.stats()
    assert max(_nw(got[j], ref["samples"][j]) for j in range(8)) <= 1e-10
    assert st.audits == 8 and st.run_max_violation <= 1e-12 * max(1.0, np.abs(p.b).max())


@pytest.mark.parametrize("prec", ["fp32", "mixed", "mixed_rs"])
@pytest.mark.parametrize("z", ZS)
@pytest.mark.parametrize("n", NS)
def test_reduced_precision_edges(n, z, prec):
    p = _body(n)
    steps = 5
    X0 = np.tile(p.x0, (z, 1))
    pure = oracle.mhar_run(p.A, p.b, X0, steps=steps, thin=1, seed=3)
    with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=3, audit_every=1) as s:
        for j in range(steps):
            start = X0 if j == 0 else pure["samples"][j - 1]
            ref = mixed.mixed_run(p.A, p.b, start, 1, prec, seed=3, step0=j, trace=True)
            s.set_state(start, j)
            got = s.run(1, thin=1)[0]
            assert _nw(got, ref["samples"][0]) <= 1e-4, (j, _nw(got, ref["samples"][0]))
            lo, hi, t = s.chord()
            span = np.maximum(1.0, ref["lmax"][0] - ref["lmin"][0])
            assert np.all(np.abs(lo - ref["lmin"][0]) <= 1e-4 * span)
            assert np.all(np.abs(hi - ref["lmax"][0]) <= 1e-4 * span)
        st = s.stats()
    assert st.run_max_violation <= 1e-10 * max(1.0, np.abs(p.b).max())
