"""The law of the GPU walk at the scale of the paper's own check (Section
6.4): Friedman-Rafsky two-sample MST tests of the tensor-core sampler's
points against exact uniform draws on hypercubes and simplexes, burn-in n^3
(hypercube) and (n-1)^3 (simplex) iterations as in the paper, acceptance
W >= -1.64.  Walkers are independent chains (Section 4.1), so the z walkers'
points after burn-in are an iid sample.  The paper compares 5000 points; here
2000 (per replicate) keep the dense MST small.
"""
import numpy as np
import pytest

from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl
from stats_util import friedman_rafsky

pytestmark = pytest.mark.gpu

Z = 2000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()


def _fr_replicates(body, burn, draw, n, reps=3):
    Ws = []
    for rep in range(reps):
        with mhar.Sampler(body.A, body.b, body.x0, Z, AE=body.AE, bE=body.bE,
                          precision="mixed_rs", seed=1000 + rep) as s:
            s.run(burn)
            X = s.state()[0]
            st = s.check()
        assert st.max_violation <= 1e-6
        Ws.append(friedman_rafsky(X, draw(n, Z, seed=500 + rep)))
    return Ws


@pytest.mark.parametrize("n", [5, 15, 25])
def test_friedman_rafsky_hypercube(n):
    Ws = _fr_replicates(wl.cube(n), n ** 3, wl.uniform_cube_points, n)
    assert np.median(Ws) >= -1.64 and sum(w >= -1.64 for w in Ws) >= 2, Ws


@pytest.mark.parametrize("n", [5, 15, 25])
def test_friedman_rafsky_simplex(n):
    Ws = _fr_replicates(wl.simplex(n), (n - 1) ** 3, wl.uniform_simplex_points, n)
    assert np.median(Ws) >= -1.64 and sum(w >= -1.64 for w in Ws) >= 2, Ws
