"""The split R_hat convergence check used with the ESS (CPU only)."""
import numpy as np

from paper_2104_07097_gb300 import diagnostics


def test_split_rhat_of_stationary_chains_is_one():
    rng = np.random.default_rng(0)
    tr = rng.standard_normal((2000, 64, 3))
    r = diagnostics.split_rhat(tr)
    assert np.all(np.abs(r - 1.0) < 0.01), r


def test_split_rhat_flags_a_transient():
    # A drift through the trace (a chain still leaving its start) puts the
    # two halves' means apart.
    rng = np.random.default_rng(1)
    T = 1000
    drift = np.linspace(0.0, 3.0, T)[:, None, None]
    tr = rng.standard_normal((T, 32, 2)) + drift
    assert np.all(diagnostics.split_rhat(tr) > 1.2)


def test_split_rhat_flags_chains_stuck_apart():
    rng = np.random.default_rng(2)
    tr = rng.standard_normal((500, 40, 1))
    tr[:, :20] += 2.0
    assert diagnostics.split_rhat(tr)[0] > 1.3
    # ... and is invariant under an affine change of the coordinate
    np.testing.assert_allclose(diagnostics.split_rhat(5 * tr - 7), diagnostics.split_rhat(tr))
