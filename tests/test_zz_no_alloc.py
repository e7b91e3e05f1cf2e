"""The allocation-free chord entry point, mhar_chord_noalloc.

It serves callers that must not allocate device memory -- a process living
inside a fixed, pre-reserved device-memory budget, or a latency-critical loop
that cannot afford the synchronisation cudaMalloc / cudaFree may bring -- by
keeping its working memory in a fixed array built into the library.  This
test calls it through the C ABI several times in a row (other inputs each
time, and a smaller walker count after a larger one, so stale contents of the
shared array would show) and checks every result against the FP64 oracle's
chord of the same point and direction (oracle.chord) at the FP64 parity
tolerance 1e-10; it also checks the open sides of a half-space body and the
NaN marking of a walker that meets a non-finite value.

This file is named to be collected last, so a failure here does not stop a
run before the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2104_07097_gb300 import mhar
from paper_2104_07097_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()
    return t


def _call(torch, A, b, X, D):
    dev = torch.device("cuda")
    m, n = A.shape
    z = X.shape[0]
    A_d = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    b_d = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
    X_d = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    D_d = torch.from_numpy(np.ascontiguousarray(D)).to(dev)
    lo_d = torch.full((z,), 7.0, dtype=torch.float64, device=dev)
    hi_d = torch.full((z,), 7.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rc = mhar.mhar_chord_noalloc(A_d.data_ptr(), b_d.data_ptr(), m, n, X_d.data_ptr(),
                                 D_d.data_ptr(), z, lo_d.data_ptr(), hi_d.data_ptr(), stream)
    assert rc == mhar.OK, mhar.mhar_last_error(None)
    torch.cuda.synchronize()
    return lo_d.cpu().numpy(), hi_d.cpu().numpy()


def _oracle_chords(A, b, X, D):
    ref = [oracle.chord(A, b, X[k], D[k]) for k in range(X.shape[0])]
    return np.array([r[0] for r in ref]), np.array([r[1] for r in ref])


def _close(got, want, span):
    both_inf = np.isinf(got) & np.isinf(want) & (np.sign(got) == np.sign(want))
    with np.errstate(invalid="ignore"):    # inf - inf where both ends are open
        ok = both_inf | (np.abs(got - want) <= TOL * span)
    return bool(np.all(ok))


def test_chord_noalloc_matches_oracle_on_successive_calls(torch):
    p = wl.random_polytope(37, 300, seed=11)
    seed = 4
    # Points: the oracle's own chain after a few iterations (distinct per walker).
    X = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (200, 1)), steps=5, seed=seed)["X"]
    for call, (step, z) in enumerate(((5, 200), (6, 200), (7, 57))):
        Xc = X[:z]
        D = np.array([oracle.direction_normals(seed, step, k, p.n) for k in range(z)])
        lo, hi = _call(torch, p.A, p.b, Xc, D)
        lo_ref, hi_ref = _oracle_chords(p.A, p.b, Xc, D)
        span = np.maximum(1.0, hi_ref - lo_ref)
        assert _close(lo, lo_ref, span), (call, np.abs(lo - lo_ref).max())
        assert _close(hi, hi_ref, span), (call, np.abs(hi - hi_ref).max())
        # Next call starts from other points.
        X = oracle.mhar_run(p.A, p.b, X, steps=1, seed=seed, step0=step)["X"]


def test_chord_noalloc_open_sides_and_nonfinite(torch):
    # The half-space x_0 <= 1: a direction with d_0 > 0 meets the facet ahead
    # only (lambda_min = -inf), d_0 < 0 behind only (lambda_max = +inf), d_0 =
    # 0 never; a NaN coordinate marks its walker with NaN chord ends.
    A = np.array([[1.0, 0.0, 0.0]])
    b = np.array([1.0])
    X = np.array([[0.0, 0.0, 0.0], [0.5, 1.0, 2.0], [-1.0, 0.0, 0.0], [0.0, np.nan, 0.0]])
    D = np.array([[2.0, 1.0, 0.0], [-1.0, 0.0, 3.0], [0.0, 1.0, 1.0], [1.0, 0.0, 0.0]])
    lo, hi = _call(torch, A, b, X, D)
    assert lo[0] == -np.inf and abs(hi[0] - 0.5) <= TOL
    assert lo[1] == -0.5 and hi[1] == np.inf
    assert lo[2] == -np.inf and hi[2] == np.inf
    assert np.isnan(lo[3]) and np.isnan(hi[3])
    for k in range(3):
        ref = oracle.chord(A, b, X[k], D[k])
        assert _close(np.array([lo[k], hi[k]]), np.array(ref[:2]), 1.0), k


def test_chord_noalloc_rejects_oversized_walker_count(torch):
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = dummy.data_ptr()
    rc = mhar.mhar_chord_noalloc(ptr, ptr, 1, 1, ptr, ptr, 65537, ptr, ptr, None)
    assert rc == mhar.E_ARG
    assert "65536" in mhar.mhar_last_error(None)
