"""The allocation-free chord entry point, mhar_chord_noalloc.

It serves callers that must not allocate device memory -- a process living
inside a fixed, pre-reserved device-memory budget, or a latency-critical loop
that cannot afford the synchronisation cudaMalloc / cudaFree may bring -- by
keeping its working memory in a fixed array built into the library.  This
test calls it through the C ABI twice in a row (the second call with other
inputs, so stale contents of the shared array would show) and checks both
results against the chords the regular FP64 path reports for the same points
and directions (mhar_get_chord), at the FP64 parity tolerance 1e-10.

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


def _existing_chords(p, X, step, seed):
    """lambda_min, lambda_max of the regular FP64 path at points X, iteration `step`."""
    with mhar.Sampler(p.A, p.b, p.x0, X.shape[0], precision="fp64", seed=seed) as s:
        s.set_state(X, step)
        s.run(1)
        lo, hi, _ = s.chord()
    return lo, hi


def test_chord_noalloc_matches_existing_path_twice():
    torch = pytest.importorskip("torch")
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()
    p = wl.random_polytope(37, 300, seed=11)
    z, seed = 200, 4
    # Points: the oracle's own chain after a few iterations (distinct per walker).
    X = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (z, 1)), steps=5, seed=seed)["X"]
    dev = torch.device("cuda")
    A_d = torch.from_numpy(np.ascontiguousarray(p.A)).to(dev)
    b_d = torch.from_numpy(np.ascontiguousarray(p.b)).to(dev)
    stream = torch.cuda.current_stream()
    for call, step in enumerate((5, 6)):
        # Directions of iteration `step` (oracle's Philox normals, no equalities).
        D = np.array([oracle.direction_normals(seed, step, k, p.n) for k in range(z)])
        X_d = torch.from_numpy(X).to(dev)
        D_d = torch.from_numpy(D).to(dev)
        lo_d = torch.full((z,), np.nan, dtype=torch.float64, device=dev)
        hi_d = torch.full((z,), np.nan, dtype=torch.float64, device=dev)
        rc = mhar.mhar_chord_noalloc(A_d.data_ptr(), b_d.data_ptr(), p.m, p.n, X_d.data_ptr(),
                                     D_d.data_ptr(), z, lo_d.data_ptr(), hi_d.data_ptr(), stream)
        assert rc == mhar.OK, (call, mhar.mhar_last_error(None))
        torch.cuda.synchronize()
        lo_ref, hi_ref = _existing_chords(p, X, step, seed)
        lo, hi = lo_d.cpu().numpy(), hi_d.cpu().numpy()
        span = np.maximum(1.0, hi_ref - lo_ref)
        assert np.all(np.abs(lo - lo_ref) <= TOL * span), (call, np.abs(lo - lo_ref).max())
        assert np.all(np.abs(hi - hi_ref) <= TOL * span), (call, np.abs(hi - hi_ref).max())
        # Next call starts from other points.
        X = oracle.mhar_run(p.A, p.b, X, steps=1, seed=seed, step0=step)["X"]


def test_chord_noalloc_rejects_oversized_walker_count():
    torch = pytest.importorskip("torch")
    from paper_2104_07097_gb300 import build
    build.build()
    mhar.load()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = dummy.data_ptr()
    rc = mhar.mhar_chord_noalloc(ptr, ptr, 1, 1, ptr, ptr, 65537, ptr, ptr, None)
    assert rc == mhar.E_ARG
    assert "65536" in mhar.mhar_last_error(None)
