"""Chebyshev's center (Section 4.2, Model CCHC) against closed forms."""
import math

import numpy as np
import pytest

import oracle
from paper_2104_07097_gb300 import start
from paper_2104_07097_gb300 import workloads as wl


def test_cube_center_is_origin_radius_one():
    p = wl.cube(6)
    x, r = start.chebyshev_center(p.A, p.b)
    np.testing.assert_allclose(x, 0.0, atol=1e-9)
    assert r == pytest.approx(1.0, abs=1e-9)


def test_right_triangle_incenter():
    # Triangle (0,0), (1,0), (0,1): inradius (a + b - c) / 2 = 1 - 1/sqrt(2), center (r, r).
    A = np.array([[-1.0, 0.0], [0.0, -1.0], [1.0, 1.0]])
    b = np.array([0.0, 0.0, 1.0])
    x, r = start.chebyshev_center(A, b)
    want = 1.0 - 1.0 / math.sqrt(2.0)
    assert r == pytest.approx(want, abs=1e-9)
    np.testing.assert_allclose(x, [want, want], atol=1e-9)


def test_simplex_center_with_equality():
    # x >= 0, sum x = 1 with the printed row norms ||e_i|| = 1: x = 1/n, r = 1/n.
    n = 9
    p = wl.simplex(n)
    x, r = start.chebyshev_center(p.A, p.b, p.AE, p.bE)
    np.testing.assert_allclose(x, 1.0 / n, atol=1e-9)
    assert r == pytest.approx(1.0 / n, abs=1e-9)


def test_random_polytope_center_is_a_valid_start():
    p = wl.random_polytope(12, 80, seed=3)
    x, r = start.chebyshev_center(p.A, p.b)
    assert r >= 1.0 - 1e-9            # the unit ball at 0 fits (unit rows, b = 1)
    norms = np.linalg.norm(p.A, axis=1)
    assert np.all(p.A @ x + r * norms <= p.b + 1e-9)
    res = oracle.mhar_run(p.A, p.b, np.tile(x, (16, 1)), 20, thin=20, seed=1)
    assert np.all(res["X"] @ p.A.T <= p.b + 1e-12)


def test_no_interior_and_infeasible_are_rejected():
    with pytest.raises(ValueError):
        start.chebyshev_center(np.array([[1.0], [-1.0]]), np.array([0.0, 0.0]))   # {0}
    with pytest.raises(ValueError):
        start.chebyshev_center(np.array([[1.0], [-1.0]]), np.array([-1.0, -1.0]))  # empty
