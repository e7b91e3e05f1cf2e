"""Starting point: Chebyshev's center (Section 4.2, Model CCHC).

MHAR needs a point in the relative interior of the body.  The paper suggests
the center of the largest inscribed ball, the linear program

    max r  subject to  A_E x = b_E,  a_i^T x + r ||a_i||_2 <= b_i  (all i),

solved once on the host (the sampling path never calls it).  The linear
program is handed to a general LP solver (scipy's HiGHS).
"""
from __future__ import annotations

import numpy as np


def chebyshev_center(A, b, AE=None, bE=None):
    """(x, r): Chebyshev's center of {A x <= b, AE x = bE} and the radius r of
    the inscribed ball (Model CCHC: row norms ||a_i||_2 as printed).  Raises
    ValueError when the program is infeasible or unbounded, or r <= 0 (the
    body has no interior point for Algorithm 2 to start from)."""
    from scipy.optimize import linprog

    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    norms = np.linalg.norm(A, axis=1)
    c = np.zeros(n + 1)
    c[-1] = -1.0                                   # maximise r
    A_ub = np.hstack([A, norms[:, None]])
    A_eq = b_eq = None
    if AE is not None and np.size(AE) > 0:
        AE = np.atleast_2d(np.asarray(AE, dtype=np.float64))
        A_eq = np.hstack([AE, np.zeros((AE.shape[0], 1))])
        b_eq = np.atleast_1d(np.asarray(bE, dtype=np.float64))
    bounds = [(None, None)] * n + [(0.0, None)]
    res = linprog(c, A_ub=A_ub, b_ub=b, A_eq=A_eq, b_eq=b_eq, bounds=bounds, method="highs")
    if res.status != 0:
        raise ValueError(f"Chebyshev center: linear program failed ({res.message})")
    x, r = res.x[:n], float(res.x[n])
    if not r > 0.0:
        raise ValueError("Chebyshev center: the body has no interior (r = 0)")
    return x, r
