"""Statistics used by the tests: Friedman-Rafsky two-sample MST test, exact
areas of convex polygons clipped to grid cells, and a chi-square helper.

None of this is the sampler's arithmetic; it is how the tests judge samples.
"""
from __future__ import annotations

import numpy as np
from scipy import stats
from scipy.sparse.csgraph import minimum_spanning_tree
from scipy.spatial.distance import pdist, squareform


def friedman_rafsky(S: np.ndarray, U: np.ndarray) -> float:
    """Friedman & Rafsky (1979) two-sample test, the independence check of
    Section 6.4: build the Euclidean MST of the pooled sample, count edges R
    joining points from different samples, and standardise R by its
    permutation mean and variance.  Returns the z-value W; the paper accepts
    "same distribution" when W >= -1.64."""
    m, n = len(S), len(U)
    N = m + n
    P = np.vstack([S, U])
    lab = np.concatenate([np.zeros(m, int), np.ones(n, int)])
    D = squareform(pdist(P))
    # Ties at zero distance would be dropped by the sparse MST; nudge them.
    D[D == 0] = 1e-300
    np.fill_diagonal(D, 0.0)
    T = minimum_spanning_tree(D).tocoo()
    R = int(np.sum(lab[T.row] != lab[T.col]))
    deg = np.bincount(np.concatenate([T.row, T.col]), minlength=N)
    C = int(np.sum(deg * (deg - 1) // 2))
    ER = 2.0 * m * n / N + 1.0
    VR = (2.0 * m * n / (N * (N - 1))) * (
        (2.0 * m * n - N) / N
        + (C - N + 2.0) / ((N - 2.0) * (N - 3.0)) * (N * (N - 1.0) - 4.0 * m * n + 2.0))
    return (R - ER) / np.sqrt(VR)


def _clip(poly: np.ndarray, axis: int, val: float, keep_le: bool) -> np.ndarray:
    """Sutherland-Hodgman clip of a convex polygon (k x 2) by x_axis <= val
    (keep_le) or x_axis >= val."""
    if len(poly) == 0:
        return poly
    out = []
    k = len(poly)
    for i in range(k):
        P, Q = poly[i], poly[(i + 1) % k]
        inP = P[axis] <= val if keep_le else P[axis] >= val
        inQ = Q[axis] <= val if keep_le else Q[axis] >= val
        if inP:
            out.append(P)
        if inP != inQ:
            t = (val - P[axis]) / (Q[axis] - P[axis])
            out.append(P + t * (Q - P))
    return np.array(out) if out else np.zeros((0, 2))


def polygon_area(poly: np.ndarray) -> float:
    if len(poly) < 3:
        return 0.0
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def cell_areas(vertices: np.ndarray, xe: np.ndarray, ye: np.ndarray) -> np.ndarray:
    """Exact area of (convex polygon) intersect (grid cell) for the grid with
    edges xe, ye; shape (len(xe)-1, len(ye)-1)."""
    out = np.zeros((len(xe) - 1, len(ye) - 1))
    for i in range(len(xe) - 1):
        for j in range(len(ye) - 1):
            p = _clip(vertices, 0, xe[i], False)
            p = _clip(p, 0, xe[i + 1], True)
            p = _clip(p, 1, ye[j], False)
            p = _clip(p, 1, ye[j + 1], True)
            out[i, j] = polygon_area(p)
    return out


def halfspaces_of_polygon(vertices: np.ndarray):
    """A, b with A x <= b describing a convex polygon given counter-clockwise."""
    k = len(vertices)
    A, b = [], []
    for i in range(k):
        P, Q = vertices[i], vertices[(i + 1) % k]
        e = Q - P
        nrm = np.array([e[1], -e[0]])  # outward normal for CCW order
        A.append(nrm)
        b.append(nrm @ P)
    return np.array(A), np.array(b)


def chi2_pvalue(counts: np.ndarray, probs: np.ndarray) -> float:
    counts = counts.ravel().astype(float)
    probs = probs.ravel() / probs.sum()
    keep = probs > 0
    exp = probs[keep] * counts.sum()
    chi2 = np.sum((counts[keep] - exp) ** 2 / exp)
    return float(stats.chi2.sf(chi2, df=int(keep.sum()) - 1))
