"""Seeded synthetic polytopes for Matrix Hit-and-Run.

This module holds input generators only -- none of the sampler's arithmetic.
Both the CUDA path's tests/benchmark and the CPU oracle draw their inputs from
here, so the two sides see identical arrays.

Bodies (all bounded, with a strictly interior start):
  * ``cube``           -- [-1,1]^n as A = [I; -I], b = 1 (the paper's Section 6
                          n-hypercube), x0 = 0;
  * ``simplex``        -- {x >= 0, sum x = 1} (Section 6 n-simplex), x0 = 1/n;
  * ``random_polytope``-- m unit-norm Gaussian rows, b = 1 (contains the unit
                          ball), x0 = 0; boundedness is checked by an LP;
  * ``simplex_cuts``   -- the simplex plus unit-norm Gaussian cuts a.x <= 1;
  * ``ill_conditioned``-- a random polytope mapped by diag(s), log s uniform;
  * ``batch``          -- many random polytopes of uneven size.
"""
from __future__ import annotations

import dataclasses

import math

import numpy as np


@dataclasses.dataclass
class Polytope:
    """{x : A x <= b, AE x = bE} with a strictly interior start x0."""

    A: np.ndarray          # m x n, row-major float64
    b: np.ndarray          # m
    x0: np.ndarray         # n
    AE: np.ndarray | None = None  # mE x n or None
    bE: np.ndarray | None = None  # mE or None
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.A.shape[0])

    @property
    def n(self) -> int:
        return int(self.A.shape[1])

    @property
    def mE(self) -> int:
        return 0 if self.AE is None else int(self.AE.shape[0])


def _unit_rows(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    G = rng.standard_normal((m, n))
    G /= np.linalg.norm(G, axis=1, keepdims=True)
    return G


def is_bounded(A: np.ndarray) -> bool:
    """{x : A x <= b} (b > 0) is bounded iff the rows positively span R^n, i.e.
    iff some y >= 1 has A^T y = 0 (Gordan's alternative).  One LP."""
    from scipy.optimize import linprog

    m, n = A.shape
    res = linprog(c=np.zeros(m), A_eq=A.T, b_eq=np.zeros(n), bounds=[(1.0, None)] * m,
                  method="highs")
    return bool(res.status == 0)


def cube(n: int) -> Polytope:
    A = np.vstack([np.eye(n), -np.eye(n)])
    return Polytope(A=A, b=np.ones(2 * n), x0=np.zeros(n), name=f"cube{n}")


def simplex(n: int) -> Polytope:
    A = -np.eye(n)
    return Polytope(A=A, b=np.zeros(n), x0=np.full(n, 1.0 / n), AE=np.ones((1, n)),
                    bE=np.ones(1), name=f"simplex{n}")


def unbounded_probability(m: int, n: int) -> float:
    """Wendel (1962): m iid symmetric random vectors in R^n lie in a common
    half-space with probability 2^-(m-1) sum_{k<n} C(m-1, k); for unit
    Gaussian rows that is the probability that {A x <= 1} is unbounded."""
    if m <= n:
        return 1.0
    return float(sum(math.comb(m - 1, k) for k in range(n)) / 2 ** (m - 1))


def random_polytope(n: int, m: int, seed: int, check_bounded="yes") -> Polytope:
    """m rows iid N(0, I_n) normalised to unit length, b = 1, x0 = 0.  Redraws
    with the next seed until the body is bounded.  check_bounded: "yes" (one LP
    per draw), "no", or "auto" (the LP only when Wendel's probability of an
    unbounded draw exceeds 1e-12, i.e. for m near 2n)."""
    if check_bounded is True:
        check_bounded = "yes"
    elif check_bounded is False:
        check_bounded = "no"
    s = seed
    while True:
        rng = np.random.default_rng(s)
        A = _unit_rows(rng, m, n)
        need = check_bounded == "yes" or (check_bounded == "auto" and
                                          unbounded_probability(m, n) > 1e-12)
        if not need or is_bounded(A):
            return Polytope(A=A, b=np.ones(m), x0=np.zeros(n), name=f"rand{n}x{m}s{s}")
        s += 1_000_003


def simplex_cuts(n: int, cuts: int, seed: int) -> Polytope:
    """{x >= 0, sum x = 1} plus `cuts` rows a.x <= 1 with a unit-norm Gaussian.
    x0 = 1/n is interior: |a.x0| <= |x0| = n^-1/2 < 1."""
    rng = np.random.default_rng(seed)
    C = _unit_rows(rng, cuts, n)
    A = np.vstack([-np.eye(n), C])
    b = np.concatenate([np.zeros(n), np.ones(cuts)])
    return Polytope(A=A, b=b, x0=np.full(n, 1.0 / n), AE=np.ones((1, n)), bE=np.ones(1),
                    name=f"simplex{n}+{cuts}cuts")


def ill_conditioned(n: int, m: int, seed: int, smin: float = 1e-3) -> Polytope:
    """Random polytope y = diag(s) x with log s ~ U[ln smin, 0]: A' = A diag(1/s),
    b = 1, x0 = 0 (rows are not re-normalised)."""
    rng = np.random.default_rng(seed)
    A = _unit_rows(rng, m, n)
    s = np.exp(rng.uniform(np.log(smin), 0.0, size=n))
    return Polytope(A=A / s[None, :], b=np.ones(m), x0=np.zeros(n), name=f"illcond{n}x{m}")


def batch(count: int, seed: int, nmin: int = 20, nmax: int = 400,
          mfac: tuple[int, int] = (2, 20)) -> list[Polytope]:
    """`count` random polytopes, n ~ U{nmin..nmax}, m ~ U{mfac0 n .. mfac1 n}."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        m = int(rng.integers(mfac[0] * n, mfac[1] * n + 1))
        out.append(random_polytope(n, m, seed=seed * 100_003 + p, check_bounded="auto"))
    return out


def uniform_cube_points(n: int, count: int, seed: int) -> np.ndarray:
    """Exact uniform draws on [-1,1]^n (test reference samples)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(count, n))


def uniform_simplex_points(n: int, count: int, seed: int) -> np.ndarray:
    """Exact uniform draws on the simplex: normalised iid Exp(1) (Dirichlet(1))."""
    E = np.random.default_rng(seed).exponential(size=(count, n))
    return E / E.sum(axis=1, keepdims=True)


# The five workloads the benchmark and the parity tests are sized from.
WORKLOADS = {
    "cube10": dict(body=lambda: cube(10), z=100, steps=1000, precision="fp64"),
    "rand100x2000": dict(body=lambda: random_polytope(100, 2000, seed=2, check_bounded=False),
                         z=4096, steps=2000, precision="mixed"),
    "simplex1000+4000": dict(body=lambda: simplex_cuts(1000, 4000, seed=3), z=8192, steps=1000,
                             precision="mixed"),
    "illcond500x10000": dict(body=lambda: ill_conditioned(500, 10000, seed=5), z=16384,
                             steps=5000, precision="mixed"),
}
