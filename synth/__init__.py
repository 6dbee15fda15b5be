"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module builds only *inputs* of the method: knot vectors, control nets,
the random amplitudes of the deformation field and right-hand-side vectors.
It performs none of the method's arithmetic (no basis evaluation, no
quadrature, no assembly, no eigen-solve, no preconditioner, no Krylov step),
so both sides can consume the same arrays without sharing computation.

Workload recipes (Section 6 of the paper uses the unit square/cube and
b = randn; the deformed cube stands in for the paper's curved domains, whose
control nets are not given):

* identity map: control points at the Greville abscissae of the
  discretisation's own knots (splines of degree >= 1 reproduce linear
  functions there, so F is the identity);
* deformed cube: the same net displaced by
  phi(g) * (1, 1, 1), phi(x) = sum_k a_k sin(k pi x) sin(k pi y) sin(k pi z),
  a_k ~ U(-amp, amp), k = 1..3; phi vanishes on every face, so the physical
  domain stays the unit cube and manufactured solutions remain exact;
* right-hand sides: i.i.d. N(0, 1) vectors (as the paper's cube test).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20160222


def rng(seed: int) -> np.random.Generator:
    """Counter-free seeded generator (PCG64) used for every random input."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(seed)))


def uniform_open_knots(nel: int, p: int) -> np.ndarray:
    """Open knot vector on [0,1] with nel uniform elements, end knots repeated
    p+1 times, interior knots simple (C^{p-1} splines, Section 2.1)."""
    if nel < 1 or p < 1:
        raise ValueError("need nel >= 1 and p >= 1")
    inner = np.linspace(0.0, 1.0, nel + 1)
    return np.concatenate([np.zeros(p), inner, np.ones(p)])


def nel_for_dofs(n: int, p: int) -> int:
    """Elements per direction giving n dofs after Dirichlet removal
    (m = nel + p basis functions, n = m - 2)."""
    nel = n - p + 2
    if nel < 1:
        raise ValueError(f"n={n} too small for p={p}")
    return nel


def greville(knots: np.ndarray, p: int) -> np.ndarray:
    """Greville abscissae: the mean of the p interior knots of each local knot
    vector. Used only to place control points of the input geometry."""
    m = len(knots) - p - 1
    return np.array([knots[i + 1:i + p + 1].mean() for i in range(m)])


def control_net(knots_per_dir, p: int, amplitudes=None) -> np.ndarray:
    """Control net C[c][i_d]...[i_1] (coordinate c, direction 1 fastest) of a
    degree-p spline map on the given knots.

    amplitudes=None gives the identity map. Otherwise `amplitudes` (length 3,
    3D only) are the a_k of the displacement phi(g)(1,1,1) applied at the
    Greville points g.
    """
    g = [greville(np.asarray(k), p) for k in knots_per_dir]
    d = len(g)
    grids = np.meshgrid(*g[::-1], indexing="ij")  # slowest direction first
    coords = [grids[d - 1 - c] for c in range(d)]  # coords[c] varies along dir c
    net = np.stack(coords).astype(np.float64)
    if amplitudes is not None:
        if d != 3:
            raise ValueError("deformation field is defined for 3D")
        x, y, z = coords
        phi = np.zeros_like(x)
        for k, a in enumerate(amplitudes, start=1):
            phi += a * np.sin(k * np.pi * x) * np.sin(k * np.pi * y) * np.sin(k * np.pi * z)
        net = net + phi[None]
    return np.ascontiguousarray(net)


def deformation_amplitudes(seed: int, amp: float = 0.05, kmax: int = 3) -> np.ndarray:
    """a_k ~ U(-amp, amp), k = 1..kmax."""
    return rng(seed).uniform(-amp, amp, size=kmax)


def random_rhs(shape, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) FP64 right-hand side, direction 1 fastest (C order with
    the slowest direction first)."""
    return rng(seed + 7919).standard_normal(size=shape)


def random_vector(shape, seed: int) -> np.ndarray:
    """Generic seeded N(0,1) test vector."""
    return rng(seed + 104729).standard_normal(size=shape)


class Problem:
    """A complete synthetic single-patch problem description (inputs only)."""

    def __init__(self, dim: int, n, p: int, amplitudes=None, kappa: float = 1.0):
        if isinstance(n, int):
            n = (n,) * dim
        self.dim = dim
        self.n = tuple(int(v) for v in n)          # dofs per direction (dir 1 first)
        self.p = int(p)
        self.nel = tuple(nel_for_dofs(v, p) for v in self.n)
        self.knots = [uniform_open_knots(e, p) for e in self.nel]
        self.amplitudes = None if amplitudes is None else np.asarray(amplitudes, float)
        self.ctrl = control_net(self.knots, p, self.amplitudes)
        self.kappa = float(kappa)

    @property
    def shape(self):
        """Tensor shape of a dof vector, slowest direction first."""
        return tuple(reversed(self.n))

    @property
    def N(self):
        return int(np.prod(self.n))


def unit_square(n: int = 64, p: int = 3) -> Problem:
    """2D Poisson on the unit square, identity map, kappa = 1."""
    return Problem(2, n, p)


def deformed_cube(n: int = 128, p: int = 3, seed: int = 0, amp: float = 0.05) -> Problem:
    """3D Poisson on the deformed unit cube, kappa = 1."""
    return Problem(3, n, p, deformation_amplitudes(seed, amp))
