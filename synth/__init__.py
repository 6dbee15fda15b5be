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
    """A complete synthetic single-patch problem description (inputs only).

    By default the geometry map is a degree-p spline on the discretisation's
    own knots (isoparametric) and the coefficient is the constant kappa. A
    separate geometry net (geo_knots, geo_p, ctrl) and a spline coefficient
    field (kappa_knots, kappa_p, kappa_ctrl; K(x) = kappa * kappa_field I)
    can be attached."""

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
        self.geo_knots = None
        self.geo_p = None
        self.kappa_knots = None
        self.kappa_p = None
        self.kappa_ctrl = None

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


# ---- learned-scaling workload: coarse random geometry, random coefficient ----

def smooth5(a, axis):
    """Separable binomial [1, 4, 6, 4, 1] / 16 smoothing along one axis with
    zero padding (applied to displacements whose boundary values are zero)."""
    w = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0
    a = np.moveaxis(a, axis, -1)
    pad = np.zeros(a.shape[:-1] + (a.shape[-1] + 4,))
    pad[..., 2:-2] = a
    out = sum(w[j] * pad[..., j:j + a.shape[-1]] for j in range(5))
    return np.moveaxis(out, -1, axis)


def coarse_random_net(seed: int, gp: int = 3, gn: int = 8, sigma: float = 0.15):
    """Degree-gp geometry net with gn control points per direction on the unit
    cube: interior points displaced by N(0, (sigma * spacing)^2) per
    coordinate, displacements smoothed by the 5-point binomial kernel along
    each axis, boundary points fixed. Returns (knots, gp, ctrl[3][gn][gn][gn])."""
    kn = [uniform_open_knots(gn - gp, gp) for _ in range(3)]
    base = control_net(kn, gp)
    g = rng(seed + 31337)
    disp = g.normal(0.0, sigma / (gn - 1), size=base.shape)
    interior = np.zeros(base.shape[1:], bool)
    interior[1:-1, 1:-1, 1:-1] = True
    disp[:, ~interior] = 0.0
    for ax in (1, 2, 3):
        disp = smooth5(disp, ax)
    disp[:, ~interior] = 0.0
    return kn, gp, np.ascontiguousarray(base + disp)


def grf_kappa(seed: int, nel: int = 16, kp: int = 3, contrast: float = 100.0,
              lengthscale: float = 0.2, features: int = 512):
    """Coefficient kappa = exp(g) for a Gaussian random field g (random Fourier
    features: `features` cosines, frequencies N(0, lengthscale^-2 I), phases
    U(0, 2 pi)) sampled at the Greville points of a degree-kp spline on nel
    uniform elements per direction, affinely rescaled so that the control
    values span exactly [1, contrast]. Returns (knots, kp, ctrl[m][m][m])."""
    kn = [uniform_open_knots(nel, kp) for _ in range(3)]
    gr = [greville(k, kp) for k in kn]
    z, y, x = np.meshgrid(gr[2], gr[1], gr[0], indexing="ij")
    g = rng(seed + 4242)
    om = g.normal(0.0, 1.0 / lengthscale, size=(features, 3))
    ph = g.uniform(0.0, 2 * np.pi, size=features)
    pts = np.stack([x, y, z], axis=-1)
    field = np.sqrt(2.0 / features) * np.cos(pts @ om.T + ph).sum(axis=-1)
    field = (field - field.min()) / (field.max() - field.min()) * np.log(contrast)
    return kn, kp, np.ascontiguousarray(np.exp(field))


def learned_workload_problem(seed: int, n: int = 96, p: int = 3) -> Problem:
    """3D patch of the learned-scaling workload: coarse random geometry net
    and a random coefficient of contrast 100."""
    pr = Problem(3, n, p)
    pr.geo_knots, pr.geo_p, pr.ctrl = coarse_random_net(seed)
    pr.kappa_knots, pr.kappa_p, pr.kappa_ctrl = grf_kappa(seed)
    return pr


def mlp_init(seed: int, sizes=(6, 64, 64, 2)) -> np.ndarray:
    """Initial parameters of the scaling network (flat, float32): weights
    Xavier-uniform per layer (layout W1, b1, W2, b2, W3, b3; W as [out][in]),
    biases zero."""
    g = rng(seed + 777)
    parts = []
    for i in range(len(sizes) - 1):
        fan_in, fan_out = sizes[i], sizes[i + 1]
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(g.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)
