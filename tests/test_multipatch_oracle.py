"""Pins of the multi-patch oracle (Section 6, the L-shaped domain of
Section 7.3): the glued global matrix against facts of the spline space, the
subdomain matrices against a single-patch assembly of each two-patch
subdomain, the spectrum of the exact additive Schwarz operator, and the CG
iteration counts of Table "L". CPU only."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import multipatch as mpm, pcg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table_L():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_L.txt")) if l.strip() and l[0] != "#"]
    return {(int(h), int(p)): (int(e), int(i)) for h, p, e, i in rows}


@pytest.mark.parametrize("nel,p", [(4, 1), (4, 2), (6, 3)])
def test_glued_matrix_annihilates_constants_and_is_spd(nel, p):
    """Before the Dirichlet conditions, the glued C^0 space contains the
    constants, whose gradient is zero: every row of the full matrix sums to
    0. With them, A is symmetric positive definite."""
    L = mpm.LShape(synth.uniform_open_knots(nel, p), p)
    Kp = np.kron(L.M1d, L.K1d) + np.kron(L.K1d, L.M1d)
    Af = np.zeros((L.n_full, L.n_full))
    for q in (1, 2, 3):
        g = L.local_to_global[q].ravel()
        Af[np.ix_(g, g)] += Kp
    assert np.abs(Af.sum(axis=1)).max() <= 1e-12 * np.abs(Af).max()
    A = L.A.toarray()
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    # degrees of freedom: 3 patches of m^2 functions, two shared edges of m,
    # minus the boundary of the L
    m = L.m
    assert L.n_full == 3 * m * m - 2 * m
    assert L.N == L.n_full - (8 * (m - 1))


@pytest.mark.parametrize("nel,p", [(3, 1), (4, 2), (3, 3)])
def test_subdomain_matrix_equals_single_patch_bruteforce(nel, p):
    """A_i = R_i A R_i^T equals the stiffness matrix of Theta_i as one patch
    (merged knot vector, C^0 at 1/2, stretched map), assembled by brute-force
    quadrature (Section 6: each subdomain is a single-patch domain)."""
    L = mpm.LShape(synth.uniform_open_knots(nel, p), p)
    for i in range(2):
        R = L.restriction(i)
        Ai = (R @ L.A @ R.T).toarray()
        disc = L.merged_discretization(i)
        Ab = disc.dense_A_bruteforce()
        assert Ai.shape == Ab.shape
        assert np.abs(Ai - Ab).max() <= 1e-13 * np.abs(Ab).max()


def test_merged_knot_vector():
    kn = synth.uniform_open_knots(4, 3)
    km = mpm.merged_knots(kn, 3)
    assert np.allclose(km, [0, 0, 0, 0, 0.125, 0.25, 0.375, 0.5, 0.5, 0.5, 0.625, 0.75, 0.875, 1, 1, 1, 1])


def test_exact_schwarz_spectrum():
    """P_EAS A = P_1 + P_2 with A-orthogonal projections P_i: eigenvalues in
    (0, 2], and 2 exactly on V_1 n V_2 (the functions of the corner patch
    that vanish on both of its interfaces: (m - 2)^2 of them)."""
    L = mpm.LShape(synth.uniform_open_knots(6, 2), 2)
    E = mpm.AdditiveSchwarz(L, exact=True)
    PE = np.column_stack([E.apply(e) for e in np.eye(L.N)])
    ev = np.sort(sla.eigvals(PE @ L.A.toarray()).real)
    assert ev[0] > 0 and ev[-1] <= 2 + 1e-10
    assert np.sum(np.abs(ev - 2) < 1e-8) == (L.m - 2) ** 2


def test_inexact_schwarz_iterations_match_table_L():
    """CG with P_IAS (local inverses by fast diagonalization) needs a number
    of iterations independent of h and p, within 3 of Table "L" at
    h^-1 = 128."""
    tab = _table_L()
    counts = {}
    for nel in (32, 64, 128):
        for p in (1, 2, 3, 4, 5):
            if nel < 128 and p > 3:
                continue
            L = mpm.LShape(synth.uniform_open_knots(nel, p), p)
            b = synth.random_rhs(L.N, 3)
            res = pcg.pcg(lambda v: L.A @ v, b, mpm.AdditiveSchwarz(L, exact=False).apply,
                          tol=1e-8, max_iter=500)
            assert res.converged
            counts[(nel, p)] = res.iters
            if nel == 128:
                assert abs(res.iters - tab[(128, p)][1]) <= 3, (p, res.iters)
    assert max(counts.values()) - min(counts.values()) <= 2


def test_exact_schwarz_converges_faster_than_inexact():
    L = mpm.LShape(synth.uniform_open_knots(32, 2), 2)
    b = synth.random_rhs(L.N, 3)
    re = pcg.pcg(lambda v: L.A @ v, b, mpm.AdditiveSchwarz(L, exact=True).apply, tol=1e-8)
    ri = pcg.pcg(lambda v: L.A @ v, b, mpm.AdditiveSchwarz(L, exact=False).apply, tol=1e-8)
    x = np.linalg.solve(L.A.toarray(), b)
    assert re.converged and ri.converged and re.iters < ri.iters
    assert np.linalg.norm(re.x - x) <= 1e-7 * np.linalg.norm(x)
