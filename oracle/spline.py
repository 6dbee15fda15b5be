"""Section 2.1: B-splines on open knot vectors (oracle; test infrastructure).

Cox-de Boor recursion, Eqs. (cox-deboor-1) and (cox-deboor-2), with the
convention 0/0 = 0; derivatives by the textbook degree-reduction formula.
Reading of the half-open indicator: a point equal to the last knot is placed
in the last non-empty span, so the basis does not vanish at zeta = 1.
"""
from __future__ import annotations

import numpy as np


def _safe_div(num, den):
    """0/0 = 0 (and x/0 = 0, which only occurs with a zero numerator factor)."""
    out = np.zeros(np.broadcast(num, den).shape)
    nz = den != 0
    np.divide(num, den, out=out, where=nz)
    return out


def basis_table(knots, p, z, deriv=False):
    """Values (or first derivatives) of all m = len(knots)-p-1 degree-p
    B-splines at the points z. Returns an array [len(z), m]."""
    xi = np.asarray(knots, dtype=np.float64)
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    nk = len(xi)
    last_span = max(j for j in range(nk - 1) if xi[j] < xi[j + 1])
    # degree 0: indicator of [xi_j, xi_{j+1})
    N = np.zeros((len(z), nk - 1))
    for j in range(nk - 1):
        if xi[j] < xi[j + 1]:
            N[:, j] = (xi[j] <= z) & (z < xi[j + 1])
    N[z == xi[-1], last_span] = 1.0
    Nprev = N
    for q in range(1, p + 1):
        Nq = np.zeros((len(z), nk - 1 - q))
        for j in range(nk - 1 - q):
            left = _safe_div(z - xi[j], xi[j + q] - xi[j]) * Nprev[:, j]
            right = _safe_div(xi[j + q + 1] - z, xi[j + q + 1] - xi[j + 1]) * Nprev[:, j + 1]
            Nq[:, j] = left + right
        if q == p and deriv:
            # derivative of degree-p functions from the degree p-1 ones
            D = np.zeros_like(Nq)
            for j in range(nk - 1 - q):
                D[:, j] = (_safe_div(q, xi[j + q] - xi[j]) * Nprev[:, j]
                           - _safe_div(q, xi[j + q + 1] - xi[j + 1]) * Nprev[:, j + 1])
            return D
        Nprev = Nq
    if p == 0 and deriv:
        return np.zeros_like(Nprev)
    return Nprev


def elements(knots):
    """Non-empty knot spans [xi_s, xi_{s+1}) as a list of span indices s."""
    xi = np.asarray(knots)
    return [s for s in range(len(xi) - 1) if xi[s] < xi[s + 1]]


def gauss_points(knots, nq):
    """nq-point Gauss-Legendre rule on every element (reading: the paper does
    not state its rule; (p+1) points per direction is exact for the pencils).
    Returns (z[E, nq], w[E, nq], spans[E])."""
    xg, wg = np.polynomial.legendre.leggauss(nq)
    xi = np.asarray(knots)
    spans = elements(knots)
    z = np.empty((len(spans), nq))
    w = np.empty((len(spans), nq))
    for e, s in enumerate(spans):
        a, b = xi[s], xi[s + 1]
        z[e] = 0.5 * (a + b) + 0.5 * (b - a) * xg
        w[e] = 0.5 * (b - a) * wg
    return z, w, np.array(spans)
