"""ADI solvers of the Kronecker-sum system P s = r (oracle; test
infrastructure only).

Two variables (Section 4.2): the Peaceman-Rachford iteration of Eq. (ADI) in
the mass-scaled form of Algorithm 2, its error operator T_J of Eqs. (ADIerr)
and (Tj), the iteration count of Eq. (ADIits), and its use as the
preconditioner P_J of Theorem 1. Three variables (Section 5.2): the Douglas
iteration of Eq. (ADI3D) in the form of Eq. (ADI3D2) / Algorithm 4, with the
parameters of the greedy rule of Eqs. (greedy1)-(greedy2) and the stopping
rule rho_J <= eps.

Readings where the paper is silent, garbled or cites instead of stating:
 - Eq. (ADI) prints omega_k in the first half step; the iteration index j is
   meant (Algorithm 2 has omega_j there).
 - The optimal two-variable parameters are cited, not printed. With equal
   spectral intervals [a, b] = [c, d] (the case Eq. (ADIits) assumes; unequal
   intervals are replaced here by their hull) the bound of Eq. (Tjnorm) with
   gamma_j = omega_j = w_j is the square of the one-variable minimax
   max_{x in [a, b]} prod_j |(x - w_j) / (x + w_j)|, whose classical
   elliptic-function solution (Wachspress; Zolotarev's problem) is
   w_j = b dn((2j - 1) K / (2J), k), k^2 = 1 - (a / b)^2, K = K(k). dn and K
   are evaluated by the arithmetic-geometric-mean method (Abramowitz and
   Stegun 16.4 and 17.6), started from the complementary modulus a / b itself
   so that nothing cancels when a / b is tiny; for (2j - 1) > J the identity
   dn(K - u) = k' / dn(u) is used (w_j = a / dn(K - u_j)). Near u = K / 2 the
   last arcsine of the method has an argument within ~k' of 1, so w_j carries
   a relative rounding error of order 1e-16 b / a (2e-8 at b / a = 7e8); the
   minimax value depends on the parameters only to second order at the
   optimum, so that error does not show in the ADI bound.
 - [a, b] (and [c, d]) are the exact extreme generalized eigenvalues of the
   pencils; the paper estimated them by ten power iterations.
 - Algorithm 4 sets v_0 = 0, but its first iteration reads v_1, which is
   (I (x) I (x) M3^{-1} K3) s_0 = 0: the vector v is zero before the first
   iteration.
 - rho_J, and the argmax of Eq. (greedy1), are taken over the triples of
   computed eigenvalues of M_k^{-1} K_k (Algorithm 4 computes all of them);
   over those triples rho_J equals ||T_J|| exactly, since T_J acts on the
   eigenvector triple (l1, l2, l3) by the product of the Douglas factors
   g(w; l) = 1 - 2 w^2 (l1 + l2 + l3) / ((w + l1)(w + l2)(w + l3)).
 - Eq. (greedy1) at k = 0 has an empty product, equal to 1 at every triple;
   the first parameter is taken at the triple of smallest eigenvalues
   (l1, l2, l3) = (a1, a2, a3).
 - Eq. (greedy2): over w > 0, w^2 / prod(w + l_i) has one stationary point,
   the positive root of w^3 - e2 w - 2 e3 (e2, e3 the elementary symmetric
   functions of l), where g is smallest. If g >= 0 there, that root is the
   minimiser of |g|; otherwise |g| = 0 at the two positive roots of
   w^3 - (l1 + l2 + l3) w^2 + e2 w + e3, and of those the one that gives the
   smaller rho_{k+1} is taken.
 - The paper calls the 3D T_J positive definite. Its eigenvalues are products
   of Douglas factors, which lie in (-1, 1) but can be negative when the three
   eigenvalues are spread apart; I - T_J, and with it P_J, is still symmetric
   positive definite, which is what CG needs.
"""
from __future__ import annotations

import math

import numpy as np

from .fd import generalized_eig, mode_product


# ------------------------------------------------------------ helpers ----

def mode_solve(X, A, k, d):
    """Solve along direction k (0-based; direction 1 is the last array axis):
    Y with A Y_(k) = X_(k), i.e. (I (x) .. A .. (x) I) y = x."""
    ax = d - 1 - k
    Xm = np.moveaxis(X, ax, 0)
    sh = Xm.shape
    Y = np.linalg.solve(A, Xm.reshape(sh[0], -1)).reshape(sh)
    return np.moveaxis(Y, 0, ax)


def pencil_spectrum(K, M):
    """All generalized eigenvalues of (K, M), ascending."""
    return generalized_eig(K, M)[0]


# ------------------------------------------ two-variable parameters ----

def adi_iterations_2d(a, b, eps):
    """Eq. (ADIits): J = ceil(ln(4 b / a) ln(4 / eps) / pi^2)."""
    return int(math.ceil(math.log(4.0 * b / a) * math.log(4.0 / eps) / math.pi ** 2))


def _agm_K(kp):
    """Complete elliptic integral K(k), k^2 = 1 - kp^2, by the AGM of 1 and kp
    (Abramowitz and Stegun 17.6: K = pi / (2 AGM(1, k')))."""
    a, b = 1.0, kp
    for _ in range(64):
        if abs(a - b) <= 1e-16 * a:
            break
        a, b = 0.5 * (a + b), math.sqrt(a * b)
    return math.pi / (2.0 * a)


def _agm_dn(u, kp):
    """Jacobi dn(u, k), k^2 = 1 - kp^2, by the AGM method (Abramowitz and
    Stegun 16.4): a_0 = 1, b_0 = k', c_0 = k, c_{n+1} = c_n^2 / (4 a_{n+1}),
    until c_N is negligible; phi_N = 2^N a_N u; then
    sin(2 phi_{n-1} - phi_n) = (c_n / a_n) sin(phi_n) down to phi_0, and
    dn = cos(phi_0) / cos(phi_1 - phi_0)."""
    k = math.sqrt((1.0 - kp) * (1.0 + kp))
    a, c = [1.0], [k]
    b = kp
    while c[-1] > 1e-16 * a[-1]:
        an = a[-1]
        a.append(0.5 * (an + b))
        c.append(c[-1] * c[-1] / (4.0 * a[-1]))     # (a_n - b_n)/2 without cancellation
        b = math.sqrt(an * b)
    n_steps = len(a) - 1
    phi = (2.0 ** n_steps) * a[-1] * u
    phis = [phi]
    for n in range(n_steps, 0, -1):
        phi = 0.5 * (phi + math.asin(c[n] / a[n] * math.sin(phi)))
        phis.append(phi)
    if n_steps == 0:                     # k = 0: dn = 1
        return 1.0
    return math.cos(phis[-1]) / math.cos(phis[-2] - phis[-1])


def wachspress_parameters(a, b, J):
    """Optimal parameters w_1 > ... > w_J of the one-variable minimax on
    [a, b] (see the module's readings): w_j = b dn((2j - 1) K / (2J), k)."""
    if not (0.0 < a <= b):
        raise ValueError("need 0 < a <= b")
    if a == b:
        return np.full(J, a)
    kp = a / b
    K = _agm_K(kp)
    w = np.empty(J)
    for j in range(1, J + 1):
        u = (2 * j - 1) * K / (2.0 * J)
        if 2 * j - 1 <= J:
            w[j - 1] = b * _agm_dn(u, kp)
        else:
            w[j - 1] = a / _agm_dn(K - u, kp)
    return w


def zolotarev_error(w, x):
    """prod_j (x - w_j) / (x + w_j) at the points x (signed)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    for wj in w:
        out = out * (x - wj) / (x + wj)
    return out


def t_norm_2d(omega, gamma, lam1, lam2):
    """||T_J|| of Eq. (Tj) on the computed spectra: the largest
    |prod_j (l - gamma_j)/(l + omega_j) * (m - omega_j)/(m + gamma_j)| over
    eigenvalue pairs (l of pencil 1, m of pencil 2)."""
    f1 = np.ones(len(lam1))
    f2 = np.ones(len(lam2))
    for om, ga in zip(omega, gamma):
        f1 = f1 * (lam1 - ga) / (lam1 + om)
        f2 = f2 * (lam2 - om) / (lam2 + ga)
    return float(np.abs(f1).max() * np.abs(f2).max())


# ---------------------------------------------- two-variable solver ----

class ADI2D:
    """Algorithm 2 on the pencils (K1, M1), (K2, M2): J iterations of Eq. (ADI)
    in the mass-scaled variables, from s~_0 = 0. Applying it to r is P_J^{-1} r
    (Theorem 1)."""

    def __init__(self, pencils, eps=None, J=None, omega=None, gamma=None):
        (K1, M1), (K2, M2) = pencils
        self.K1, self.M1, self.K2, self.M2 = K1, M1, K2, M2
        self.n = (K1.shape[0], K2.shape[0])
        self.lam1 = pencil_spectrum(K1, M1)
        self.lam2 = pencil_spectrum(K2, M2)
        a = min(self.lam1[0], self.lam2[0])
        b = max(self.lam1[-1], self.lam2[-1])
        self.a, self.b = a, b
        if omega is None:
            if J is None:
                J = adi_iterations_2d(a, b, eps)
            omega = wachspress_parameters(a, b, J)
        self.omega = np.asarray(omega, dtype=np.float64)
        self.gamma = self.omega.copy() if gamma is None else np.asarray(gamma, dtype=np.float64)
        self.J = len(self.omega)

    def apply(self, r):
        d = 2
        R = np.asarray(r, dtype=np.float64).reshape(self.n[1], self.n[0])
        S = np.zeros_like(R)                                       # s~_0 = 0
        for om, ga in zip(self.omega, self.gamma):
            rj = R - mode_product(S, self.K2 - om * self.M2, 1, d)     # r - (I (x) (K2 - w M2)) s~
            S = mode_solve(rj, self.K1 + om * self.M1, 0, d)           # ((K1 + w M1) (x) I) s~_{j-1/2}
            rh = R - mode_product(S, self.K1 - ga * self.M1, 0, d)     # r - ((K1 - g M1) (x) I) s~_{j-1/2}
            S = mode_solve(rh, self.K2 + ga * self.M2, 1, d)           # (I (x) (K2 + g M2)) s~_j
        return mode_solve(S, self.M1, 0, d).ravel()                    # s_J = (M1 (x) I)^{-1} s~_J


# -------------------------------------------- three-variable solver ----

def douglas_factor(w, l1, l2, l3):
    """Amplification of the Douglas step on the eigenvector triple (l1, l2, l3):
    1 - 2 w^2 (l1 + l2 + l3) / ((w + l1)(w + l2)(w + l3))."""
    return 1.0 - 2.0 * w * w * (l1 + l2 + l3) / ((w + l1) * (w + l2) * (w + l3))


def _triples(lams):
    L1, L2, L3 = lams
    g3, g2, g1 = np.meshgrid(L3, L2, L1, indexing="ij")   # [i3, i2, i1]
    return g1, g2, g3


def rho_3d(omega, lams):
    """rho_J of Section 5.2 over the computed eigenvalue triples (= ||T_J||)."""
    l1, l2, l3 = _triples(lams)
    prod = np.ones_like(l1)
    for w in omega:
        prod = prod * douglas_factor(w, l1, l2, l3)
    return float(np.abs(prod).max())


def _greedy_candidates(l1, l2, l3):
    """Minimisers over w > 0 of |g(w; l)| (Eq. (greedy2)); one value, or the
    two zeros of g when g < 0 at its stationary point."""
    S = l1 + l2 + l3
    e2 = l1 * l2 + l1 * l3 + l2 * l3
    e3 = l1 * l2 * l3
    roots = np.roots([1.0, 0.0, -e2, -2.0 * e3])
    w_st = max(float(z.real) for z in roots if abs(z.imag) <= 1e-12 * abs(z) and z.real > 0)
    if douglas_factor(w_st, l1, l2, l3) >= 0.0:
        return [w_st]
    zs = np.roots([1.0, -S, e2, e3])
    return sorted(float(z.real) for z in zs if abs(z.imag) <= 1e-9 * abs(z) and z.real > 0)


def greedy_parameters_3d(lams, eps, max_J=400):
    """Parameters w_1, ..., w_J by Eqs. (greedy1)-(greedy2), J the first index
    with rho_J <= eps (the stopping rule of Section 5.2)."""
    l1, l2, l3 = _triples(lams)
    prod = np.ones_like(l1)
    omega = []
    star = (lams[0][0], lams[1][0], lams[2][0])            # start: the smallest triple
    while len(omega) < max_J:
        best = None
        for w in _greedy_candidates(*star):
            nxt = prod * douglas_factor(w, l1, l2, l3)
            val = np.abs(nxt).max()
            if best is None or val < best[0]:
                best = (val, w, nxt)
        val, w, prod = best
        omega.append(w)
        if val <= eps:
            break
        idx = np.unravel_index(np.argmax(np.abs(prod)), prod.shape)
        star = (l1[idx], l2[idx], l3[idx])                  # Eq. (greedy1)
    return np.array(omega)


class ADI3D:
    """Algorithm 4 on the pencils (K_k, M_k), k = 1, 2, 3, from s_0 = 0: the
    Douglas iteration of Eq. (ADI3D) in the form of Eq. (ADI3D2), with the
    quantities u_j, v_j, b_j of Section 5.2. Applying it to r is P_J^{-1} r."""

    def __init__(self, pencils, eps=None, omega=None, max_J=400):
        (self.K1, self.M1), (self.K2, self.M2), (self.K3, self.M3) = pencils
        self.n = tuple(K.shape[0] for K, _ in pencils)
        self.lams = [pencil_spectrum(K, M) for K, M in pencils]       # all eigenvalues
        if omega is None:
            omega = greedy_parameters_3d(self.lams, eps, max_J)
        self.omega = np.asarray(omega, dtype=np.float64)
        self.J = len(self.omega)

    def apply(self, r):
        d = 3
        R = np.asarray(r, dtype=np.float64).reshape(self.n[2], self.n[1], self.n[0])
        rt = 2.0 * mode_solve(mode_solve(R, self.M2, 1, d), self.M3, 2, d)   # r~ = 2 (I (x) M2 (x) M3)^{-1} r
        s = np.zeros_like(R)                                                 # s_0 = 0
        v = np.zeros_like(R)                                                 # v_1 = 0
        for w in self.omega:
            u = mode_solve(mode_product(s, self.K2, 1, d), self.M2, 1, d)    # u_j = (I (x) M2^{-1}K2 (x) I) s_{j-1}
            r1 = (rt - mode_product(s, self.K1 - w * self.M1, 0, d)
                  - mode_product(2.0 * (u + v), self.M1, 0, d))              # r*_j, Eq. (ADI3D2a)
            s1 = mode_solve(r1, self.K1 + w * self.M1, 0, d)                 # s*_j
            r2 = mode_product(u + w * s1, self.M2, 1, d)                     # r**_j, Eq. (ADI3D2b)
            s2 = mode_solve(r2, self.K2 + w * self.M2, 1, d)                 # s**_j
            bj = v + w * s2                                                  # b_j
            r3 = mode_product(bj, self.M3, 2, d)                             # r_j, Eq. (ADI3D2c)
            s = mode_solve(r3, self.K3 + w * self.M3, 2, d)                  # s_j
            v = bj - w * s                                                   # v_{j+1} = b_j - w_j s_j
        return s.ravel()
