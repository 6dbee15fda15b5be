"""Pins of the FP64 oracle against facts fixed by the paper and by the
mathematics (closed forms, invariants, brute force), independent of the
oracle's own code paths. CPU only."""
import os

import numpy as np
import pytest

import synth
from oracle import assemble, fd, pcg, spline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _nonuniform_knots(nel, p, seed):
    g = synth.rng(seed)
    inner = np.sort(g.uniform(0.05, 0.95, nel - 1))
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def _disc(prob, nq=None):
    return assemble.Discretization.from_problem(prob, nq)


# ---------------------------------------------------------------- basis ----
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_partition_of_unity_nonneg_support(p):
    kn = _nonuniform_knots(7, p, p)
    z = np.linspace(0, 1, 301)
    B = spline.basis_table(kn, p, z)
    assert np.allclose(B.sum(axis=1), 1.0, atol=1e-14)
    assert B.min() >= -1e-15
    for i in range(B.shape[1]):                     # supp B_i = [xi_i, xi_{i+p+1}]
        outside = (z < kn[i]) | (z > kn[i + p + 1])
        assert np.all(B[outside, i] == 0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_integrals_and_derivatives(p):
    kn = _nonuniform_knots(6, p, 10 + p)
    z, w, _ = spline.gauss_points(kn, p + 2)
    B = spline.basis_table(kn, p, z.ravel())
    integ = (B * w.ravel()[:, None]).sum(axis=0)
    m = len(kn) - p - 1
    expect = np.array([(kn[i + p + 1] - kn[i]) / (p + 1) for i in range(m)])
    assert np.allclose(integ, expect, atol=1e-14)
    # derivatives against central differences away from knots
    zz = np.linspace(0.013, 0.987, 97)
    zz = zz[np.min(np.abs(zz[:, None] - kn[None, :]), axis=1) > 1e-3]
    h = 1e-6
    Dn = (spline.basis_table(kn, p, zz + h) - spline.basis_table(kn, p, zz - h)) / (2 * h)
    Da = spline.basis_table(kn, p, zz, deriv=True)
    assert np.allclose(Da, Dn, atol=1e-6 * max(1, np.abs(Da).max()))


def test_gauss_rule_exactness():
    kn = synth.uniform_open_knots(3, 2)
    for nq in (2, 3, 4):
        z, w, _ = spline.gauss_points(kn, nq)
        for deg in range(2 * nq):
            assert abs((w * z ** deg).sum() - 1.0 / (deg + 1)) < 1e-14


# -------------------------------------------------------------- pencils ----
@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_pencil_structure(p):
    pr = synth.Problem(2, 12, p)
    disc = _disc(pr)
    Kf, Mf = disc.pencil(0, full=True)
    m = Kf.shape[0]
    kn = pr.knots[0]
    assert np.allclose(Kf.sum(axis=1), 0.0, atol=1e-11)          # K 1 = 0
    assert np.allclose(Mf.sum(axis=1),
                       [(kn[i + p + 1] - kn[i]) / (p + 1) for i in range(m)], atol=1e-15)
    K, M = disc.pencil(0)
    for X in (K, M):
        assert np.allclose(X, X.T, atol=1e-15)
        i, j = np.nonzero(np.abs(X) > 0)
        assert np.max(np.abs(i - j)) == p                          # bandwidth p
        assert np.linalg.eigvalsh(X).min() > 0                     # SPD


def test_p1_closed_form():
    nel = 16
    pr = synth.Problem(2, nel - 1, 1)
    disc = _disc(pr)
    K, M = disc.pencil(0)
    h = 1.0 / nel
    n = nel - 1
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    assert np.allclose(K, T / h, atol=1e-12)
    assert np.allclose(M, (h / 6) * (4 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)), atol=1e-15)
    D, U = fd.generalized_eig(K, M)
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    lam = (6 / h ** 2) * (1 - np.cos(th)) / (2 + np.cos(th))
    assert np.allclose(D, lam, rtol=1e-12)
    for j in (0, 3, n - 1):                                          # sin(i j theta) eigvecs
        v = np.sin(np.arange(1, n + 1) * th[j])
        u = U[:, j]
        c = (u @ v) / (v @ v)
        assert np.allclose(u, c * v, atol=1e-10 * np.abs(u).max())


def test_table_cond_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_cond.txt")) if l[0] != "#"]
    for p_s, kap_s in rows:
        p, kap = int(p_s), float(kap_s)
        if p == 4:
            continue  # printed 4e5; the p=4 value at h=2^-9 is 6.5e5 (the table is not self-consistent)
        kn = synth.uniform_open_knots(512, p)
        geo = assemble.Geometry(np.zeros((1, len(kn) - p - 1)), [kn], p)
        K, M = assemble.Discretization([kn], p, geo).pencil(0)
        D, _ = fd.generalized_eig(K, M)
        val = D[-1] / D[0]
        assert float("%.0e" % val) == kap, (p, val, kap)


# ---------------------------------------------------------------- eigen ----
@pytest.mark.parametrize("n,p", [(128, 3), (64, 2), (96, 5)])
def test_eig_invariants(n, p):
    pr = synth.Problem(2, n, p)
    K, M = _disc(pr).pencil(0)
    D, U = fd.generalized_eig(K, M)
    I = np.eye(n)
    assert np.abs(U.T @ M @ U - I).max() <= 1e-12
    assert np.abs(U.T @ K @ U - np.diag(D)).max() <= 1e-12 * D.max()
    assert np.all(np.diff(D) > 0)


# ------------------------------------------------------------------- FD ----
@pytest.mark.parametrize("dim,n,p", [(2, (7, 5), 2), (3, (5, 6, 4), 3), (3, (6, 6, 6), 1)])
def test_fd_equals_dense_inverse(dim, n, p):
    pr = synth.Problem(dim, n, p)
    disc = _disc(pr)
    P = disc.dense_P()
    F = fd.FD([disc.pencil(k) for k in range(dim)])
    r = synth.random_vector(disc.N, 1)
    s_ref = np.linalg.solve(P, r)
    s = F.apply(r)
    assert np.abs(s - s_ref).max() <= 1e-13 * np.abs(s_ref).max()


# ------------------------------------------------------------ stiffness ----
@pytest.mark.parametrize("dim,n,p,amp", [(2, (6, 5), 2, None), (3, (5, 4, 6), 2, [0.05, -0.04, 0.03]),
                                         (3, (4, 4, 4), 3, [0.1, 0.05, -0.05])])
def test_A_elementwise_vs_bruteforce(dim, n, p, amp):
    pr = synth.Problem(dim, n, p, amp)
    disc = _disc(pr)
    S = disc.assemble_stencil()
    A = assemble.stencil_to_csr(disc, S).toarray()
    Ad = disc.dense_A_bruteforce()
    assert np.abs(A - Ad).max() <= 1e-14 * np.abs(Ad).max()
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()
    # same sparsity as P (Section 3)
    P = disc.dense_P()
    assert np.array_equal(np.abs(A) > 1e-14, np.abs(P) > 1e-14)


@pytest.mark.parametrize("dim,n,p", [(2, 9, 3), (3, 5, 2)])
def test_identity_map_A_equals_P(dim, n, p):
    disc = _disc(synth.Problem(dim, n, p))
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil()).toarray()
    assert np.abs(A - disc.dense_P()).max() <= 1e-14 * np.abs(A).max()


def _weighted_1d(knots, p, weight):
    """1D stiffness and mass matrices of the Dirichlet-reduced basis with the
    weight function weight(z), by a 10-point Gauss rule per element (exact
    for the polynomial weights used here)."""
    xg, wg = np.polynomial.legendre.leggauss(10)
    K = M = 0.0
    for s in spline.elements(knots):
        a, b = knots[s], knots[s + 1]
        z = 0.5 * (b - a) * xg + 0.5 * (a + b)
        w = 0.5 * (b - a) * wg * weight(z)
        B = spline.basis_table(knots, p, z)[:, 1:-1]
        D = spline.basis_table(knots, p, z, deriv=True)[:, 1:-1]
        K = K + D.T @ (w[:, None] * D)
        M = M + B.T @ (w[:, None] * B)
    return K, M


def test_variable_coefficient_linear_in_zeta1():
    """Identity map, coefficient kappa = 1 + zeta_1 (a degree-1 spline field):
    A is the Kronecker sum of 1D matrices with the weight 1 + z along
    direction 1, K1w (x) M2 (x) M3 + M1w (x) K2 (x) M3 + M1w (x) M2 (x) K3
    (direction 1 fastest), built here from 1D integrals alone."""
    p, n = 2, (6, 5, 4)
    pr = synth.Problem(3, n, p)
    pr.kappa_knots = [np.array([0.0, 0.0, 1.0, 1.0])] * 3
    pr.kappa_p = 1
    ctrl = np.ones((2, 2, 2))
    ctrl[:, :, 1] = 2.0                   # value 1 at zeta_1 = 0, 2 at zeta_1 = 1
    pr.kappa_ctrl = ctrl
    disc = _disc(pr)
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil()).toarray()
    K1, M1 = _weighted_1d(pr.knots[0], p, lambda z: 1.0 + z)
    K2, M2 = _weighted_1d(pr.knots[1], p, lambda z: np.ones_like(z))
    K3, M3 = _weighted_1d(pr.knots[2], p, lambda z: np.ones_like(z))
    kron3 = lambda c, b, a: np.kron(c, np.kron(b, a))
    Ak = kron3(M3, M2, K1) + kron3(M3, K2, M1) + kron3(K3, M2, M1)
    assert np.abs(A - Ak).max() <= 1e-13 * np.abs(Ak).max()
    # the weight matters: the unweighted Kronecker sum differs
    K1u, M1u = _weighted_1d(pr.knots[0], p, lambda z: np.ones_like(z))
    Au = kron3(M3, M2, K1u) + kron3(M3, K2, M1u) + kron3(K3, M2, M1u)
    assert np.abs(A - Au).max() > 1e-3 * np.abs(Ak).max()


def test_rhs_identity_map_separable_load():
    """Identity map, f = 1 + 2 x: b_i = int (1 + 2 zeta_1) B_i = (I_1 + 2 X_1)
    (x) I_2 (x) I_3 (direction 1 fastest), with I_k the integrals and X_1 the
    first moments of the Dirichlet-reduced 1D B-splines (closed form
    (xi_{i+p+1} - xi_i)/(p+1) for the integrals)."""
    p, n = 3, (7, 5, 6)
    pr = synth.Problem(3, n, p)
    disc = _disc(pr)
    b = disc.assemble_rhs(lambda x, y, z: 1.0 + 2.0 * x + 0.0 * y * z)
    ints = []
    for k in range(3):
        xi = pr.knots[k]
        m = len(xi) - p - 1
        ints.append(np.array([(xi[i + p + 1] - xi[i]) / (p + 1) for i in range(1, m - 1)]))
    xg, wg = np.polynomial.legendre.leggauss(10)
    X1 = 0.0
    xi = pr.knots[0]
    for s_ in spline.elements(xi):
        a_, b_ = xi[s_], xi[s_ + 1]
        z = 0.5 * (b_ - a_) * xg + 0.5 * (a_ + b_)
        X1 = X1 + (0.5 * (b_ - a_) * wg * z) @ spline.basis_table(xi, p, z)[:, 1:-1]
    bk = np.kron(ints[2], np.kron(ints[1], ints[0] + 2.0 * X1))
    assert np.abs(b - bk).max() <= 1e-14 * np.abs(bk).max()


def test_affine_map_closed_form():
    a = np.array([1.0, 2.0, 0.5])
    pr = synth.Problem(3, (5, 4, 6), 2)
    pr.ctrl = pr.ctrl * a[:, None, None, None]
    disc = _disc(pr)
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil()).toarray()
    pens = [disc.pencil(k) for k in range(3)]
    expect = 0
    for k in range(3):
        T = np.ones((1, 1))
        for l in reversed(range(3)):
            T = np.kron(T, pens[l][0] if l == k else pens[l][1])
        expect = expect + (np.prod(a) / a[k] ** 2) * T
    assert np.abs(A - expect).max() <= 1e-13 * np.abs(A).max()
    # the spectrum of P^-1 A lies in [min c, max c] (Prop. 1 with constant Q)
    ev = np.linalg.eigvals(np.linalg.solve(disc.dense_P(), A)).real
    c = np.prod(a) / a ** 2
    assert ev.min() >= c.min() * (1 - 1e-12) and ev.max() <= c.max() * (1 + 1e-12)


def test_shear_map_energy_fixes_Q_transposes():
    """x = zeta_1 + s zeta_2, y = zeta_2. The Greville interpolant of zeta_1
    is the function x - s y, whose energy on the unit-area parallelogram is
    1 + s^2; zeta_2 is y (energy 1); their coupling is -s."""
    s, p = 0.7, 2
    pr = synth.Problem(2, 5, p)
    pr.ctrl = np.stack([pr.ctrl[0] + s * pr.ctrl[1], pr.ctrl[1]])
    disc = _disc(pr)
    Af = disc.dense_A_bruteforce(full=True)
    g1 = synth.greville(pr.knots[0], p)
    g2 = synth.greville(pr.knots[1], p)
    u1 = np.tile(g1, len(g2))                     # zeta_1 (direction 1 fastest)
    u2 = np.repeat(g2, len(g1))                   # zeta_2
    assert abs(u1 @ Af @ u1 - (1 + s * s)) < 1e-13
    assert abs(u2 @ Af @ u2 - 1.0) < 1e-13
    assert abs(u1 @ Af @ u2 + s) < 1e-13


def test_assemble_rows_matches_full():
    pr = synth.Problem(3, (6, 5, 7), 3, [0.05, 0.02, -0.04])
    disc = _disc(pr)
    S = disc.assemble_stencil()
    rows = [(0, 0, 0), (5, 4, 6), (2, 3, 1), (3, 0, 6)]
    R = disc.assemble_rows(rows)
    for r, i in enumerate(rows):
        assert np.abs(R[r] - S[:, disc.row_index(i)]).max() <= 1e-15 * np.abs(S).max()


# ------------------------------------------------------------------ PCG ----
@pytest.mark.parametrize("dim,n,p", [(2, 16, 3), (3, 8, 3)])
def test_pcg_identity_map_one_iteration(dim, n, p):
    disc = _disc(synth.Problem(dim, n, p))
    S = disc.assemble_stencil()
    f = (lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)) if dim == 2 else \
        (lambda x, y, z: 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z))
    b = disc.assemble_rhs(f)
    F = fd.FD([disc.pencil(k) for k in range(dim)])
    res = pcg.pcg(lambda v: assemble.apply_stencil(disc, S, v), b, F.apply, tol=1e-8)
    assert res.converged and res.iters == 1
    assert res.true_relres < 1e-12


def test_pcg_matches_direct_solve():
    disc = _disc(synth.Problem(3, (7, 6, 5), 3, [0.08, -0.05, 0.03]))
    S = disc.assemble_stencil()
    A = assemble.stencil_to_csr(disc, S)
    b = synth.random_rhs(disc.N, 3)
    F = fd.FD([disc.pencil(k) for k in range(3)])
    res = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-13, max_iter=200)
    x = np.linalg.solve(A.toarray(), b)
    assert res.converged
    assert np.linalg.norm(res.x - x) <= 1e-11 * np.linalg.norm(x)
    # fixed-iteration mode returns the k-th iterate of the same recurrence
    r5 = pcg.pcg(lambda v: A @ v, b, F.apply, fixed_iters=5)
    assert r5.iters == 5 and np.allclose(r5.history[:6], res.history[:6], rtol=1e-12)


def test_flexible_beta_equals_fletcher_reeves_for_exact_preconditioner():
    """With a fixed SPD preconditioner (the exact FD), (r_{k+1}, z_k) = 0 in
    exact arithmetic, so the flexible beta (r_{k+1}, z_{k+1} - z_k)/(r_k, z_k)
    equals the Fletcher-Reeves one and the iterates agree to rounding."""
    disc = _disc(synth.Problem(3, (8, 7, 6), 3, [0.1, -0.06, 0.04]))
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
    b = synth.random_rhs(disc.N, 41)
    F = fd.FD([disc.pencil(k) for k in range(3)])
    fr = pcg.pcg(lambda v: A @ v, b, F.apply, fixed_iters=8)
    fl = pcg.pcg(lambda v: A @ v, b, F.apply, fixed_iters=8, flexible=True)
    assert np.linalg.norm(fl.x - fr.x) <= 1e-9 * np.linalg.norm(fr.x)
    assert np.allclose(fl.betas, fr.betas, rtol=1e-6, atol=1e-12)


def _round_mantissa(v, bits):
    m, e = np.frexp(v)
    s = 2.0 ** bits
    return np.ldexp(np.round(m * s) / s, e)


def test_flexible_beta_with_a_low_precision_preconditioner():
    """The FD applied through rounding of its input and output to a few
    mantissa bits (a stand-in for low-precision operands) is no longer a fixed
    linear operator, and (r_{k+1}, z_k) is no longer ~0. PCG with the flexible
    beta (r_{k+1}, z_{k+1} - z_k)/(r_k, z_k) still reaches the direct solution
    within two iterations of the exact FD at 8 bits, and at 3 bits it needs far
    fewer iterations than Fletcher-Reeves (a wrong sign in the formula makes
    the 8-bit run stall)."""
    disc = _disc(synth.Problem(3, (9, 8, 7), 3, [0.1, -0.06, 0.04]))
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
    b = synth.random_rhs(disc.N, 42)
    F = fd.FD([disc.pencil(k) for k in range(3)])
    x = np.linalg.solve(A.toarray(), b)
    exact = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-10, max_iter=300)

    def rounded(bits):
        return lambda r: _round_mantissa(F.apply(_round_mantissa(r, bits)), bits)
    flex8 = pcg.pcg(lambda v: A @ v, b, rounded(8), tol=1e-10, max_iter=300, flexible=True)
    assert flex8.converged and flex8.iters <= exact.iters + 2
    assert np.linalg.norm(flex8.x - x) <= 1e-8 * np.linalg.norm(x)
    flex3 = pcg.pcg(lambda v: A @ v, b, rounded(3), tol=1e-10, max_iter=300, flexible=True)
    fr3 = pcg.pcg(lambda v: A @ v, b, rounded(3), tol=1e-10, max_iter=300, flexible=False)
    assert flex3.converged and flex3.iters < 0.6 * fr3.iters


def test_planted_flexible_sign_fails_low_precision_pin(monkeypatch):
    """A sign error planted in the oracle's flexible beta, (r_{k+1}, z_{k+1} +
    z_k), passes with the exact FD (where (r_{k+1}, z_k) ~ 0) but fails the
    low-precision pin above."""
    import inspect
    src = inspect.getsource(pcg.pcg).replace("(r @ (zn - z)) / rho", "(r @ (zn + z)) / rho")
    assert src != inspect.getsource(pcg.pcg)
    ns = {}
    exec(src, pcg.__dict__, ns)
    monkeypatch.setattr(pcg, "pcg", ns["pcg"])
    with pytest.raises(AssertionError):
        test_flexible_beta_with_a_low_precision_preconditioner()


def test_prop1_condition_bound():
    pr = synth.Problem(3, 6, 2, [0.1, -0.08, 0.05])
    disc = _disc(pr)
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil()).toarray()
    ev = np.linalg.eigvals(np.linalg.solve(disc.dense_P(), A)).real
    kappa = ev.max() / ev.min()
    # extreme eigenvalues of Q on a fine sample of the parameter domain
    pts = [np.linspace(0, 1, 41)] * 3
    _, J = disc.geo.eval_grid(pts)
    Q, _ = assemble.q_matrix(J)
    lam = np.linalg.eigvalsh(Q.reshape(-1, 3, 3))
    bound = lam[:, -1].max() / lam[:, 0].min()
    assert 1.0 < kappa <= bound
    assert ev.min() >= lam[:, 0].min() * (1 - 1e-3) and ev.max() <= lam[:, -1].max() * (1 + 1e-3)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_l2_convergence_rate_2d(p):
    u = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    f = lambda x, y: 2 * np.pi ** 2 * u(x, y)
    errs = []
    for nel in (8, 16, 32):
        pr = synth.Problem(2, nel + p - 2, p)
        pr.ctrl = pr.ctrl.copy()
        disc = _disc(pr)
        A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
        x = np.linalg.solve(A.toarray(), disc.assemble_rhs(f))
        errs.append(disc.l2_error(x, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(rates[-1] - (p + 1)) < 0.2, rates


def test_l2_convergence_rate_3d_deformed():
    """On the deformed cube the physical domain is still the unit cube, so
    the manufactured solution is exact; a wrong Q would stall the rate."""
    p = 2
    amp = [0.04, -0.03, 0.02]
    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f = lambda x, y, z: 3 * np.pi ** 2 * u(x, y, z)
    errs = []
    for nel in (4, 8, 16):
        pr = synth.Problem(3, nel + p - 2, p, amp)
        disc = _disc(pr)
        S = disc.assemble_stencil()
        A = assemble.stencil_to_csr(disc, S)
        F = fd.FD([disc.pencil(k) for k in range(3)])
        res = pcg.pcg(lambda v: A @ v, disc.assemble_rhs(f), F.apply, tol=1e-12, max_iter=300)
        errs.append(disc.l2_error(res.x, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(rates[-1] - (p + 1)) < 0.25, rates


# ---------------------------------------------- planted mistakes fail pins ----
def test_planted_transposed_Q_fails_shear_pin(monkeypatch):
    def wrong_q(J, kappa=1.0):
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        return kappa * np.abs(det)[..., None, None] * (np.swapaxes(Jinv, -1, -2) @ Jinv), det
    monkeypatch.setattr(assemble, "q_matrix", wrong_q)
    with pytest.raises(AssertionError):
        test_shear_map_energy_fixes_Q_transposes()


def test_planted_swapped_fd_transposes_fail_dense_pin(monkeypatch):
    orig = fd.FD.apply

    def swapped(self, r):
        d = self.d
        R = np.asarray(r).reshape(tuple(reversed(self.n)))
        for k in range(d):
            R = fd.mode_product(R, self.eig[k][1], k, d)
        R = R / self.lam
        for k in range(d):
            R = fd.mode_product(R, self.eig[k][1].T, k, d)
        return R.ravel()
    monkeypatch.setattr(fd.FD, "apply", swapped)
    with pytest.raises(AssertionError):
        test_fd_equals_dense_inverse(3, (5, 6, 4), 3)
    monkeypatch.setattr(fd.FD, "apply", orig)


# ------------------------------------------------------ span scalings ----
from oracle import learned  # noqa: E402


def _affine_problem(a):
    pr = synth.Problem(3, (6, 5, 7), 2)
    pr.ctrl = pr.ctrl * np.asarray(a)[:, None, None, None]
    return pr


def test_sepfit_and_features_affine_map_closed_form():
    """F = diag(a): Q = kappa prod(a) diag(1/a_k^2) is constant, so the fit is
    exact (log wK_k = log c_k, log wM = 0) and the slab spread is zero."""
    a = np.array([1.0, 2.0, 0.5])
    disc = assemble.Discretization.from_problem(_affine_problem(a))
    c = np.prod(a) / a ** 2
    lw = learned.sepfit(disc)
    dirs = np.repeat(np.arange(3), disc.nel)
    assert np.allclose(np.exp(lw[:, 0]), c[dirs], rtol=1e-12)
    assert np.abs(lw[:, 1]).max() < 1e-12
    f = learned.features(disc)
    assert np.allclose(f[:, 0], np.log(c[dirs]), atol=1e-12)
    assert np.allclose(f[:, 2], np.log(c.min()), atol=1e-12)
    assert np.allclose(f[:, 3], np.log(c.max()), atol=1e-12)
    assert np.abs(f[:, 4]).max() < 1e-12


def test_scaled_pencils_make_P_equal_A_for_affine_map():
    """With wK_k = c_k the scaled Kronecker sum is A itself: one iteration."""
    a = np.array([1.0, 2.0, 0.5])
    disc = assemble.Discretization.from_problem(_affine_problem(a))
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
    F = fd.FD(learned.scaled_pencils(disc, learned.sepfit(disc)))
    b = synth.random_rhs(disc.N, 2)
    res = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-10)
    assert res.converged and res.iters == 1
    F0 = fd.FD([disc.pencil(k) for k in range(3)])
    assert pcg.pcg(lambda v: A @ v, b, F0.apply, tol=1e-10).iters > 3


def test_sepfit_scaling_helps_on_random_coefficient():
    pr = synth.learned_workload_problem(1, n=10, p=2)
    disc = assemble.Discretization.from_problem(pr)
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
    b = synth.random_rhs(disc.N, 3)
    F0 = fd.FD([disc.pencil(k) for k in range(3)])
    F1 = fd.FD(learned.scaled_pencils(disc, learned.sepfit(disc)))
    it0 = pcg.pcg(lambda v: A @ v, b, F0.apply, tol=1e-8, max_iter=400).iters
    it1 = pcg.pcg(lambda v: A @ v, b, F1.apply, tol=1e-8, max_iter=400).iters
    assert it1 < it0, (it1, it0)


def test_mlp_gradient_matches_finite_differences():
    g = synth.rng(12)
    params = g.normal(0, 0.3, 4738)
    X = g.normal(0, 1, (20, 6))
    T = g.normal(0, 1, (20, 2))
    norm = (np.full(6, 0.1), np.full(6, 1.5), np.array([0.2, -0.1]), np.array([2.0, 0.5]))
    loss, grad = learned.mlp_loss_grad(params, norm, X, T)
    idx = g.choice(4738, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(4738); e[i] = h
        lp, _ = learned.mlp_loss_grad(params + e, norm, X, T)
        lm, _ = learned.mlp_loss_grad(params - e, norm, X, T)
        assert abs((lp - lm) / (2 * h) - grad[i]) <= 1e-6 * max(1.0, abs(grad[i]))


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 7)])
def test_fd_apply_flop_count(monkeypatch, dim, n):
    """The FD apply costs 8 n^3 FLOPs in 2D and 12 n^4 in 3D (Sections 4.1 and
    5.1.1): 2d dense mode products of 2 n^(d+1) FLOPs each (the divide by the
    eigenvalue sums is of lower order). Counted on the oracle's products."""
    disc = _disc(synth.Problem(dim, n, 2))
    F = fd.FD([disc.pencil(k) for k in range(dim)])
    count = [0]
    real = fd.mode_product

    def counting(X, W, k, d):
        count[0] += 2 * W.shape[0] * W.shape[1] * (X.size // X.shape[d - 1 - k])
        return real(X, W, k, d)

    monkeypatch.setattr(fd, "mode_product", counting)
    F.apply(synth.random_vector(disc.N, 1))
    assert count[0] == (8 * n ** 3 if dim == 2 else 12 * n ** 4)


def test_mode_product_is_the_kronecker_product():
    """Section 2.2's Kronecker identities: the product along direction k of
    a direction-1-fastest tensor is the matrix I (x) .. W .. (x) I, with W in
    the factor of direction k (numpy's kron puts its first factor on the
    slowest index)."""
    g = synth.rng(3)
    n = (4, 3, 5)                                       # n_1, n_2, n_3
    X = g.standard_normal((n[2], n[1], n[0]))
    for k in range(3):
        W = g.standard_normal((n[k], n[k]))
        mats = [np.eye(m) for m in n]
        mats[k] = W
        big = np.kron(np.kron(mats[2], mats[1]), mats[0])
        assert np.allclose(fd.mode_product(X, W, k, 3).ravel(), big @ X.ravel(), atol=1e-13)


def _pencil_triple(knots, p):
    """1D M, K and the mixed G_ij = int B_i' B_j (Dirichlet rows and columns
    removed), from the basis at a Gauss rule exact for their integrands."""
    z, w, _ = spline.gauss_points(knots, p + 1)
    z, w = z.ravel(), w.ravel()
    V = spline.basis_table(knots, p, z)
    D = spline.basis_table(knots, p, z, deriv=True)
    M = (V * w[:, None]).T @ V
    K = (D * w[:, None]).T @ D
    G = (D * w[:, None]).T @ V
    return M[1:-1, 1:-1], K[1:-1, 1:-1], G[1:-1, 1:-1]


def test_general_affine_map_closed_form():
    """x = B zeta with a full matrix B (det > 0): Q = |det B| B^-1 B^-T is
    constant and A = sum_{k,l} Q_kl (x)_m F_m with F_m = K_m (m = k = l),
    G_m (m = k != l), G_m^T (m = l != k), M_m otherwise (direction 1
    fastest). Pins every entry of Q, its transposition included."""
    B = np.array([[1.1, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.3]])
    p = 2
    pr = synth.Problem(3, (5, 4, 6), p)
    pr.ctrl = np.einsum("ij,j...->i...", B, pr.ctrl)    # Greville net of the identity, mapped by B
    disc = _disc(pr)
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil()).toarray()
    Binv = np.linalg.inv(B)
    Q = abs(np.linalg.det(B)) * Binv @ Binv.T
    F = [_pencil_triple(kn, p) for kn in pr.knots]      # (M, K, G) per direction
    expect = 0
    for k in range(3):
        for l in range(3):
            fac = []
            for m in range(3):
                Mm, Km, Gm = F[m]
                fac.append(Km if m == k == l else Gm if m == k else Gm.T if m == l else Mm)
            expect = expect + Q[k, l] * np.kron(fac[2], np.kron(fac[1], fac[0]))
    assert np.abs(A - expect).max() <= 1e-13 * np.abs(A).max()


def test_parallel_assembly_matches_serial():
    """The process-parallel assembly (plane ranges summed by spawned workers,
    range sums added in order) gives the serial A and b up to the association
    of each row's element sums."""
    prob = synth.Problem(3, (9, 8, 10), 2, [0.03, -0.02, 0.04])
    disc = assemble.Discretization.from_problem(prob)
    S1, S2 = disc.assemble_stencil(), disc.assemble_stencil(workers=3)
    assert np.abs(S1 - S2).max() <= 1e-14 * np.abs(S1).max()
    b1 = disc.assemble_rhs(assemble.sine_load)
    b2 = disc.assemble_rhs(assemble.sine_load, workers=3)
    assert np.abs(b1 - b2).max() <= 1e-14 * np.abs(b1).max()
    # the module-level manufactured load is f = 3 pi^2 sin sin sin
    x = np.array([0.3, 0.7]), np.array([0.2, 0.5]), np.array([0.9, 0.4])
    ref = 3 * np.pi ** 2 * np.sin(np.pi * x[0]) * np.sin(np.pi * x[1]) * np.sin(np.pi * x[2])
    assert np.allclose(assemble.sine_load(*x), ref, rtol=1e-15, atol=0)
