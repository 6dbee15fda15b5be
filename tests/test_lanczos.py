"""CG-Lanczos condition estimate of P^-1 A (label search of the learned
scalings; Section 4 bounds the spread of this spectrum).

CPU pins: the library's tridiagonal extremes against numpy's eigenvalues of
the same tridiagonal, and the Lanczos relation itself: CG on a small SPD
system runs to convergence, and the extreme eigenvalues of its tridiagonal
match those of the dense pencil (A, P) of the oracle. GPU: the library's
recorded coefficients give the same estimate as the oracle's CG."""
import numpy as np
import pytest

import synth
from oracle import assemble, fd, pcg


def lanczos_tridiagonal(alphas, betas):
    m = len(alphas)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < m - 1:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return T


def small_case():
    prob = synth.Problem(3, (6, 5, 7), 2, [0.05, -0.03, 0.02])
    disc = assemble.Discretization.from_problem(prob)
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil()).toarray()
    Pd = disc.dense_P()
    F = fd.FD([disc.pencil(k) for k in range(3)])
    return prob, disc, A, Pd, F


def test_tridiagonal_extremes_match_numpy():
    from paper_1602_01636_gb300 import igafd
    g = np.random.default_rng(5)
    for m in (1, 2, 7, 40):
        a = g.uniform(0.1, 2.0, m)
        b = g.uniform(0.0, 0.9, max(m - 1, 0))
        lo, hi = igafd.lanczos_extremes(a, b)
        ev = np.linalg.eigvalsh(lanczos_tridiagonal(a, b))
        assert abs(lo - ev[0]) <= 1e-12 * ev[-1] and abs(hi - ev[-1]) <= 1e-12 * ev[-1]
    with pytest.raises(igafd.IgafdError):
        igafd.lanczos_extremes(np.array([1.0, -1.0]), np.array([0.5]))


def test_cg_lanczos_relation_on_oracle():
    """The Lanczos relation itself: n steps of CG on an n x n SPD system give a
    tridiagonal whose eigenvalues are those of P^-1 A (here with P a
    diagonal, so P^-1 A's eigenvalues are the pencil's); fewer steps give
    Ritz values inside the spectrum."""
    from paper_1602_01636_gb300 import igafd
    import scipy.linalg
    g = np.random.default_rng(11)
    n = 12
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    A = Q @ np.diag(np.geomspace(1.0, 50.0, n)) @ Q.T
    Pd = np.diag(g.uniform(0.5, 2.0, n))
    ev = scipy.linalg.eigh(A, Pd, eigvals_only=True)
    b = g.standard_normal(n)
    res = pcg.pcg(lambda v: A @ v, b, lambda r: r / np.diag(Pd), fixed_iters=n, true_every=0)
    lo, hi = igafd.lanczos_extremes(res.alphas, res.betas[:n - 1])
    assert abs(lo - ev[0]) <= 1e-8 * ev[-1] and abs(hi - ev[-1]) <= 1e-8 * ev[-1]
    # all n Ritz values (the formula, checked independently of the library)
    assert np.allclose(np.linalg.eigvalsh(lanczos_tridiagonal(res.alphas, res.betas[:n - 1])), ev,
                       rtol=1e-8, atol=1e-8 * ev[-1])
    # a planted mistake (beta_j shifted by one step) breaks it
    bad = res.betas[1:n] + [res.betas[0]]
    blo, bhi = igafd.lanczos_extremes(res.alphas, bad[:n - 1])
    assert abs(blo - ev[0]) > 1e-6 * ev[-1] or abs(bhi - ev[-1]) > 1e-6 * ev[-1]
    # the deformed-cube system: Ritz extremes lie inside the pencil's spectrum
    prob, disc, A3, Pd3, F = small_case()
    r3 = pcg.pcg(lambda v: A3 @ v, synth.random_rhs(disc.N, 3), F.apply, tol=1e-12,
                 max_iter=400, true_every=0)
    e3 = scipy.linalg.eigh(A3, Pd3, eigvals_only=True)
    l3, h3 = igafd.lanczos_extremes(r3.alphas, r3.betas[:len(r3.alphas) - 1])
    assert e3[0] * (1 - 1e-12) <= l3 < h3 <= e3[-1] * (1 + 1e-12)


@pytest.mark.gpu
def test_gpu_condition_estimate_matches_oracle():
    from gpu_util import need_gpu, make_patch, to_dev
    need_gpu()
    prob, disc, A, Pd, F = small_case()
    b = synth.random_rhs(disc.N, 3)
    res = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-12, max_iter=400, true_every=0)
    patch = make_patch(prob)
    x, info = patch.pcg(to_dev(b), tol=1e-12, max_iter=400, dtype="fp64", true_every=0)
    assert info.status == 0
    from paper_1602_01636_gb300 import igafd
    for steps in (10, 0):
        k, lo, hi = patch.condition_estimate(steps)
        m = steps or info.iterations
        m = min(m, len(res.alphas))
        lo_o, hi_o = igafd.lanczos_extremes(res.alphas[:m], res.betas[:m - 1])
        assert abs(lo - lo_o) <= 1e-8 * lo_o and abs(hi - hi_o) <= 1e-8 * hi_o
        assert abs(k - hi / lo) <= 1e-12 * k
    patch.close()
