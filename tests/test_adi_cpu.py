"""The library's host-side greedy ADI parameter search (igafd_adi_greedy,
the core of igafd_adi_parameters) against the oracle's Eqs. (greedy1)-
(greedy2) on the same spectra. CPU only: the search needs no GPU."""
import numpy as np
import pytest

import synth
from oracle import adi, assemble


@pytest.fixture(scope="module")
def igafd():
    from paper_1602_01636_gb300 import build, igafd as mod
    build.build()
    return mod


@pytest.mark.parametrize("n,p,eps", [((12, 10, 14), 3, 0.1), ((12, 10, 14), 3, 1e-6),
                                     ((20, 20, 20), 2, 1e-8), ((9, 30, 5), 4, 1e-3)])
def test_library_greedy_matches_oracle(igafd, n, p, eps):
    prob = synth.Problem(3, n, p, [0.04, 0.02, -0.03])
    disc = assemble.Discretization.from_problem(prob)
    lams = [adi.pencil_spectrum(K, M) for K, M in (disc.pencil(k) for k in range(3))]
    w = igafd.adi_greedy(*lams, eps)
    w_ref = adi.greedy_parameters_3d(lams, eps)
    assert abs(len(w) - len(w_ref)) <= 1
    m = min(len(w), len(w_ref))
    assert np.allclose(w[:m], w_ref[:m], rtol=1e-10, atol=0)
    assert adi.rho_3d(w, lams) <= eps * (1 + 1e-9)


def test_library_greedy_large_and_threaded(igafd):
    """n = 96 per direction (884,736 triples, split over threads): the same
    count and parameters as the oracle."""
    kn = synth.uniform_open_knots(95, 3)
    geo = assemble.Geometry(np.zeros((1, len(kn) - 4)), [kn], 3)
    lam = adi.pencil_spectrum(*assemble.Discretization([kn], 3, geo).pencil(0))
    w = igafd.adi_greedy(lam, lam, lam, 1e-4)
    w_ref = adi.greedy_parameters_3d([lam, lam, lam], 1e-4)
    assert len(w) == len(w_ref)
    assert np.allclose(w, w_ref, rtol=1e-10, atol=0)


def test_library_greedy_rejects_bad_input(igafd):
    with pytest.raises(igafd.IgafdError):
        igafd.adi_greedy([1.0, -2.0], [1.0], [1.0], 0.1)
    with pytest.raises(igafd.IgafdError):
        igafd.adi_greedy([1.0], [1.0], [1.0], 1.5)
    with pytest.raises(igafd.IgafdError):           # max_J too small to reach eps
        igafd.adi_greedy([1.0, 1e4], [1.0, 1e4], [1.0, 1e4], 1e-12, max_J=2)


@pytest.mark.parametrize("ratio", [1.0, 4.0, 1e2, 3.2e5, 1e8])
@pytest.mark.parametrize("eps", [1e-1, 1e-8])
def test_library_wachspress_matches_oracle(igafd, ratio, eps):
    """Two-variable parameters: J of Eq. (ADIits) and the elliptic-function
    parameters, the library's C against the oracle's Python (both by the
    AGM method; rounding near u = K/2 grows like 1e-16 b/a)."""
    a, b = 3.0, 3.0 * ratio
    w = igafd.adi_wachspress(a, b, eps)
    J = adi.adi_iterations_2d(a, b, eps) if ratio > 1 else max(1, adi.adi_iterations_2d(a, b, eps))
    assert len(w) == J
    w_ref = adi.wachspress_parameters(a, b, J)
    assert np.allclose(w, w_ref, rtol=1e-14 + 4e-16 * ratio, atol=0)


def test_library_wachspress_table_square(igafd):
    """The library reproduces the iteration counts of Table "square" from the
    closed-form p = 1 spectra (as the oracle's pin does)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table_adi_square.txt")
    for h_s, p_s, J_s, _ in (l.split() for l in open(path) if l.strip() and l[0] != "#"):
        if int(p_s) != 1:
            continue
        nel = int(h_s)
        t = np.array([1, nel - 1]) * np.pi / nel
        lam = 6.0 * nel ** 2 * (1 - np.cos(t)) / (2 + np.cos(t))
        assert len(igafd.adi_wachspress(lam[0], lam[1], 1e-8)) == int(J_s)


def test_library_wachspress_table_square_all_degrees(igafd):
    """Every printed J of Table "square" at h^-1 = 512 from the library's
    Eq. (ADIits) on the exact pencil extremes, and ||T_J|| of the library's
    parameters within the printed final error and 1e-8 (Table "relerr")."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table_adi_square.txt")
    for h_s, p_s, J_s, err_s in (l.split() for l in open(path) if l.strip() and l[0] != "#"):
        if int(h_s) != 512:
            continue
        p = int(p_s)
        kn = synth.uniform_open_knots(512, p)
        geo = assemble.Geometry(np.zeros((1, len(kn) - p - 1)), [kn], p)
        lam = adi.pencil_spectrum(*assemble.Discretization([kn], p, geo).pencil(0))
        w = igafd.adi_wachspress(lam[0], lam[-1], 1e-8)
        assert len(w) == int(J_s)
        assert float(err_s) <= adi.t_norm_2d(w, w, lam, lam) <= 1e-8
