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
