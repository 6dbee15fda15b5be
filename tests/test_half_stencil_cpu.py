"""The reading behind the half-stored stencil (IGAFD_SETUP_HALF_STENCIL),
pinned on the oracle's own assembly (CPU): A is symmetric (Eq. (A): the
bilinear form of the Laplacian with an SPD coefficient matrix Q), so in the
offset-major stencil the coupling delta of row i equals the coupling -delta
of row i + off(delta), off(delta) = delta_1 + delta_2 n_1 + delta_3 n_1 n_2;
and a coupling leaves the index box exactly when its mirror does (the zero
halos of the half layout stand for rows outside [0, N))."""
import itertools

import numpy as np
import pytest

import synth
from oracle import assemble

CASES = [
    synth.Problem(3, (6, 5, 7), 2, [0.05, -0.03, 0.02]),
    synth.Problem(3, (4, 5, 3), 3, [0.03, 0.01, -0.02]),
    synth.Problem(2, (9, 7), 3),
]


@pytest.mark.parametrize("prob", CASES, ids=["3d-p2", "3d-narrow-p3", "2d-p3"])
def test_mirrored_couplings(prob):
    disc = assemble.Discretization.from_problem(prob)
    S = disc.assemble_stencil()
    n = list(disc.n) + [1] * (3 - prob.dim)
    p, dim, N = prob.p, prob.dim, disc.N
    W = 2 * p + 1
    n_off = W ** dim
    assert S.shape == (n_off, N)
    scale = np.abs(S).max()
    rows = np.arange(N)
    coords = np.stack([rows % n[0], (rows // n[0]) % n[1], rows // (n[0] * n[1])], axis=1)
    for o in range(n_off):
        d = [(o // W ** k) % W - p for k in range(dim)] + [0] * (3 - dim)
        off = d[0] + d[1] * n[0] + d[2] * n[0] * n[1]
        om = n_off - 1 - o
        inside = np.all((coords + np.array(d) >= 0) & (coords + np.array(d) < np.array(n)), axis=1)
        q = rows + off
        inq = (q >= 0) & (q < N)
        # a coupling exists only if the row it reaches is in range and sees the mirror
        assert not np.any(inside & ~inq)
        mirrored = np.zeros(N)
        mirrored[inq] = S[om, q[inq]]
        assert np.abs(S[o] - mirrored).max() <= 1e-14 * scale, o
        assert np.all(S[o][~inside] == 0.0) and np.all(mirrored[~inside] == 0.0)


def test_mirror_index_reverses_every_digit():
    """The offset index o = sum_k (delta_k + p) W^k has its mirror (-delta) at
    W^d - 1 - o, and the centre (delta = 0) at (W^d - 1) / 2."""
    for dim, p in itertools.product((2, 3), (1, 2, 5)):
        W = 2 * p + 1
        for d in itertools.product(range(-p, p + 1), repeat=dim):
            o = sum((d[k] + p) * W ** k for k in range(dim))
            om = sum((-d[k] + p) * W ** k for k in range(dim))
            assert om == W ** dim - 1 - o
        assert sum(p * W ** k for k in range(dim)) == (W ** dim - 1) // 2
