"""The stiffness stencil stored by its symmetry (IGAFD_SETUP_HALF_STENCIL,
A_ij = A_ji of Eq. (A)): its entries written out in the full layout, the
product A x with one and two rows per compute thread, PCG solves and batched
solves, against the oracle's assembly and against the full stencil. Cases
span ragged sizes, several tiles, p = 1..5, 2D and 3D, and directions with
fewer dofs than the stencil's reach (n_k <= 2p)."""
import numpy as np
import pytest

import synth
from oracle import assemble
from gpu_util import need_gpu, to_dev, maxrel, rel

pytestmark = pytest.mark.gpu

CASES = [
    ("2d-ragged", lambda: synth.Problem(2, (70, 45), 3)),
    ("2d-p1", lambda: synth.Problem(2, (17, 9), 1)),
    ("3d-deformed", lambda: synth.Problem(3, (13, 9, 11), 3, [0.05, -0.03, 0.02])),
    ("3d-p2-tiles", lambda: synth.Problem(3, (30, 17, 22), 2, [0.04, 0.02, -0.03])),
    ("3d-p5", lambda: synth.Problem(3, (8, 7, 9), 5, [0.02, -0.03, 0.04])),
    ("3d-narrow", lambda: synth.Problem(3, (4, 5, 3), 3, [0.03, 0.01, -0.02])),
]


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request, torch):
    from paper_1602_01636_gb300 import igafd
    prob = request.param[1]()
    disc = assemble.Discretization.from_problem(prob)
    S = disc.assemble_stencil()
    half = igafd.Patch.from_problem(prob, half_stencil=True)
    full = igafd.Patch.from_problem(prob)
    yield prob, disc, S, half, full
    half.close()
    full.close()


def test_half_layout_bytes_and_entries(case):
    prob, disc, S, half, full = case
    n_off = S.shape[0]
    assert half.info.stencil_half == 1 and full.info.stencil_half == 0
    assert half.info.stencil_bytes == (n_off + 1) // 2 * disc.N * 8
    assert full.info.stencil_bytes == n_off * disc.N * 8
    Sh = half.stencil().cpu().numpy()
    assert np.abs(Sh - S).max() <= 1e-13 * np.abs(S).max()
    # the lower offsets are the upper ones of the rows they reach: zero where
    # a coupling leaves the box, exactly as in the full layout
    Sf = full.stencil().cpu().numpy()
    assert np.array_equal(Sh == 0.0, Sf == 0.0)


def test_half_apply_A(case):
    prob, disc, S, half, full = case
    x = synth.random_vector(disc.N, 21)
    yo = assemble.apply_stencil(disc, S, x)
    for rows in ((1, 2) if prob.dim == 3 else (1,)):
        half.set_stencil_rows(rows)
        y = half.apply_A(to_dev(x)).cpu().numpy()
        assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max(), rows
        yf = full.apply_A(to_dev(x)).cpu().numpy()
        assert np.abs(y - yf).max() <= 1e-12 * np.abs(yf).max(), rows
    half.set_stencil_rows(1)


def test_half_pcg(case):
    """PCG with the half-stored A: the full stencil's iteration count (or one
    more) and its solution to 1e-10, true residual below the tolerance."""
    prob, disc, S, half, full = case
    b = to_dev(synth.random_rhs(disc.N, 22))
    xh, ih = half.pcg(b, tol=1e-10, max_iter=500)
    xf, i_f = full.pcg(b, tol=1e-10, max_iter=500)
    assert ih.status == 0 and abs(ih.iterations - i_f.iterations) <= 1
    assert ih.true_relres <= 1e-10
    assert maxrel(xh.cpu().numpy(), xf.cpu().numpy()) <= 1e-9
    assert rel(xh.cpu().numpy(), xf.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("groups", [1, 0])
def test_half_batched_matches_single(torch, groups):
    """A batch of half-stored and full patches: every member's iterates and
    iteration count are those of its own single solve, bitwise."""
    from paper_1602_01636_gb300 import igafd
    g = synth.rng(707)
    probs = [synth.Problem(3, tuple(int(v) for v in g.integers(9, 20, 3)), int(g.integers(2, 5)),
                           g.uniform(-0.05, 0.05, 3)) for _ in range(4)]
    probs.append(synth.Problem(2, (31, 26), 2))
    patches = [igafd.Patch.from_problem(pr, half_stencil=(i % 2 == 0)) for i, pr in enumerate(probs)]
    bs = [to_dev(synth.random_rhs(p.N, 80 + i)) for i, p in enumerate(patches)]
    batch = igafd.Batch(patches, tol=1e-10, dtype="bf16", groups=groups)
    xs, infos = batch.solve(bs)
    batch.close()
    for p, b, x, inf in zip(patches, bs, xs, infos):
        xr, ir = p.pcg(b, tol=1e-10, dtype="bf16")
        assert inf.status == ir.status == 0 and inf.iterations == ir.iterations
        assert torch.equal(x, xr)
    for p in patches:
        p.close()
