"""Parity of the ADI preconditioners (two variables: Section 4.2, Algorithm 2;
three variables: Section 5.2, Algorithm 4) through the C ABI with the
oracle's ADI on the same inputs and parameters.

Tolerances: in FP64 both sides run J contracting Douglas iterations on the
same pencils; the library solves the shifted systems by banded Cholesky, the
oracle by dense LU, so entries agree to rounding, 1e-12 of max|z|. The FP32
variant keeps factors, scratch and arithmetic in FP32: 1e-5 relative (a few
hundred FP32 ulps over J iterations of n-step recurrences)."""
import numpy as np
import pytest

import synth
from oracle import adi, assemble, pcg
from gpu_util import need_gpu, to_dev, rel, maxrel

pytestmark = pytest.mark.gpu

CASES = [
    ("ragged-p3", (37, 9, 11), 3, [0.05, -0.03, 0.02], [0.7, 25.0, 3.0]),
    ("one-iteration", (5, 40, 6), 2, None, [2.0]),
    ("p1", (33, 34, 35), 1, None, [1.0, 50.0]),
    ("p4-long-dir3", (8, 7, 70), 4, None, [3.0, 0.5, 80.0, 9.0]),
]


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _patch(prob):
    from paper_1602_01636_gb300 import igafd
    return igafd.Patch.from_problem(prob, stencil=False)


@pytest.mark.parametrize("name,n,p,amp,omega", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_adi_matches_oracle(torch, name, n, p, amp, omega, dtype):
    prob = synth.Problem(3, n, p, amp)
    disc = assemble.Discretization.from_problem(prob)
    pens = [disc.pencil(k) for k in range(3)]
    r = synth.random_vector(disc.N, 21)
    z_ref = adi.ADI3D(pens, omega=np.array(omega)).apply(r)
    patch = _patch(prob)
    patch.adi_setup(omega, dtype)
    z = patch.apply_prec_adi(to_dev(r)).cpu().numpy()
    if dtype == "fp64":
        assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()
    else:
        assert np.linalg.norm(z - z_ref) <= 1e-5 * np.linalg.norm(z_ref)
        assert maxrel(z, z_ref) <= 1e-5


def test_adi_greedy_parameters_and_apply(torch):
    """The library's greedy parameters meet rho_J <= eps on the oracle's own
    spectra, start where the oracle starts, and the apply with them matches
    the oracle's ADI with the same parameters."""
    prob = synth.Problem(3, (12, 10, 14), 3, [0.04, 0.02, -0.03])
    disc = assemble.Discretization.from_problem(prob)
    pens = [disc.pencil(k) for k in range(3)]
    lams = [adi.pencil_spectrum(K, M) for K, M in pens]
    patch = _patch(prob)
    for eps in (0.1, 1e-6):
        w = patch.adi_parameters(eps)
        w_ref = adi.greedy_parameters_3d(lams, eps)
        assert abs(w[0] - w_ref[0]) <= 1e-10 * w_ref[0]
        assert abs(len(w) - len(w_ref)) <= 1
        assert adi.rho_3d(w, lams) <= eps * (1 + 1e-9)
    patch.adi_setup(w, "fp64")
    r = synth.random_vector(disc.N, 4)
    z = patch.apply_prec_adi(to_dev(r)).cpu().numpy()
    z_ref = adi.ADI3D(pens, omega=w).apply(r)
    assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()


def test_adi_full_size_deformed_cube(torch):
    """The 3D deformed cube at n = 128, p = 3 with the greedy parameters for
    eps = 0.1: the whole FP64 apply against the oracle."""
    prob = synth.Problem(3, 128, 3, synth.deformation_amplitudes(0))
    disc = assemble.Discretization.from_problem(prob)
    pens = [disc.pencil(k) for k in range(3)]
    patch = _patch(prob)
    w = patch.adi_parameters(0.1)
    patch.adi_setup(w, "fp64")
    r = synth.random_vector(disc.N, 9)
    z = patch.apply_prec_adi(to_dev(r)).cpu().numpy()
    z_ref = adi.ADI3D(pens, omega=w).apply(r)
    assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()


def test_pcg_with_adi_preconditioner(torch):
    """PCG with P_J (igafd_pcg_solve, prec_dtype IGAFD_ADI, flexible beta):
    fixed-k iterates equal the oracle's PCG with the oracle's ADI (same
    parameters) to 1e-10; the converged solution matches the direct solve;
    Theorem 1 keeps the iteration count near the FD's; apply_prec with the
    ADI dtype is the ADI apply."""
    from paper_1602_01636_gb300 import igafd
    prob = synth.Problem(3, (14, 11, 12), 3, [0.06, -0.04, 0.03])
    disc = assemble.Discretization.from_problem(prob)
    pens = [disc.pencil(k) for k in range(3)]
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
    b = synth.random_rhs(disc.N, 5)
    patch = igafd.Patch.from_problem(prob)
    w = patch.adi_parameters(0.1)
    patch.adi_setup(w, "fp64")
    P_J = adi.ADI3D(pens, omega=w)
    k = 6
    ro = pcg.pcg(lambda v: A @ v, b, P_J.apply, fixed_iters=k, flexible=True)
    x, info = patch.pcg(to_dev(b), tol=0.0, max_iter=k, dtype="adi")
    assert info.iterations == k
    assert rel(x.cpu().numpy(), ro.x) <= 1e-10 and maxrel(x.cpu().numpy(), ro.x) <= 1e-10
    x, info = patch.pcg(to_dev(b), tol=1e-10, max_iter=500, dtype="adi")
    xd = np.linalg.solve(A.toarray(), b)
    assert rel(x.cpu().numpy(), xd) <= 1e-8 and maxrel(x.cpu().numpy(), xd) <= 1e-8
    _, info_fd = patch.pcg(to_dev(b), tol=1e-10, max_iter=500, dtype="fp64")
    assert info.iterations <= info_fd.iterations + 3
    r = to_dev(synth.random_vector(disc.N, 2))
    assert torch.equal(patch.apply_prec(r, dtype="adi"), patch.apply_prec_adi(r))
    # a new set-up (FP32) replaces the state the captured loop used
    patch.adi_setup(w, "fp32")
    x32, info32 = patch.pcg(to_dev(b), tol=1e-10, max_iter=500, dtype="adi")
    assert rel(x32.cpu().numpy(), xd) <= 1e-8 and maxrel(x32.cpu().numpy(), xd) <= 1e-8


CASES_2D = [
    ("2d-ragged-p3", (70, 45), 3, [0.7, 25.0, 3.0, 400.0]),
    ("2d-one-iteration", (33, 40), 2, [2.0]),
    ("2d-p1-long", (9, 100), 1, [1.0, 50.0]),
    ("2d-p4", (40, 8), 4, [3.0, 0.5, 80.0]),
]


@pytest.mark.parametrize("name,n,p,omega", CASES_2D, ids=[c[0] for c in CASES_2D])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_adi_2d_matches_oracle(torch, name, n, p, omega, dtype):
    """Two-variable ADI (Algorithm 2, gamma_j = omega_j). The right-hand sides
    r - (K - w M) s~ cancel and the result passes through a final M_1 solve,
    so FP64 entries agree to 1e-11 of max|z| (3e-13 observed in a CPU
    emulation of the kernels' arithmetic) and FP32 to 1e-3 in the 2-norm
    (FP32 solves with K_k + w M_k of condition up to ~1e4 here: 2.3e-4
    observed in the same emulation run in FP32)."""
    prob = synth.Problem(2, n, p)
    disc = assemble.Discretization.from_problem(prob)
    pens = [disc.pencil(k) for k in range(2)]
    r = synth.random_vector(disc.N, 21)
    z_ref = adi.ADI2D(pens, omega=np.array(omega)).apply(r)
    patch = _patch(prob)
    patch.adi_setup(omega, dtype)
    z = patch.apply_prec_adi(to_dev(r)).cpu().numpy()
    if dtype == "fp64":
        assert np.abs(z - z_ref).max() <= 1e-11 * np.abs(z_ref).max()
    else:
        assert np.linalg.norm(z - z_ref) <= 1e-3 * np.linalg.norm(z_ref)
        assert maxrel(z, z_ref) <= 1e-3


def test_adi_2d_parameters_and_pcg(torch):
    """The patch's two-variable parameters equal the oracle's (J of
    Eq. (ADIits) on the hull of the two spectra); the apply with them matches
    the oracle's Algorithm 2 with eps = 1e-8 in M-norm terms; PCG with P_J
    on a deformed 2D patch: fixed-k iterates equal the oracle's, and the
    converged solution the direct solve."""
    from paper_1602_01636_gb300 import igafd
    prob = synth.Problem(2, (30, 26), 3)
    x, y = prob.ctrl
    prob.ctrl = prob.ctrl + (0.06 * np.sin(np.pi * x) * np.sin(np.pi * y))[None]
    disc = assemble.Discretization.from_problem(prob)
    pens = [disc.pencil(k) for k in range(2)]
    patch = igafd.Patch.from_problem(prob)
    ref = adi.ADI2D(pens, eps=0.1)
    w = patch.adi_parameters(0.1)
    assert len(w) == ref.J and np.allclose(w, ref.omega, rtol=1e-9, atol=0)
    patch.adi_setup(w, "fp64")
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
    b = synth.random_rhs(disc.N, 5)
    k = 6
    ro = pcg.pcg(lambda v: A @ v, b, ref.apply, fixed_iters=k, flexible=True)
    xk, info = patch.pcg(to_dev(b), tol=0.0, max_iter=k, dtype="adi")
    assert info.iterations == k
    assert rel(xk.cpu().numpy(), ro.x) <= 1e-10 and maxrel(xk.cpu().numpy(), ro.x) <= 1e-10
    xs, info = patch.pcg(to_dev(b), tol=1e-10, max_iter=500, dtype="adi")
    xd = np.linalg.solve(A.toarray(), b)
    assert rel(xs.cpu().numpy(), xd) <= 1e-8 and maxrel(xs.cpu().numpy(), xd) <= 1e-8


def test_adi_rejects_bad_calls(torch):
    from paper_1602_01636_gb300 import igafd
    patch3 = _patch(synth.Problem(3, (6, 5, 7), 2))
    r = to_dev(np.ones(6 * 5 * 7))
    with pytest.raises(igafd.IgafdError):
        patch3.apply_prec_adi(r)                       # no set-up yet
    with pytest.raises(igafd.IgafdError):
        patch3.apply_prec(r, dtype="adi")
    with pytest.raises(igafd.IgafdError):
        patch3.adi_setup([1.0, -2.0])                  # parameters must be positive
    with pytest.raises(igafd.IgafdError):
        patch3.adi_setup([1.0], dtype="bf16")          # FP64 or FP32 only
    with pytest.raises(igafd.IgafdError):
        patch3.adi_parameters(1.5)                     # 0 < eps < 1


@pytest.mark.parametrize("groups", [1, 0])
def test_batched_solve_with_adi(torch, groups):
    """A batched solve with P_J as every member's preconditioner (the ADI
    line kernels launched per problem inside the device loop) gives the
    iterates and iteration counts of the members' single solves, bitwise,
    in one lockstep loop and in one loop per problem."""
    from paper_1602_01636_gb300 import igafd
    probs = [synth.Problem(3, (12, 10, 11), 2, [0.05, -0.03, 0.02]),
             synth.Problem(3, (9, 13, 10), 3, [-0.04, 0.02, 0.05]),
             synth.Problem(3, (11, 11, 14), 3, [0.03, 0.04, -0.02])]
    patches = []
    for pr in probs:
        patch = igafd.Patch.from_problem(pr)
        patch.adi_setup(patch.adi_parameters(0.1), "fp64")
        patches.append(patch)
    bs = [to_dev(synth.random_rhs(p.N, 30 + i)) for i, p in enumerate(patches)]
    batch = igafd.Batch(patches, tol=1e-10, max_iter=300, dtype="adi", groups=groups)
    xs, infos = batch.solve(bs)
    batch.close()
    for p, b, x, inf in zip(patches, bs, xs, infos):
        xr, ir = p.pcg(b, tol=1e-10, max_iter=300, dtype="adi")
        assert inf.status == ir.status == 0 and inf.iterations == ir.iterations
        assert torch.equal(x, xr)
    for p in patches:
        p.close()
