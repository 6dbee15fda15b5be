"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs.

Tolerances (FP64 path): the GPU and the oracle evaluate the same sums in a
different order, so entries agree to a few ulps of the largest term:
stencil 1e-13 of max|A|, products with A 1e-12 of max|y|, the FD apply
1e-11 relative (two triangular-factor eigenbases, six dense products),
PCG iterates and converged solutions 1e-10 relative. Every vector is
compared entry by entry (max|a - b| <= tol max|b|) and, where the bound was
derived for it, also in the 2-norm.
"""
import numpy as np
import pytest

import synth
from oracle import assemble, fd, pcg
from gpu_util import need_gpu, make_patch, to_dev, rel, maxrel

pytestmark = pytest.mark.gpu

CASES = [
    ("2d-ragged", lambda: synth.Problem(2, (70, 45), 3)),
    ("2d-p1", lambda: synth.Problem(2, (17, 9), 1)),
    ("3d-deformed", lambda: synth.Problem(3, (13, 9, 11), 3, [0.05, -0.03, 0.02])),
    ("3d-p2", lambda: synth.Problem(3, (10, 12, 7), 2, [0.08, 0.02, -0.04])),
    ("3d-p4", lambda: synth.Problem(3, (9, 8, 10), 4, [-0.03, 0.04, 0.01])),
    ("3d-p5", lambda: synth.Problem(3, (8, 7, 9), 5, [0.02, -0.03, 0.04])),
]


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request, torch):
    prob = request.param[1]()
    disc = assemble.Discretization.from_problem(prob)
    S = disc.assemble_stencil()
    patch = make_patch(prob)
    yield prob, disc, S, patch
    patch.close()


def test_sizes(case):
    prob, disc, S, patch = case
    assert patch.n == tuple(disc.n)
    assert patch.info.n_offsets == S.shape[0]


def test_eigen_invariants_and_values(case):
    prob, disc, S, patch = case
    for k in range(prob.dim):
        K, M = disc.pencil(k)
        D, U = patch.eigen(k)
        Do, _ = fd.generalized_eig(K, M)
        assert np.abs(D - Do).max() <= 1e-12 * Do.max()
        assert np.abs(U.T @ M @ U - np.eye(len(D))).max() <= 1e-12
        assert np.abs(U.T @ K @ U - np.diag(D)).max() <= 1e-12 * D.max()


def test_eigen_routes(case):
    """Both eigen routes (FP32 Jacobi + FP64 refinement, and FP64 Jacobi) meet
    the oracle's invariants; a re-setup of P is bitwise reproducible."""
    prob, disc, S, patch = case
    assert list(patch.info.eig_refined)[:prob.dim] == [1] * prob.dim
    fast = [patch.eigen(k) for k in range(prob.dim)]
    patch.setup_prec()
    for k in range(prob.dim):
        D, U = patch.eigen(k)
        assert np.array_equal(D, fast[k][0]) and np.array_equal(U, fast[k][1])
    patch.set_eig_route(1)
    patch.setup_prec()
    try:
        assert list(patch.info.eig_refined)[:prob.dim] == [0] * prob.dim
        for k in range(prob.dim):
            K, M = disc.pencil(k)
            D, U = patch.eigen(k)
            Do, _ = fd.generalized_eig(K, M)
            assert np.abs(D - Do).max() <= 1e-12 * Do.max()
            assert np.abs(U.T @ M @ U - np.eye(len(D))).max() <= 1e-12
            assert np.abs(U.T @ K @ U - np.diag(D)).max() <= 1e-12 * D.max()
            assert np.abs(D - fast[k][0]).max() <= 1e-12 * D.max()
    finally:
        patch.set_eig_route(0)
        patch.setup_prec()
    for k in range(prob.dim):
        D, U = patch.eigen(k)
        assert np.array_equal(D, fast[k][0]) and np.array_equal(U, fast[k][1])


def test_stencil_entries(case):
    prob, disc, S, patch = case
    Sg = patch.stencil().cpu().numpy()
    assert np.abs(Sg - S).max() <= 1e-13 * np.abs(S).max()


def test_apply_A(case):
    prob, disc, S, patch = case
    x = synth.random_vector(disc.N, 11)
    y = patch.apply_A(to_dev(x)).cpu().numpy()
    yo = assemble.apply_stencil(disc, S, x)
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


def test_apply_prec_fp64(case):
    prob, disc, S, patch = case
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    r = synth.random_vector(disc.N, 12)
    z = patch.apply_prec(to_dev(r)).cpu().numpy()
    zo = F.apply(r)
    assert rel(z, zo) <= 1e-11 and maxrel(z, zo) <= 1e-11


def test_apply_prec_fp32(case):
    prob, disc, S, patch = case
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    r = synth.random_vector(disc.N, 13)
    z = patch.apply_prec(to_dev(r), dtype="fp32").cpu().numpy()
    zo = F.apply(r)
    assert rel(z, zo) <= 1e-4 and maxrel(z, zo) <= 1e-4


TC_TOL = {"tf32": 1e-2, "fp16": 1e-2, "bf16": 4e-2}


@pytest.mark.parametrize("dtype", ["tf32", "bf16", "fp16"])
def test_apply_prec_tensor_core(case, dtype):
    """tcgen05 FD: operands rounded to the dtype, FP32 accumulation; the
    error is a few operand roundings (2^-11 for TF32/FP16, 2^-8 for BF16)
    per product, six products."""
    prob, disc, S, patch = case
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    r = synth.random_vector(disc.N, 14)
    z = patch.apply_prec(to_dev(r), dtype=dtype).cpu().numpy()
    zo = F.apply(r)
    err, emax = rel(z, zo), maxrel(z, zo)
    print(f"{dtype} FD rel err {err:.2e} entry-wise {emax:.2e}")
    assert err <= TC_TOL[dtype] and emax <= TC_TOL[dtype]


@pytest.mark.parametrize("dtype", ["tf32", "bf16"])
def test_apply_prec_fused_matches_per_mode(case, dtype):
    """The fused three-kernel FD (two mode products per kernel, the
    intermediate kept on chip) and the one-kernel-per-mode-product FD round
    the same operands to the same type; they differ only in the order of the
    backward products, so they agree to a few operand roundings, and each
    meets the oracle bound."""
    prob, disc, S, patch = case
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    r = synth.random_vector(disc.N, 15)
    zo = F.apply(r)
    from paper_1602_01636_gb300 import igafd
    rd = to_dev(r)
    patch.set_fd_fused(0)
    l0 = igafd.kernel_launches()
    z_pass = patch.apply_prec(rd, dtype=dtype).cpu().numpy()
    l1 = igafd.kernel_launches()
    patch.set_fd_fused(1)
    z_fused = patch.apply_prec(rd, dtype=dtype).cpu().numpy()
    l2 = igafd.kernel_launches()
    # one kernel per mode product, against one per pair of them
    assert (l1 - l0, l2 - l1) == (2 * prob.dim, prob.dim)
    e_pass, e_fused, e_mut = maxrel(z_pass, zo), maxrel(z_fused, zo), maxrel(z_fused, z_pass)
    print(f"{dtype} entry-wise: per-mode {e_pass:.2e} fused {e_fused:.2e} mutual {e_mut:.2e}")
    assert e_pass <= TC_TOL[dtype] and e_fused <= TC_TOL[dtype]
    assert e_mut <= TC_TOL[dtype]
    assert rel(z_pass, zo) <= TC_TOL[dtype] and rel(z_fused, zo) <= TC_TOL[dtype]


@pytest.mark.parametrize("dtype", ["tf32", "bf16", "fp16"])
def test_pcg_tensor_core_preconditioner(case, dtype):
    prob, disc, S, patch = case
    A = assemble.stencil_to_csr(disc, S)
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    b = synth.random_rhs(disc.N, 8)
    ro = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-13, max_iter=500)
    r8 = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-8, max_iter=500)
    x, info = patch.pcg(to_dev(b), tol=1e-8, max_iter=500, dtype=dtype)
    assert info.status == 0
    # at most two more iterations than the exact preconditioner; when P = A
    # (identity map) the exact one needs a single step and an inexact FD with
    # relative error eps needs about log(1e-8)/log(eps) steps instead
    bound = r8.iters + 2 if r8.iters > 2 else 8
    assert info.iterations <= bound, (info.iterations, r8.iters)
    xg = x.cpu().numpy()
    assert rel(xg, ro.x) <= 1e-7 and maxrel(xg, ro.x) <= 1e-7


def test_rhs_sine(case):
    prob, disc, S, patch = case
    f = {2: lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y),
         3: lambda x, y, z: 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)}
    bo = disc.assemble_rhs(f[prob.dim])
    b = patch.load_rhs_sine().cpu().numpy()
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()


def test_quad_points_and_general_rhs(case):
    """igafd_quad_points gives the oracle's physical quadrature points (the map
    F on the tensor Gauss grid), and igafd_load_rhs with a load sampled there
    gives the oracle's right-hand side for that load (not a manufactured one)."""
    prob, disc, S, patch = case
    torch = pytest.importorskip("torch")
    X = patch.quad_points()
    pts = [disc.qz[k].ravel() for k in range(prob.dim)]
    Fo, _ = disc.geo.eval_grid(pts)                  # [c][q_d]..[q_1], direction 1 fastest
    Fo = Fo.reshape(prob.dim, -1)
    assert X.shape == Fo.shape
    assert np.abs(X.cpu().numpy() - Fo).max() <= 1e-14
    if prob.dim == 2:
        f_np = lambda x, y: np.exp(x) * np.cos(3.0 * y) + 2.0 * x * y
        f_t = lambda x, y: torch.exp(x) * torch.cos(3.0 * y) + 2.0 * x * y
    else:
        f_np = lambda x, y, z: np.exp(x) * np.cos(3.0 * y) + 2.0 * x * y * z - z
        f_t = lambda x, y, z: torch.exp(x) * torch.cos(3.0 * y) + 2.0 * x * y * z - z
    fq = f_t(*[X[c] for c in range(prob.dim)]).contiguous()
    b = patch.load_rhs(fq).cpu().numpy()
    bo = disc.assemble_rhs(f_np)
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()


def test_pcg_fixed_iterates(case):
    """x_k after exactly k iterations (no stopping test) equals the oracle's."""
    prob, disc, S, patch = case
    A = assemble.stencil_to_csr(disc, S)
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    b = synth.random_rhs(disc.N, 5)
    k = 6
    ro = pcg.pcg(lambda v: A @ v, b, F.apply, fixed_iters=k)
    x, info = patch.pcg(to_dev(b), tol=0.0, max_iter=k)
    assert info.iterations == k
    xg = x.cpu().numpy()
    assert rel(xg, ro.x) <= 1e-10 and maxrel(xg, ro.x) <= 1e-10


@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_fixed_iterates_periodic_true_residual(case, flexible):
    """The periodic true residual r = b - A x (every 3 iterations here, so it
    replaces the recurrence residual at k = 3 and 6 of 8) gives the oracle's
    x_8 on both sides, with Fletcher-Reeves and with the flexible beta (whose
    (r, z_old) must then come from the recomputed residual); a wrong
    predicate on the iteration counter or a stale scalar would move x_8."""
    prob, disc, S, patch = case
    A = assemble.stencil_to_csr(disc, S)
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    b = synth.random_rhs(disc.N, 15)
    k = 8
    ro = pcg.pcg(lambda v: A @ v, b, F.apply, fixed_iters=k, true_every=3, flexible=flexible)
    x, info = patch.pcg(to_dev(b), tol=0.0, max_iter=k, true_every=3, flexible=flexible)
    assert info.iterations == k
    xg = x.cpu().numpy()
    assert rel(xg, ro.x) <= 1e-10 and maxrel(xg, ro.x) <= 1e-10
    # on a deformed geometry the iterate without the recomputation differs
    # from this one (so the pin catches a predicate that never fires); with
    # the identity map P = A and the iterates stop moving after one step
    if prob.amplitudes is not None:
        rn = pcg.pcg(lambda v: A @ v, b, F.apply, fixed_iters=k, true_every=0, flexible=flexible)
        assert not np.array_equal(rn.x, ro.x)


def test_pcg_converged_solution(case):
    prob, disc, S, patch = case
    A = assemble.stencil_to_csr(disc, S)
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    b = synth.random_rhs(disc.N, 6)
    # 1e-12 is above the rounding floor of both solvers up to p = 5
    ro = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-12, max_iter=500)
    assert ro.converged
    x, info = patch.pcg(to_dev(b), tol=1e-12, max_iter=500)
    assert info.status == 0 and info.true_relres <= 1e-12
    xg = x.cpu().numpy()
    assert rel(xg, ro.x) <= 1e-10 and maxrel(xg, ro.x) <= 1e-10
    # the iteration count equals the oracle's at the same tolerance
    r8 = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-8, max_iter=500)
    _, i8 = patch.pcg(to_dev(b), tol=1e-8, max_iter=500)
    assert i8.iterations == r8.iters


def test_pcg_fp32_preconditioner(case):
    prob, disc, S, patch = case
    A = assemble.stencil_to_csr(disc, S)
    F = fd.FD([disc.pencil(k) for k in range(prob.dim)])
    b = synth.random_rhs(disc.N, 7)
    ro = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-13, max_iter=500)
    r8 = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-8, max_iter=500)
    x, info = patch.pcg(to_dev(b), tol=1e-8, max_iter=500, dtype="fp32")
    assert info.status == 0
    assert info.iterations <= r8.iters + 2
    xg = x.cpu().numpy()
    assert rel(xg, ro.x) <= 1e-7 and maxrel(xg, ro.x) <= 1e-7


def test_identity_map_one_iteration(torch):
    """Config-1 workload: 2D unit square, n = 64, p = 3: P = A, one iteration."""
    prob = synth.unit_square(64, 3)
    disc = assemble.Discretization.from_problem(prob)
    patch = make_patch(prob)
    b = patch.load_rhs_sine()
    x, info = patch.pcg(b, tol=1e-8)
    assert info.status == 0 and info.iterations == 1
    S = disc.assemble_stencil()
    A = assemble.stencil_to_csr(disc, S)
    bo = disc.assemble_rhs(lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y))
    xo = np.linalg.solve(A.toarray(), bo)
    assert rel(x.cpu().numpy(), xo) <= 1e-10 and maxrel(x.cpu().numpy(), xo) <= 1e-10
    patch.close()


def test_zero_rhs_and_errors(torch):
    from paper_1602_01636_gb300 import igafd
    prob = synth.Problem(3, (8, 7, 9), 2, [0.02, 0.01, -0.02])
    patch = make_patch(prob)
    b = torch.zeros(patch.N, dtype=torch.float64, device="cuda")
    x, info = patch.pcg(b)
    assert info.status == 0 and info.iterations == 0 and float(x.abs().max()) == 0.0
    # iteration cap
    b = to_dev(synth.random_rhs(patch.N, 1))
    x, info = patch.pcg(b, tol=1e-14, max_iter=2, raise_on_error=False)
    assert info.status == igafd.ERR_NOT_CONVERGED and info.iterations == 2
    # non-finite right-hand side -> breakdown status, no trap
    b[3] = float("nan")
    x, info = patch.pcg(b, raise_on_error=False)
    assert info.status == igafd.ERR_BREAKDOWN
    patch.close()
    # folded geometry is reported at set-up
    bad = synth.Problem(3, (8, 8, 8), 2, [1.5, 1.5, 1.5])
    with pytest.raises(igafd.IgafdError) as e:
        make_patch(bad)
    assert e.value.status == igafd.ERR_FOLDED


def test_full_size_sampled(torch):
    """3D deformed cube, n = 128, p = 3 (2.1M dofs, 5.75 GB stencil): sampled
    stencil rows against the oracle's per-row assembly, the full FD apply
    against the oracle's FD, and the FP64 solve's residual on sampled rows."""
    prob = synth.deformed_cube(128, 3, seed=0)
    disc = assemble.Discretization.from_problem(prob)
    patch = make_patch(prob)
    g = synth.rng(99)
    rows = [tuple(int(v) for v in g.integers(0, 128, 3)) for _ in range(12)]
    rows += [(0, 0, 0), (127, 127, 127), (0, 64, 127), (3, 2, 1)]
    So = disc.assemble_rows(rows)
    Sg = patch.stencil()
    idx = torch.tensor([disc.row_index(i) for i in rows], device="cuda")
    Sg_rows = Sg[:, idx].T.cpu().numpy()
    del Sg
    assert np.abs(Sg_rows - So).max() <= 1e-13 * np.abs(So).max()
    F = fd.FD([disc.pencil(k) for k in range(3)])
    r = synth.random_vector(disc.N, 21)
    zo = F.apply(r)
    z = patch.apply_prec(to_dev(r)).cpu().numpy()
    assert rel(z, zo) <= 1e-11 and maxrel(z, zo) <= 1e-11
    for dt, tol in TC_TOL.items():
        zt = patch.apply_prec(to_dev(r), dtype=dt).cpu().numpy()
        print(f"n=128 {dt} FD: 2-norm {rel(zt, zo):.2e} entry-wise {maxrel(zt, zo):.2e}")
        assert rel(zt, zo) <= tol and maxrel(zt, zo) <= tol
    b = synth.random_rhs(disc.N, 22)
    x, info = patch.pcg(to_dev(b), tol=1e-8)
    assert info.status == 0 and info.true_relres <= 1e-8
    xh = x.cpu().numpy().reshape(128, 128, 128)
    res = []
    for r_i, i in enumerate(rows):
        acc = 0.0
        for o in range(343):
            d1, d2, d3 = o % 7 - 3, (o // 7) % 7 - 3, o // 49 - 3
            j = (i[0] + d1, i[1] + d2, i[2] + d3)
            if all(0 <= j[k] < 128 for k in range(3)):
                acc += So[r_i, o] * xh[j[2], j[1], j[0]]
        res.append(b[disc.row_index(i)] - acc)
    assert np.abs(res).max() <= 1e-6 * np.abs(b).max()
    patch.close()


@pytest.mark.parametrize("dtype", ["tf32", "bf16"])
def test_fd_n128_kernels(torch, dtype):
    """Every n_k = 128 in 3D takes the compile-time-sized fused kernels (three
    launches): they meet the oracle bound and agree with the per-mode path
    (p = 1 keeps the stencil small; the FD depends only on the pencils)."""
    from paper_1602_01636_gb300 import igafd
    prob = synth.deformed_cube(128, 1, seed=0)
    disc = assemble.Discretization.from_problem(prob)
    patch = make_patch(prob)
    F = fd.FD([disc.pencil(k) for k in range(3)])
    r = synth.random_vector(disc.N, 31)
    zo = F.apply(r)
    rd = to_dev(r)
    patch.set_fd_fused(0)
    z_pass = patch.apply_prec(rd, dtype=dtype).cpu().numpy()
    patch.set_fd_fused(1)
    l0 = igafd.kernel_launches()
    z = patch.apply_prec(rd, dtype=dtype).cpu().numpy()
    assert igafd.kernel_launches() - l0 == 3
    e, e_pass, e_mut = maxrel(z, zo), maxrel(z_pass, zo), maxrel(z, z_pass)
    print(f"n=128 {dtype} entry-wise: fused {e:.2e} per-mode {e_pass:.2e} mutual {e_mut:.2e}")
    assert e <= TC_TOL[dtype] and e_pass <= TC_TOL[dtype] and e_mut <= TC_TOL[dtype]
    assert rel(z, zo) <= TC_TOL[dtype] and rel(z_pass, zo) <= TC_TOL[dtype]
    # a second call on the same input gives the same bits
    z2 = patch.apply_prec(rd, dtype=dtype).cpu().numpy()
    assert np.array_equal(z, z2)
    patch.close()


def test_batched_solve_matches_single_solves(torch):
    """Config-4-like batch (uneven n per axis, p in {2,3,4}, a_k ~ U(-0.1, 0.1),
    N(0,1) right-hand sides): one batched solve gives bitwise the iterates
    and iteration counts of one-by-one solves, for the FP64 and a tensor-core
    preconditioner."""
    from paper_1602_01636_gb300 import igafd
    g = synth.rng(404)
    probs = []
    for i in range(5):
        n = tuple(int(v) for v in g.integers(10, 24, 3))
        p = int(g.integers(2, 5))
        probs.append(synth.Problem(3, n, p, g.uniform(-0.1, 0.1, 3)))
    probs.append(synth.Problem(2, (33, 17), 3))
    patches = [make_patch(pr) for pr in probs]
    bs = [to_dev(synth.random_rhs(p.N, 50 + i)) for i, p in enumerate(patches)]
    for dt in ("fp64", "bf16"):
        xs, infos = igafd.batch_pcg(patches, bs, tol=1e-10, dtype=dt)
        for p, b, x, inf in zip(patches, bs, xs, infos):
            xr, ir = p.pcg(b, tol=1e-10, dtype=dt)
            assert inf.status == 0 and inf.iterations == ir.iterations
            assert torch.equal(x, xr)
    # and against the oracle for one member
    disc = assemble.Discretization.from_problem(probs[0])
    A = assemble.stencil_to_csr(disc, disc.assemble_stencil())
    F = fd.FD([disc.pencil(k) for k in range(3)])
    ro = pcg.pcg(lambda v: A @ v, bs[0].cpu().numpy(), F.apply, tol=1e-13, max_iter=500)
    xs, _ = igafd.batch_pcg(patches, bs, tol=1e-12, dtype="fp64")
    assert rel(xs[0].cpu().numpy(), ro.x) <= 1e-10 and maxrel(xs[0].cpu().numpy(), ro.x) <= 1e-10
    for p in patches:
        p.close()


@pytest.mark.parametrize("groups,ppl", [(1, 0), (3, 0), (0, 0), (0, 2), (3, 5)])
def test_batched_solve_device_loop(torch, groups, ppl):
    """The device-driven batched loop against single solves, bitwise: a
    periodic true residual every 3 iterations with the flexible beta (TF32
    FD), one member on the per-mode tensor-core FD (its own launches inside the
    loop), one with b = 0 (finished before the loop), a reused batch object
    (two solves, the same bits), and an iteration cap that stops one member
    (NOT_CONVERGED) while the others converge; in one group, in three
    concurrently looping groups and in one loop per problem, each with the
    whole loop in one graph launch or a few passes per launch (relaunched by
    the host). With one group a pass of the loop is a fixed number of
    launches, not one set per problem."""
    from paper_1602_01636_gb300 import igafd
    g = synth.rng(505)
    probs = [synth.Problem(3, tuple(int(v) for v in g.integers(9, 20, 3)), int(g.integers(2, 5)),
                           g.uniform(-0.05, 0.05, 3)) for _ in range(6)]
    probs.append(synth.Problem(2, (40, 23), 2))
    patches = [make_patch(pr) for pr in probs]
    patches[1].set_fd_fused(0)                    # per-mode FD: launched on its own
    bs = [to_dev(synth.random_rhs(p.N, 70 + i)) for i, p in enumerate(patches)]
    bs[3].zero_()
    opts = dict(tol=1e-10, dtype="tf32", flexible=True, true_every=3)
    batch = igafd.Batch(patches, groups=groups, passes_per_launch=ppl, **opts)
    ng, of = batch.groups()
    assert ng == (groups or len(patches)) and sorted(set(of)) == list(range(ng))
    l0 = igafd.kernel_launches()
    xs1, inf1 = batch.solve(bs)
    launches = igafd.kernel_launches() - l0
    xs2, inf2 = batch.solve(bs)
    for i, (p, b) in enumerate(zip(patches, bs)):
        xr, ir = p.pcg(b, tol=1e-10, dtype="tf32", flexible=True, true_every=3)
        assert inf1[i].status == ir.status == 0 and inf1[i].iterations == ir.iterations, i
        assert torch.equal(xs1[i], xr) and torch.equal(xs2[i], xr), i
        assert inf1[i].true_relres == ir.true_relres and inf1[i].relres == ir.relres, i
    assert inf1[3].iterations == 0 and float(xs1[3].abs().max()) == 0.0
    # fewer launches than one-by-one would take (7 problems x ~8 kernels per iteration)
    its = max(i.iterations for i in inf1)
    if groups == 1:
        assert launches < 7 * 8 * its, (launches, its)
    for gi in range(ng):                         # one record per pass of each loop
        log = batch.pass_log(gi)
        members = [i for i in range(len(patches)) if of[i] == gi]
        assert len(log["dur_us"]) >= max(inf1[i].iterations for i in members)
        assert (log["dur_us"] > 0).all() and log["active"][0] <= len(members)
    batch.close()
    # an iteration cap that only some members meet
    capped = igafd.Batch(patches, tol=1e-12, max_iter=6, dtype="fp64", groups=groups,
                         passes_per_launch=ppl)
    xs, infs = capped.solve(bs)
    for i, (p, b) in enumerate(zip(patches, bs)):
        xr, ir = p.pcg(b, tol=1e-12, max_iter=6, dtype="fp64", raise_on_error=False)
        assert infs[i].status == ir.status and infs[i].iterations == ir.iterations, i
        assert torch.equal(xs[i], xr), i
    assert any(i.status == igafd.ERR_NOT_CONVERGED for i in infs)
    capped.close()
    for p in patches:
        p.close()


def test_autotune_fd_form(torch):
    """The autotuner times the fused and the per-mode tensor-core FD for TF32
    and BF16 and keeps one per type; the apply then launches three kernels
    (fused) or six (per mode), and its result meets the oracle bound."""
    from paper_1602_01636_gb300 import igafd
    prob = synth.Problem(3, (40, 33, 37), 3, [0.05, 0.02, -0.03])
    patch = make_patch(prob)
    disc = assemble.Discretization.from_problem(prob)
    F = fd.FD([disc.pencil(k) for k in range(3)])
    r = synth.random_vector(disc.N, 78)
    zo = F.apply(r)
    patch.autotune(force=True)
    forms = list(patch.info.fd_fused)
    assert forms[0] in (0, 1) and forms[1] in (0, 1) and forms[2] == 0
    for i, dt in enumerate(["tf32", "bf16"]):
        l0 = igafd.kernel_launches()
        z = patch.apply_prec(to_dev(r), dtype=dt).cpu().numpy()
        assert igafd.kernel_launches() - l0 == (3 if forms[i] else 6)
        assert rel(z, zo) <= TC_TOL[dt] and maxrel(z, zo) <= TC_TOL[dt]
    patch.set_fd_fused(1)          # an explicit choice replaces the tuned one
    assert list(patch.query().fd_fused)[:2] == [1, 1]
    patch.close()


@pytest.mark.parametrize("n,p", [((40, 33, 37), 3), ((150, 24, 20), 2)])
def test_fd_tile_shapes_match_oracle(torch, n, p):
    """Every tile shape of the tensor-core FD (rows per CTA 128 or 64, one or
    two column tiles, two or three K stages where some n_k > 128, the fused
    pencil kernel's 128 or 64 columns per CTA) meets the oracle bound entry by
    entry for TF32, BF16 and FP16; the autotuner keeps one of them."""
    from paper_1602_01636_gb300 import igafd
    prob = synth.Problem(3, n, p, [0.04, -0.02, 0.03])
    patch = make_patch(prob)
    disc = assemble.Discretization.from_problem(prob)
    F = fd.FD([disc.pencil(k) for k in range(3)])
    r = synth.random_vector(disc.N, 91)
    zo = F.apply(r)
    rd = to_dev(r)
    fusable = max(n) <= 128
    checked = 0
    for dt in ("tf32", "bf16", "fp16"):
        for m in (128, 64):
            for nd in (1, 2):
                for stg in (2, 3):
                    try:
                        patch.set_fd_tile(dt, (m, nd, stg, 128))
                    except igafd.IgafdError:
                        assert stg == 3      # a third stage of 256 TF32 columns does not fit
                        continue
                    patch.set_fd_fused(0)
                    z = patch.apply_prec(rd, dtype=dt).cpu().numpy()
                    assert maxrel(z, zo) <= TC_TOL[dt], (dt, m, nd, stg)
                    checked += 1
        if fusable and dt != "fp16":
            for pm in (128, 64):
                patch.set_fd_tile(dt, (128, 1, 2, pm))
                patch.set_fd_fused(1)
                z = patch.apply_prec(rd, dtype=dt).cpu().numpy()
                assert maxrel(z, zo) <= TC_TOL[dt], (dt, "fused", pm)
                checked += 1
    assert checked >= 20
    with pytest.raises(igafd.IgafdError):
        patch.set_fd_tile("tf32", (96, 1, 2, 128))
    patch.autotune(force=True)
    for dt in ("tf32", "bf16", "fp16"):
        t = patch.fd_tile(dt)
        assert t[0] in (64, 128) and t[1] in (1, 2) and t[2] in (2, 3) and t[3] in (64, 128)
        z = patch.apply_prec(rd, dtype=dt).cpu().numpy()
        assert maxrel(z, zo) <= TC_TOL[dt]
    print("autotuned tiles", [patch.fd_tile(dt) for dt in ("tf32", "bf16", "fp16")],
          "fused", list(patch.info.fd_fused))
    patch.close()


def test_autotune_picks_a_candidate_and_every_depth_agrees(torch):
    """The autotuner keeps one of the measured configurations; every ring
    depth and both row counts per thread give bitwise the same product with A
    (and the oracle's, to tolerance)."""
    prob = synth.Problem(3, (40, 33, 37), 3, [0.05, 0.02, -0.03])
    patch = make_patch(prob)
    x = to_dev(synth.random_vector(patch.N, 77))
    y0 = patch.apply_A(x)
    assert patch.autotune(force=True) in (3, 4, 6)
    assert patch.info.stencil_rows in (1, 2)
    for rows in (1, 2):
        patch.set_stencil_rows(rows)
        for st in (3, 4, 6):
            patch.set_stencil_stages(st)
            assert (patch.info.stencil_stages, patch.info.stencil_rows) == (st, rows)
            assert torch.equal(patch.apply_A(x), y0)
    disc = assemble.Discretization.from_problem(prob)
    yo = assemble.apply_stencil(disc, disc.assemble_stencil(), x.cpu().numpy())
    assert np.abs(y0.cpu().numpy() - yo).max() <= 1e-12 * np.abs(yo).max()
    from paper_1602_01636_gb300 import igafd
    with pytest.raises(igafd.IgafdError):
        patch.set_stencil_stages(5)
    with pytest.raises(igafd.IgafdError):
        patch.set_stencil_rows(3)
    patch.close()


def test_batch_grouping_and_argument_errors(torch):
    """Grouping arguments: more groups than problems gives one per problem,
    negative counts and an out-of-range pass record are rejected, and the
    groups hold problems of like size (consecutive in the order of the
    stencil work of an iteration)."""
    import ctypes as C
    from paper_1602_01636_gb300 import igafd
    g = synth.rng(606)
    probs = [synth.Problem(3, tuple(int(v) for v in g.integers(9, 18, 3)), int(g.integers(2, 4)),
                           g.uniform(-0.05, 0.05, 3)) for _ in range(5)]
    patches = [make_patch(pr) for pr in probs]
    batch = igafd.Batch(patches, groups=9)
    ng, of = batch.groups()
    assert ng == 5 and sorted(of) == list(range(5))
    batch.close()
    batch = igafd.Batch(patches, groups=2)
    ng, of = batch.groups()
    work = [p.N * (2 * p.info.p + 1) ** 3 for p in patches]
    order = sorted(range(5), key=lambda i: -work[i])
    assert ng == 2 and [of[i] for i in order] == sorted(of[i] for i in order)
    n = C.c_int()
    st = igafd.lib().igafd_batch_pass_log(batch.h, 2, 0, None, None, None, C.byref(n))
    assert st == igafd.ERR_ARG
    batch.close()
    for kw in (dict(groups=-1), dict(passes_per_launch=-1)):
        with pytest.raises(igafd.IgafdError) as e:
            igafd.Batch(patches, **kw)
        assert e.value.status == igafd.ERR_ARG
    for p in patches:
        p.close()


def test_probed_peaks_are_plausible(torch):
    """igafd_probe_peaks: the FP64 FMA rate lies near the pipe's unit count
    (152 SMs x 2 FMA/clk at the SM clock), the BF16 tensor rate near the
    measured cuBLAS BF16 rate, and TF32 below BF16 (each MMA step carries half
    the K of a BF16 one)."""
    import json
    import os
    from paper_1602_01636_gb300 import igafd
    pk = igafd.probe_peaks(0)
    derived = 152 * 2 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
    assert 0.5 * derived <= pk["fp64_tflops"] <= 1.1 * derived, pk
    assert 0 < pk["tf32_tflops"] < pk["bf16_tflops"], pk
    path = os.path.join(os.path.dirname(__file__), "..", "MEASURED_PEAKS.json")
    if os.path.exists(path):
        bf16 = json.load(open(path))["bf16_tflops"]
        assert 0.5 * bf16 <= pk["bf16_tflops"] <= 1.5 * bf16, (pk, bf16)
    print("probed peaks", pk)
