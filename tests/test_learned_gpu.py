"""Learned span scalings on the GPU against the oracle: features, separable
fit, scaled preconditioner, network forward/gradient; and the gain of the
trained network over the unscaled preconditioner on held-out patches."""
import numpy as np
import pytest

import synth
from oracle import assemble, fd, learned as olearned, pcg
from gpu_util import need_gpu, make_patch, to_dev, rel, maxrel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def kcase(torch):
    prob = synth.learned_workload_problem(2, n=12, p=2)
    disc = assemble.Discretization.from_problem(prob)
    patch = make_patch(prob)
    yield prob, disc, patch
    patch.close()


def test_variable_coefficient_stencil_and_solve(kcase):
    """Coarse geometry net on its own knots plus a spline coefficient."""
    prob, disc, patch = kcase
    S = disc.assemble_stencil()
    Sg = patch.stencil().cpu().numpy()
    assert np.abs(Sg - S).max() <= 1e-13 * np.abs(S).max()
    A = assemble.stencil_to_csr(disc, S)
    F = fd.FD([disc.pencil(k) for k in range(3)])
    b = synth.random_rhs(disc.N, 4)
    ro = pcg.pcg(lambda v: A @ v, b, F.apply, tol=1e-13, max_iter=800)
    x, info = patch.pcg(to_dev(b), tol=1e-12, max_iter=800)
    assert info.status == 0 and rel(x.cpu().numpy(), ro.x) <= 1e-10
    assert maxrel(x.cpu().numpy(), ro.x) <= 1e-10


def test_features_and_sepfit_match_oracle(kcase):
    prob, disc, patch = kcase
    f = patch.features().cpu().numpy()
    fo = olearned.features(disc)
    assert f.shape == fo.shape
    assert np.abs(f - fo).max() <= 1e-4 * max(1.0, np.abs(fo).max())
    lw = patch.sepfit().cpu().numpy()
    lwo = olearned.sepfit(disc)
    assert np.abs(lw - lwo).max() <= 1e-4


def test_patch_without_stencil(kcase):
    """A patch built without A gives the same features, separable fit and FD
    apply as the full patch; the calls that need A return an argument error."""
    from paper_1602_01636_gb300 import igafd
    prob, disc, patch = kcase
    g = igafd.Patch.from_problem(prob, stencil=False)
    assert g.info.stencil_bytes == 0 and patch.info.stencil_bytes > 0
    assert np.array_equal(g.features().cpu().numpy(), patch.features().cpu().numpy())
    assert np.array_equal(g.sepfit().cpu().numpy(), patch.sepfit().cpu().numpy())
    r = to_dev(synth.random_vector(disc.N, 5))
    assert np.array_equal(g.apply_prec(r).cpu().numpy(), patch.apply_prec(r).cpu().numpy())
    for call in (lambda: g.apply_A(r), lambda: g.pcg(r), lambda: g.stencil()):
        with pytest.raises(igafd.IgafdError) as e:
            call()
        assert e.value.status == igafd.ERR_ARG
    g.close()


def test_scaled_preconditioner_matches_oracle_and_affine_pin(torch):
    a = np.array([1.0, 2.0, 0.5])
    prob = synth.Problem(3, (9, 8, 10), 2)
    prob.ctrl = prob.ctrl * a[:, None, None, None]
    patch = make_patch(prob)
    disc = assemble.Discretization.from_problem(prob)
    lw = patch.sepfit()
    patch.set_scalings(lw)
    r = synth.random_vector(disc.N, 8)
    Fs = fd.FD(olearned.scaled_pencils(disc, lw.double().cpu().numpy()))
    zs = patch.apply_prec(to_dev(r)).cpu().numpy()
    assert rel(zs, Fs.apply(r)) <= 1e-10 and maxrel(zs, Fs.apply(r)) <= 1e-10
    b = to_dev(synth.random_rhs(disc.N, 9))
    # the scaled P equals A up to the float32 rounding of the log scalings
    # (~1e-7), so one iteration reaches 1e-6
    _, info = patch.pcg(b, tol=1e-6)
    assert info.status == 0 and info.iterations == 1
    patch.set_scalings(None)
    _, info0 = patch.pcg(b, tol=1e-6)
    assert info0.iterations > 3
    patch.close()


def test_fallback_when_the_scaled_solve_exceeds_the_unscaled_budget(kcase, torch):
    """Span scalings of the wrong sign (the separable fit negated and tripled)
    make P a poor model of A: the scaled solve runs out of the unscaled
    solve's iteration budget and the unscaled preconditioner's solve is
    returned, bitwise that of the plain solve. With the fit itself the scaled
    solve is kept whenever it converges within the budget."""
    from paper_1602_01636_gb300 import learned
    prob, disc, patch = kcase
    b = to_dev(synth.random_rhs(disc.N, 12))
    patch.set_scalings(None)
    x0, i0 = patch.pcg(b, tol=1e-8)
    assert i0.status == 0
    fit = patch.sepfit()
    x, info, fell_back = learned.solve_with_scalings(patch, -3.0 * fit, b, tol=1e-8,
                                                     budget=i0.iterations)
    assert fell_back and info.status == 0 and info.iterations == i0.iterations
    assert torch.equal(x, x0)
    x, info, fell_back = learned.solve_with_scalings(patch, fit, b, tol=1e-8, budget=i0.iterations)
    assert info.status == 0
    if not fell_back:
        assert info.iterations <= i0.iterations
    patch.set_scalings(None)


def test_network_forward_and_gradient_match_oracle(torch):
    from paper_1602_01636_gb300 import igafd
    g = synth.rng(5)
    params = synth.mlp_init(3) + g.normal(0, 0.05, 4738).astype(np.float32)
    norm = (np.full(6, 0.2), np.full(6, 1.3), np.array([0.5, -0.2]), np.array([1.5, 0.7]))
    net = igafd.MLP(params)
    net.set_normalization(*norm)
    X = g.normal(0, 1, (300, 6)).astype(np.float32)
    T = g.normal(0, 1, (300, 2)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    p16 = params.astype(np.float16).astype(np.float64)      # the forward pass uses FP16 weights
    Yo, _ = olearned.mlp_forward(p16, norm, X.astype(np.float64))
    assert np.abs(net.forward(Xd).cpu().numpy() - Yo).max() <= 1e-4 * max(1.0, np.abs(Yo).max())
    loss, grad = net.gradient(Xd, Td)
    lo, go = olearned.mlp_loss_grad(p16, norm, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - lo) <= 1e-4 * lo
    assert np.linalg.norm(grad - go) <= 1e-3 * np.linalg.norm(go)
    net.close()


def test_trained_network_reduces_iterations_on_held_out_patches(torch):
    """Contrast-100 coefficient on randomly deformed cubes: the network's
    span scalings need fewer iterations than the paper's unscaled
    preconditioner on held-out patches."""
    from paper_1602_01636_gb300 import learned
    def maker(seed):
        def make():
            patch = make_patch(synth.learned_workload_problem(100 + seed, n=14, p=2))
            return patch, to_dev(synth.random_rhs(patch.N, seed))
        return make
    from paper_1602_01636_gb300 import igafd

    def geo(seed):      # further training patches, labelled from the geometry alone
        return lambda: igafd.Patch.from_problem(synth.learned_workload_problem(100 + seed, n=14, p=2),
                                                stencil=False)
    X, T, gamma, totals, records = learned.build_dataset([maker(s) for s in range(16)],
                                                         geo_makers=[geo(s) for s in range(16, 24)])
    assert X.shape[0] == 24 * 3 * 14 and T.shape[0] == X.shape[0]    # 3 directions x 14 spans
    assert totals[gamma] <= totals[0.0]          # the labels beat the unscaled P
    # the condition-estimate refinement never costs iterations on its patch
    assert all(r["its"][1] <= r["its"][0] and r["kappa"][1] <= r["kappa"][0] for r in records)
    print("refinement records", records)
    net, losses = learned.train(X, T, synth.mlp_init(0), steps=1500)
    assert losses[-1] < 0.5 * losses[0]
    plain, scaled = [], []
    for seed in range(4):
        patch = make_patch(synth.learned_workload_problem(9000 + seed, n=14, p=2))
        b = to_dev(synth.random_rhs(patch.N, 50 + seed))
        _, i0 = patch.pcg(b, tol=1e-8, max_iter=1000)
        x, i1, fell_back, _ = learned.scaled_solve(patch, net, b, tol=1e-8, max_iter=1000)
        assert i0.status == 0 and i1.status == 0
        plain.append(i0.iterations)
        scaled.append(i1.iterations)
        patch.close()
    print("held-out iterations plain", plain, "learned", scaled, "gamma", gamma)
    assert np.mean(scaled) < 0.9 * np.mean(plain)
