"""Parity of the GPU additive Schwarz preconditioner P_IAS (Eq. (Pias)) on
the three-patch L-shaped domain with the oracle's, on the same inputs: the
library's own numbering and subdomain rows (host C, checked against the
oracle on the CPU), one patch per two-patch subdomain (merged knot vector,
stretched rectangle, no stencil) and the library's FD on each.

Tolerance: two FD applies (each within 1e-11 of the oracle's) summed by the
scatter: 1e-11 of max|z| in FP64; the TF32 FD is an inexact P_i with a few
operand roundings (2^-11) per mode product, four products in 2D: 1e-2 in
the 2-norm, the bound of the single-patch tensor-core FD parity tests."""
import numpy as np
import pytest

import synth
from oracle import multipatch as mpm
from gpu_util import need_gpu, to_dev, maxrel

pytestmark = pytest.mark.gpu

GLUE = [(1, 3, 0, 2, 0), (1, 1, 2, 0, 0)]    # Omega_2 top = Omega_1 bottom, Omega_2 right = Omega_3 left
SUBS = [(1, 0, 1), (1, 2, 0)]                # (patch a, patch b, direction merged)


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _merged(kn, p):
    inner = kn[p + 1:len(kn) - p - 1]
    return np.concatenate([np.zeros(p + 1), 0.5 * inner, np.full(p, 0.5), 0.5 + 0.5 * inner,
                           np.ones(p + 1)])


def _schwarz(igafd, kn, p):
    m = len(kn) - p - 1
    glob, fixed = igafd.mp_numbering([[m, m]] * 3, GLUE)
    free_index = np.cumsum(~fixed) - 1
    patches, rows = [], []
    for qa, qb, d in SUBS:
        r_full, _ = igafd.mp_subdomain([[m, m]] * 3, glob, fixed, qa, qb, d)
        rows.append(free_index[r_full])
        knots = [kn, _merged(kn, p)] if d == 1 else [_merged(kn, p), kn]
        sx, sy = (1.0, 2.0) if d == 1 else (2.0, 1.0)
        ctrl = np.array([[[0.0, sx], [0.0, sx]], [[0.0, 0.0], [sy, sy]]])
        patches.append(igafd.Patch(knots, p, ctrl, geo_knots=[np.array([0, 0, 1, 1.0])] * 2, geo_p=1,
                                   stencil=False))
    return igafd.Schwarz(patches, rows, int((~fixed).sum())), glob, fixed


def _to_oracle_order(L, glob, fixed):
    """perm[j] = the oracle's free index of the library's j-th free function."""
    lib_ids = np.concatenate([g.ravel() for g in glob])
    ora_ids = np.concatenate([L.local_to_global[q].ravel() for q in (1, 2, 3)])
    to_oracle = dict(zip(lib_ids.tolist(), ora_ids.tolist()))
    lib_free = np.flatnonzero(~fixed)
    return L.index[[to_oracle[g] for g in lib_free.tolist()]]


@pytest.mark.parametrize("nel,p", [(8, 2), (20, 3), (128, 3)])
def test_schwarz_apply_matches_oracle(torch, nel, p):
    from paper_1602_01636_gb300 import igafd
    kn = synth.uniform_open_knots(nel, p)
    L = mpm.LShape(kn, p)
    S, glob, fixed = _schwarz(igafd, kn, p)
    perm = _to_oracle_order(L, glob, fixed)
    assert S.n == L.N and sorted(perm.tolist()) == list(range(L.N))
    r = synth.random_vector(L.N, 13)                      # in the library's order
    r_o = np.empty(L.N)
    r_o[perm] = r
    z_o = mpm.AdditiveSchwarz(L, exact=False).apply(r_o)[perm]
    z = S.apply(to_dev(r)).cpu().numpy()
    assert np.abs(z - z_o).max() <= 1e-11 * np.abs(z_o).max()
    if 2 * L.m - 3 <= 256:                                # the tensor-core FD takes n_k <= 256
        z32 = S.apply(to_dev(r), dtype="tf32").cpu().numpy()
        assert np.linalg.norm(z32 - z_o) <= 1e-2 * np.linalg.norm(z_o)
        assert maxrel(z32, z_o) <= 1e-2


def test_schwarz_rejects_bad_rows(torch):
    from paper_1602_01636_gb300 import igafd
    kn = synth.uniform_open_knots(6, 2)
    S, glob, fixed = _schwarz(igafd, kn, 2)
    bad = [S._rows[0].copy(), S._rows[1].copy()]
    bad[0][1] = bad[0][0]                                 # a repeated row
    with pytest.raises(igafd.IgafdError):
        igafd.Schwarz(S._patches, bad, S.n)
    with pytest.raises(igafd.IgafdError):
        igafd.Schwarz(S._patches, S._rows, S.n - 5)       # rows out of range
    with pytest.raises(ValueError):
        igafd.Schwarz(S._patches, [S._rows[0][:-1], S._rows[1]], S.n)   # one row short


def _operator(igafd, kn, p, glob, fixed):
    """Full-space patches of the L (library patch q = the oracle's Omega_{q+1},
    each its parameter square translated: a degree-1 net) and the global free
    index of each of their local functions (-1: Dirichlet)."""
    free_index = np.where(fixed, -1, np.cumsum(~fixed) - 1)
    ops, maps = [], []
    for q in range(3):
        ox, oy = mpm.ORIGINS[q + 1]
        ctrl = np.array([[[ox, ox + 1.0], [ox, ox + 1.0]], [[oy, oy], [oy + 1.0, oy + 1.0]]])
        ops.append(igafd.Patch([kn, kn], p, ctrl, geo_knots=[np.array([0, 0, 1, 1.0])] * 2, geo_p=1,
                               full_space=True))
        maps.append(free_index[glob[q].ravel()])
    return ops, maps


@pytest.mark.parametrize("nel,p", [(32, 2), (64, 3)])
def test_multipatch_operator_and_solve_match_oracle(torch, nel, p):
    """Section 6 on the L (Table "L" workload): the glued stiffness A applied
    on the GPU (gather per patch, the patch's full-space stencil, scatter-add)
    equals the oracle's C^0 assembly entry by entry, and PCG with P_IAS takes
    the oracle's iteration count to 1e-8 with its iterate to 1e-10; solved to
    1e-12 it matches the oracle's direct solve."""
    import scipy.sparse.linalg as spla
    from oracle import pcg as opcg
    from paper_1602_01636_gb300 import igafd
    kn = synth.uniform_open_knots(nel, p)
    L = mpm.LShape(kn, p)
    S, glob, fixed = _schwarz(igafd, kn, p)
    ops, maps = _operator(igafd, kn, p, glob, fixed)
    S.set_operator(ops, maps)
    perm = _to_oracle_order(L, glob, fixed)
    x = synth.random_vector(L.N, 41)
    x_o = np.empty(L.N)
    x_o[perm] = x
    y = S.apply_A(to_dev(x)).cpu().numpy()
    y_o = (L.A @ x_o)[perm]
    assert maxrel(y, y_o) <= 1e-12
    b = synth.random_rhs(L.N, 42)
    b_o = np.empty(L.N)
    b_o[perm] = b
    P_ias = mpm.AdditiveSchwarz(L, exact=False)
    ro = opcg.pcg(lambda v: L.A @ v, b_o, P_ias.apply, tol=1e-8)
    xg, info = S.pcg(to_dev(b), tol=1e-8)
    print(f"L h^-1={nel} p={p}: oracle {ro.iters} it, GPU {info.iterations} it")
    assert info.status == 0 and info.iterations == ro.iters
    assert maxrel(xg.cpu().numpy(), ro.x[perm]) <= 1e-10
    xd = spla.spsolve(L.A.tocsc(), b_o)[perm]
    x12, i12 = S.pcg(to_dev(b), tol=1e-12)
    assert i12.status == 0 and maxrel(x12.cpu().numpy(), xd) <= 1e-10
    # the TF32 tensor-core FD inside P_IAS (flexible beta): at most two more
    # iterations, and a 1e-8 solution of the same system (the residual
    # bounds the error by kappa(A) 1e-8; the observed difference is printed)
    xt, it = S.pcg(to_dev(b), tol=1e-8, dtype="tf32")
    et = maxrel(xt.cpu().numpy(), xd)
    print(f"  TF32 FD in P_IAS: {it.iterations} it, max rel. difference from the direct solve {et:.1e}")
    assert it.status == 0 and it.iterations <= ro.iters + 2
    assert et <= 1e-6
    S.close()
    for q in ops:
        q.close()
