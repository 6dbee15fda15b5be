"""The allocation-free FP64 FD entry point (igafd_apply_prec_static), for
callers that cannot call cudaMalloc, against the oracle's fast
diagonalization and against the patch's own FD apply.

This file sorts after every other test file on purpose: it uses the
library's static device scratch, and a run that stops at the first failure
has then already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import assemble, fd
from gpu_util import need_gpu, to_dev, maxrel

pytestmark = pytest.mark.gpu

MAX_DOFS = 1048576          # IGAFD_STATIC_FD_MAX_DOFS in include/igafd.h


def _call_static(L, dim, n, U_dev, D_dev, r, z, stream):
    vp = C.c_void_p
    fn = L.igafd_apply_prec_static
    fn.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(vp), C.POINTER(vp), vp, vp, vp]
    fn.restype = C.c_int
    n_arr = (C.c_int * dim)(*n)
    u_arr = (vp * dim)(*[vp(t.data_ptr()) for t in U_dev])
    d_arr = (vp * dim)(*[vp(t.data_ptr()) for t in D_dev])
    return fn(dim, n_arr, u_arr, d_arr, vp(r.data_ptr()), vp(z.data_ptr()), vp(stream))


@pytest.mark.parametrize("dim,n,p,amp", [(3, (40, 36, 44), 3, [0.05, -0.03, 0.02]),
                                         (2, (130, 97), 2, None),
                                         (3, (128, 128, 64), 2, [0.02, 0.01, -0.03])])
def test_static_fd_matches_oracle_and_patch_fd(dim, n, p, amp):
    """Two calls in a row with different inputs share the static scratch;
    (128, 128, 64) has exactly the limit of 1,048,576 dofs, so the second
    half of the scratch is filled to its end."""
    torch = need_gpu()
    from paper_1602_01636_gb300 import igafd
    L = igafd.lib()
    prob = synth.Problem(dim, n, p, amp)
    patch = igafd.Patch.from_problem(prob, stencil=False)
    disc = assemble.Discretization.from_problem(prob)
    F = fd.FD([disc.pencil(k) for k in range(dim)])
    eig = [patch.eigen(k) for k in range(dim)]
    D_dev = [to_dev(D) for D, _ in eig]
    U_dev = [to_dev(U) for _, U in eig]
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (31, 32):
        r_h = synth.random_vector(patch.N, seed)
        r = to_dev(r_h)
        z = torch.full_like(r, float("nan"))
        assert _call_static(L, dim, patch.n, U_dev, D_dev, r, z, stream) == igafd.OK
        z_patch = patch.apply_prec(r)
        torch.cuda.synchronize()
        zs = z.cpu().numpy()
        assert maxrel(zs, F.apply(r_h)) <= 1e-11
        assert maxrel(zs, z_patch.cpu().numpy()) <= 1e-11
    patch.close()


def test_static_fd_rejects_oversize():
    torch = need_gpu()
    from paper_1602_01636_gb300 import igafd
    L = igafd.lib()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # one dof over the limit (17 x 61681 = 1,048,577), and far over it; both
    # are rejected on the host before any pointer is used
    for dim, n in ((2, (17, 61681)), (3, (128, 128, 128))):
        assert np.prod(n) > MAX_DOFS
        st = _call_static(L, dim, n, [dummy] * dim, [dummy] * dim, dummy, dummy + 0, stream)
        assert st == igafd.ERR_ARG
