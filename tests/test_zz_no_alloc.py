"""The allocation-free FP64 FD entry point (igafd_apply_prec_static), for
callers that cannot call cudaMalloc, against the patch's own FD apply.

Collected last on purpose: it uses the library's static device scratch, and
a run that stops at the first failure has then already run every other test.
"""
import ctypes as C

import pytest

import synth
from gpu_util import need_gpu, make_patch, to_dev, rel

pytestmark = pytest.mark.gpu


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
                                         (2, (130, 97), 2, None)])
def test_static_fd_matches_patch_fd(dim, n, p, amp):
    torch = need_gpu()
    from paper_1602_01636_gb300 import igafd
    L = igafd.lib()
    patch = make_patch(synth.Problem(dim, n, p, amp))
    eig = [patch.eigen(k) for k in range(dim)]
    D_dev = [to_dev(D) for D, _ in eig]
    U_dev = [to_dev(U) for _, U in eig]
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different inputs reuse the same static scratch
    for seed in (31, 32):
        r = to_dev(synth.random_vector(patch.N, seed))
        z = torch.full_like(r, float("nan"))
        assert _call_static(L, dim, patch.n, U_dev, D_dev, r, z, stream) == igafd.OK
        z_ref = patch.apply_prec(r)
        torch.cuda.synchronize()
        assert rel(z.cpu().numpy(), z_ref.cpu().numpy()) <= 1e-11
    patch.close()


def test_static_fd_rejects_oversize():
    torch = need_gpu()
    from paper_1602_01636_gb300 import igafd
    L = igafd.lib()
    n = (128, 128, 128)                     # 2,097,152 dofs > the static limit
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = _call_static(L, 3, n, [dummy] * 3, [dummy] * 3, dummy, dummy + 0,
                      torch.cuda.current_stream().cuda_stream)
    assert st == igafd.ERR_ARG
