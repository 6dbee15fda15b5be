"""ctypes binding of the igafd C ABI (include/igafd.h).

Argument marshalling only: every computation runs in libigafd.so. Device
vectors are torch CUDA tensors (float64, contiguous); streams are taken from
torch's current stream. There is no CPU fallback: if the library is missing
or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libigafd.so")

FP64, FP32, BF16, FP16, TF32, ADI = 0, 1, 2, 3, 4, 5
DTYPES = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16, "tf32": TF32, "adi": ADI}

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error",
          -3: "1D mass matrix not positive definite", -4: "eigen-solve did not converge",
          -5: "geometry map folds (det J <= 0)", -6: "PCG breakdown",
          -7: "PCG did not converge", -8: "device wait timed out", -9: "out of device memory"}
OK, ERR_ARG, ERR_CUDA, ERR_NOT_SPD, ERR_EIG, ERR_FOLDED, ERR_BREAKDOWN, ERR_NOT_CONVERGED, \
    ERR_TIMEOUT, ERR_OOM = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9


class IgafdError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"igafd {what}: {STATUS.get(status, status)} ({status})")


class PatchDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int),
                ("n_knots", C.POINTER(C.c_int)), ("knots", C.POINTER(C.POINTER(C.c_double))),
                ("geo_p", C.c_int), ("geo_n_knots", C.POINTER(C.c_int)),
                ("geo_knots", C.POINTER(C.POINTER(C.c_double))),
                ("ctrl", C.POINTER(C.c_double)), ("kappa", C.c_double),
                ("kappa_p", C.c_int), ("kappa_n_knots", C.POINTER(C.c_int)),
                ("kappa_knots", C.POINTER(C.POINTER(C.c_double))),
                ("kappa_ctrl", C.POINTER(C.c_double)), ("flags", C.c_int)]

SETUP_NO_STENCIL = 1
SETUP_FULL_SPACE = 2
SETUP_HALF_STENCIL = 4


class PatchInfo(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("n", C.c_int * 3), ("N", C.c_longlong),
                ("nel", C.c_int * 3), ("n_offsets", C.c_int), ("min_detJ", C.c_double),
                ("q_bound", C.c_double), ("setup_ms", C.c_double), ("eig_ms", C.c_double),
                ("stencil_bytes", C.c_longlong), ("stencil_stages", C.c_int),
                ("stencil_rows", C.c_int), ("eig_refined", C.c_int * 3),
                ("eig_check", (C.c_double * 2) * 3), ("fd_fused", C.c_int * 3),
                ("fd_tile", (C.c_int * 4) * 3), ("stencil_half", C.c_int)]


class PCGOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("true_every", C.c_int),
                ("prec_dtype", C.c_int), ("flexible", C.c_int), ("x0_given", C.c_int),
                ("check_every", C.c_int), ("timing", C.c_int)]


class PCGInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("relres", C.c_double),
                ("true_relres", C.c_double), ("true_checks", C.c_int),
                ("solve_ms", C.c_double), ("stencil_ms", C.c_double), ("prec_ms", C.c_double)]


_lib = None

EXPORTS = ["igafd_setup_patch", "igafd_destroy_patch", "igafd_patch_query", "igafd_get_eigen",
           "igafd_copy_stencil", "igafd_apply_A", "igafd_apply_prec", "igafd_load_rhs_sine",
           "igafd_pcg_solve", "igafd_pcg_default_opts", "igafd_status_str",
           "igafd_kernel_launches", "igafd_batch_pcg_solve", "igafd_autotune",
           "igafd_set_stencil_stages", "igafd_set_stencil_rows", "igafd_setup_prec", "igafd_set_eig_route",
           "igafd_pcg_condition_estimate", "igafd_lanczos_extremes", "igafd_set_fd_fused", "igafd_scaling_rows", "igafd_patch_features",
           "igafd_patch_sepfit", "igafd_set_scalings", "igafd_mlp_create", "igafd_mlp_destroy",
           "igafd_mlp_set_normalization", "igafd_mlp_get_params", "igafd_mlp_set_params",
           "igafd_mlp_forward", "igafd_mlp_gradient", "igafd_mlp_train_step",
           "igafd_adi_parameters", "igafd_adi_setup", "igafd_apply_prec_adi", "igafd_adi_greedy",
           "igafd_adi_wachspress", "igafd_mp_numbering", "igafd_mp_subdomain", "igafd_mp_create",
           "igafd_mp_destroy", "igafd_mp_apply_ias", "igafd_quad_points", "igafd_load_rhs",
           "igafd_batch_create", "igafd_batch_solve", "igafd_batch_destroy", "igafd_batch_pass_log",
           "igafd_batch_create_grouped", "igafd_batch_groups", "igafd_probe_peaks",
           "igafd_mp_set_operator", "igafd_mp_apply_A", "igafd_mp_pcg_solve", "igafd_set_fd_tile"]

MLP_PARAMS = 4738


def lib():
    """Load libigafd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1602_01636_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.igafd_setup_patch.argtypes = [C.POINTER(PatchDesc), vp, C.POINTER(vp)]
    L.igafd_destroy_patch.argtypes = [vp]
    L.igafd_destroy_patch.restype = None
    L.igafd_patch_query.argtypes = [vp, C.POINTER(PatchInfo)]
    L.igafd_get_eigen.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.igafd_copy_stencil.argtypes = [vp, vp, vp]
    L.igafd_apply_A.argtypes = [vp, vp, vp, vp]
    L.igafd_apply_prec.argtypes = [vp, C.c_int, vp, vp, vp]
    L.igafd_load_rhs_sine.argtypes = [vp, vp, vp]
    L.igafd_load_rhs.argtypes = [vp, vp, vp, vp]
    L.igafd_quad_points.argtypes = [vp, vp, vp]
    L.igafd_pcg_solve.argtypes = [vp, C.POINTER(PCGOpts), vp, vp, C.POINTER(PCGInfo), vp]
    L.igafd_batch_pcg_solve.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(vp),
                                        C.POINTER(PCGOpts), C.POINTER(PCGInfo), vp]
    L.igafd_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(PCGOpts), C.POINTER(vp)]
    L.igafd_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(PCGInfo), vp]
    L.igafd_batch_destroy.argtypes = [vp]
    L.igafd_batch_pass_log.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.igafd_batch_create_grouped.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(PCGOpts), C.c_int,
                                             C.c_int, C.POINTER(vp)]
    L.igafd_batch_groups.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.igafd_probe_peaks.argtypes = [C.c_int, C.POINTER(Peaks)]
    L.igafd_batch_destroy.restype = None
    L.igafd_autotune.argtypes = [vp, C.c_int, vp]
    L.igafd_set_stencil_stages.argtypes = [vp, C.c_int]
    L.igafd_set_fd_fused.argtypes = [vp, C.c_int]
    L.igafd_set_fd_tile.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
    L.igafd_set_stencil_rows.argtypes = [vp, C.c_int]
    L.igafd_setup_prec.argtypes = [vp, vp]
    dp = C.POINTER(C.c_double)
    L.igafd_pcg_condition_estimate.argtypes = [vp, C.c_int, dp, dp, dp]
    L.igafd_lanczos_extremes.argtypes = [dp, dp, C.c_int, dp, dp]
    L.igafd_set_eig_route.argtypes = [vp, C.c_int]
    L.igafd_scaling_rows.argtypes = [vp, C.POINTER(C.c_int)]
    L.igafd_patch_features.argtypes = [vp, vp, vp]
    L.igafd_patch_sepfit.argtypes = [vp, C.c_int, vp, vp]
    L.igafd_set_scalings.argtypes = [vp, vp, vp]
    fp = C.POINTER(C.c_float)
    L.igafd_mlp_create.argtypes = [fp, C.POINTER(vp)]
    L.igafd_mlp_destroy.argtypes = [vp]
    L.igafd_mlp_destroy.restype = None
    L.igafd_mlp_set_normalization.argtypes = [vp, fp, fp, fp, fp]
    L.igafd_mlp_get_params.argtypes = [vp, fp]
    L.igafd_mlp_set_params.argtypes = [vp, fp]
    L.igafd_mlp_forward.argtypes = [vp, vp, C.c_int, vp, vp]
    L.igafd_mlp_gradient.argtypes = [vp, vp, vp, C.c_int, fp, fp, vp]
    L.igafd_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, fp, vp]
    L.igafd_adi_parameters.argtypes = [vp, C.c_double, C.c_int, dp, C.POINTER(C.c_int)]
    L.igafd_adi_setup.argtypes = [vp, dp, C.c_int, C.c_int, vp]
    L.igafd_mp_numbering.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_longlong), C.POINTER(C.c_ubyte), C.POINTER(C.c_longlong)]
    L.igafd_mp_subdomain.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                     C.POINTER(C.c_ubyte), C.c_int, C.c_int, C.c_int,
                                     C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
    L.igafd_mp_create.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(C.POINTER(C.c_longlong)),
                                  C.c_longlong, C.POINTER(vp)]
    L.igafd_mp_destroy.argtypes = [vp]
    L.igafd_mp_destroy.restype = None
    L.igafd_mp_apply_ias.argtypes = [vp, C.c_int, vp, vp, vp]
    L.igafd_mp_set_operator.argtypes = [vp, C.c_int, C.POINTER(vp), C.POINTER(C.POINTER(C.c_longlong))]
    L.igafd_mp_apply_A.argtypes = [vp, vp, vp, vp]
    L.igafd_mp_pcg_solve.argtypes = [vp, C.POINTER(PCGOpts), vp, vp, C.POINTER(PCGInfo), vp]
    L.igafd_adi_wachspress.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, dp,
                                       C.POINTER(C.c_int)]
    L.igafd_adi_greedy.argtypes = [dp, C.c_int, dp, C.c_int, dp, C.c_int, C.c_double, C.c_int, dp,
                                   C.POINTER(C.c_int)]
    L.igafd_apply_prec_adi.argtypes = [vp, vp, vp, vp]
    L.igafd_pcg_default_opts.argtypes = [C.POINTER(PCGOpts)]
    L.igafd_pcg_default_opts.restype = None
    L.igafd_status_str.argtypes = [C.c_int]
    L.igafd_status_str.restype = C.c_char_p
    L.igafd_kernel_launches.argtypes = []
    L.igafd_kernel_launches.restype = C.c_longlong
    for name in EXPORTS:
        if name not in ("igafd_destroy_patch", "igafd_pcg_default_opts", "igafd_status_str",
                        "igafd_kernel_launches", "igafd_mlp_destroy", "igafd_mp_destroy",
                        "igafd_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def lanczos_extremes(alpha, beta):
    """Extreme eigenvalues of the CG-Lanczos tridiagonal of len(alpha) steps
    (host arithmetic in the library; no GPU needed)."""
    import numpy as _np
    a = _np.ascontiguousarray(alpha, dtype=_np.float64)
    b = _np.ascontiguousarray(beta if len(beta) else [0.0], dtype=_np.float64)
    lo, hi = C.c_double(), C.c_double()
    dp = C.POINTER(C.c_double)
    _check(lib().igafd_lanczos_extremes(a.ctypes.data_as(dp), b.ctypes.data_as(dp), len(a),
                                        C.byref(lo), C.byref(hi)), "lanczos_extremes")
    return lo.value, hi.value


def adi_greedy(L1, L2, L3, eps, max_J=400):
    """Greedy three-variable ADI parameters on the spectra L1, L2, L3 (host
    arithmetic in the library; no GPU needed). Raises when max_J parameters
    do not reach eps."""
    import numpy as _np
    ls = [_np.ascontiguousarray(v, dtype=_np.float64) for v in (L1, L2, L3)]
    w = _np.zeros(max_J, dtype=_np.float64)
    J = C.c_int()
    dp = C.POINTER(C.c_double)
    _check(lib().igafd_adi_greedy(ls[0].ctypes.data_as(dp), len(ls[0]), ls[1].ctypes.data_as(dp),
                                  len(ls[1]), ls[2].ctypes.data_as(dp), len(ls[2]), float(eps),
                                  int(max_J), w.ctypes.data_as(dp), C.byref(J)), "adi_greedy")
    return w[:J.value].copy()


def adi_wachspress(a, b, eps, max_J=400):
    """Two-variable ADI: J of Eq. (ADIits) and the optimal parameters for the
    spectral interval [a, b] (host arithmetic in the library; no GPU needed)."""
    import numpy as _np
    w = _np.zeros(max_J, dtype=_np.float64)
    J = C.c_int()
    _check(lib().igafd_adi_wachspress(float(a), float(b), float(eps), int(max_J),
                                      w.ctypes.data_as(C.POINTER(C.c_double)), C.byref(J)),
           "adi_wachspress")
    return w[:J.value].copy()


def mp_numbering(m, glue):
    """Multi-patch numbering (host arithmetic in the library; no GPU needed).
    m: [npatch][dim] functions per direction; glue: [(patch a, side a,
    patch b, side b, orientation), ...]. Returns (global ids per patch as a
    list of arrays shaped [m_d..m_1], fixed flags per global function)."""
    import numpy as _np
    m = _np.ascontiguousarray(m, dtype=_np.int32)
    npatch, dim = m.shape
    g = _np.ascontiguousarray(glue, dtype=_np.int32).reshape(-1, 5)
    sizes = [int(_np.prod(row)) for row in m]
    total = sum(sizes)
    glob = _np.zeros(total, dtype=_np.int64)
    fixed = _np.zeros(total, dtype=_np.uint8)
    ng = C.c_longlong()
    ip = C.POINTER(C.c_int)
    _check(lib().igafd_mp_numbering(dim, npatch, m.ctypes.data_as(ip), len(g), g.ctypes.data_as(ip),
                                    glob.ctypes.data_as(C.POINTER(C.c_longlong)),
                                    fixed.ctypes.data_as(C.POINTER(C.c_ubyte)), C.byref(ng)),
           "mp_numbering")
    out, o = [], 0
    for q in range(npatch):
        out.append(glob[o:o + sizes[q]].reshape(tuple(int(v) for v in m[q][::-1])))
        o += sizes[q]
    return out, fixed[:ng.value].astype(bool)


def mp_subdomain(m, glob, fixed, qa, qb, direction):
    """Rows of R_i for the subdomain of glued patches qa, qb merged along
    `direction` (host arithmetic in the library): (global ids in the merged
    patch's interior order, interior shape per direction)."""
    import numpy as _np
    m = _np.ascontiguousarray(m, dtype=_np.int32)
    npatch, dim = m.shape
    gl = _np.ascontiguousarray(_np.concatenate([g.ravel() for g in glob]), dtype=_np.int64)
    fx = _np.ascontiguousarray(fixed, dtype=_np.uint8)
    cap = int(_np.prod([m[qa][k] + (m[qb][k] if k == direction else 0) for k in range(dim)]))
    rows = _np.zeros(cap, dtype=_np.int64)
    shape = (C.c_int * 3)()
    _check(lib().igafd_mp_subdomain(dim, npatch, m.ctypes.data_as(C.POINTER(C.c_int)),
                                    gl.ctypes.data_as(C.POINTER(C.c_longlong)),
                                    fx.ctypes.data_as(C.POINTER(C.c_ubyte)), qa, qb, direction,
                                    rows.ctypes.data_as(C.POINTER(C.c_longlong)), shape),
           "mp_subdomain")
    shp = tuple(int(shape[k]) for k in range(dim))
    return rows[:int(_np.prod(shp))].copy(), shp


class Peaks(C.Structure):
    _fields_ = [("fp64_tflops", C.c_double), ("tf32_tflops", C.c_double),
                ("bf16_tflops", C.c_double), ("sm_max_mhz", C.c_double)]


def probe_peaks(device=0):
    """Measured FP64-pipe and tensor-core (TF32, BF16) rates of the device,
    TFLOP/s (igafd_probe_peaks)."""
    pk = Peaks()
    _check(lib().igafd_probe_peaks(int(device), C.byref(pk)), "probe_peaks")
    return {"fp64_tflops": pk.fp64_tflops, "tf32_tflops": pk.tf32_tflops,
            "bf16_tflops": pk.bf16_tflops, "sm_max_mhz": pk.sm_max_mhz}


def kernel_launches():
    """Kernels the library has enqueued in this process so far."""
    return int(lib().igafd_kernel_launches())


def _check(st, what):
    if st != OK:
        raise IgafdError(st, what)


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_ptr(t, n=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _opts(tol, max_iter, dtype, flexible, true_every, check_every, timing=False):
    o = PCGOpts()
    lib().igafd_pcg_default_opts(C.byref(o))
    o.tol, o.max_iter, o.true_every, o.check_every = tol, max_iter, true_every, check_every
    o.prec_dtype = DTYPES[dtype]
    o.flexible = int(dtype != "fp64") if flexible is None else int(flexible)
    o.timing = int(bool(timing))
    return o


class Batch:
    """A batched solver for a fixed set of patches and options: the device
    tables and the device-driven loop graph are built once (igafd_batch_create);
    each solve() allocates nothing on the library side."""

    def __init__(self, patches, tol=1e-8, max_iter=1000, dtype="fp64", flexible=None,
                 true_every=50, groups=1, passes_per_launch=0):
        """groups: problems split into that many concurrently looping groups
        (0: one per problem); passes_per_launch: passes per launch of a
        group's loop graph, relaunched from the host while members are
        unfinished (0: the whole loop in one launch)."""
        self._patches = list(patches)
        self.n = len(self._patches)
        o = _opts(tol, max_iter, dtype, flexible, true_every, 4)
        vp = C.c_void_p
        hp = (vp * self.n)(*[p.h for p in self._patches])
        h = C.c_void_p()
        _check(lib().igafd_batch_create_grouped(hp, self.n, C.byref(o), int(groups),
                                                int(passes_per_launch), C.byref(h)), "batch_create")
        self.h = h

    def groups(self):
        """(number of groups, each problem's group)."""
        g = C.c_int()
        of = (C.c_int * self.n)()
        _check(lib().igafd_batch_groups(self.h, C.byref(g), of), "batch_groups")
        return g.value, list(of)

    def solve(self, bs, xs=None, raise_on_error=True):
        """Solve patches[i] x_i = bs[i] for all i; returns (xs, infos)."""
        import torch
        if xs is None:
            xs = [torch.zeros_like(b) for b in bs]
        vp = C.c_void_p
        hb = (vp * self.n)(*[_dev_ptr(b, p.N) for p, b in zip(self._patches, bs)])
        hx = (vp * self.n)(*[_dev_ptr(x, p.N) for p, x in zip(self._patches, xs)])
        infos = (PCGInfo * self.n)()
        st = lib().igafd_batch_solve(self.h, hb, hx, infos, _stream())
        if raise_on_error and st not in (OK, ERR_NOT_CONVERGED):
            raise IgafdError(st, "batch_solve")
        return xs, list(infos)

    def pass_log(self, group=0):
        """Per pass of group `group`'s device loop in the last solve: start
        (from the earliest pass of any group) and length (us, on the device
        clock) and the number of unfinished members."""
        import numpy as np
        L, n = lib(), C.c_int()
        _check(L.igafd_batch_pass_log(self.h, group, 0, None, None, None, C.byref(n)),
               "batch_pass_log")
        m = n.value
        st, du, ac = (C.c_double * m)(), (C.c_double * m)(), (C.c_int * m)()
        _check(L.igafd_batch_pass_log(self.h, group, m, st, du, ac, C.byref(n)), "batch_pass_log")
        return {"start_us": np.array(st[:]), "dur_us": np.array(du[:]), "active": np.array(ac[:])}

    def close(self):
        if getattr(self, "h", None):
            lib().igafd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_pcg(patches, bs, xs=None, tol=1e-8, max_iter=1000, dtype="fp64", flexible=None,
              true_every=50, check_every=4, raise_on_error=True):
    """Solve patches[i] x_i = bs[i] for all i in one batched solve (the
    device-driven loop over every unfinished problem; creates and frees a
    Batch). Returns (xs, infos)."""
    import torch
    n = len(patches)
    if xs is None:
        xs = [torch.zeros_like(b) for b in bs]
    o = _opts(tol, max_iter, dtype, flexible, true_every, check_every)
    vp = C.c_void_p
    hp = (vp * n)(*[p.h for p in patches])
    hb = (vp * n)(*[_dev_ptr(b, p.N) for p, b in zip(patches, bs)])
    hx = (vp * n)(*[_dev_ptr(x, p.N) for p, x in zip(patches, xs)])
    infos = (PCGInfo * n)()
    st = lib().igafd_batch_pcg_solve(hp, n, hb, hx, C.byref(o), infos, _stream())
    if raise_on_error and st not in (OK, ERR_NOT_CONVERGED):
        raise IgafdError(st, "batch_pcg_solve")
    return xs, list(infos)


class Patch:
    """A single-patch problem set up on the current CUDA device."""

    def __init__(self, knots, p, ctrl, kappa=1.0, geo_knots=None, geo_p=None, kappa_field=None,
                 stencil=True, full_space=False, half_stencil=False):
        """kappa_field: optional (knots, degree, control values) of a positive
        spline coefficient c(zeta); K = kappa * c. stencil=False builds the
        patch without A (geometry, features, separable fit and P only).
        full_space=True keeps every B-spline (no Dirichlet removal) and builds
        no preconditioner: a piece of a multi-patch operator. half_stencil=True
        stores A by its symmetry (about half the bytes)."""
        L = lib()
        dim = len(knots)
        geo_knots = knots if geo_knots is None else geo_knots
        geo_p = p if geo_p is None else geo_p
        self._keep = []
        kn = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
        gk = [np.ascontiguousarray(k, dtype=np.float64) for k in geo_knots]
        ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
        self._keep += kn + gk + [ctrl]
        dp = C.POINTER(C.c_double)
        d = PatchDesc()
        d.dim, d.p, d.geo_p, d.kappa = dim, p, geo_p, float(kappa)
        d.n_knots = (C.c_int * dim)(*[len(k) for k in kn])
        d.knots = (dp * dim)(*[k.ctypes.data_as(dp) for k in kn])
        d.geo_n_knots = (C.c_int * dim)(*[len(k) for k in gk])
        d.geo_knots = (dp * dim)(*[k.ctypes.data_as(dp) for k in gk])
        d.ctrl = ctrl.ctypes.data_as(dp)
        d.flags = ((0 if stencil else SETUP_NO_STENCIL) | (SETUP_FULL_SPACE if full_space else 0) |
                   (SETUP_HALF_STENCIL if half_stencil else 0))
        if kappa_field is not None:
            kk, kpd, kc = kappa_field
            kk = [np.ascontiguousarray(k, dtype=np.float64) for k in kk]
            kc = np.ascontiguousarray(kc, dtype=np.float64)
            self._keep += kk + [kc]
            d.kappa_p = int(kpd)
            d.kappa_n_knots = (C.c_int * dim)(*[len(k) for k in kk])
            d.kappa_knots = (dp * dim)(*[k.ctypes.data_as(dp) for k in kk])
            d.kappa_ctrl = kc.ctypes.data_as(dp)
        h = C.c_void_p()
        _check(L.igafd_setup_patch(C.byref(d), _stream(), C.byref(h)), "setup_patch")
        self.h = h
        self.info = self.query()
        self.dim = dim
        self.n = tuple(self.info.n[k] for k in range(dim))
        self.N = int(self.info.N)

    @classmethod
    def from_problem(cls, prob, stencil=True, half_stencil=False):
        kf = None
        if getattr(prob, "kappa_ctrl", None) is not None:
            kf = (prob.kappa_knots, prob.kappa_p, prob.kappa_ctrl)
        return cls(prob.knots, prob.p, prob.ctrl, prob.kappa,
                   geo_knots=getattr(prob, "geo_knots", None), geo_p=getattr(prob, "geo_p", None),
                   kappa_field=kf, stencil=stencil, half_stencil=half_stencil)

    def query(self):
        info = PatchInfo()
        _check(lib().igafd_patch_query(self.h, C.byref(info)), "patch_query")
        return info

    def eigen(self, k):
        n = self.info.n[k]
        U = np.empty((n, n))
        D = np.empty(n)
        dp = C.POINTER(C.c_double)
        _check(lib().igafd_get_eigen(self.h, k, U.ctypes.data_as(dp), D.ctypes.data_as(dp)),
               "get_eigen")
        return D, U

    def autotune(self, force=False):
        """Measure the stencil pipeline's candidates on this patch (ring depth,
        and in 3D one or two rows per thread) and the tensor-core FD's forms
        (fused or one kernel per mode product, for TF32 and BF16) and keep the
        fastest; returns the chosen depth (`info.stencil_rows` holds the rows,
        `info.fd_fused` the FD form per operand type)."""
        _check(lib().igafd_autotune(self.h, int(bool(force)), _stream()), "autotune")
        self.info = self.query()
        return self.info.stencil_stages

    # ---- span scalings of the pencils -------------------------------------
    def scaling_rows(self):
        r = C.c_int()
        _check(lib().igafd_scaling_rows(self.h, C.byref(r)), "scaling_rows")
        return r.value

    def features(self):
        """float32 CUDA tensor [rows][6] of per-span features of Q."""
        import torch
        out = torch.empty((self.scaling_rows(), 6), dtype=torch.float32, device="cuda")
        _check(lib().igafd_patch_features(self.h, C.c_void_p(out.data_ptr()), _stream()), "features")
        return out

    def sepfit(self, sweeps=20):
        """float32 CUDA tensor [rows][2] of separable-fit log scalings."""
        import torch
        out = torch.empty((self.scaling_rows(), 2), dtype=torch.float32, device="cuda")
        _check(lib().igafd_patch_sepfit(self.h, int(sweeps), C.c_void_p(out.data_ptr()), _stream()),
               "sepfit")
        return out

    def set_scalings(self, logw=None):
        """Rebuild the preconditioner from span-scaled pencils (logw: float32
        CUDA tensor [rows][2]) or, with None, from the unscaled ones."""
        ptr = None
        if logw is not None:
            logw = logw.contiguous()
            assert logw.is_cuda and logw.shape == (self.scaling_rows(), 2)
            ptr = C.c_void_p(logw.data_ptr())
        _check(lib().igafd_set_scalings(self.h, ptr, _stream()), "set_scalings")

    def set_stencil_stages(self, stages):
        _check(lib().igafd_set_stencil_stages(self.h, int(stages)), "set_stencil_stages")
        self.info = self.query()

    def setup_prec(self):
        """Redo P's setup (pencils, eigendecompositions, FD tables) in place."""
        _check(lib().igafd_setup_prec(self.h, _stream()), "setup_prec")
        self.info = self.query()

    def condition_estimate(self, steps=0):
        """(kappa, lambda_min, lambda_max) of P^-1 A from the last solve's CG-Lanczos
        tridiagonal (its first `steps` iterations when steps > 0)."""
        k, lo, hi = C.c_double(), C.c_double(), C.c_double()
        _check(lib().igafd_pcg_condition_estimate(self.h, int(steps), C.byref(k), C.byref(lo),
                                                  C.byref(hi)), "condition_estimate")
        return k.value, lo.value, hi.value

    def set_eig_route(self, route):
        """0: FP32 Jacobi + FP64 refinement where n_k <= 128 (default); 1: FP64 Jacobi.
        Takes effect at the next setup_prec()."""
        _check(lib().igafd_set_eig_route(self.h, int(route)), "set_eig_route")

    def set_stencil_rows(self, rows):
        _check(lib().igafd_set_stencil_rows(self.h, int(rows)), "set_stencil_rows")
        self.info = self.query()

    def set_fd_fused(self, fused):
        _check(lib().igafd_set_fd_fused(self.h, int(fused)), "set_fd_fused")

    def set_fd_tile(self, dtype, tile):
        """Tile shape of the tensor-core FD for dtype: (rows per CTA of the
        per-mode kernel, its column tiles, its K stages, columns per CTA of
        the fused pencil kernel)."""
        t = (C.c_int * 4)(*[int(v) for v in tile])
        _check(lib().igafd_set_fd_tile(self.h, DTYPES[dtype], t), "set_fd_tile")
        self.info = self.query()

    def fd_tile(self, dtype):
        o = {"tf32": 0, "bf16": 1, "fp16": 2}[dtype]
        return tuple(self.info.fd_tile[o][i] for i in range(4))

    def stencil(self):
        import torch
        out = torch.empty((self.info.n_offsets, self.N), dtype=torch.float64, device="cuda")
        _check(lib().igafd_copy_stencil(self.h, C.c_void_p(out.data_ptr()), _stream()),
               "copy_stencil")
        return out

    def apply_A(self, x, y=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(lib().igafd_apply_A(self.h, _dev_ptr(x, self.N), _dev_ptr(y, self.N), _stream()),
               "apply_A")
        return y

    def apply_prec(self, r, z=None, dtype="fp64"):
        import torch
        z = torch.empty_like(r) if z is None else z
        _check(lib().igafd_apply_prec(self.h, DTYPES[dtype], _dev_ptr(r, self.N),
                                      _dev_ptr(z, self.N), _stream()), "apply_prec")
        return z

    def adi_parameters(self, eps, max_J=400):
        """ADI parameters w_1..w_J for the tolerance eps: the optimal
        two-variable parameters in 2D, the greedy three-variable ones in 3D
        (host arithmetic in the library over the patch's eigenvalues)."""
        import numpy as _np
        w = _np.zeros(max_J, dtype=_np.float64)
        J = C.c_int()
        _check(lib().igafd_adi_parameters(self.h, float(eps), int(max_J),
                                          w.ctypes.data_as(C.POINTER(C.c_double)), C.byref(J)),
               "adi_parameters")
        return w[:J.value].copy()

    def adi_setup(self, omega, dtype="fp64"):
        """Set up the ADI preconditioner P_J with the parameters omega."""
        import numpy as _np
        w = _np.ascontiguousarray(omega, dtype=_np.float64)
        _check(lib().igafd_adi_setup(self.h, w.ctypes.data_as(C.POINTER(C.c_double)), len(w),
                                     DTYPES[dtype], _stream()), "adi_setup")

    def apply_prec_adi(self, r, z=None):
        """z = P_J^{-1} r by the ADI iterations set up with adi_setup."""
        import torch
        z = torch.empty_like(r) if z is None else z
        _check(lib().igafd_apply_prec_adi(self.h, _dev_ptr(r, self.N), _dev_ptr(z, self.N),
                                          _stream()), "apply_prec_adi")
        return z

    def n_quad_points(self):
        return int(np.prod([self.info.nel[k] * (self.info.p + 1) for k in range(self.dim)]))

    def quad_points(self):
        """float64 CUDA tensor [dim][Q]: physical coordinates of the patch's
        quadrature points (order of igafd_quad_points)."""
        import torch
        x = torch.empty((self.dim, self.n_quad_points()), dtype=torch.float64, device="cuda")
        _check(lib().igafd_quad_points(self.h, C.c_void_p(x.data_ptr()), _stream()), "quad_points")
        return x

    def load_rhs(self, f_qp, b=None):
        """b_i = int f B_i |det J| from f at the quadrature points (a float64
        CUDA tensor of n_quad_points() values, order of quad_points())."""
        import torch
        b = torch.empty(self.N, dtype=torch.float64, device="cuda") if b is None else b
        _check(lib().igafd_load_rhs(self.h, _dev_ptr(f_qp.reshape(-1), self.n_quad_points()),
                                    _dev_ptr(b, self.N), _stream()), "load_rhs")
        return b

    def load_rhs_sine(self, b=None):
        import torch
        b = torch.empty(self.N, dtype=torch.float64, device="cuda") if b is None else b
        _check(lib().igafd_load_rhs_sine(self.h, _dev_ptr(b, self.N), _stream()), "load_rhs")
        return b

    def pcg(self, b, x=None, x0=False, tol=1e-8, max_iter=1000, dtype="fp64", flexible=None,
            true_every=50, check_every=4, timing=False, raise_on_error=True):
        """Solve A x = b; returns (x, PCGInfo). x is the output buffer (allocated
        when None); its contents are the initial guess only when x0=True."""
        import torch
        o = PCGOpts()
        lib().igafd_pcg_default_opts(C.byref(o))
        o.tol, o.max_iter, o.true_every, o.check_every = tol, max_iter, true_every, check_every
        o.prec_dtype = DTYPES[dtype]
        o.flexible = int(dtype != "fp64") if flexible is None else int(flexible)
        o.x0_given = int(bool(x0) and x is not None)
        o.timing = int(bool(timing))
        x = torch.zeros_like(b) if x is None else x
        info = PCGInfo()
        st = lib().igafd_pcg_solve(self.h, C.byref(o), _dev_ptr(b, self.N), _dev_ptr(x, self.N),
                                   C.byref(info), _stream())
        if raise_on_error and st not in (OK, ERR_NOT_CONVERGED):
            raise IgafdError(st, "pcg_solve")
        return x, info

    def close(self):
        if getattr(self, "h", None):
            lib().igafd_destroy_patch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Schwarz:
    """The additive Schwarz preconditioner P_IAS = sum_i R_i^T P_i^{-1} R_i
    (Eq. (Pias)) on the GPU: patches[i] is subdomain i as one patch, rows[i]
    the global (free) index of each of its dofs, n the global size."""

    def __init__(self, patches, rows, n):
        import numpy as _np
        k = len(patches)
        self._patches = list(patches)
        self._rows = [_np.ascontiguousarray(r, dtype=_np.int64) for r in rows]
        if len(self._rows) != k or any(len(r) != pt.N for r, pt in zip(self._rows, self._patches)):
            raise ValueError("rows[i] must hold one global index per dof of patches[i]")
        lp = C.POINTER(C.c_longlong)
        hs = (C.c_void_p * k)(*[pt.h for pt in self._patches])
        rp = (lp * k)(*[r.ctypes.data_as(lp) for r in self._rows])
        h = C.c_void_p()
        _check(lib().igafd_mp_create(k, hs, rp, int(n), C.byref(h)), "mp_create")
        self.h, self.n = h, int(n)

    def apply(self, r, z=None, dtype="fp64"):
        import torch
        z = torch.empty_like(r) if z is None else z
        _check(lib().igafd_mp_apply_ias(self.h, DTYPES[dtype], _dev_ptr(r, self.n), _dev_ptr(z, self.n),
                                        _stream()), "mp_apply_ias")
        return z

    def set_operator(self, patches, free_of_local):
        """The multi-patch A: full-space patches (Patch(..., full_space=True))
        and, per patch, the global free index of each local function (-1 for
        Dirichlet ones)."""
        import numpy as _np
        self._ops = list(patches)
        self._maps = [_np.ascontiguousarray(m, dtype=_np.int64).ravel() for m in free_of_local]
        if len(self._maps) != len(self._ops) or any(len(m) != pt.N for m, pt in zip(self._maps, self._ops)):
            raise ValueError("free_of_local[q] must hold one index per local function of patches[q]")
        lp = C.POINTER(C.c_longlong)
        hs = (C.c_void_p * len(self._ops))(*[pt.h for pt in self._ops])
        mp = (lp * len(self._ops))(*[m.ctypes.data_as(lp) for m in self._maps])
        _check(lib().igafd_mp_set_operator(self.h, len(self._ops), hs, mp), "mp_set_operator")

    def apply_A(self, x, y=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(lib().igafd_mp_apply_A(self.h, _dev_ptr(x, self.n), _dev_ptr(y, self.n), _stream()),
               "mp_apply_A")
        return y

    def pcg(self, b, x=None, tol=1e-8, max_iter=1000, dtype="fp64", flexible=None, true_every=50,
            raise_on_error=True):
        """Solve A x = b by PCG with P_IAS; returns (x, PCGInfo)."""
        import torch
        o = _opts(tol, max_iter, dtype, flexible, true_every, 1)
        x = torch.zeros_like(b) if x is None else x
        info = PCGInfo()
        st = lib().igafd_mp_pcg_solve(self.h, C.byref(o), _dev_ptr(b, self.n), _dev_ptr(x, self.n),
                                      C.byref(info), _stream())
        if raise_on_error and st not in (OK, ERR_NOT_CONVERGED):
            raise IgafdError(st, "mp_pcg_solve")
        return x, info

    def close(self):
        if getattr(self, "h", None):
            lib().igafd_mp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The scaling network (6 -> 64 -> 64 -> 2, tanh) on the GPU."""

    def __init__(self, params=None):
        fp = C.POINTER(C.c_float)
        h = C.c_void_p()
        arr = None
        if params is not None:
            arr = np.ascontiguousarray(params, dtype=np.float32)
            assert arr.size == MLP_PARAMS
        _check(lib().igafd_mlp_create(None if arr is None else arr.ctypes.data_as(fp), C.byref(h)),
               "mlp_create")
        self.h = h

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        fp = C.POINTER(C.c_float)
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (in_mean, in_std, out_mean, out_std)]
        self._norm = arrs
        _check(lib().igafd_mlp_set_normalization(self.h, *[a.ctypes.data_as(fp) for a in arrs]),
               "mlp_set_normalization")

    def params(self):
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(lib().igafd_mlp_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float))),
               "mlp_get_params")
        return out

    def set_params(self, params):
        arr = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().igafd_mlp_set_params(self.h, arr.ctypes.data_as(C.POINTER(C.c_float))),
               "mlp_set_params")

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
        _check(lib().igafd_mlp_forward(self.h, C.c_void_p(X.data_ptr()), int(X.shape[0]),
                                       C.c_void_p(Y.data_ptr()), _stream()), "mlp_forward")
        return Y

    def gradient(self, X, T):
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = C.c_float()
        fp = C.POINTER(C.c_float)
        _check(lib().igafd_mlp_gradient(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                        int(X.shape[0]), g.ctypes.data_as(fp), C.byref(loss),
                                        _stream()), "mlp_gradient")
        return float(loss.value), g

    def train_step(self, X, T, lr):
        loss = C.c_float()
        _check(lib().igafd_mlp_train_step(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                          int(X.shape[0]), float(lr), C.byref(loss), _stream()),
               "mlp_train_step")
        return float(loss.value)

    def close(self):
        if getattr(self, "h", None):
            lib().igafd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
