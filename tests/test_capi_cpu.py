"""CPU-side checks of the C-ABI library: it loads without a GPU and exports
every entry point declared in include/igafd.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "igafd.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(igafd_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1602_01636_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    syms = declared_symbols()
    assert len(syms) >= 10
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_1602_01636_gb300 import igafd
    assert set(igafd.EXPORTS) <= set(declared_symbols())
    L = igafd.lib()
    assert L.igafd_status_str(-5) == b"geometry map folds (det J <= 0)"


def test_struct_layouts_match_header(libpath):
    """The ctypes mirrors have the field order and count of the C structs."""
    from paper_1602_01636_gb300 import igafd
    text = open(HEADER).read()
    for cname, py in [("igafd_pcg_opts", igafd.PCGOpts), ("igafd_pcg_info", igafd.PCGInfo),
                      ("igafd_patch_info", igafd.PatchInfo), ("igafd_patch_desc", igafd.PatchDesc)]:
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                nm = re.findall(r"\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*((?:\[\d+\])*)\s*$", part.strip())
                names.append(nm[0][0])
        assert names == [f[0] for f in py._fields_], (cname, names)


def test_invalid_arguments_are_rejected_without_gpu_work(libpath):
    """Argument validation happens on the host before any CUDA call."""
    from paper_1602_01636_gb300 import igafd
    L = igafd.lib()
    h = ctypes.c_void_p()
    assert L.igafd_setup_patch(None, None, ctypes.byref(h)) == igafd.ERR_ARG
    d = igafd.PatchDesc()
    d.dim = 4
    assert L.igafd_setup_patch(ctypes.byref(d), None, ctypes.byref(h)) == igafd.ERR_ARG
    assert L.igafd_apply_A(None, None, None, None) == igafd.ERR_ARG
    assert L.igafd_pcg_solve(None, None, None, None, None, None) == igafd.ERR_ARG
    J = ctypes.c_int()
    assert L.igafd_adi_parameters(None, 0.1, 10, None, ctypes.byref(J)) == igafd.ERR_ARG
    assert L.igafd_adi_setup(None, None, 1, igafd.FP64, None) == igafd.ERR_ARG
    assert L.igafd_apply_prec_adi(None, None, None, None) == igafd.ERR_ARG
