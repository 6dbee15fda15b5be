"""Helpers shared by the GPU tests: device availability and patch set-up."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_01636_gb300 import build
    build.build()
    return torch


def make_patch(prob):
    from paper_1602_01636_gb300 import igafd
    return igafd.Patch.from_problem(prob)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    """2-norm relative difference ||a - b|| / ||b||."""
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def maxrel(a, b):
    """Entry-wise difference max_i |a_i - b_i| / max_i |b_i|: a few wrong
    entries (a boundary slab of a tile, a ragged edge) cannot hide in it."""
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())
