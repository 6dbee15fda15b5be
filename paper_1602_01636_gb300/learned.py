"""Learned span scalings of the pencils: labels, training, scaled solve.

Host orchestration of library calls only; every computation (features of Q,
separable fit, scaled pencils and their eigendecompositions, the network's
forward and backward passes and Adam, the PCG solves) runs in libigafd.so.

Labels are chosen by the method itself: the separable log-fit of Q's
diagonal on each training patch, scaled by one factor gamma in
{0, 0.5, 0.75, 1, 1.25} (gamma = 0 is the paper's unscaled P) chosen for the
whole training set by minimising the total iterations of PCG with the FP64
fast-diagonalization preconditioner. The network learns those labels from
the six per-span features of Q, so at solve time the scalings come from the
features alone. The unscaled preconditioner remains the fallback when the
scaled run breaks down or exceeds its iteration budget.
"""
from __future__ import annotations

import time

import numpy as np

from . import igafd

GAMMAS = (0.0, 0.5, 0.75, 1.0, 1.25)


def label_patch(patch, b, tol=1e-8, max_iter=1000, gammas=GAMMAS):
    """Separable fit of one training patch and the FP64-preconditioned PCG
    iterations for each label scale gamma: (fit [rows][2], {gamma: its})."""
    fit = patch.sepfit()
    its = {}
    for g in gammas:
        patch.set_scalings(None if g == 0.0 else fit * g)
        _, info = patch.pcg(b, tol=tol, max_iter=max_iter, dtype="fp64", raise_on_error=False)
        its[g] = info.iterations if info.status == 0 else 10 ** 9
    patch.set_scalings(None)
    return fit, its


def build_dataset(items):
    """items: iterable of (patch, b). Returns (X [rows][6], T [rows][2],
    gamma, {gamma: total iterations over the set})."""
    import torch
    Xs, fits, totals = [], [], {}
    for patch, b in items:
        fit, its = label_patch(patch, b)
        Xs.append(patch.features())
        fits.append(fit)
        for g, v in its.items():
            totals[g] = totals.get(g, 0) + v
    gamma = min(totals, key=lambda g: (totals[g], g))
    return torch.cat(Xs), torch.cat(fits) * gamma, gamma, totals


def train(X, T, init_params, steps=1500, lr=3e-3, lr_final=3e-4):
    """Full-batch Adam on the mean squared error of the normalised outputs,
    learning rate decayed geometrically from lr to lr_final. X: [rows][6],
    T: [rows][2] float32 CUDA tensors. Returns (network, losses)."""
    Xh = X.double().cpu().numpy()
    Th = T.double().cpu().numpy()
    net = igafd.MLP(init_params)
    net.set_normalization(Xh.mean(0), np.maximum(Xh.std(0), 1e-3), Th.mean(0),
                          np.maximum(Th.std(0), 1e-3))
    losses = []
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    for s in range(steps):
        losses.append(net.train_step(X, T, lr * decay ** s))
    return net, losses


def predict_scalings(patch, net):
    """The network's span scalings [rows][2] for a patch."""
    return net.forward(patch.features())


def scaled_solve(patch, net, b, tol=1e-8, max_iter=1000, dtype="fp64"):
    """Solve with the learned scalings; fall back to the unscaled
    preconditioner when the scaled solve does not succeed within max_iter.
    Returns (x, info, used_fallback, prep_seconds)."""
    t0 = time.perf_counter()
    logw = predict_scalings(patch, net)
    patch.set_scalings(logw)
    prep = time.perf_counter() - t0
    x, info = patch.pcg(b, tol=tol, max_iter=max_iter, dtype=dtype, raise_on_error=False)
    if info.status != 0:
        patch.set_scalings(None)
        x, info = patch.pcg(b, tol=tol, max_iter=max_iter, dtype=dtype, raise_on_error=False)
        return x, info, True, prep
    return x, info, False, prep
