"""Learned span scalings of the pencils: labels, training, scaled solve.

Host orchestration of library calls only; every computation (features of Q,
separable fit, scaled pencils and their eigendecompositions, the network's
forward and backward passes and Adam, the PCG solves) runs in libigafd.so.

Labels are chosen by the method itself: the separable log-fit of Q's
diagonal on each training patch, scaled by one factor gamma in
{0, 0.5, 0.75, 1, 1.25} (gamma = 0 is the paper's unscaled P) chosen for the
whole training set by minimising the total iterations of PCG with the FP64
fast-diagonalization preconditioner; then, per patch, a coordinate search
over one multiplier per direction minimises the condition estimate of
P^-1 A from 30 PCG steps (the CG-Lanczos tridiagonal), and the refined label
is kept when full PCG needs no more iterations than before. The network
learns the labels from the six per-span features of Q, so at solve time the
scalings come from the features alone. The unscaled preconditioner remains
the fallback when the scaled run breaks down or exceeds the unscaled
preconditioner's iteration budget (or the scaled pencils cannot be set up).
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


def kappa_estimate(patch, b, steps=30, dtype="fp32"):
    """Condition estimate of P^-1 A with the patch's current scalings from
    `steps` PCG steps (Fletcher-Reeves beta, so the CG-Lanczos relation holds;
    the FP32 fast diagonalization is P to ~1e-6, plenty for an estimate)."""
    _, info = patch.pcg(b, tol=1e-30, max_iter=steps, dtype=dtype, flexible=False,
                        true_every=0, raise_on_error=False)
    return patch.condition_estimate(steps)[0]


def direction_rows(patch):
    """Row ranges of the scaling rows of each direction."""
    out, r0 = [], 0
    for k in range(patch.dim):
        nel = patch.info.nel[k]
        out.append((r0, r0 + nel))
        r0 += nel
    return out


def refine_label(patch, b, label, factors=(0.5, 0.75, 1.25, 1.5), steps=30, tol=1e-8,
                 max_iter=1000):
    """Coordinate search over one multiplier c_k per direction of the label's
    log-scalings (rows of direction k times c_k), each step keeping the
    multiplier that lowers the 30-step condition estimate; the refined label
    is kept only if full FP64-preconditioned PCG needs no more iterations.
    Returns (label, {"kappa": (start, refined), "its": (start, refined)})."""
    rows = direction_rows(patch)

    def scaled(c):
        L = label.clone()
        for (r0, r1), ck in zip(rows, c):
            L[r0:r1] *= ck
        return L

    def kappa(c):
        patch.set_scalings(scaled(c))
        return kappa_estimate(patch, b, steps)

    c = [1.0] * patch.dim
    k0 = best = kappa(c)
    for k in range(patch.dim):
        ck = c[k]
        for f in factors:
            trial = list(c)
            trial[k] = ck * f
            kt = kappa(trial)
            if kt < best:
                best, c = kt, trial

    def iterations(L):
        patch.set_scalings(L)
        _, info = patch.pcg(b, tol=tol, max_iter=max_iter, dtype="fp64", raise_on_error=False)
        return info.iterations if info.status == 0 else 10 ** 9

    it0 = iterations(label)
    refined = scaled(c)
    it1 = iterations(refined) if c != [1.0] * patch.dim else it0
    patch.set_scalings(None)
    if it1 <= it0:
        return refined, {"kappa": (k0, best), "its": (it0, it1)}
    return label, {"kappa": (k0, best), "its": (it0, it0)}


def build_dataset(makers, refine=True, geo_makers=()):
    """makers: list of callables, each returning a fresh (patch, b) of one
    training problem (patches are closed after use, so a large set never
    holds all stencils at once; the refinement pass builds them again); gamma
    is selected on these by PCG iterations and their labels are refined.
    geo_makers: callables returning a patch of a further training problem
    built without the stencil (features and separable fit need only the
    geometry); its label is the separable fit times the selected gamma.
    Returns (X [rows][6], T [rows][2], gamma, {gamma: total iterations over
    the selection set}, per-patch refinement records)."""
    import torch
    Xs, fits, totals = [], [], {}
    for make in makers:
        patch, b = make()
        fit, its = label_patch(patch, b)
        Xs.append(patch.features())
        fits.append(fit)
        for g, v in its.items():
            totals[g] = totals.get(g, 0) + v
        patch.close()
    gamma = min(totals, key=lambda g: (totals[g], g))
    labels, records = [f * gamma for f in fits], []
    if refine and gamma != 0.0:
        for i, make in enumerate(makers):
            patch, b = make()
            labels[i], rec = refine_label(patch, b, labels[i])
            records.append(rec)
            patch.close()
    for make in geo_makers:
        patch = make()
        Xs.append(patch.features())
        labels.append(patch.sepfit() * gamma)
        patch.close()
    return torch.cat(Xs), torch.cat(labels), gamma, totals, records


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


def solve_with_scalings(patch, logw, b, tol=1e-8, max_iter=1000, dtype="fp64", budget=None):
    """PCG with the span scalings logw ([rows][2] CUDA tensor), capped at
    `budget` iterations (the unscaled preconditioner's iteration budget;
    default max_iter). Falls back to the paper's unscaled P -- a fresh solve
    from x0 = 0 with up to max_iter iterations -- when the scalings cannot be
    set up (a pencil that is not positive definite or an eigen-solve that
    fails), or when the scaled solve breaks down or has not converged within
    the budget. Returns (x, info, used_fallback)."""
    cap = max_iter if budget is None else min(int(budget), max_iter)
    try:
        patch.set_scalings(logw)
    except igafd.IgafdError:
        patch.set_scalings(None)
        x, info = patch.pcg(b, tol=tol, max_iter=max_iter, dtype=dtype, raise_on_error=False)
        return x, info, True
    x, info = patch.pcg(b, tol=tol, max_iter=cap, dtype=dtype, raise_on_error=False)
    if info.status != igafd.OK:
        patch.set_scalings(None)
        x, info = patch.pcg(b, tol=tol, max_iter=max_iter, dtype=dtype, raise_on_error=False)
        return x, info, True
    return x, info, False


def scaled_solve(patch, net, b, tol=1e-8, max_iter=1000, dtype="fp64", budget=None):
    """Solve with the network's span scalings, under the fallback rule of
    solve_with_scalings. Returns (x, info, used_fallback, prep_seconds)."""
    t0 = time.perf_counter()
    logw = predict_scalings(patch, net)
    prep = time.perf_counter() - t0
    x, info, fell_back = solve_with_scalings(patch, logw, b, tol=tol, max_iter=max_iter,
                                             dtype=dtype, budget=budget)
    return x, info, fell_back, prep
