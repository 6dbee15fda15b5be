"""Preconditioned conjugate gradients (oracle; test infrastructure).

The paper runs CG preconditioned by P (Section 3) but prints neither the
algorithm nor its stopping rule. Readings used here: x_0 = 0 unless given;
stop when ||r_k||_2 <= tol ||b||_2, confirmed by the true residual b - A x_k
(which replaces the recurrence residual when it does not confirm); the true
residual is also recomputed every `true_every` iterations; the iteration
count is the number of products with A inside the loop. beta is
Fletcher-Reeves (r_{k+1}, z_{k+1}) / (r_k, z_k) for a fixed SPD
preconditioner, or the flexible (r_{k+1}, z_{k+1} - z_k) / (r_k, z_k) for an
inexact one.
"""
from __future__ import annotations

import numpy as np


class PCGResult:
    def __init__(self, x, iters, converged, relres, true_relres, history, alphas=(), betas=()):
        self.x, self.iters, self.converged = x, iters, converged
        self.relres, self.true_relres, self.history = relres, true_relres, history
        # step lengths alpha_k and direction factors beta_k (p_{k+1} = z_{k+1} + beta_k p_k)
        self.alphas, self.betas = list(alphas), list(betas)


def pcg(apply_A, b, apply_P, tol=1e-8, max_iter=1000, x0=None, flexible=False,
        true_every=50, fixed_iters=None):
    """Solve A x = b. With fixed_iters set, run exactly that many iterations
    without a convergence test (used to compare iterates)."""
    b = np.asarray(b, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    if bnorm == 0.0:
        return PCGResult(x, 0, True, 0.0, 0.0, [0.0])
    z = apply_P(r)
    pdir = z.copy()
    rho = r @ z
    hist = [np.linalg.norm(r) / bnorm]
    iters = 0
    limit = fixed_iters if fixed_iters is not None else max_iter
    converged = False
    alphas, betas = [], []
    for k in range(1, limit + 1):
        q = apply_A(pdir)
        alpha = rho / (pdir @ q)
        alphas.append(alpha)
        x = x + alpha * pdir
        r = r - alpha * q
        iters = k
        rn = np.linalg.norm(r) / bnorm
        hist.append(rn)
        if fixed_iters is None and rn <= tol:
            rt = b - apply_A(x)
            if np.linalg.norm(rt) / bnorm <= tol:
                converged = True
                break
            r = rt
        elif true_every and k % true_every == 0:
            r = b - apply_A(x)
        zn = apply_P(r)
        rho_new = r @ zn
        beta = (r @ (zn - z)) / rho if flexible else rho_new / rho
        betas.append(beta)
        rho = rho_new
        pdir = zn + beta * pdir
        z = zn
    true_rel = np.linalg.norm(b - apply_A(x)) / bnorm
    return PCGResult(x, iters, converged, hist[-1], true_rel, hist, alphas, betas)
