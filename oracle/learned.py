"""Span scalings of the 1D pencils (oracle; test infrastructure).

Prop. 1 bounds kappa(P^{-1} A) by the spread of the eigenvalues of Q. With
per-span weights, K~_k = sum_e wK_{k,e} K_k^(e) and M~_k = sum_e wM_{k,e}
M_k^(e), term k of the Kronecker sum carries wK_k(zeta_k) prod_{l != k}
wM_l(zeta_l) at each quadrature point. This module evaluates, by plain numpy
over the full quadrature grid:
  * the per-span features of Q (means, extremes and spread over the slab of
    quadrature points whose direction-k coordinate lies in span e);
  * the separable least-squares fit of log Q_kk by
    log wK_k(zeta_k) + sum_{l != k} log wM_l(zeta_l) (backfitting with slab
    means, gauge: the mean of each log wM_l is 0);
  * a 6 -> 64 -> 64 -> 2 tanh network with its mean-squared-error gradient.
Rows r <-> (direction k, span e), direction-major.
"""
from __future__ import annotations

import numpy as np

from . import assemble


def qdiag(disc: assemble.Discretization):
    """log Q_kk (k < d), log lambda_min(Q), log lambda_max(Q) on the tensor
    grid of quadrature points, each as an array [t_d, ..., t_1]."""
    pts = [disc.qz[k].ravel() for k in range(disc.d)]
    _, J = disc.geo.eval_grid(pts)
    Q, _ = assemble.q_matrix(J, disc.kappa_grid(pts))
    lam = np.linalg.eigvalsh(Q)
    out = [np.log(Q[..., k, k]) for k in range(disc.d)]
    out.append(np.log(lam[..., 0]))
    out.append(np.log(lam[..., -1]))
    return out


def _slab(arr, k, e, d, nq):
    """Values of a grid array on the slab of span e in direction k."""
    ax = d - 1 - k
    sl = [slice(None)] * d
    sl[ax] = slice(e * nq, (e + 1) * nq)
    return arr[tuple(sl)]


def features(disc: assemble.Discretization):
    d, nq = disc.d, disc.nq
    y = qdiag(disc)
    rows = []
    for k in range(d):
        for e in range(disc.nel[k]):
            lq = _slab(y[k], k, e, d, nq)
            oth = np.mean([np.exp(_slab(y[l], k, e, d, nq)) for l in range(d) if l != k], axis=0)
            s = disc.spans[k][e]
            rows.append([np.log(np.exp(lq).mean()), np.log(oth.mean()),
                         _slab(y[d], k, e, d, nq).min(), _slab(y[d + 1], k, e, d, nq).max(),
                         lq.std(), 0.5 * (disc.knots[k][s] + disc.knots[k][s + 1])])
    return np.array(rows)


def sepfit(disc: assemble.Discretization, sweeps=20):
    """(log wK, log wM) per row by backfitting; returns an array [rows][2]."""
    d, nq = disc.d, disc.nq
    y = qdiag(disc)[:d]
    a = [np.zeros(disc.nel[k]) for k in range(d)]
    m = [np.zeros(disc.nel[k]) for k in range(d)]

    def grid(v, l):
        e = np.repeat(v, nq)
        shape = [1] * d
        shape[d - 1 - l] = len(e)
        return e.reshape(shape)

    def slab_means(arr, l):
        ax = tuple(i for i in range(d) if i != d - 1 - l)
        return arr.mean(axis=ax).reshape(-1, nq).mean(axis=1)

    for _ in range(sweeps):
        for k in range(d):
            r = y[k] - sum(grid(m[l], l) for l in range(d) if l != k)
            a[k] = slab_means(r, k)
        for l in range(d):
            acc = 0.0
            for k in range(d):
                if k == l:
                    continue
                r = y[k] - grid(a[k], k) - sum(grid(m[j], j) for j in range(d) if j not in (k, l))
                acc = acc + slab_means(r, l)
            m[l] = acc / (d - 1)
        for l in range(d):
            c = m[l].mean()
            m[l] = m[l] - c
            for k in range(d):
                if k != l:
                    a[k] = a[k] + c
    return np.stack([np.concatenate(a), np.concatenate(m)], axis=1)


def split_rows(disc, logw):
    """Per-direction (wK, wM) weight arrays from a [rows][2] log array."""
    out, r = [], 0
    for k in range(disc.d):
        seg = np.asarray(logw[r:r + disc.nel[k]], dtype=np.float64)
        out.append((np.exp(seg[:, 0]), np.exp(seg[:, 1])))
        r += disc.nel[k]
    return out


def scaled_pencils(disc, logw):
    return [disc.pencil(k, wK=wK, wM=wM) for k, (wK, wM) in enumerate(split_rows(disc, logw))]


# ---- network ---------------------------------------------------------------
SIZES = (6, 64, 64, 2)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + 64 * 6].reshape(64, 6); o += 64 * 6
    b1 = p[o:o + 64]; o += 64
    W2 = p[o:o + 64 * 64].reshape(64, 64); o += 64 * 64
    b2 = p[o:o + 64]; o += 64
    W3 = p[o:o + 2 * 64].reshape(2, 64); o += 2 * 64
    b3 = p[o:o + 2]; o += 2
    assert o == len(p)
    return W1, b1, W2, b2, W3, b3


def mlp_forward(params, norm, X):
    in_mean, in_std, out_mean, out_std = norm
    W1, b1, W2, b2, W3, b3 = unpack(params)
    xn = (np.asarray(X, dtype=np.float64) - in_mean) / in_std
    h1 = np.tanh(xn @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    o = h2 @ W3.T + b3
    return out_mean + out_std * o, (xn, h1, h2, o)


def mlp_loss_grad(params, norm, X, T):
    """Mean over rows and outputs of (o - t_n)^2 (t_n the normalised target)
    and its gradient with respect to the flat parameter vector."""
    _, out_mean, out_std = None, norm[2], norm[3]
    W1, b1, W2, b2, W3, b3 = unpack(params)
    _, (xn, h1, h2, o) = mlp_forward(params, norm, X)
    tn = (np.asarray(T, dtype=np.float64) - out_mean) / out_std
    R = o.shape[0]
    diff = o - tn
    loss = np.mean(diff ** 2)
    do = 2.0 * diff / (R * 2)
    gW3 = do.T @ h2
    gb3 = do.sum(axis=0)
    dz2 = (do @ W3) * (1 - h2 ** 2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1 - h1 ** 2)
    gW1 = dz1.T @ xn
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
