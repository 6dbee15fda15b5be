"""Eqs. (A), (Q), (prec) and the right-hand side (oracle; test infrastructure).

Readings of the paper used here:
* Eq. (Q) is printed as det(J) J^{-T} K J^{-1}; the chain rule with
  J_ij = d x_i / d zeta_j gives grad_x u = J^{-T} grad_zeta u, hence
  Q = |det J| J^{-1} K J^{-T}. This module uses the latter (K = kappa I).
* The scalar index of Eq. (Vh) makes direction 1 the fastest; P is built by
  that index: the 1D factor K_k (or M_k) acts on i_k.
* Quadrature: (p+1)-point Gauss per element per direction (the paper's rule
  is not stated); exact for the 1D pencils.
* The stiffness matrix is held as a (2p+1)^d offset ("stencil") array
  S[o, row], o = sum_k (delta_k + p) (2p+1)^(k-1), row = sum_k i_k n^(k-1),
  entry A[row, row + delta]; couplings that leave the index box are 0.
"""
from __future__ import annotations

import itertools
import os

import numpy as np
import scipy.sparse as sp

from . import spline


class Geometry:
    """Spline map F(zeta) = sum_i C_i B_i(zeta) (Section 2.1)."""

    def __init__(self, ctrl, knots, p):
        self.ctrl = np.asarray(ctrl, dtype=np.float64)    # [c][i_d]..[i_1]
        self.knots = [np.asarray(k, dtype=np.float64) for k in knots]
        self.p = int(p)
        self.d = len(self.knots)

    def eval_grid(self, pts):
        """F and its Jacobian on the tensor grid of 1D point sets pts[k]
        (direction k). Returns F[c, q_d, ..., q_1] and J[q_d, ..., q_1, c, j]
        with J_cj = dF_c / dzeta_j."""
        d = self.d
        vals, ders, lo = [], [], []
        for k in range(d):
            V = spline.basis_table(self.knots[k], self.p, pts[k])
            D = spline.basis_table(self.knots[k], self.p, pts[k], deriv=True)
            nz = np.nonzero(np.any(V != 0, axis=0) | np.any(D != 0, axis=0))[0]
            a, b = nz.min(), nz.max() + 1
            vals.append(V[:, a:b]); ders.append(D[:, a:b]); lo.append((a, b))
        # restrict the net to the control points that can be nonzero
        sl = (slice(None),) + tuple(slice(*lo[k]) for k in reversed(range(d)))
        C = self.ctrl[sl]

        def contract(tables):
            # tables[k] acts on direction k; array axes are [c, dir d, ..., dir 1]
            T = C
            for k in range(d):
                ax = d - k  # axis of direction k in T
                T = np.moveaxis(np.tensordot(T, tables[k], axes=([ax], [1])), -1, ax)
            return T

        F = contract(vals)
        J = np.empty(F.shape[1:] + (F.shape[0], d))
        for j in range(d):
            tabs = [ders[k] if k == j else vals[k] for k in range(d)]
            Tj = contract(tabs)
            for c in range(F.shape[0]):
                J[..., c, j] = Tj[c]
        return F, J


def q_matrix(J, kappa=1.0):
    """Q = kappa |det J| J^{-1} J^{-T} at every point (reading of Eq. (Q));
    kappa is a scalar or an array over the points. Also returns det J."""
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    kap = np.asarray(kappa, dtype=np.float64)
    Q = (kap * np.abs(det))[..., None, None] * (Jinv @ np.swapaxes(Jinv, -1, -2))
    return Q, det


class ScalarSpline:
    """Scalar tensor spline field c(zeta) = sum_i c_i B_i(zeta) (used for a
    variable coefficient K(x) = kappa(zeta) I of Eq. (poisson))."""

    def __init__(self, ctrl, knots, p):
        self._g = Geometry(np.asarray(ctrl, dtype=np.float64)[None], knots, p)

    def eval_grid(self, pts):
        F, _ = self._g.eval_grid(pts)
        return F[0]


class Discretization:
    """Degree-p tensor B-spline space with homogeneous Dirichlet conditions on
    a spline-mapped patch (Eqs. (Vh), (A))."""

    def __init__(self, knots, p, geometry: Geometry, kappa=1.0, nq=None, kappa_field=None):
        self.knots = [np.asarray(k, dtype=np.float64) for k in knots]
        self.p = int(p)
        self.d = len(self.knots)
        self.geo = geometry
        self.kappa = float(kappa)
        self.kappa_field = kappa_field          # ScalarSpline or None
        self.nq = self.p + 1 if nq is None else int(nq)
        self.m = [len(k) - self.p - 1 for k in self.knots]   # 1D space dims
        self.n = [mk - 2 for mk in self.m]                   # Dirichlet dofs
        self.N = int(np.prod(self.n))
        self.qz, self.qw, self.spans = [], [], []
        for k in self.knots:
            z, w, s = spline.gauss_points(k, self.nq)
            self.qz.append(z); self.qw.append(w); self.spans.append(s)
        self.nel = [len(s) for s in self.spans]

    @classmethod
    def from_problem(cls, prob, nq=None):
        geo = Geometry(prob.ctrl, getattr(prob, "geo_knots", None) or prob.knots,
                       getattr(prob, "geo_p", None) or prob.p)
        kf = None
        if getattr(prob, "kappa_ctrl", None) is not None:
            kf = ScalarSpline(prob.kappa_ctrl, prob.kappa_knots, prob.kappa_p)
        return cls(prob.knots, prob.p, geo, prob.kappa, nq, kf)

    def kappa_grid(self, pts):
        """kappa at the tensor grid of 1D point sets (scalar if constant)."""
        if self.kappa_field is None:
            return self.kappa
        return self.kappa * self.kappa_field.eval_grid(pts)

    # ---- 1D pencils (Section 3) -------------------------------------------
    def pencil(self, k, full=False, wK=None, wM=None):
        """(K_k, M_k): 1D stiffness and mass matrices of direction k by
        Gauss quadrature; Dirichlet rows/columns removed unless full.
        Optional per-element weights wK, wM give the span-scaled pencils
        sum_e wK_e K^(e), sum_e wM_e M^(e)."""
        z, w = self.qz[k].ravel(), self.qw[k].ravel()
        V = spline.basis_table(self.knots[k], self.p, z)
        D = spline.basis_table(self.knots[k], self.p, z, deriv=True)
        nq = self.nq
        wk = w if wK is None else w * np.repeat(np.asarray(wK, dtype=np.float64), nq)
        wm = w if wM is None else w * np.repeat(np.asarray(wM, dtype=np.float64), nq)
        M = (V * wm[:, None]).T @ V
        K = (D * wk[:, None]).T @ D
        if not full:
            M, K = M[1:-1, 1:-1], K[1:-1, 1:-1]
        return K, M

    # ---- element-by-element quantities ------------------------------------
    def _box(self, elo, ehi, need_q=True):
        """Quadrature data on a box of elements [elo_k, ehi_k) per direction:
        local basis values/derivatives, weights, det J and (need_q) Q on the
        box grid."""
        p, nq, d = self.p, self.nq, self.d
        V, D, W, I0, pts = [], [], [], [], []
        for k in range(d):
            z = self.qz[k][elo[k]:ehi[k]]
            s = self.spans[k][elo[k]:ehi[k]]
            Vt = spline.basis_table(self.knots[k], p, z.ravel()).reshape(z.shape + (-1,))
            Dt = spline.basis_table(self.knots[k], p, z.ravel(), deriv=True).reshape(z.shape + (-1,))
            cols = s[:, None] - p + np.arange(p + 1)[None, :]       # full indices
            V.append(np.take_along_axis(Vt, cols[:, None, :].repeat(nq, 1), 2))
            D.append(np.take_along_axis(Dt, cols[:, None, :].repeat(nq, 1), 2))
            W.append(self.qw[k][elo[k]:ehi[k]])
            I0.append(s - p)
            pts.append(z.ravel())
        F, J = self.geo.eval_grid(pts)
        if need_q:
            Q, det = q_matrix(J, self.kappa_grid(pts))
        else:
            Q, det = None, np.linalg.det(J)
        return dict(V=V, D=D, W=W, I0=I0, F=F, Q=Q, det=det)

    @staticmethod
    def _tprod(factors):
        """Tensor product over directions of per-element factors f_k[E, g, a]
        -> [E, G, A] with direction 1 fastest in G and A."""
        T = np.ones((factors[0].shape[0], 1, 1))
        for f in reversed(factors):          # slowest direction first
            E, G, A = T.shape
            T = (T[:, :, None, :, None] * f[:, None, :, None, :]).reshape(
                E, G * f.shape[1], A * f.shape[2])
        return T

    def _element_lists(self, box, elo, ehi):
        d = self.d
        ranges = [np.arange(ehi[k] - elo[k]) for k in range(d)]
        grid = np.meshgrid(*ranges[::-1], indexing="ij")
        return [grid[d - 1 - k].ravel() for k in range(d)]   # local element idx per dir

    def _gather_grid(self, arr, eidx):
        """Values of a box-grid array arr[q_d..q_1, ...] at each element's
        own quadrature points -> [E, G, ...] (G with direction 1 fastest)."""
        d, nq = self.d, self.nq
        g = np.arange(nq)
        idx = []
        for k in reversed(range(d)):   # slowest direction first
            gi = eidx[k][:, None] * nq + g[None, :]
            shape = [len(eidx[k])] + [1] * d
            shape[1 + (d - 1 - k)] = nq
            idx.append(gi.reshape(shape))
        out = arr[tuple(idx)]
        return out.reshape((len(eidx[0]), nq ** d) + arr.shape[d:])

    def element_matrices(self, box, eidx):
        """Local matrices L[e, a, b] = sum_q w_q grad B_a^T Q grad B_b
        (Eq. (A)) for the elements eidx of a box."""
        d = self.d
        V = [box["V"][k][eidx[k]] for k in range(d)]
        D = [box["D"][k][eidx[k]] for k in range(d)]
        W = self._tprod([box["W"][k][eidx[k]][:, :, None] for k in range(d)])[:, :, 0]
        # dB_a/dzeta_r at the element's quadrature points g: G[e, a, r, g]
        G = np.stack([self._tprod([D[k] if k == r else V[k] for k in range(d)])
                      for r in range(d)], axis=-1)
        G = np.ascontiguousarray(G.transpose(0, 2, 3, 1))
        Qe = self._gather_grid(box["Q"], eidx)                # [E, g, r, s]
        QW = np.ascontiguousarray((Qe * W[:, :, None, None]).transpose(0, 2, 3, 1))  # [E, r, s, g]
        # H[e, b, r, g] = w_g sum_s Q_rs(g) dB_b/dzeta_s(g), the d-term sum written out
        H = sum(QW[:, None, :, s, :] * G[:, :, s, None, :] for s in range(d))
        E, A, _, Gn = G.shape
        # L[e, a, b] = sum_{r, g} G[e, a, r, g] H[e, b, r, g]
        L = np.matmul(G.reshape(E, A, d * Gn), H.reshape(E, A, d * Gn).transpose(0, 2, 1))
        return L

    def _local_full_indices(self, box, eidx):
        """Full (Dirichlet-included) multi-index of each local function:
        list over directions of [E, A] arrays."""
        d, p = self.d, self.p
        out = []
        for k in range(d):
            base = box["I0"][k][eidx[k]]                     # [E]
            ak = np.arange(p + 1)
            shape = [1] * d
            shape[d - 1 - k] = p + 1
            loc = np.broadcast_to(ak.reshape(shape), [p + 1] * d).ravel()
            out.append(base[:, None] + loc[None, :])
        return out

    # ---- stiffness matrix ---------------------------------------------------
    def n_offsets(self):
        return (2 * self.p + 1) ** self.d

    def offset_index(self, delta):
        """o = sum_k (delta_k + p) (2p+1)^(k-1) for a list/array of deltas."""
        w = 2 * self.p + 1
        return sum((np.asarray(delta[k]) + self.p) * w ** k for k in range(self.d))

    def row_index(self, i):
        """Scalar Dirichlet index of Eq. (Vh) (0-based), direction 1 fastest."""
        r, s = 0, 1
        for k in range(self.d):
            r = r + np.asarray(i[k]) * s
            s *= self.n[k]
        return r

    def assemble_stencil(self, chunk_planes=1, workers=1):
        """Full stiffness matrix A as the offset array S[o, row]: the element
        matrices of Eq. (A) summed into the rows of their basis functions,
        element planes of the slowest direction in increasing order (each
        plane in blocks along the next direction).

        workers > 1 splits the planes into that many contiguous ranges, each
        summed by its own (spawned) process from zero in plane order; the
        range sums are then added in range order. Only the association of the
        per-row sums changes (entries agree with workers=1 to rounding)."""
        d = self.d
        last = d - 1
        planes = [(e0, min(e0 + chunk_planes, self.nel[last]))
                  for e0 in range(0, self.nel[last], chunk_planes)]
        S = np.zeros((self.n_offsets(), self.N))
        workers = max(1, min(int(workers), len(planes)))
        if workers == 1:
            for e0, e1 in planes:
                for elo, ehi in self._plane_boxes(e0, e1):
                    self._scatter_box(S, elo, ehi)
            return S
        for r0, part in _spawn_map(_assemble_planes, [self] * workers, _split(planes, workers)):
            if part is not None:
                S[:, r0:r0 + part.shape[1]] += part
        return S

    def _plane_box_full(self, e0, e1):
        """Element box of whole planes [e0, e1) of the slowest direction."""
        elo = [0] * self.d
        ehi = list(self.nel)
        elo[-1], ehi[-1] = e0, e1
        return elo, ehi

    def _plane_boxes(self, e0, e1, max_elems=4096):
        """Element boxes covering planes [e0, e1) of the slowest direction,
        the next-slowest direction cut into blocks so that a box holds about
        max_elems elements at most (bounds the temporaries of one box)."""
        d = self.d
        per_line = int(np.prod(self.nel[:d - 2])) * (e1 - e0) if d > 2 else (e1 - e0)
        n2 = self.nel[d - 2]
        step = max(1, min(n2, max_elems // max(per_line, 1)))
        out = []
        for b0 in range(0, n2, step):
            elo = [0] * d
            ehi = list(self.nel)
            elo[-1], ehi[-1] = e0, e1
            elo[-2], ehi[-2] = b0, min(b0 + step, n2)
            out.append((elo, ehi))
        return out

    def _row_range(self, e0, e1):
        """Half-open range of scalar rows that the elements of planes
        [e0, e1) of the slowest direction couple to."""
        last, p = self.d - 1, self.p
        stride = int(np.prod(self.n[:last]))
        i_lo = max(int(self.spans[last][e0]) - p - 1, 0)
        i_hi = min(int(self.spans[last][e1 - 1]) - 1, self.n[last] - 1)
        return i_lo * stride, (i_hi + 1) * stride

    def _scatter_box(self, S, elo, ehi, rows=None, row0=0):
        """Add the element matrices of a box into S[o, row - row0] (S 2D, its
        columns a contiguous range of rows starting at row0); with `rows`,
        only into those rows."""
        d = self.d
        box = self._box(elo, ehi)
        eidx = self._element_lists(box, elo, ehi)
        L = self.element_matrices(box, eidx)
        I = self._local_full_indices(box, eidx)               # full indices
        valid_r = np.ones(L.shape[:2], bool)
        for k in range(d):
            valid_r &= (I[k] >= 1) & (I[k] <= self.m[k] - 2)
        row = self.row_index([I[k] - 1 for k in range(d)])      # [E, A]
        # pairs (a, b): row from a, column offset from b - a
        rowp = np.broadcast_to(row[:, :, None], L.shape)
        valid = valid_r[:, :, None] & valid_r[:, None, :]
        # the offset of a local pair (a, b) is I_b - I_a, the same in every
        # element (local indices are consecutive from the element's first)
        delta = [I[k][0, None, :] - I[k][0, :, None] for k in range(d)]
        o = np.broadcast_to(self.offset_index(delta), L.shape)
        if rows is not None:
            valid &= np.isin(rowp, rows)
            np.add.at(S, (o[valid], rowp[valid] - row0), L[valid])
            return S
        if not valid.any():
            return S
        rsel = rowp[valid]
        r0, r1 = int(rsel.min()), int(rsel.max()) + 1
        R = r1 - r0
        part = np.bincount(o[valid] * R + (rsel - r0), weights=L[valid],
                           minlength=S.shape[0] * R)
        S[:, r0 - row0:r1 - row0] += part.reshape(S.shape[0], R)
        return S

    def assemble_rows(self, rows_multi):
        """Rows of A for the given Dirichlet multi-indices (list of tuples,
        direction 1 first), computed from the elements of each row's support
        only. Returns S_rows[len(rows), n_offsets]."""
        d, p = self.d, self.p
        out = np.zeros((len(rows_multi), self.n_offsets()))
        for r, i in enumerate(rows_multi):
            # full index I_k = i_k + 1; support elements s - p <= I <= s
            elo, ehi = [], []
            for k in range(d):
                I = i[k] + 1
                es = [e for e, s in enumerate(self.spans[k]) if s - p <= I <= s]
                elo.append(min(es)); ehi.append(max(es) + 1)
            row = int(self.row_index(i))
            S = np.zeros((self.n_offsets(), 1))
            self._scatter_box(S, elo, ehi, rows=np.array([row]), row0=row)
            out[r] = S[:, 0]
        return out

    # ---- right-hand side ----------------------------------------------------
    def assemble_rhs(self, f, chunk_planes=4, workers=1):
        """b_i = int f(F(zeta)) B_i(zeta) |det J| dzeta with f a callable of
        the physical coordinates (x_1, ..., x_d). workers > 1: contiguous
        plane ranges summed by spawned processes (f must then be picklable,
        e.g. a module-level function), range sums added in order."""
        last = self.d - 1
        planes = [(e0, min(e0 + chunk_planes, self.nel[last]))
                  for e0 in range(0, self.nel[last], chunk_planes)]
        workers = max(1, min(int(workers), len(planes)))
        b = np.zeros(self.N)
        if workers == 1:
            r0, part = _rhs_planes(self, f, planes)
            b[r0:r0 + len(part)] += part
            return b
        for r0, part in _spawn_map(_rhs_planes, [self] * workers, [f] * workers,
                                   _split(planes, workers)):
            if part is not None:
                b[r0:r0 + len(part)] += part
        return b

    def _rhs_box(self, f, elo, ehi, out, row0):
        """Add the element load vectors of a box into out[row - row0]."""
        d = self.d
        box = self._box(elo, ehi, need_q=False)
        eidx = self._element_lists(box, elo, ehi)
        V = [box["V"][k][eidx[k]] for k in range(d)]
        W = self._tprod([box["W"][k][eidx[k]][:, :, None] for k in range(d)])[:, :, 0]
        Bh = self._tprod(V)                                   # [E, G, A]
        X = [self._gather_grid(box["F"][c], eidx) for c in range(d)]
        det = self._gather_grid(box["det"], eidx)
        fv = f(*X) * np.abs(det) * W                          # [E, G]
        loc = np.einsum("eg,ega->ea", fv, Bh)
        I = self._local_full_indices(box, eidx)
        valid = np.ones(loc.shape, bool)
        for k in range(d):
            valid &= (I[k] >= 1) & (I[k] <= self.m[k] - 2)
        row = self.row_index([I[k] - 1 for k in range(d)])
        out += np.bincount(row[valid] - row0, weights=loc[valid], minlength=len(out))

    # ---- discretization error ------------------------------------------------
    def l2_error(self, u_dofs, u_exact, extra_q=2, chunk_planes=4):
        """|| u - u_h ||_{L2(Omega)} with u_h = sum_i u_i B_i (Dirichlet dofs
        zero), by a Gauss rule with p+1+extra_q points per direction."""
        fine = Discretization(self.knots, self.p, self.geo, self.kappa, self.p + 1 + extra_q,
                              self.kappa_field)
        d = self.d
        U = np.zeros(tuple(reversed(self.m)))
        U[tuple(slice(1, -1) for _ in range(d))] = np.asarray(u_dofs).reshape(tuple(reversed(self.n)))
        err2 = 0.0
        last = d - 1
        for e0 in range(0, fine.nel[last], chunk_planes):
            elo = [0] * d
            ehi = list(fine.nel)
            elo[last], ehi[last] = e0, min(e0 + chunk_planes, fine.nel[last])
            box = fine._box(elo, ehi, need_q=False)
            eidx = fine._element_lists(box, elo, ehi)
            V = [box["V"][k][eidx[k]] for k in range(d)]
            W = fine._tprod([box["W"][k][eidx[k]][:, :, None] for k in range(d)])[:, :, 0]
            Bh = fine._tprod(V)
            I = fine._local_full_indices(box, eidx)
            coef = U[tuple(I[k] for k in reversed(range(d)))]          # [E, A]
            uh = np.einsum("ega,ea->eg", Bh, coef)
            X = [fine._gather_grid(box["F"][c], eidx) for c in range(d)]
            det = fine._gather_grid(box["det"], eidx)
            err2 += np.sum(W * np.abs(det) * (u_exact(*X) - uh) ** 2)
        return float(np.sqrt(err2))

    # ---- dense reference objects for tiny problems --------------------------
    def dense_A_bruteforce(self, full=False):
        """A by one global quadrature sum over the whole tensor grid of
        quadrature points with global (not element-local) basis tables:
        A = sum_q w_q G(q)^T Q(q) G(q). Tiny problems only."""
        d = self.d
        pts = [self.qz[k].ravel() for k in range(d)]
        wts = [self.qw[k].ravel() for k in range(d)]
        V = [spline.basis_table(self.knots[k], self.p, pts[k]) for k in range(d)]
        Dr = [spline.basis_table(self.knots[k], self.p, pts[k], deriv=True) for k in range(d)]
        if not full:
            V = [v[:, 1:-1] for v in V]
            Dr = [x[:, 1:-1] for x in Dr]
        _, J = self.geo.eval_grid(pts)
        Q, _ = q_matrix(J, self.kappa_grid(pts))
        Q = Q.reshape(-1, d, d)

        def kron_all(tabs):  # rows: q (dir 1 fastest), cols: dof (dir 1 fastest)
            T = tabs[-1]
            for k in range(d - 2, -1, -1):
                T = np.einsum("qi,rj->qrij", T, tabs[k]).reshape(
                    T.shape[0] * tabs[k].shape[0], T.shape[1] * tabs[k].shape[1])
            return T

        Wq = kron_all([w[:, None] for w in wts])[:, 0]
        G = np.stack([kron_all([Dr[k] if k == r else V[k] for k in range(d)])
                      for r in range(d)], axis=-1)                 # [q, dof, r]
        return np.einsum("q,qir,qrs,qjs->ij", Wq, G, Q, G)

    def dense_P(self):
        """Eq. (prec) in Kronecker form with K_k acting on index i_k:
        P = sum_k (x)_{l} (K_l if l == k else M_l), direction 1 fastest."""
        pens = [self.pencil(k) for k in range(self.d)]
        P = 0
        for k in range(self.d):
            T = np.ones((1, 1))
            for l in reversed(range(self.d)):
                T = np.kron(T, pens[l][0] if l == k else pens[l][1])
            P = P + T
        return P


_BLAS_THREAD_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def sine_load(*x):
    """The manufactured load f = d pi^2 prod_k sin(pi x_k) of u = prod_k
    sin(pi x_k) (-Laplace u = f, kappa = 1; the right-hand side used for the
    3D workloads, which the paper does not state)."""
    v = len(x) * np.pi ** 2
    for xk in x:
        v = v * np.sin(np.pi * xk)
    return v


def _split(items, parts):
    """items cut into `parts` contiguous, nearly equal runs."""
    bounds = np.linspace(0, len(items), parts + 1).round().astype(int)
    return [items[bounds[w]:bounds[w + 1]] for w in range(parts)]


def _spawn_map(fn, *iterables):
    """fn over the iterables in spawned worker processes (one per item), in
    order, each with a single BLAS thread (the workers use every core)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    n = len(iterables[0])
    saved = {v: os.environ.get(v) for v in _BLAS_THREAD_VARS}
    os.environ.update({v: "1" for v in _BLAS_THREAD_VARS})
    try:
        with cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(fn, *iterables))
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val


def _rhs_planes(disc: Discretization, f, planes):
    """Load-vector sum over the given element planes of the slowest
    direction, from zero in plane order, over the rows they couple to.
    Returns (first row, b_part)."""
    if not planes:
        return 0, None
    r0, r1 = disc._row_range(planes[0][0], planes[-1][1])
    part = np.zeros(r1 - r0)
    for e0, e1 in planes:
        elo, ehi = disc._plane_box_full(e0, e1)
        disc._rhs_box(f, elo, ehi, part, r0)
    return r0, part


def _assemble_planes(disc: Discretization, planes):
    """One worker of Discretization.assemble_stencil: the sum, from zero and
    in plane order, of the element matrices of the given planes of the
    slowest direction, over the contiguous rows they couple to.
    Returns (first row, S_part[o, rows])."""
    if not planes:
        return 0, None
    r0, r1 = disc._row_range(planes[0][0], planes[-1][1])
    part = np.zeros((disc.n_offsets(), r1 - r0))
    for e0, e1 in planes:
        for elo, ehi in disc._plane_boxes(e0, e1):
            disc._scatter_box(part, elo, ehi, row0=r0)
    return r0, part


def stencil_to_csr(disc: Discretization, S):
    """Sparse CSR form of an offset array S[o, row]."""
    d, p, N = disc.d, disc.p, disc.N
    rows, cols, vals = [], [], []
    idx = np.arange(N)
    multi = []
    rem = idx.copy()
    for k in range(d):
        multi.append(rem % disc.n[k]); rem //= disc.n[k]
    for delta in itertools.product(range(-p, p + 1), repeat=d):
        delta = delta[::-1]  # product varies the last slot fastest; keep dir 1 fastest
        o = int(disc.offset_index(delta))
        ok = np.ones(N, bool)
        for k in range(d):
            ok &= (multi[k] + delta[k] >= 0) & (multi[k] + delta[k] < disc.n[k])
        col = disc.row_index([multi[k] + delta[k] for k in range(d)])
        rows.append(idx[ok]); cols.append(col[ok]); vals.append(S[o][ok])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def apply_stencil(disc: Discretization, S, x):
    """y[row] = sum_o S[o, row] x[row + delta(o)], zero outside the box."""
    d, p = disc.d, disc.p
    X = x.reshape(tuple(reversed(disc.n)))
    Y = np.zeros_like(X)
    Sv = S.reshape((-1,) + tuple(reversed(disc.n)))
    for delta in itertools.product(range(-p, p + 1), repeat=d):
        delta = delta[::-1]
        o = int(disc.offset_index(delta))
        dst, src = [], []
        for k in reversed(range(d)):          # array axes: slowest first
            dk, nk = delta[k], disc.n[k]
            dst.append(slice(max(0, -dk), min(nk, nk - dk)))
            src.append(slice(max(0, dk), min(nk, nk + dk)))
        Y[tuple(dst)] += Sv[o][tuple(dst)] * X[tuple(src)]
    return Y.ravel()
