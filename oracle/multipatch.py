"""Multi-patch problems and the overlapping Schwarz preconditioners of
Section 6 (Eqs. (Peas), (Pias)) on the three-patch L-shaped domain of
Section 7.3 (oracle; test infrastructure only).

Domain: the L made of three unit squares, Omega_1 = [0,1] x [1,2] (top),
Omega_2 = [0,1] x [0,1] (corner), Omega_3 = [1,2] x [0,1] (right); each patch
is its parameter square translated (identity Jacobian), carries the same
open knot vector in both directions and degree p, and neighbouring patches
are glued C^0 (their shared edges carry the same control points), with
homogeneous Dirichlet conditions on the boundary of the L.

Subdomains (Section 6): Theta_1 = Omega_1 u Omega_2 = [0,1] x [0,2] and
Theta_2 = Omega_2 u Omega_3 = [0,2] x [0,1]; R_i restricts to the degrees of
freedom of Theta_i's basis functions that vanish on its boundary, so that
A_i = R_i A R_i^T is the stiffness matrix of the Poisson problem on Theta_i
with homogeneous Dirichlet conditions. Theta_i is one patch over [0,1]^2 with
the merged knot vector (the two halves rescaled to [0, 1/2] and [1/2, 1], the
interface knot 1/2 repeated p times: C^0) in its long direction.

Readings (the paper gives Figure "L" but no coordinates, tolerance or load):
 - the unit-square layout above, with h the knot spacing of each patch;
 - P_i of Eq. (prec) for Theta_i is built from the parametric pencils of its
   merged knot vectors, without the factor-2 stretch of the long direction
   (the paper leaves the stretch out of the preconditioner on purpose);
 - CG to a relative residual of 1e-8 from x_0 = 0 with a right-hand side of
   i.i.d. N(0, 1) entries (as in the paper's cube test).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble
from .fd import FD

# patch origins in the L; shared edges: (Omega_2 top, Omega_1 bottom),
# (Omega_2 right, Omega_3 left)
ORIGINS = {1: (0, 1), 2: (0, 0), 3: (1, 0)}
INTERFACE_EDGES = {1: {"bottom"}, 2: {"top", "right"}, 3: {"left"}}


def pencils_1d(knots, p, full):
    """1D stiffness and mass matrices on the knot vector (Section 3)."""
    m = len(knots) - p - 1
    geo = assemble.Geometry(np.zeros((1, m)), [knots], p)
    return assemble.Discretization([knots], p, geo).pencil(0, full=full)


def merged_knots(knots, p):
    """Knot vector on [0, 1] of two copies of `knots` (on [0, 1]) placed on
    [0, 1/2] and [1/2, 1], with the interface knot 1/2 repeated p times."""
    kn = np.asarray(knots, dtype=np.float64)
    inner = kn[p + 1:len(kn) - p - 1]
    return np.concatenate([np.zeros(p + 1), 0.5 * inner, np.full(p, 0.5), 0.5 + 0.5 * inner,
                           np.ones(p + 1)])


class LShape:
    """Global C^0 multi-patch space on the L, its stiffness matrix A and the
    subdomain restrictions of Section 6."""

    def __init__(self, knots, p):
        self.knots = np.asarray(knots, dtype=np.float64)
        self.p = int(p)
        self.m = len(self.knots) - self.p - 1          # functions per direction per patch
        K, M = pencils_1d(self.knots, self.p, full=True)
        self.K1d, self.M1d = K, M
        m = self.m
        # global numbering: a patch's control point (i1, i2) sits at
        # origin + (i1, i2) / (m - 1) on a lattice where shared edges coincide
        key_of = {}
        self.local_to_global = {}
        for q in (1, 2, 3):
            ox, oy = ORIGINS[q]
            g = np.empty((m, m), dtype=np.int64)       # [i2, i1]
            for i2 in range(m):
                for i1 in range(m):
                    key = (ox * (m - 1) + i1, oy * (m - 1) + i2)
                    if key not in key_of:
                        key_of[key] = len(key_of)
                    g[i2, i1] = key_of[key]
            self.local_to_global[q] = g
        self.n_full = len(key_of)
        # Dirichlet: a global function is fixed when any of its patch copies
        # lies on a patch edge that is not an interface
        fixed = np.zeros(self.n_full, dtype=bool)
        for q in (1, 2, 3):
            g = self.local_to_global[q]
            edges = {"bottom": g[0, :], "top": g[-1, :], "left": g[:, 0], "right": g[:, -1]}
            for name, ids in edges.items():
                if name not in INTERFACE_EDGES[q]:
                    fixed[ids] = True
        self.free = np.flatnonzero(~fixed)
        self.index = -np.ones(self.n_full, dtype=np.int64)
        self.index[self.free] = np.arange(len(self.free))
        self.N = len(self.free)
        # A = sum over patches of the scattered patch stiffness (identity
        # Jacobian: the Kronecker sum of the full 1D pencils, Eq. (A))
        Kp = (sp.kron(sp.csr_matrix(M), sp.csr_matrix(K)) + sp.kron(sp.csr_matrix(K), sp.csr_matrix(M))).tocoo()
        rows, cols, vals = [], [], []
        for q in (1, 2, 3):
            g = self.local_to_global[q].ravel()          # local index i1 + m i2
            rows.append(g[Kp.row]); cols.append(g[Kp.col]); vals.append(Kp.data)
        Af = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(self.n_full, self.n_full))
        self.A = Af[self.free][:, self.free].tocsr()
        self.sub = [self._subdomain(1), self._subdomain(2)]

    def _subdomain(self, i):
        """Global free indices of Theta_i's interior functions, in the order of
        the merged single patch (direction 1 fastest, Dirichlet removed)."""
        m = self.m
        if i == 1:     # Theta_1 = Omega_2 (lower half) u Omega_1 (upper half), long direction 2
            n1, n2 = m - 2, 2 * m - 3
            out = np.empty((n2, n1), dtype=np.int64)
            for j2 in range(1, 2 * m - 2):
                for j1 in range(1, m - 1):
                    if j2 <= m - 1:
                        gid = self.local_to_global[2][j2, j1]
                    else:
                        gid = self.local_to_global[1][j2 - (m - 1), j1]
                    out[j2 - 1, j1 - 1] = gid
        else:          # Theta_2 = Omega_2 (left half) u Omega_3 (right half), long direction 1
            n1, n2 = 2 * m - 3, m - 2
            out = np.empty((n2, n1), dtype=np.int64)
            for j2 in range(1, m - 1):
                for j1 in range(1, 2 * m - 2):
                    if j1 <= m - 1:
                        gid = self.local_to_global[2][j2, j1]
                    else:
                        gid = self.local_to_global[3][j2, j1 - (m - 1)]
                    out[j2 - 1, j1 - 1] = gid
        idx = self.index[out.ravel()]
        if np.any(idx < 0):
            raise AssertionError("a subdomain interior function is fixed")
        return idx, (n1, n2)

    def restriction(self, i):
        """R_i as a sparse matrix (rows: Theta_i's functions)."""
        idx, _ = self.sub[i]
        return sp.csr_matrix((np.ones(len(idx)), (np.arange(len(idx)), idx)), shape=(len(idx), self.N))

    def merged_pencils(self, i):
        """Parametric pencils [(K_1, M_1), (K_2, M_2)] of Theta_i as one patch
        over [0, 1]^2 (merged knot vector in the long direction)."""
        kn = self.knots
        km = merged_knots(kn, self.p)
        dirs = [kn, km] if i == 0 else [km, kn]
        return [pencils_1d(k, self.p, full=False) for k in dirs]

    def merged_discretization(self, i):
        """Theta_i as a single patch with the physical map
        F(zeta) = (zeta_1, 2 zeta_2) (i = 0) or (2 zeta_1, zeta_2) (i = 1)."""
        kn = self.knots
        km = merged_knots(kn, self.p)
        knots = [kn, km] if i == 0 else [km, kn]
        sx, sy = (1.0, 2.0) if i == 0 else (2.0, 1.0)
        ctrl = np.array([[[0.0, sx], [0.0, sx]], [[0.0, 0.0], [sy, sy]]])   # degree-1 net
        geo = assemble.Geometry(ctrl, [np.array([0, 0, 1, 1.0])] * 2, 1)
        return assemble.Discretization(knots, self.p, geo)


class AdditiveSchwarz:
    """Eq. (Peas) (exact local solves) or Eq. (Pias) with the local inverse
    approximated by the fast-diagonalization P_i of Theta_i."""

    def __init__(self, L: LShape, exact: bool):
        self.L = L
        self.R = [L.restriction(i) for i in range(2)]
        if exact:
            self.local = [spla.splu((R @ L.A @ R.T).tocsc()).solve for R in self.R]
        else:
            self.local = [FD(L.merged_pencils(i)).apply for i in range(2)]

    def apply(self, r):
        z = np.zeros_like(r)
        for R, solve in zip(self.R, self.local):
            z += R.T @ solve(R @ r)
        return z
