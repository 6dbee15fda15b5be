// Device-side geometry of a patch: views of the per-direction tables,
// B-spline evaluation, the map F and its Jacobian, the coefficient field and
// Q = kappa |det J| J^{-1} J^{-T} at quadrature points. Shared by the set-up
// kernels and the learned-scaling kernels.
#pragma once

#include "common.cuh"

namespace igafd_geom {

// Device-visible view of the patch tables (passed by value to kernels).
struct PV {
  int dim, p, gp, nq, kp;
  int ds;                        // first function kept per direction (1: Dirichlet removed, 0: full)
  int n[3], nel[3], gm[3], km[3];
  const int *span[3];
  const double *w[3], *bv[3], *bd[3], *gv[3], *gd[3], *kv[3];
  const int *gspan[3], *kspan[3];
  const double *ctrl, *kctrl;
  double kappa;
};

inline PV make_view(const igafd_patch *P) {
  PV v{};
  v.dim = P->dim; v.p = P->p; v.gp = P->geo_p; v.nq = P->p + 1; v.kp = P->kappa_p;
  v.ds = P->dshift;
  for (int k = 0; k < 3; ++k) {
    v.n[k] = P->n[k]; v.nel[k] = P->nel[k]; v.gm[k] = P->dir[k].gm;
    v.span[k] = P->dir[k].span; v.w[k] = P->dir[k].w;
    v.bv[k] = P->dir[k].bv; v.bd[k] = P->dir[k].bd;
    v.gv[k] = P->dir[k].gv; v.gd[k] = P->dir[k].gd; v.gspan[k] = P->dir[k].gspan;
    v.km[k] = P->dir[k].km; v.kv[k] = P->dir[k].kv; v.kspan[k] = P->dir[k].kspan;
  }
  v.ctrl = P->ctrl; v.kctrl = P->kctrl; v.kappa = P->kappa;
  return v;
}

// Nonzero degree-p B-splines B_{s-p..s} and their derivatives at u in span s
// (triangular Cox-de Boor scheme; derivatives from the degree p-1 values).
__device__ inline void bspline_local(const double *xi, int s, double u, int p, double *N, double *dN) {
  double left[IGAFD_MAXP + 1], right[IGAFD_MAXP + 1], prev[IGAFD_MAXP + 1];
  N[0] = 1.0;
  prev[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = u - xi[s + 1 - j];
    right[j] = xi[s + j] - u;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double den = right[r + 1] + left[j - r];
      double t = den != 0.0 ? N[r] / den : 0.0;
      N[r] = saved + right[r + 1] * t;
      saved = left[j - r] * t;
    }
    N[j] = saved;
    if (j == p - 1)
      for (int r = 0; r <= j; ++r) prev[r] = N[r];
  }
  // prev[b] = B_{s-p+1+b, p-1}, b = 0..p-1
  for (int a = 0; a <= p; ++a) {
    int i = s - p + a;
    double d = 0.0;
    if (a >= 1) {
      double den = xi[i + p] - xi[i];
      if (den != 0.0) d += p * prev[a - 1] / den;
    }
    if (a <= p - 1) {
      double den = xi[i + p + 1] - xi[i + 1];
      if (den != 0.0) d -= p * prev[a] / den;
    }
    dN[a] = d;
  }
}

// x = F(zeta) and J = dF/dzeta at the quadrature point with 1D indices t[k].
template <int DIM>
__device__ void geo_eval(const PV &v, const int *t, double *x, double (*J)[3]) {
  const int gp = v.gp, ga = gp + 1;
  const double *gv[3], *gd[3];
  int g0[3];
  for (int k = 0; k < DIM; ++k) {
    gv[k] = v.gv[k] + (size_t)t[k] * ga;
    gd[k] = v.gd[k] + (size_t)t[k] * ga;
    g0[k] = v.gspan[k][t[k]] - gp;
  }
  for (int c = 0; c < DIM; ++c) {
    x[c] = 0.0;
    for (int j = 0; j < DIM; ++j) J[c][j] = 0.0;
  }
  if (DIM == 2) {
    for (int c = 0; c < 2; ++c) {
      const double *C = v.ctrl + (size_t)c * v.gm[0] * v.gm[1];
      for (int a2 = 0; a2 < ga; ++a2) {
        const double *row = C + (size_t)(g0[1] + a2) * v.gm[0] + g0[0];
        double s0 = 0.0, s1 = 0.0;
        for (int a1 = 0; a1 < ga; ++a1) {
          s0 += row[a1] * gv[0][a1];
          s1 += row[a1] * gd[0][a1];
        }
        x[c] += s0 * gv[1][a2];
        J[c][0] += s1 * gv[1][a2];
        J[c][1] += s0 * gd[1][a2];
      }
    }
  } else {
    for (int c = 0; c < 3; ++c) {
      const double *C = v.ctrl + (size_t)c * v.gm[0] * v.gm[1] * v.gm[2];
      for (int a3 = 0; a3 < ga; ++a3) {
        double v3 = gv[2][a3], d3 = gd[2][a3];
        for (int a2 = 0; a2 < ga; ++a2) {
          const double *row =
              C + ((size_t)(g0[2] + a3) * v.gm[1] + (g0[1] + a2)) * v.gm[0] + g0[0];
          double s0 = 0.0, s1 = 0.0;
          for (int a1 = 0; a1 < ga; ++a1) {
            s0 += row[a1] * gv[0][a1];
            s1 += row[a1] * gd[0][a1];
          }
          double v2 = gv[1][a2], d2 = gd[1][a2];
          x[c] += s0 * v2 * v3;
          J[c][0] += s1 * v2 * v3;
          J[c][1] += s0 * d2 * v3;
          J[c][2] += s0 * v2 * d3;
        }
      }
    }
  }
}

// Q = kappa |det J| J^{-1} J^{-T}; returns det J. Q stored symmetric:
// 2D [00, 11, 01], 3D [00, 11, 22, 01, 02, 12].
template <int DIM>
__device__ double q_from_J(const double (*J)[3], double kappa, double *Q) {
  if (DIM == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double id = 1.0 / det;
    double Ji[2][2] = {{J[1][1] * id, -J[0][1] * id}, {-J[1][0] * id, J[0][0] * id}};
    double sc = kappa * fabs(det);
    Q[0] = sc * (Ji[0][0] * Ji[0][0] + Ji[0][1] * Ji[0][1]);
    Q[1] = sc * (Ji[1][0] * Ji[1][0] + Ji[1][1] * Ji[1][1]);
    Q[2] = sc * (Ji[0][0] * Ji[1][0] + Ji[0][1] * Ji[1][1]);
    return det;
  } else {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    double id = 1.0 / det;
    double Ji[3][3];
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    double sc = kappa * fabs(det);
    const int rr[6] = {0, 1, 2, 0, 0, 1}, ss[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
      double acc = 0.0;
      for (int c = 0; c < 3; ++c) acc += Ji[rr[q]][c] * Ji[ss[q]][c];
      Q[q] = sc * acc;
    }
    return det;
  }
}

__device__ __forceinline__ int qidx(int r, int s, int dim) {
  if (r == s) return r;
  if (dim == 2) return 2;
  int lo = r < s ? r : s, hi = r < s ? s : r;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// Extreme eigenvalues of a symmetric 2x2 / 3x3 matrix (closed form).
template <int DIM>
__device__ void sym_eig_extremes(const double *Q, double *lmin, double *lmax) {
  if (DIM == 2) {
    double m = 0.5 * (Q[0] + Q[1]);
    double d = sqrt(0.25 * (Q[0] - Q[1]) * (Q[0] - Q[1]) + Q[2] * Q[2]);
    *lmin = m - d; *lmax = m + d;
  } else {
    double a = Q[0], b = Q[1], c = Q[2], d = Q[3], e = Q[5], f = Q[4];
    double p1 = d * d + f * f + e * e;
    double q = (a + b + c) / 3.0;
    double p2 = (a - q) * (a - q) + (b - q) * (b - q) + (c - q) * (c - q) + 2.0 * p1;
    double pp = sqrt(p2 / 6.0);
    if (pp < 1e-300) { *lmin = *lmax = q; return; }
    double B00 = (a - q) / pp, B11 = (b - q) / pp, B22 = (c - q) / pp;
    double B01 = d / pp, B02 = f / pp, B12 = e / pp;
    double detB = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) +
                  B02 * (B01 * B12 - B11 * B02);
    double r = fmin(1.0, fmax(-1.0, 0.5 * detB));
    double phi = acos(r) / 3.0;
    double e1 = q + 2.0 * pp * cos(phi);
    double e3 = q + 2.0 * pp * cos(phi + 2.0 * M_PI / 3.0);
    *lmax = e1; *lmin = e3;
  }
}

// Coefficient kappa(zeta) = kappa * sum_i c_i B_i(zeta) at the quadrature
// point with 1D indices t[k] (the constant kappa when no field is given).
template <int DIM>
__device__ double kappa_eval(const PV &v, const int *t) {
  if (!v.kctrl) return v.kappa;
  const int ka = v.kp + 1;
  const double *kv[3];
  int k0[3];
  for (int k = 0; k < DIM; ++k) {
    kv[k] = v.kv[k] + (size_t)t[k] * ka;
    k0[k] = v.kspan[k][t[k]] - v.kp;
  }
  double acc = 0.0;
  if (DIM == 2) {
    for (int a2 = 0; a2 < ka; ++a2) {
      const double *row = v.kctrl + (size_t)(k0[1] + a2) * v.km[0] + k0[0];
      double s0 = 0.0;
      for (int a1 = 0; a1 < ka; ++a1) s0 += row[a1] * kv[0][a1];
      acc += s0 * kv[1][a2];
    }
  } else {
    for (int a3 = 0; a3 < ka; ++a3)
      for (int a2 = 0; a2 < ka; ++a2) {
        const double *row =
            v.kctrl + ((size_t)(k0[2] + a3) * v.km[1] + (k0[1] + a2)) * v.km[0] + k0[0];
        double s0 = 0.0;
        for (int a1 = 0; a1 < ka; ++a1) s0 += row[a1] * kv[0][a1];
        acc += s0 * kv[1][a2] * kv[2][a3];
      }
  }
  return v.kappa * acc;
}


}  // namespace igafd_geom
