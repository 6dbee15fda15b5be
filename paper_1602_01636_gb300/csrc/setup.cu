// Patch setup on the device: per-direction quadrature/basis tables, the
// geometry map, the (2p+1)^d stiffness stencil of Eq. (A) and the
// manufactured right-hand side.
//
// Quadrature: (p+1)-point Gauss-Legendre per element and direction.
// Q = kappa |det J| J^{-1} J^{-T} (chain rule with J_ij = dx_i/dzeta_j; the
// paper prints the transposes the other way round in Eq. (Q)).
#include "common.cuh"

#include <algorithm>
#include "geom.cuh"

#include <cmath>
#include <vector>

namespace {

using namespace igafd_geom;


// i-th node (ascending) and weight of the nq-point Gauss-Legendre rule on
// [-1, 1] by Newton's method on the Legendre polynomial P_nq.
__device__ void gauss_node(int nq, int i, double *x, double *w) {
  int ir = nq - 1 - i;  // Newton guess ordering is descending
  double z = cos(M_PI * (ir + 0.75) / (nq + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= nq; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1; p1 = p2;
    }
    if (nq == 1) { p1 = z; p0 = 1.0; }
    dp = nq * (z * p1 - p0) / (z * z - 1.0);
    double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= nq; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1; p1 = p2;
    }
    dp = nq * (z * p1 - p0) / (z * z - 1.0);
  }
  *x = z;
  *w = 2.0 / ((1.0 - z * z) * dp * dp);
}

// Span s of a knot vector with xi_s <= z < xi_{s+1}, s in [deg, m-1].
__device__ int find_span(const double *xi, int deg, int m, double z) {
  int lo = deg, hi = m - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (xi[mid] <= z) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One thread per 1D quadrature point of one direction.
__global__ void tables_kernel(Dir1D D, int p, int gp, int kp) {
  int nq = p + 1;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D.nel * nq) return;
  int e = t / nq, g = t % nq;
  int s = D.span[e];
  double a = D.knots[s], b = D.knots[s + 1];
  double xg, wg;
  gauss_node(nq, g, &xg, &wg);
  double z = 0.5 * (a + b) + 0.5 * (b - a) * xg;
  D.z[t] = z;
  D.w[t] = 0.5 * (b - a) * wg;
  double N[IGAFD_MAXP + 1], dN[IGAFD_MAXP + 1];
  bspline_local(D.knots, s, z, p, N, dN);
  for (int i = 0; i <= p; ++i) {
    D.bv[t * (p + 1) + i] = N[i];
    D.bd[t * (p + 1) + i] = dN[i];
  }
  // geometry span: xi_gs <= z < xi_{gs+1}, gs in [gp, gm-1]
  const int gs = find_span(D.gknots, gp, D.gm, z);
  D.gspan[t] = gs;
  bspline_local(D.gknots, gs, z, gp, N, dN);
  for (int i = 0; i <= gp; ++i) {
    D.gv[t * (gp + 1) + i] = N[i];
    D.gd[t * (gp + 1) + i] = dN[i];
  }
  if (D.kknots) {   // coefficient field
    const int ks = find_span(D.kknots, kp, D.km, z);
    D.kspan[t] = ks;
    bspline_local(D.kknots, ks, z, kp, N, dN);
    for (int i = 0; i <= kp; ++i) D.kv[t * (kp + 1) + i] = N[i];
  }
}

// Geometry diagnostics over every quadrature point: min det J and the Prop. 1
// extremes sup lambda_max(Q), inf lambda_min(Q) (per-block partials).
template <int DIM>
__global__ void geo_check_kernel(PV v, long long nqp, double *part) {
  __shared__ double sh[32];
  double mdet = 1e300, lmin = 1e300, lmax = -1e300;
  const int nq = v.nq;
  const long long tot1 = (long long)v.nel[0] * nq, tot2 = (long long)v.nel[1] * nq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nqp;
       i += (long long)gridDim.x * blockDim.x) {
    int t[3];
    t[0] = (int)(i % tot1);
    t[1] = (int)((i / tot1) % tot2);
    t[2] = DIM == 3 ? (int)(i / (tot1 * tot2)) : 0;
    double x[3], J[3][3], Q[6];
    geo_eval<DIM>(v, t, x, J);
    double det = q_from_J<DIM>(J, kappa_eval<DIM>(v, t), Q);
    mdet = fmin(mdet, det);
    double a, b;
    sym_eig_extremes<DIM>(Q, &a, &b);
    lmin = fmin(lmin, a);
    lmax = fmax(lmax, b);
  }
  // block min/max via negation trick on sums is not possible; use shuffles
  for (int o = 16; o > 0; o >>= 1) {
    mdet = fmin(mdet, __shfl_xor_sync(0xffffffffu, mdet, o));
    lmin = fmin(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  }
  __shared__ double s3[3][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s3[0][wid] = mdet; s3[1][wid] = lmin; s3[2][wid] = lmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mdet = fmin(mdet, s3[0][w]); lmin = fmin(lmin, s3[1][w]); lmax = fmax(lmax, s3[2][w]);
    }
    part[3 * blockIdx.x + 0] = mdet;
    part[3 * blockIdx.x + 1] = lmin;
    part[3 * blockIdx.x + 2] = lmax;
  }
  (void)sh;
}

// Stiffness assembly, one thread block per element of one colour class
// (element index = colour mod (p+1) per direction), so that no two blocks of
// a launch touch the same stencil entry: plain read-modify-write, fixed
// summation order, deterministic.
//
// Local matrix L[a][b] = sum_g sum_{r,s} Q_rs(g) dB_a/dzeta_r dB_b/dzeta_s,
// evaluated by sum factorisation over the tensor quadrature points: for each
// (r, s) contract direction 1, then direction 2, and accumulate by the
// derivative pattern of direction 3 (or 2 in 2D), then contract the last
// direction per output entry.
//
// PERPAT: keep the partial sums of one derivative pattern of direction 3 at
// a time in shared memory (each (r, s) term belongs to exactly one pattern,
// so nothing is recomputed; the stencil is accumulated once per pattern).
// Needed for p >= 5 in 3D, where all four patterns would not fit.
// The stencil entry of offset index o and row i goes to
// stencil[(o - o_min) ld + H + i]; offsets below o_min are not stored (the
// full layout: o_min = 0, H = 0, ld = Np; the half layout: o_min the centre).
template <int DIM, bool PERPAT>
__global__ void assemble_kernel(PV v, int c1, int c2, int c3, int ne1, int ne2,
                                double *__restrict__ stencil, long long ld, int o_min,
                                long long H) {
  extern __shared__ double sm[];
  const int p = v.p, A = p + 1, nq = p + 1, W = 2 * p + 1;
  const int nqd = DIM == 3 ? nq * nq * nq : nq * nq;
  const int nQ = DIM == 3 ? 6 : 3;
  // element of this block
  int bid = blockIdx.x;
  int e1 = c1 + (p + 1) * (bid % ne1);
  int e2 = c2 + (p + 1) * ((bid / ne1) % ne2);
  int e3 = DIM == 3 ? c3 + (p + 1) * (bid / (ne1 * ne2)) : 0;
  int e[3] = {e1, e2, e3};
  double *Qs = sm;                          // [nQ][nqd]
  double *F = Qs + nQ * nqd;                // [DIM][2][A][nq]: basis value/deriv per direction
  double *T1 = F + DIM * 2 * A * nq;        // 3D: [A*A][nq][nq], 2D: unused
  double *G = T1 + (DIM == 3 ? A * A * nq * nq : 0);  // 3D: [4][A*A][A*A][nq], 2D: [4][A*A][nq]
  const int AA = A * A;
  constexpr int kSlots = PERPAT ? 1 : 4;
  const int Gsz = DIM == 3 ? kSlots * AA * AA * nq : 4 * AA * nq;
  // tables
  for (int i = threadIdx.x; i < DIM * 2 * A * nq; i += blockDim.x) {
    int g = i % nq, a = (i / nq) % A, vd = (i / (nq * A)) % 2, k = i / (2 * nq * A);
    size_t t = (size_t)e[k] * nq + g;
    F[i] = (vd ? v.bd[k] : v.bv[k])[t * A + a];
  }
  // Q at the element's quadrature points, with weights folded in
  for (int g = threadIdx.x; g < nqd; g += blockDim.x) {
    int gq[3] = {g % nq, (g / nq) % nq, DIM == 3 ? g / (nq * nq) : 0};
    int t[3];
    for (int k = 0; k < DIM; ++k) t[k] = e[k] * nq + gq[k];
    double x[3], J[3][3], Q[6];
    geo_eval<DIM>(v, t, x, J);
    q_from_J<DIM>(J, kappa_eval<DIM>(v, t), Q);
    double wt = 1.0;
    for (int k = 0; k < DIM; ++k) wt *= v.w[k][t[k]];
    for (int q = 0; q < nQ; ++q) Qs[q * nqd + g] = Q[q] * wt;
  }
  __syncthreads();
#define FV(k, vd, a, g) F[(((k) * 2 + (vd)) * A + (a)) * nq + (g)]
  for (int pp = 0; pp < (PERPAT ? 4 : 1); ++pp) {
  for (int i = threadIdx.x; i < Gsz; i += blockDim.x) G[i] = 0.0;
  __syncthreads();
  for (int r = 0; r < DIM; ++r) {
    for (int s = 0; s < DIM; ++s) {
      if (PERPAT && 2 * (r == 2) + (s == 2) != pp) continue;
      const double *Qrs = Qs + qidx(r, s, DIM) * nqd;
      const int ra = (r == 0), sa = (s == 0);       // derivative pattern, dir 1
      const int rb = (r == 1), sb = (s == 1);       // dir 2
      if (DIM == 3) {
        // T1[a1b1][g2][g3] = sum_g1 f1(a1,g1) f1'(b1,g1) Q(g1,g2,g3)
        for (int i = threadIdx.x; i < AA * nq * nq; i += blockDim.x) {
          int g23 = i % (nq * nq), ab = i / (nq * nq);
          int a1 = ab % A, b1 = ab / A;
          double acc = 0.0;
          for (int g1 = 0; g1 < nq; ++g1)
            acc += FV(0, ra, a1, g1) * FV(0, sa, b1, g1) * Qrs[g23 * nq + g1];
          T1[i] = acc;
        }
        __syncthreads();
        // G[pat3][a1b1][a2b2][g3] += sum_g2 f2(a2,g2) f2'(b2,g2) T1[a1b1][g2][g3]
        const int pat = PERPAT ? 0 : 2 * (r == 2) + (s == 2);
        double *Gp = G + (size_t)pat * AA * AA * nq;
        for (int i = threadIdx.x; i < AA * AA * nq; i += blockDim.x) {
          int g3 = i % nq, ab2 = (i / nq) % AA, ab1 = i / (nq * AA);
          int a2 = ab2 % A, b2 = ab2 / A;
          double acc = 0.0;
          for (int g2 = 0; g2 < nq; ++g2)
            acc += FV(1, rb, a2, g2) * FV(1, sb, b2, g2) * T1[(ab1 * nq + g3) * nq + g2];
          Gp[i] += acc;
        }
        __syncthreads();
      } else {
        // G[pat2][a1b1][g2] += sum_g1 f1 f1' Q(g1, g2)
        const int pat = 2 * (r == 1) + (s == 1);
        double *Gp = G + (size_t)pat * AA * nq;
        for (int i = threadIdx.x; i < AA * nq; i += blockDim.x) {
          int g2 = i % nq, ab = i / nq;
          int a1 = ab % A, b1 = ab / A;
          double acc = 0.0;
          for (int g1 = 0; g1 < nq; ++g1)
            acc += FV(0, ra, a1, g1) * FV(0, sa, b1, g1) * Qrs[g2 * nq + g1];
          Gp[i] += acc;
        }
        __syncthreads();
      }
    }
  }
  // Output entries (a, delta): consecutive threads take consecutive a_1 with
  // the same offset, so their stencil addresses are contiguous.
  const int last = DIM - 1;
  int nent = 1;
  for (int k = 0; k < DIM; ++k) nent *= A * W;
  for (int i = threadIdx.x; i < nent; i += blockDim.x) {
    int rem = i;
    int a[3], dl[3], b[3];
    bool ok = true;
    for (int k = 0; k < DIM; ++k) {
      a[k] = rem % A; rem /= A;
      dl[k] = rem % W - p; rem /= W;
      b[k] = a[k] + dl[k];
      ok = ok && b[k] >= 0 && b[k] < A;
    }
    if (!ok) continue;
    // global indices: full index I = span - p + a, kept i = I - ds (ds = 1:
    // Dirichlet functions removed, 0: the full space)
    long long row = 0, stride = 1;
    for (int k = 0; k < DIM; ++k) {
      int I = v.span[k][e[k]] - p + a[k];
      int J = I + dl[k];
      if (I < v.ds || I >= v.ds + v.n[k] || J < v.ds || J >= v.ds + v.n[k]) { ok = false; break; }
      row += (long long)(I - v.ds) * stride;
      stride *= v.n[k];
    }
    if (!ok) continue;
    double val = 0.0;
    if (DIM == 3) {
      int ab1 = a[0] + A * b[0], ab2 = a[1] + A * b[1];
      for (int pat = (PERPAT ? pp : 0); pat < (PERPAT ? pp + 1 : 4); ++pat) {
        const double *Gp = G + (((size_t)(PERPAT ? 0 : pat) * AA + ab1) * AA + ab2) * nq;
        int da = pat >> 1, db = pat & 1;
        for (int g3 = 0; g3 < nq; ++g3)
          val += FV(last, da, a[2], g3) * FV(last, db, b[2], g3) * Gp[g3];
      }
    } else {
      int ab1 = a[0] + A * b[0];
      for (int pat = 0; pat < 4; ++pat) {
        const double *Gp = G + ((size_t)pat * AA + ab1) * nq;
        int da = pat >> 1, db = pat & 1;
        for (int g2 = 0; g2 < nq; ++g2)
          val += FV(last, da, a[1], g2) * FV(last, db, b[1], g2) * Gp[g2];
      }
    }
    int o = 0, ws = 1;
    for (int k = 0; k < DIM; ++k) { o += (dl[k] + p) * ws; ws *= W; }
    if (o >= o_min) stencil[(size_t)(o - o_min) * ld + H + row] += val;
  }
  __syncthreads();
  }   // pattern pass
#undef FV
}

// Right-hand side b_i = sum_q f(x_q) B_i(zeta_q) |det J(zeta_q)| w_q, one
// block per element of a colour class (same colouring as the stiffness
// assembly): f from fq[q] at the tensor quadrature point q = t_1 + T_1 (t_2 +
// T_2 t_3) (T_k = nel_k (p + 1) 1D points of direction k), or, with fq null,
// the manufactured f = d pi^2 prod sin(pi x_k).
template <int DIM>
__global__ void rhs_kernel(PV v, int c1, int c2, int c3, int ne1, int ne2, const double *fq,
                           double *b) {
  extern __shared__ double sm[];
  const int p = v.p, A = p + 1, nq = p + 1;
  const int nqd = DIM == 3 ? nq * nq * nq : nq * nq;
  int bid = blockIdx.x;
  int e[3];
  e[0] = c1 + (p + 1) * (bid % ne1);
  e[1] = c2 + (p + 1) * ((bid / ne1) % ne2);
  e[2] = DIM == 3 ? c3 + (p + 1) * (bid / (ne1 * ne2)) : 0;
  double *fw = sm;  // [nqd]
  for (int g = threadIdx.x; g < nqd; g += blockDim.x) {
    int gq[3] = {g % nq, (g / nq) % nq, DIM == 3 ? g / (nq * nq) : 0};
    int t[3];
    for (int k = 0; k < DIM; ++k) t[k] = e[k] * nq + gq[k];
    double x[3], J[3][3], Q[6];
    geo_eval<DIM>(v, t, x, J);
    double det = q_from_J<DIM>(J, 1.0, Q);
    double f;
    if (fq) {
      const long long T0 = (long long)v.nel[0] * nq, T1 = (long long)v.nel[1] * nq;
      f = fq[t[0] + T0 * (t[1] + (DIM == 3 ? T1 * t[2] : 0))];
    } else {
      f = DIM * M_PI * M_PI;
      for (int k = 0; k < DIM; ++k) f *= sin(M_PI * x[k]);
    }
    double wt = fabs(det);
    for (int k = 0; k < DIM; ++k) wt *= v.w[k][t[k]];
    fw[g] = f * wt;
  }
  __syncthreads();
  int nloc = 1;
  for (int k = 0; k < DIM; ++k) nloc *= A;
  for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
    int a[3] = {i % A, (i / A) % A, DIM == 3 ? i / (A * A) : 0};
    long long row = 0, stride = 1;
    bool ok = true;
    for (int k = 0; k < DIM; ++k) {
      int I = v.span[k][e[k]] - p + a[k];
      if (I < v.ds || I >= v.ds + v.n[k]) { ok = false; break; }
      row += (long long)(I - v.ds) * stride;
      stride *= v.n[k];
    }
    if (!ok) continue;
    double acc = 0.0;
    for (int g = 0; g < nqd; ++g) {
      int gq[3] = {g % nq, (g / nq) % nq, DIM == 3 ? g / (nq * nq) : 0};
      double bv = 1.0;
      for (int k = 0; k < DIM; ++k) bv *= v.bv[k][((size_t)e[k] * nq + gq[k]) * A + a[k]];
      acc += bv * fw[g];
    }
    b[row] += acc;
  }
}

// Physical coordinates x = F(zeta_q) of every tensor quadrature point,
// x[c * Qn + q] with q as in rhs_kernel.
template <int DIM>
__global__ void quad_points_kernel(PV v, long long Qn, double *xout) {
  const int nq = v.p + 1;
  const long long T0 = (long long)v.nel[0] * nq, T1 = (long long)v.nel[1] * nq;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Qn;
       q += (long long)gridDim.x * blockDim.x) {
    int t[3] = {(int)(q % T0), (int)((q / T0) % T1), DIM == 3 ? (int)(q / (T0 * T1)) : 0};
    double x[3], J[3][3];
    geo_eval<DIM>(v, t, x, J);
    for (int c = 0; c < DIM; ++c) xout[c * Qn + q] = x[c];
  }
}

size_t assemble_smem(int dim, int p, bool perpat) {
  size_t A = p + 1, nq = p + 1, AA = A * A;
  size_t nqd = dim == 3 ? nq * nq * nq : nq * nq;
  size_t nQ = dim == 3 ? 6 : 3;
  size_t s = nQ * nqd + dim * 2 * A * nq;
  if (dim == 3) s += AA * nq * nq + (perpat ? 1 : 4) * AA * AA * nq;
  else s += 4 * AA * nq;
  return s * sizeof(double);
}

}  // namespace

// ---------------------------------------------------------------------------
static igafd_status dalloc(void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return IGAFD_ERR_OOM;
  }
  return IGAFD_OK;
}

igafd_status igafd_setup_tables(igafd_patch *P, const igafd_patch_desc *d, cudaStream_t s) {
  const int p = P->p, gp = P->geo_p, nq = p + 1;
  size_t ctrl_count = (size_t)P->dim;
  for (int k = 0; k < 3; ++k) {
    Dir1D &D = P->dir[k];
    if (k >= P->dim) {
      continue;
    }
    std::vector<int> spans;
    const double *kn = d->knots[k];
    int nk = d->n_knots[k];
    for (int i = p; i < nk - p - 1; ++i)
      if (kn[i] < kn[i + 1]) spans.push_back(i);
    D.m = nk - p - 1;
    D.n = D.m - 2 * P->dshift;
    D.nel = (int)spans.size();
    D.gm = d->geo_n_knots[k] - gp - 1;
    ctrl_count *= D.gm;
    int nt = D.nel * nq;
    IGAFD_TRY(dalloc((void **)&D.knots, nk * sizeof(double)));
    IGAFD_TRY(dalloc((void **)&D.gknots, d->geo_n_knots[k] * sizeof(double)));
    IGAFD_TRY(dalloc((void **)&D.span, D.nel * sizeof(int)));
    IGAFD_TRY(dalloc((void **)&D.z, nt * sizeof(double)));
    IGAFD_TRY(dalloc((void **)&D.w, nt * sizeof(double)));
    IGAFD_TRY(dalloc((void **)&D.bv, (size_t)nt * (p + 1) * sizeof(double)));
    IGAFD_TRY(dalloc((void **)&D.bd, (size_t)nt * (p + 1) * sizeof(double)));
    IGAFD_TRY(dalloc((void **)&D.gspan, nt * sizeof(int)));
    IGAFD_TRY(dalloc((void **)&D.gv, (size_t)nt * (gp + 1) * sizeof(double)));
    IGAFD_TRY(dalloc((void **)&D.gd, (size_t)nt * (gp + 1) * sizeof(double)));
    if (d->kappa_ctrl) {
      const int kp = d->kappa_p;
      D.km = d->kappa_n_knots[k] - kp - 1;
      IGAFD_TRY(dalloc((void **)&D.kknots, d->kappa_n_knots[k] * sizeof(double)));
      IGAFD_TRY(dalloc((void **)&D.kspan, nt * sizeof(int)));
      IGAFD_TRY(dalloc((void **)&D.kv, (size_t)nt * (kp + 1) * sizeof(double)));
      IGAFD_CUDA(cudaMemcpyAsync(D.kknots, d->kappa_knots[k], d->kappa_n_knots[k] * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    }
    IGAFD_CUDA(cudaMemcpyAsync(D.knots, kn, nk * sizeof(double), cudaMemcpyHostToDevice, s));
    IGAFD_CUDA(cudaMemcpyAsync(D.gknots, d->geo_knots[k], d->geo_n_knots[k] * sizeof(double),
                               cudaMemcpyHostToDevice, s));
    IGAFD_CUDA(cudaMemcpyAsync(D.span, spans.data(), D.nel * sizeof(int),
                               cudaMemcpyHostToDevice, s));
    // the host vector must outlive the async copy
    IGAFD_CUDA(cudaStreamSynchronize(s));
    tables_kernel<<<(nt + 127) / 128, 128, 0, s>>>(D, p, gp, P->kappa_p);
    IGAFD_CUDA(cudaGetLastError());
    P->n[k] = D.n;
    P->nel[k] = D.nel;
    // directions with identical knot vectors have identical pencils K_k, M_k
    P->twin[k] = k;
    for (int j = 0; j < k; ++j)
      if (P->twin[j] == j && d->n_knots[j] == nk &&
          std::equal(kn, kn + nk, d->knots[j])) {
        P->twin[k] = j;
        break;
      }
  }
  IGAFD_TRY(dalloc((void **)&P->ctrl, ctrl_count * sizeof(double)));
  IGAFD_CUDA(cudaMemcpyAsync(P->ctrl, d->ctrl, ctrl_count * sizeof(double),
                             cudaMemcpyHostToDevice, s));
  if (d->kappa_ctrl) {
    size_t kc = 1;
    for (int k = 0; k < P->dim; ++k) kc *= P->dir[k].km;
    IGAFD_TRY(dalloc((void **)&P->kctrl, kc * sizeof(double)));
    IGAFD_CUDA(cudaMemcpyAsync(P->kctrl, d->kappa_ctrl, kc * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  IGAFD_CUDA(cudaStreamSynchronize(s));
  return IGAFD_OK;
}

igafd_status igafd_setup_stencil(igafd_patch *P, cudaStream_t s) {
  PV v = make_view(P);
  const int p = P->p, dim = P->dim;
  // geometry diagnostics
  long long nqp = 1;
  for (int k = 0; k < dim; ++k) nqp *= (long long)P->nel[k] * (p + 1);
  double *part = P->partial;  // >= 3 * 592 doubles available
  const int gblocks = 592;
  if (dim == 3) geo_check_kernel<3><<<gblocks, 256, 0, s>>>(v, nqp, part);
  else geo_check_kernel<2><<<gblocks, 256, 0, s>>>(v, nqp, part);
  IGAFD_CUDA(cudaGetLastError());
  std::vector<double> h(3 * gblocks);
  IGAFD_CUDA(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  double mdet = 1e300, lmin = 1e300, lmax = -1e300;
  for (int b = 0; b < gblocks; ++b) {
    mdet = fmin(mdet, h[3 * b]);
    lmin = fmin(lmin, h[3 * b + 1]);
    lmax = fmax(lmax, h[3 * b + 2]);
  }
  P->min_detJ = mdet;
  P->q_bound = lmax / lmin;
  if (!(mdet > 0.0)) return IGAFD_ERR_FOLDED;
  // stiffness stencil
  const int o_min = P->stencil_half ? P->n_off / 2 : 0;
  const long long ld = P->stencil_half ? P->sh_ld : P->Np, H = P->stencil_half ? P->sh_H : 0;
  IGAFD_CUDA(cudaMemsetAsync(P->stencil, 0, (size_t)(P->n_off - o_min) * ld * sizeof(double), s));
  const bool perpat = dim == 3 && assemble_smem(dim, p, false) > 200 * 1024;
  size_t smem = assemble_smem(dim, p, perpat);
  if (smem > 200 * 1024) return IGAFD_ERR_ARG;
  if (dim == 3) {
    IGAFD_CUDA(cudaFuncSetAttribute(assemble_kernel<3, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    IGAFD_CUDA(cudaFuncSetAttribute(assemble_kernel<3, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  } else {
    IGAFD_CUDA(cudaFuncSetAttribute(assemble_kernel<2, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  const int C = p + 1;
  for (int c3 = 0; c3 < (dim == 3 ? C : 1); ++c3)
    for (int c2 = 0; c2 < C; ++c2)
      for (int c1 = 0; c1 < C; ++c1) {
        int ne1 = c1 < P->nel[0] ? (P->nel[0] - c1 + C - 1) / C : 0;
        int ne2 = c2 < P->nel[1] ? (P->nel[1] - c2 + C - 1) / C : 0;
        int ne3 = dim == 3 ? (c3 < P->nel[2] ? (P->nel[2] - c3 + C - 1) / C : 0) : 1;
        long long nb = (long long)ne1 * ne2 * ne3;
        if (nb == 0) continue;
        if (dim == 3 && perpat)
          assemble_kernel<3, true><<<(unsigned)nb, 256, smem, s>>>(v, c1, c2, c3, ne1, ne2, P->stencil, ld, o_min, H);
        else if (dim == 3)
          assemble_kernel<3, false><<<(unsigned)nb, 256, smem, s>>>(v, c1, c2, c3, ne1, ne2, P->stencil, ld, o_min, H);
        else
          assemble_kernel<2, false><<<(unsigned)nb, 256, smem, s>>>(v, c1, c2, 0, ne1, ne2, P->stencil, ld, o_min, H);
        IGAFD_CUDA(cudaGetLastError());
      }
  return IGAFD_OK;
}

// dst[o][i] (o < n_off, i < N, row stride N) from a half-stored stencil: the
// stored offsets as they are, the others as the stored coupling -delta of
// row i + off(delta) (zero where that row lies outside the box: the halo).
__global__ void expand_half_kernel(const double *__restrict__ S, long long ld, long long H, int p,
                                   int dim, int n1, int n2, int n_off, long long N,
                                   double *__restrict__ dst) {
  const int W = 2 * p + 1, oc = n_off / 2;
  const long long total = (long long)n_off * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(t / N);
    const long long i = t - (long long)o * N;
    double v;
    if (o >= oc) {
      v = S[(size_t)(o - oc) * ld + H + i];
    } else {
      const int d1 = o % W - p, d2 = (o / W) % W - p, d3 = dim == 3 ? o / (W * W) - p : 0;
      const long long off = d1 + (long long)d2 * n1 + (long long)d3 * n1 * n2;
      v = S[(size_t)(n_off - 1 - o - oc) * ld + H + i + off];
    }
    dst[t] = v;
  }
}

igafd_status igafd_stencil_expand(const igafd_patch *P, double *dst, cudaStream_t s) {
  expand_half_kernel<<<1216, 256, 0, s>>>(P->stencil, P->sh_ld, P->sh_H, P->p, P->dim, P->n[0],
                                          P->n[1], P->n_off, P->N, dst);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

static igafd_status load_rhs(igafd_patch *P, const double *fq, double *b, cudaStream_t s) {
  IGAFD_CUDA(cudaSetDevice(P->dev));
  PV v = make_view(P);
  const int p = P->p, dim = P->dim, C = p + 1;
  size_t smem = (size_t)(dim == 3 ? C * C * C : C * C) * sizeof(double);
  IGAFD_CUDA(cudaMemsetAsync(b, 0, P->N * sizeof(double), s));
  for (int c3 = 0; c3 < (dim == 3 ? C : 1); ++c3)
    for (int c2 = 0; c2 < C; ++c2)
      for (int c1 = 0; c1 < C; ++c1) {
        int ne1 = c1 < P->nel[0] ? (P->nel[0] - c1 + C - 1) / C : 0;
        int ne2 = c2 < P->nel[1] ? (P->nel[1] - c2 + C - 1) / C : 0;
        int ne3 = dim == 3 ? (c3 < P->nel[2] ? (P->nel[2] - c3 + C - 1) / C : 0) : 1;
        long long nb = (long long)ne1 * ne2 * ne3;
        if (nb == 0) continue;
        if (dim == 3) rhs_kernel<3><<<(unsigned)nb, 128, smem, s>>>(v, c1, c2, c3, ne1, ne2, fq, b);
        else rhs_kernel<2><<<(unsigned)nb, 128, smem, s>>>(v, c1, c2, 0, ne1, ne2, fq, b);
        IGAFD_LAUNCHED(1);
        IGAFD_CUDA(cudaGetLastError());
      }
  return IGAFD_OK;
}

extern "C" igafd_status igafd_load_rhs_sine(igafd_patch *P, double *b, void *stream) {
  if (!P || !b) return IGAFD_ERR_ARG;
  return load_rhs(P, nullptr, b, (cudaStream_t)stream);
}

extern "C" igafd_status igafd_load_rhs(igafd_patch *P, const double *f_qp, double *b,
                                       void *stream) {
  if (!P || !f_qp || !b || (const void *)f_qp == (const void *)b) return IGAFD_ERR_ARG;
  return load_rhs(P, f_qp, b, (cudaStream_t)stream);
}

extern "C" igafd_status igafd_quad_points(const igafd_patch *P, double *x, void *stream) {
  if (!P || !x) return IGAFD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  PV v = make_view(P);
  long long Qn = 1;
  for (int k = 0; k < P->dim; ++k) Qn *= (long long)P->nel[k] * (P->p + 1);
  long long nb = (Qn + 255) / 256;
  if (nb > 4 * 1184) nb = 4 * 1184;
  if (P->dim == 3) quad_points_kernel<3><<<(unsigned)nb, 256, 0, s>>>(v, Qn, x);
  else quad_points_kernel<2><<<(unsigned)nb, 256, 0, s>>>(v, Qn, x);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}
