// Learned span scalings of the 1D pencils: features, separable log-fit
// labels, and the scaled preconditioner.
//
// Prop. 1 bounds the condition number of P^{-1} A by the spread of the
// eigenvalues of Q over the domain. Scaling the element contributions of the
// 1D pencils, K~_k = sum_e wK_{k,e} K_k^(e) and M~_k = sum_e wM_{k,e} M_k^(e),
// keeps P a Kronecker sum (so the fast diagonalization still applies) while
// letting term k of P follow Q_kk: on the quadrature grid, term k carries the
// factor wK_k(zeta_k) * prod_{l != k} wM_l(zeta_l). The separable fit chooses
// log wK, log wM by least squares of log Q_kk against that additive model
// (backfitting); it initialises the labels that a small network learns to
// predict from per-span features of Q. Each backfitting update of a span's
// log-weight is the slab mean of log Q_kk minus the element means of the
// other factors (every element carries the same number of quadrature points
// in each direction), so one pass over the quadrature grid gives both the
// features and the slab means Ybar[k][dir][e] of every log Q_kk, and the
// sweeps run on those few numbers. The pass is done once per patch and kept.
//
// Rows: r <-> (direction k, span e), direction-major: r = sum_{l<k} nel_l + e.
#include "common.cuh"
#include "geom.cuh"

#include <cmath>
#include <vector>

using namespace igafd_geom;

namespace {

// The features are FP32 logarithms of Q, so Q is evaluated in FP32 (GB300's
// FP32 pipe is 64x its FP64 pipe; one pass covers every quadrature point):
// FP32 copies of the geometry and coefficient tables, the map's Jacobian,
// Q = kappa |det J| J^{-1} J^{-T} and the extreme eigenvalues of Q.
struct PVf {
  int gp, kp;
  int nel[3], gm[3], km[3];
  const float *gv[3], *gd[3], *kv[3];
  const int *gspan[3], *kspan[3];
  const float *ctrl, *kctrl;
  float kappa;
};

template <int DIM>
__device__ void jacobian_f(const PVf &v, const int *t, float (*J)[3]) {
  const int gp = v.gp, ga = gp + 1;
  const float *gv[3], *gd[3];
  int g0[3];
  for (int k = 0; k < DIM; ++k) {
    gv[k] = v.gv[k] + (size_t)t[k] * ga;
    gd[k] = v.gd[k] + (size_t)t[k] * ga;
    g0[k] = v.gspan[k][t[k]] - gp;
  }
  for (int c = 0; c < DIM; ++c)
    for (int j = 0; j < DIM; ++j) J[c][j] = 0.0f;
  for (int c = 0; c < DIM; ++c) {
    if (DIM == 2) {
      const float *C = v.ctrl + (size_t)c * v.gm[0] * v.gm[1];
      for (int a2 = 0; a2 < ga; ++a2) {
        const float *row = C + (size_t)(g0[1] + a2) * v.gm[0] + g0[0];
        float s0 = 0.0f, s1 = 0.0f;
        for (int a1 = 0; a1 < ga; ++a1) {
          s0 += row[a1] * gv[0][a1];
          s1 += row[a1] * gd[0][a1];
        }
        J[c][0] += s1 * gv[1][a2];
        J[c][1] += s0 * gd[1][a2];
      }
    } else {
      const float *C = v.ctrl + (size_t)c * v.gm[0] * v.gm[1] * v.gm[2];
      for (int a3 = 0; a3 < ga; ++a3) {
        const float v3 = gv[2][a3], d3 = gd[2][a3];
        for (int a2 = 0; a2 < ga; ++a2) {
          const float *row = C + ((size_t)(g0[2] + a3) * v.gm[1] + (g0[1] + a2)) * v.gm[0] + g0[0];
          float s0 = 0.0f, s1 = 0.0f;
          for (int a1 = 0; a1 < ga; ++a1) {
            s0 += row[a1] * gv[0][a1];
            s1 += row[a1] * gd[0][a1];
          }
          const float v2 = gv[1][a2], d2 = gd[1][a2];
          J[c][0] += s1 * v2 * v3;
          J[c][1] += s0 * d2 * v3;
          J[c][2] += s0 * v2 * d3;
        }
      }
    }
  }
}

template <int DIM>
__device__ float kappa_f(const PVf &v, const int *t) {
  if (!v.kctrl) return v.kappa;
  const int ka = v.kp + 1;
  const float *kv[3];
  int k0[3];
  for (int k = 0; k < DIM; ++k) {
    kv[k] = v.kv[k] + (size_t)t[k] * ka;
    k0[k] = v.kspan[k][t[k]] - v.kp;
  }
  float acc = 0.0f;
  if (DIM == 2) {
    for (int a2 = 0; a2 < ka; ++a2) {
      const float *row = v.kctrl + (size_t)(k0[1] + a2) * v.km[0] + k0[0];
      float s0 = 0.0f;
      for (int a1 = 0; a1 < ka; ++a1) s0 += row[a1] * kv[0][a1];
      acc += s0 * kv[1][a2];
    }
  } else {
    for (int a3 = 0; a3 < ka; ++a3)
      for (int a2 = 0; a2 < ka; ++a2) {
        const float *row = v.kctrl + ((size_t)(k0[2] + a3) * v.km[1] + (k0[1] + a2)) * v.km[0] + k0[0];
        float s0 = 0.0f;
        for (int a1 = 0; a1 < ka; ++a1) s0 += row[a1] * kv[0][a1];
        acc += s0 * kv[1][a2] * kv[2][a3];
      }
  }
  return v.kappa * acc;
}

// Q = kappa |det J| J^{-1} J^{-T}, stored 2D [00, 11, 01], 3D [00, 11, 22, 01, 02, 12]
template <int DIM>
__device__ void q_f(const float (*J)[3], float kappa, float *Q) {
  if (DIM == 2) {
    const float det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const float id = 1.0f / det;
    const float a = J[1][1] * id, b = -J[0][1] * id, c = -J[1][0] * id, d = J[0][0] * id;
    const float sc = kappa * fabsf(det);
    Q[0] = sc * (a * a + b * b);
    Q[1] = sc * (c * c + d * d);
    Q[2] = sc * (a * c + b * d);
  } else {
    float Ji[3][3];
    const float c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const float c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const float c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const float det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const float id = 1.0f / det;
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    const float sc = kappa * fabsf(det);
    const int rr[6] = {0, 1, 2, 0, 0, 1}, ss[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) acc += Ji[rr[q]][c] * Ji[ss[q]][c];
      Q[q] = sc * acc;
    }
  }
}

// extreme eigenvalues of the symmetric Q (closed form: the 2x2 formula, and
// for 3x3 the trigonometric solution of the characteristic cubic)
template <int DIM>
__device__ void extremes_f(const float *Q, float *lmin, float *lmax) {
  if (DIM == 2) {
    const float m = 0.5f * (Q[0] + Q[1]);
    const float d = sqrtf(0.25f * (Q[0] - Q[1]) * (Q[0] - Q[1]) + Q[2] * Q[2]);
    *lmin = m - d;
    *lmax = m + d;
  } else {
    const float a = Q[0], b = Q[1], c = Q[2], d = Q[3], e = Q[5], f = Q[4];
    const float p1 = d * d + f * f + e * e;
    const float q = (a + b + c) * (1.0f / 3.0f);
    const float p2 = (a - q) * (a - q) + (b - q) * (b - q) + (c - q) * (c - q) + 2.0f * p1;
    const float pp = sqrtf(p2 * (1.0f / 6.0f));
    if (!(pp > 1e-30f * fabsf(q))) {
      *lmin = *lmax = q;
      return;
    }
    const float ip = 1.0f / pp;
    const float B00 = (a - q) * ip, B11 = (b - q) * ip, B22 = (c - q) * ip;
    const float B01 = d * ip, B02 = f * ip, B12 = e * ip;
    const float detB = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) +
                       B02 * (B01 * B12 - B11 * B02);
    const float r = fminf(1.0f, fmaxf(-1.0f, 0.5f * detB));
    const float phi = acosf(r) * (1.0f / 3.0f);
    *lmax = q + 2.0f * pp * cosf(phi);
    *lmin = q + 2.0f * pp * cosf(phi + 2.0943951f);   // + 2 pi / 3
  }
}

// Per quadrature point: log Q_kk (k < DIM), log lambda_min(Q), log lambda_max(Q).
// Layout y[c][t3][t2][t1] (global 1D quadrature indices, direction 1 fastest).
template <int DIM>
__global__ void qdiag_kernel(PVf v, int nq, long long nqp, float *y) {
  const long long T1 = (long long)v.nel[0] * nq, T2 = (long long)v.nel[1] * nq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nqp;
       i += (long long)gridDim.x * blockDim.x) {
    int t[3];
    t[0] = (int)(i % T1);
    t[1] = (int)((i / T1) % T2);
    t[2] = DIM == 3 ? (int)(i / (T1 * T2)) : 0;
    float J[3][3], Q[6];
    jacobian_f<DIM>(v, t, J);
    q_f<DIM>(J, kappa_f<DIM>(v, t), Q);
#pragma unroll
    for (int k = 0; k < DIM; ++k) y[k * nqp + i] = logf(Q[k]);
    float lo, hi;
    extremes_f<DIM>(Q, &lo, &hi);
    y[DIM * nqp + i] = logf(fmaxf(lo, 1e-30f));
    y[(DIM + 1) * nqp + i] = logf(hi);
  }
}

__global__ void narrow_kernel(const double *a, float *b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

struct Slab {
  int dim, nq;
  int nel[3];
  long long T[3];       // quadrature points per direction
  long long nqp;
  int row0[3];          // first row of each direction
};

// index of the element of direction l that quadrature point i lies in
__device__ __forceinline__ int elem_of(const Slab &S, long long i, int l) {
  long long t = l == 0 ? i % S.T[0] : l == 1 ? (i / S.T[0]) % S.T[1] : i / (S.T[0] * S.T[1]);
  return (int)(t / S.nq);
}

// one block per (direction k, span e): the slab's quadrature points, loop form
template <typename F>
__device__ void for_slab(const Slab &S, int k, int e, F f) {
  const int nq = S.nq;
  const long long cnt = (long long)nq * (S.nqp / S.T[k]);
  for (long long j = threadIdx.x; j < cnt; j += blockDim.x) {
    // j enumerates (g in the element, then the other directions' points)
    const int g = (int)(j % nq);
    const long long rest = j / nq;
    const long long tk = (long long)e * nq + g;
    long long i;
    if (k == 0) i = tk + S.T[0] * rest;
    else if (k == 1) i = (rest % S.T[0]) + S.T[0] * (tk + S.T[1] * (rest / S.T[0]));
    else i = rest + S.T[0] * S.T[1] * tk;
    f(i);
  }
}

__device__ double block_min(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 1e300;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmin(r, sh[w]);
  return r;
}

__device__ double block_total(double v, double *sh) {
  double t = block_sum(v, sh);
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// One block per row (slab direction k, span e), one pass over the slab's
// quadrature points:
//  - features of the row: [log mean Q_kk, log mean of the other diagonal
//    entries, log min lambda_min(Q), log max lambda_max(Q), std of log Q_kk,
//    span centre];
//  - ybar[j * rows + row]: the slab mean of log Q_jj for every j < dim.
__global__ void slab_stats_kernel(Slab S, const float *y, const double *const *knots,
                                  const int *const *spans, int rows, float *feat, double *ybar) {
  __shared__ double sh[32];
  const int k = blockIdx.y, e = blockIdx.x;
  if (e >= S.nel[k]) return;
  const long long nqp = S.nqp;
  double sq = 0.0, so = 0.0, sl2 = 0.0, mn = 1e300, mx = -1e300;
  double sy[3] = {0.0, 0.0, 0.0};
  for_slab(S, k, e, [&](long long i) {
    float yj[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (j < S.dim) {
        yj[j] = y[j * nqp + i];
        sy[j] += yj[j];
      }
    const float lq = k == 0 ? yj[0] : k == 1 ? yj[1] : yj[2];
    sq += expf(lq);
    sl2 += (double)lq * lq;
    float oth = 0.f;
#pragma unroll
    for (int l = 0; l < 3; ++l)
      if (l < S.dim && l != k) oth += expf(yj[l]);
    so += oth / (S.dim - 1);
    mn = fmin(mn, (double)y[S.dim * nqp + i]);
    mx = fmax(mx, (double)y[(S.dim + 1) * nqp + i]);
  });
  const double cnt = (double)S.nq * (double)(nqp / S.T[k]);
  sq = block_total(sq, sh);
  so = block_total(so, sh);
  sl2 = block_total(sl2, sh);
  for (int j = 0; j < 3; ++j) sy[j] = block_total(sy[j], sh);
  mn = block_min(mn, sh);
  mx = -block_min(-mx, sh);
  if (threadIdx.x == 0) {
    const int row = S.row0[k] + e;
    float *f = feat + (size_t)row * 6;
    const double ml = (k == 0 ? sy[0] : k == 1 ? sy[1] : sy[2]) / cnt;
    f[0] = (float)log(sq / cnt);
    f[1] = (float)log(so / cnt);
    f[2] = (float)mn;
    f[3] = (float)mx;
    f[4] = (float)sqrt(fmax(0.0, sl2 / cnt - ml * ml));
    const int s = spans[k][e];
    f[5] = (float)(0.5 * (knots[k][s] + knots[k][s + 1]));
    for (int j = 0; j < S.dim; ++j) ybar[(size_t)j * rows + row] = sy[j] / cnt;
  }
}

// The backfitting sweeps on the slab means (one thread; a few hundred rows):
// a_k(e) = Ybar[k][k][e] - sum_{l != k} mean(m_l), then for every l
// m_l(e) = mean_{k != l} (Ybar[k][l][e] - mean(a_k) - sum_{j != k, l} mean(m_j)),
// then the gauge (each m_l has mean 0, absorbed into the a_k, k != l).
__global__ void sepfit_kernel(Slab S, const double *ybar, int rows, int sweeps, double *a,
                              double *m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int dim = S.dim;
  auto mean = [&](const double *v, int l) {
    double c = 0.0;
    for (int e = 0; e < S.nel[l]; ++e) c += v[S.row0[l] + e];
    return c / S.nel[l];
  };
  for (int r = 0; r < rows; ++r) a[r] = m[r] = 0.0;
  for (int it = 0; it < sweeps; ++it) {
    for (int k = 0; k < dim; ++k) {
      double mb = 0.0;
      for (int l = 0; l < dim; ++l)
        if (l != k) mb += mean(m, l);
      for (int e = 0; e < S.nel[k]; ++e) a[S.row0[k] + e] = ybar[(size_t)k * rows + S.row0[k] + e] - mb;
    }
    for (int l = 0; l < dim; ++l) {
      double rest = 0.0;      // sum over k != l of (mean(a_k) + sum_{j != k, l} mean(m_j))
      for (int k = 0; k < dim; ++k) {
        if (k == l) continue;
        rest += mean(a, k);
        for (int j = 0; j < dim; ++j)
          if (j != k && j != l) rest += mean(m, j);
      }
      for (int e = 0; e < S.nel[l]; ++e) {
        double acc = 0.0;
        for (int k = 0; k < dim; ++k)
          if (k != l) acc += ybar[(size_t)k * rows + S.row0[l] + e];
        m[S.row0[l] + e] = (acc - rest) / (dim - 1);
      }
    }
    for (int l = 0; l < dim; ++l) {
      const double c = mean(m, l);
      for (int e = 0; e < S.nel[l]; ++e) m[S.row0[l] + e] -= c;
      for (int k = 0; k < dim; ++k)
        if (k != l)
          for (int e = 0; e < S.nel[k]; ++e) a[S.row0[k] + e] += c;
    }
  }
}

__global__ void pack_logw_kernel(const double *a, const double *m, int rows, float *logw) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  logw[2 * r] = (float)a[r];
  logw[2 * r + 1] = (float)m[r];
}

__global__ void exp_weights_kernel(const float *logw, int row0, int nel, double *wK, double *wM) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  wK[e] = exp((double)logw[2 * (row0 + e)]);
  wM[e] = exp((double)logw[2 * (row0 + e) + 1]);
}


Slab make_slab(const igafd_patch *P) {
  Slab S{};
  S.dim = P->dim;
  S.nq = P->p + 1;
  S.nqp = 1;
  int row = 0;
  for (int k = 0; k < 3; ++k) {
    S.nel[k] = k < P->dim ? P->nel[k] : 1;
    S.T[k] = k < P->dim ? (long long)P->nel[k] * S.nq : 1;
    S.nqp *= S.T[k];
    S.row0[k] = row;
    if (k < P->dim) row += P->nel[k];
  }
  return S;
}

int rows_of(const igafd_patch *P) {
  int r = 0;
  for (int k = 0; k < P->dim; ++k) r += P->nel[k];
  return r;
}

// log-diagonal table of Q on the quadrature grid (allocated here, freed by
// the caller together with *tables, the FP32 copies of the patch tables)
igafd_status make_qdiag(igafd_patch *P, cudaStream_t s, float **y, long long *nqp, float **tables) {
  Slab S = make_slab(P);
  *nqp = S.nqp;
  *y = nullptr;
  *tables = nullptr;
  const int dim = P->dim, nq = P->p + 1, ga = P->geo_p + 1, ka = P->kappa_p + 1;
  const bool kf = P->kctrl != nullptr;
  long long nctrl = dim, nkc = 1, tot = 0;
  for (int k = 0; k < dim; ++k) {
    nctrl *= P->dir[k].gm;
    nkc *= kf ? P->dir[k].km : 1;
    tot += 2LL * P->nel[k] * nq * ga + (kf ? (long long)P->nel[k] * nq * ka : 0);
  }
  tot += nctrl + (kf ? nkc : 0);
  if (cudaMalloc(y, (size_t)(dim + 2) * S.nqp * sizeof(float)) != cudaSuccess ||
      cudaMalloc(tables, (size_t)tot * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return IGAFD_ERR_OOM;
  }
  PVf v{};
  v.gp = P->geo_p; v.kp = P->kappa_p; v.kappa = (float)P->kappa;
  float *f = *tables;
  auto narrow = [&](const double *src, long long n) -> const float * {
    narrow_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, f, n);
    IGAFD_LAUNCHED(1);
    const float *out = f;
    f += n;
    return out;
  };
  for (int k = 0; k < 3; ++k) {
    v.nel[k] = k < dim ? P->nel[k] : 1;
    v.gm[k] = P->dir[k].gm;
    v.km[k] = P->dir[k].km;
    if (k >= dim) continue;
    const long long nt = (long long)P->nel[k] * nq;
    v.gv[k] = narrow(P->dir[k].gv, nt * ga);
    v.gd[k] = narrow(P->dir[k].gd, nt * ga);
    v.gspan[k] = P->dir[k].gspan;
    if (kf) {
      v.kv[k] = narrow(P->dir[k].kv, nt * ka);
      v.kspan[k] = P->dir[k].kspan;
    }
  }
  v.ctrl = narrow(P->ctrl, nctrl);
  v.kctrl = kf ? narrow(P->kctrl, nkc) : nullptr;
  if (dim == 3) qdiag_kernel<3><<<P->num_sms * 8, 256, 0, s>>>(v, nq, S.nqp, *y);
  else qdiag_kernel<2><<<P->num_sms * 8, 256, 0, s>>>(v, nq, S.nqp, *y);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

}  // namespace

extern "C" igafd_status igafd_scaling_rows(const igafd_patch *P, int *rows) {
  if (!P || !rows) return IGAFD_ERR_ARG;
  *rows = rows_of(P);
  return IGAFD_OK;
}

// Features and slab means of the patch's quadrature grid, computed on the
// first request and kept (the geometry and the coefficient are fixed).
static igafd_status ensure_stats(igafd_patch *P, cudaStream_t s) {
  if (P->lstats_valid) return IGAFD_OK;
  const int rows = rows_of(P);
  if (!P->lfeat && cudaMalloc(&P->lfeat, (size_t)rows * 6 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return IGAFD_ERR_OOM;
  }
  if (!P->lybar && cudaMalloc(&P->lybar, (size_t)P->dim * rows * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return IGAFD_ERR_OOM;
  }
  float *y = nullptr, *tables = nullptr;
  long long nqp = 0;
  igafd_status qs = make_qdiag(P, s, &y, &nqp, &tables);
  if (qs != IGAFD_OK) {
    cudaFree(y);
    cudaFree(tables);
    return qs;
  }
  Slab S = make_slab(P);
  const double *kn[3] = {P->dir[0].knots, P->dir[1].knots, P->dir[2].knots};
  const int *sp[3] = {P->dir[0].span, P->dir[1].span, P->dir[2].span};
  const double **dkn = nullptr;
  const int **dsp = nullptr;
  igafd_status st = IGAFD_OK;
  if (cudaMalloc(&dkn, sizeof(kn)) != cudaSuccess || cudaMalloc(&dsp, sizeof(sp)) != cudaSuccess) {
    cudaGetLastError();
    st = IGAFD_ERR_OOM;
  } else {
    cudaMemcpyAsync(dkn, kn, sizeof(kn), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dsp, sp, sizeof(sp), cudaMemcpyHostToDevice, s);
    int emax = 0;
    for (int k = 0; k < P->dim; ++k) emax = emax > P->nel[k] ? emax : P->nel[k];
    slab_stats_kernel<<<dim3(emax, P->dim), 256, 0, s>>>(S, y, dkn, dsp, rows, P->lfeat, P->lybar);
    IGAFD_LAUNCHED(1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = IGAFD_ERR_CUDA;
  }
  cudaFree(dkn);
  cudaFree(dsp);
  cudaFree(y);
  cudaFree(tables);
  if (st == IGAFD_OK) P->lstats_valid = 1;
  return st;
}

extern "C" igafd_status igafd_patch_features(igafd_patch *P, float *feat, void *stream) {
  if (!P || !feat) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  cudaStream_t s = (cudaStream_t)stream;
  IGAFD_TRY(ensure_stats(P, s));
  IGAFD_CUDA(cudaMemcpyAsync(feat, P->lfeat, (size_t)rows_of(P) * 6 * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  return IGAFD_OK;
}

extern "C" igafd_status igafd_patch_sepfit(igafd_patch *P, int sweeps, float *logw, void *stream) {
  if (!P || !logw || sweeps < 1 || sweeps > 1000) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  cudaStream_t s = (cudaStream_t)stream;
  IGAFD_TRY(ensure_stats(P, s));
  Slab S = make_slab(P);
  const int rows = rows_of(P);
  double *a = nullptr, *m = nullptr;
  igafd_status st = IGAFD_OK;
  if (cudaMalloc(&a, rows * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&m, rows * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    st = IGAFD_ERR_OOM;
  } else {
    sepfit_kernel<<<1, 32, 0, s>>>(S, P->lybar, rows, sweeps, a, m);
    IGAFD_LAUNCHED(1);
    pack_logw_kernel<<<(rows + 127) / 128, 128, 0, s>>>(a, m, rows, logw);
    IGAFD_LAUNCHED(1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = IGAFD_ERR_CUDA;
  }
  cudaFree(a);
  cudaFree(m);
  return st;
}

extern "C" igafd_status igafd_set_scalings(igafd_patch *P, const float *logw, void *stream) {
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // a full-space patch has no preconditioner
  if (!P) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  cudaStream_t s = (cudaStream_t)stream;
  if (logw) {
    int row0 = 0;
    for (int k = 0; k < P->dim; ++k) {
      if (!P->wK[k]) {
        if (cudaMalloc(&P->wK[k], P->nel[k] * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&P->wM[k], P->nel[k] * sizeof(double)) != cudaSuccess) {
          cudaGetLastError();
          return IGAFD_ERR_OOM;
        }
      }
      exp_weights_kernel<<<(P->nel[k] + 127) / 128, 128, 0, s>>>(logw, row0, P->nel[k], P->wK[k],
                                                                 P->wM[k]);
      IGAFD_LAUNCHED(1);
      row0 += P->nel[k];
    }
    IGAFD_CUDA(cudaGetLastError());
    P->scaled = 1;
  } else {
    P->scaled = 0;
  }
  return igafd_build_prec(P, s);
}
