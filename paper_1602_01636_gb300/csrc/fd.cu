// Fast-diagonalization apply z = P^{-1} r on SIMT cores (FP64 and FP32).
//
// Algorithm 3 (Algorithm 1 in 2D) as six (four) mode-k products:
//   forward   t = (U_1^T (x) U_2^T (x) U_3^T) r      (mode 1, 2, 3)
//   divide    t /= D_1 (+) D_2 (+) D_3              (fused into mode 3)
//   backward  z = (U_1 (x) U_2 (x) U_3) t           (mode 3, 2, 1)
// The forward step applies U_k^T and the backward step U_k: from
// U^T M U = I, U^T K U = D one has P^{-1} = (x)U_k Lambda^{-1} (x)U_k^T.
//
// Each mode-k product of the tensor X[s][a][f] (s: slower directions,
// a: direction k, f: faster directions) is a strided GEMM
//   modes 2, 3:  Y_s (n_k x F) = W (n_k x n_k) X_s (n_k x F)
//   mode 1:      Y (S x n_1)   = X (S x n_1) W^T
// with W(j, a) = U[a][j] forward and U[j][a] backward.
#include "common.cuh"

namespace {

struct GemmArgs {
  const void *A;
  const void *B;
  void *C;
  int M, N, K, batch;
  long long sam, sak, sbk, sbn, scm, scn;
  long long batA, batB, batC;
  const void *scale;   // per-element scale of C (indexed like C), or null
  const double *done;  // skip when *done != 0 (PCG has converged)
};

// 64x64 output tile, 16-deep K slices, 256 threads with 4x4 outputs each.
// Double-buffered: the next K slice is read from global memory into
// registers while the current one is multiplied out of shared memory, and
// lands in the other shared buffer (one barrier per slice). Each output sums
// over k in increasing order, as a single-buffered loop would.
template <typename TA, typename TB, typename TC, typename ACC>
__global__ void __launch_bounds__(256) mode_gemm_kernel(GemmArgs g) {
  pdl_wait();
  pdl_trigger();
  if (g.done && *g.done != 0.0) return;
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ ACC As[2][BK][BM + 1];
  __shared__ ACC Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long long b = blockIdx.z;
  const TA *A = (const TA *)g.A + b * g.batA;
  const TB *B = (const TB *)g.B + b * g.batB;
  TC *C = (TC *)g.C + b * g.batC;
  ACC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (ACC)0;
  const bool a_kfast = g.sak == 1;
  const bool b_nfast = g.sbn == 1;
  // this thread's four (row, k) entries of an A slice and (k, column) of a B slice
  int am[4], ak[4], bn[4], bk[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int t = tid + 256 * l;
    if (a_kfast) { am[l] = t / BK; ak[l] = t % BK; } else { ak[l] = t / BM; am[l] = t % BM; }
    if (b_nfast) { bk[l] = t / BN; bn[l] = t % BN; } else { bn[l] = t / BK; bk[l] = t % BK; }
  }
  ACC va[4], vb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int m = m0 + am[l], k = k0 + ak[l];
      va[l] = (m < g.M && k < g.K) ? (ACC)A[m * g.sam + k * g.sak] : (ACC)0;
      const int n = n0 + bn[l], kq = k0 + bk[l];
      vb[l] = (n < g.N && kq < g.K) ? (ACC)B[kq * g.sbk + n * g.sbn] : (ACC)0;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      As[buf][ak[l]][am[l]] = va[l];
      Bs[buf][bk[l]][bn[l]] = vb[l];
    }
  };
  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    const bool more = k0 + BK < g.K;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      ACC a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  const ACC *sc = (const ACC *)g.scale;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      long long ci = m * g.scm + n * g.scn;
      ACC v = acc[i][j];
      if (sc) v *= sc[b * g.batC + ci];
      C[ci] = (TC)v;
    }
  }
}

template <typename TA, typename TB, typename TC, typename ACC>
igafd_status launch_gemm(const GemmArgs &g, cudaStream_t s) {
  dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.batch);
  IGAFD_CUDA(igafd_launch(mode_gemm_kernel<TA, TB, TC, ACC>, grid, dim3(256), 0, s, g));
  IGAFD_LAUNCHED(1);
  return IGAFD_OK;
}

// Describe the mode-k product of the tensor with sizes n[0..dim-1]
// (direction 1 fastest): Y = W *_k X with W(j,a) = U[a][j] (forward) or
// U[j][a] (backward).
GemmArgs mode_args(const int *n, int dim, int k, const void *U, bool forward, const void *X,
                   void *Y, const void *scale) {
  long long F = 1, S = 1;
  for (int l = 0; l < k; ++l) F *= n[l];
  for (int l = k + 1; l < dim; ++l) S *= n[l];
  const long long nk = n[k];
  GemmArgs g{};
  g.scale = scale;
  if (k == 0) {
    // Y[s][j] = sum_a X[s][a] W(j, a): A = X (S x n1), B[a][j] = W(j, a)
    g.A = X; g.B = U; g.C = Y;
    g.M = (int)S; g.N = (int)nk; g.K = (int)nk; g.batch = 1;
    g.sam = nk; g.sak = 1;
    if (forward) { g.sbk = nk; g.sbn = 1; } else { g.sbk = 1; g.sbn = nk; }
    g.scm = nk; g.scn = 1;
    g.batA = g.batB = g.batC = 0;
  } else {
    // Y_s[j][f] = sum_a W(j, a) X_s[a][f]: A[j][a] = W(j, a), B = X_s
    g.A = U; g.B = X; g.C = Y;
    g.M = (int)nk; g.N = (int)F; g.K = (int)nk; g.batch = (int)S;
    if (forward) { g.sam = 1; g.sak = nk; } else { g.sam = nk; g.sak = 1; }
    g.sbk = F; g.sbn = 1;
    g.scm = F; g.scn = 1;
    g.batA = 0; g.batB = nk * F; g.batC = nk * F;
  }
  return g;
}

}  // namespace

// FP64: every product and the divide in FP64 (FD == P^{-1} up to rounding).
igafd_status igafd_fd64_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                              double *done_flag) {
  const int dim = P->dim;
  const double *in = r;
  double *bufs[2] = {P->fd_a, P->fd_b};
  int cur = 0;
  // forward modes 1..dim, divide fused into the last
  for (int k = 0; k < dim; ++k) {
    double *out = bufs[cur];
    GemmArgs g = mode_args(P->n, dim, k, P->U[k], true, in, out,
                           k == dim - 1 ? (const void *)P->inv_lam : nullptr);
    g.done = done_flag;
    IGAFD_TRY((launch_gemm<double, double, double, double>(g, s)));
    in = out;
    cur ^= 1;
  }
  // backward modes dim..1, the last writes z
  for (int k = dim - 1; k >= 0; --k) {
    double *out = k == 0 ? z : bufs[cur];
    GemmArgs g = mode_args(P->n, dim, k, P->U[k], false, in, out, nullptr);
    g.done = done_flag;
    IGAFD_TRY((launch_gemm<double, double, double, double>(g, s)));
    in = out;
    cur ^= 1;
  }
  return IGAFD_OK;
}

// FP32: products and divide in FP32 (FP64 in, FP64 out), U_k rounded to FP32.
igafd_status igafd_fd32_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                              double *done_flag) {
  const int dim = P->dim;
  float *bufs[2] = {(float *)P->fd_a, (float *)P->fd_b};
  int cur = 0;
  const void *in = r;
  for (int k = 0; k < dim; ++k) {
    float *out = bufs[cur];
    GemmArgs g = mode_args(P->n, dim, k, P->U32[k], true, in, out,
                           k == dim - 1 ? (const void *)P->inv_lam32 : nullptr);
    g.done = done_flag;
    if (k == 0) IGAFD_TRY((launch_gemm<double, float, float, float>(g, s)));
    else IGAFD_TRY((launch_gemm<float, float, float, float>(g, s)));
    in = out;
    cur ^= 1;
  }
  for (int k = dim - 1; k >= 0; --k) {
    GemmArgs g;
    if (k == 0) {
      g = mode_args(P->n, dim, k, P->U32[k], false, in, z, nullptr);
      g.done = done_flag;
      IGAFD_TRY((launch_gemm<float, float, double, float>(g, s)));
    } else {
      float *out = bufs[cur];
      g = mode_args(P->n, dim, k, P->U32[k], false, in, out, nullptr);
      g.done = done_flag;
      IGAFD_TRY((launch_gemm<float, float, float, float>(g, s)));
      in = out;
      cur ^= 1;
    }
  }
  return IGAFD_OK;
}
