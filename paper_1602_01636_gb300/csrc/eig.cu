// 1D pencils and their generalized eigendecompositions (Section 3 and
// Algorithm 1 line 1 / Eq. (eigen3d)), in FP64 on the device.
//
//   M_k, K_k: (p+1)-point Gauss quadrature of B_i B_j and B_i' B_j'
//   M = L L^T (banded Cholesky), K~ = L^{-1} K L^{-T} (banded triangular
//   solves), K~ = U~ D U~^T, U = L^{-T} U~ (Section 4.1). Eigenvalues sorted
//   ascending, each eigenvector signed so that its largest-magnitude entry is
//   positive.
//
// The symmetric eigenproblem K~ = U~ D U~^T has two routes:
//   fast (n <= 128): an FP32 start in one CTA per direction, all in shared
//     memory -- Householder tridiagonalisation T = Q^T K~ Q, every
//     eigenvalue of T by bisection on Sturm counts (one thread each),
//     eigenvectors of T by inverse iteration (3 steps; members of a cluster
//     of eigenvalues closer than 1e-5 ||T|| are solved in turn and
//     orthogonalised against each other), back-transformed by Q -- then FP64
//     iterative refinement of the eigenvector matrix (Ogita and Aishima,
//     "Iterative refinement for symmetric eigenvalue decomposition", 2018):
//     with R = I - X^T X and S = X^T K~ X, lambda_i = s_ii / (1 - r_ii) and
//     X <- X + X E, E_ii = r_ii / 2, E_ij = (s_ij + lambda_j r_ij) /
//     (lambda_j - lambda_i) for separated pairs and r_ij / 2 within a
//     cluster. Pairs closer than 1e-5 ||K~||_inf stay clusters throughout and
//     are diagonalised at the end by exact 2x2 rotations. The products are
//     dense FP64 GEMMs spread over many CTAs (GB300's FP64 rate per SM is
//     low). The result is checked (max |X^T X - I| and max |offdiag S| /
//     max |diag S| <= 1e-12); a direction that fails takes the other route.
//   FP64 (n > 128, or fallback): cyclic two-sided Jacobi in FP64 with a
//     round-robin (tournament) ordering, n/2 disjoint rotations in parallel.
#include "common.cuh"

#include <vector>

namespace {

// Dense (Dirichlet-reduced) pencils of one direction; one thread per
// (i, j) with |i - j| <= p. Full index I = i + 1. Optional per-element
// weights wK, wM (null: 1) give the span-scaled pencils
// K~ = sum_e wK_e K^(e), M~ = sum_e wM_e M^(e).
__global__ void pencil_kernel(Dir1D D, int p, double *K, double *M, const double *wK,
                              const double *wM) {
  const int n = D.n, W = 2 * p + 1, A = p + 1, nq = p + 1;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * W) return;
  int i = t / W, j = i + (t % W) - p;
  if (j < 0 || j >= n) return;
  int I = i + 1, J = j + 1;
  double m = 0.0, k = 0.0;
  for (int e = 0; e < D.nel; ++e) {
    int s = D.span[e];
    int ai = I - (s - p), aj = J - (s - p);
    if (ai < 0 || ai > p || aj < 0 || aj > p) continue;
    double me = 0.0, ke = 0.0;
    for (int g = 0; g < nq; ++g) {
      size_t q = (size_t)e * nq + g;
      double w = D.w[q];
      me += w * D.bv[q * A + ai] * D.bv[q * A + aj];
      ke += w * D.bd[q * A + ai] * D.bd[q * A + aj];
    }
    m += wM ? wM[e] * me : me;
    k += wK ? wK[e] * ke : ke;
  }
  M[(size_t)i * n + j] = m;
  K[(size_t)i * n + j] = k;
}

// One block per direction. Work arrays (global, n*n each): M (becomes L),
// K (becomes X = L^{-1} K, later scratch), A (K~, kept), V (FP64 Jacobi
// rotations), X/Xn (refined eigenvectors, ping-pong), G (X^T X), AX, S
// (X^T K~ X), E (correction). U, D: outputs. sc: per-direction scalars
// [0] = infinity norm of K~, [1] = cluster bound delta, [2] = orthogonality
// error, [3] = relative off-diagonal of S. state: 0 = refined eigenpairs
// accepted, 1 = take the FP64 Jacobi route.
struct EigJob {
  int n, p;
  double *M, *K, *A, *V;
  double *X, *Xn, *G, *AX, *S, *E;
  double *W;                          // 2 n^2: FP32 inverse-iteration scratch
  double *U, *D;
  double *sc;
  int *state;
};

constexpr int kFastMaxN = 128;       // the FP32 start keeps A and Z in shared memory
constexpr int kMaxBand = 8;          // p <= 8: the banded solves keep p values in registers

// ---- banded Cholesky, K~ = L^{-1} K L^{-T} (into A), route choice ----
__global__ void __launch_bounds__(1024) prep_kernel(EigJob *jobs, int *err, int allow_fast) {
  EigJob jb = jobs[blockIdx.x];
  const int n = jb.n, p = jb.p;
  double *M = jb.M, *K = jb.K, *A = jb.A;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  __shared__ int s_fail;
  __shared__ double s_red[32];
  // banded Cholesky M = L L^T (L in the lower band of M) by one warp: O(n p^2)
  // work, where a block-wide barrier per column would cost more than the
  // arithmetic
  if (tid < 32) {
    int fail = 0;
    for (int k = 0; k < n; ++k) {
      if (lane == 0) {
        const double d = M[(size_t)k * n + k];
        if (!(d > 0.0)) fail = 1;
        M[(size_t)k * n + k] = d > 0.0 ? sqrt(d) : 1.0;
      }
      __syncwarp();
      const double rkk = 1.0 / M[(size_t)k * n + k];
      const int bw = min(n, k + p + 1) - (k + 1);
      if (lane < bw) M[(size_t)(k + 1 + lane) * n + k] *= rkk;
      __syncwarp();
      for (int t = lane; t < bw * bw; t += 32) {
        const int i = k + 1 + t / bw, j = k + 1 + t % bw;
        if (j <= i) M[(size_t)i * n + j] -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
      }
      __syncwarp();
    }
    fail = __any_sync(0xffffffffu, fail);
    if (lane == 0) s_fail = fail;
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) {
      atomicExch(err, (int)IGAFD_ERR_NOT_SPD);
      *jb.state = 2;     // nothing further for this direction
    }
    return;
  }
  // 1 / l_ii once (an FP64 division is many FP64-pipe instructions)
  __shared__ double rdiag[kFastMaxN];
  double *rd = n <= kFastMaxN ? rdiag : jb.V;     // V is free until the FP64 route
  for (int i = tid; i < n; i += nt) rd[i] = 1.0 / M[(size_t)i * n + i];
  __syncthreads();
  // X = L^{-1} K (column-parallel forward substitution), into K; the last p
  // results of a column stay in registers (w[d] = X[i-1-d][c])
  for (int c = tid; c < n; c += nt) {
    double w[kMaxBand];
#pragma unroll
    for (int d = 0; d < kMaxBand; ++d) w[d] = 0.0;
    for (int i = 0; i < n; ++i) {
      double acc = K[(size_t)i * n + c];
#pragma unroll
      for (int d = kMaxBand - 1; d >= 0; --d)
        if (d < p && i - 1 - d >= 0) acc -= M[(size_t)i * n + i - 1 - d] * w[d];
      const double x = acc * rd[i];
      K[(size_t)i * n + c] = x;
#pragma unroll
      for (int d = kMaxBand - 1; d > 0; --d) w[d] = w[d - 1];
      w[0] = x;
    }
  }
  __syncthreads();
  // K~ = X L^{-T} (row-parallel), into A; w[d] = A[r][j-1-d]
  for (int r = tid; r < n; r += nt) {
    double w[kMaxBand];
#pragma unroll
    for (int d = 0; d < kMaxBand; ++d) w[d] = 0.0;
    for (int j = 0; j < n; ++j) {
      double acc = K[(size_t)r * n + j];
#pragma unroll
      for (int d = kMaxBand - 1; d >= 0; --d)
        if (d < p && j - 1 - d >= 0) acc -= M[(size_t)j * n + j - 1 - d] * w[d];
      const double x = acc * rd[j];
      A[(size_t)r * n + j] = x;
#pragma unroll
      for (int d = kMaxBand - 1; d > 0; --d) w[d] = w[d - 1];
      w[0] = x;
    }
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += nt) {
    int i = t / n, j = t % n;
    if (i < j) {
      double a = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = a;
      A[(size_t)j * n + i] = a;
    }
  }
  __syncthreads();
  // infinity norm of K~ (bounds its 2-norm)
  double rmax = 0.0;
  for (int i = tid; i < n; i += nt) {
    double rs = 0.0;
    for (int j = 0; j < n; ++j) rs += fabs(A[(size_t)i * n + j]);
    rmax = fmax(rmax, rs);
  }
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((tid & 31) == 0) s_red[tid >> 5] = rmax;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < nt / 32; ++w) m = fmax(m, s_red[w]);
    jb.sc[0] = m;
    jb.sc[1] = jb.sc[2] = jb.sc[3] = 0.0;
    *jb.state = (allow_fast && n <= kFastMaxN) ? 0 : 1;
  }
}

// Round-robin pairing of round `round` among ne (even) players: pair k.
__device__ __forceinline__ void tournament_pair(int round, int k, int ne, int &a, int &b) {
  if (k == 0) { a = ne - 1; b = round; }
  else { a = (round + k) % (ne - 1); b = (round - k + ne - 1) % (ne - 1); }
  if (a > b) { int t = a; a = b; b = t; }
}

// ---- fast route, step 1: FP32 eigenpairs of K~ in shared memory ----
// Scratch (global, 4 n^2 floats): per-thread rows of the inverse-iteration
// solves, interleaved by thread so that a warp's accesses are contiguous.
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kInvBatch = 32;        // clusters solved at once by inverse iteration
constexpr float kInvCluster = 1e-5f; // eigenvalues of T closer than this x ||T|| form a cluster

// shared memory of tri32_kernel (floats): A and Z (n x (n+1) each), eight
// vectors of n, and the pivot rows of kInvBatch concurrent solves
__host__ __device__ constexpr size_t tri32_smem_floats(int n) {
  return 2 * (size_t)n * (n + 1) + 8 * (size_t)n + 3 * (size_t)n * kInvBatch;
}

__global__ void __launch_bounds__(1024) tri32_kernel(EigJob *jobs) {
  EigJob jb = jobs[blockIdx.x];
  if (*jb.state != 0) return;
  const int n = jb.n, ld = n + 1;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ float t32[];
  float *As = t32;                      // K~, then the reflectors below the diagonal
  float *Zs = As + (size_t)n * ld;      // eigenvectors of T, then of K~
  float *vv = Zs + (size_t)n * ld;      // current reflector v
  float *pw = vv + n;                   // beta K~ v; later beta v^T Z
  float *dd = pw + n, *ee = dd + n, *e2 = ee + n, *bet = e2 + n, *lam = bet + n;
  float *Ub = lam + 2 * n;              // [3][n][kInvBatch] pivot rows of the batch's solves
  __shared__ float s_f[4];
  __shared__ int s_start[kFastMaxN];
  for (int t = tid; t < n * n; t += nt) As[(t / n) * ld + t % n] = (float)jb.A[t];
  __syncthreads();
  // -- Householder tridiagonalisation: step k zeroes A[k+2..][k] --
  for (int k = 0; k < n - 2; ++k) {
    const int m = n - k - 1;            // length of x = A[k+1..n-1][k]
    if (warp == 0) {
      float x2 = 0.0f, t2 = 0.0f;
      for (int i = lane; i < m; i += 32) {
        const float x = As[(k + 1 + i) * ld + k];
        x2 += x * x;
        if (i > 0) { t2 += x * x; vv[i] = x; }
      }
      x2 = warp_sum_f(x2);
      t2 = warp_sum_f(t2);
      if (lane == 0) {
        const float x0 = As[(k + 1) * ld + k];
        float beta = 0.0f, alpha = x0;
        if (t2 > 0.0f) {
          const float nx = sqrtf(x2);
          alpha = x0 >= 0.0f ? -nx : nx;
          const float v0 = x0 - alpha;
          beta = 2.0f / (t2 + v0 * v0);
          vv[0] = v0;
        }
        s_f[0] = beta;
        dd[k] = As[k * ld + k];
        ee[k] = alpha;
        bet[k] = beta;
      }
    }
    __syncthreads();
    const float beta = s_f[0];
    if (beta == 0.0f) continue;        // already tridiagonal in this column
    // p = beta A_sub v, eight threads per row
    {
      const int r = tid >> 3, sub = tid & 7;
      float acc = 0.0f;
      if (r < m)
        for (int j = sub; j < m; j += 8) acc += As[(k + 1 + r) * ld + k + 1 + j] * vv[j];
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (r < m && sub == 0) pw[r] = beta * acc;
    }
    __syncthreads();
    // K = beta/2 v.p (every warp computes it), w = p - K v, A_sub -= v w^T + w v^T
    float vp = 0.0f;
    for (int i = lane; i < m; i += 32) vp += vv[i] * pw[i];
    const float K = 0.5f * beta * warp_sum_f(vp);
    for (int i = warp; i < m; i += nt / 32) {
      const float vi = vv[i], wi = pw[i] - K * vi;
      float *row = As + (k + 1 + i) * ld + k + 1;
      for (int j = lane; j < m; j += 32) row[j] -= vi * (pw[j] - K * vv[j]) + wi * vv[j];
    }
    for (int i = tid; i < m; i += nt) As[(k + 1 + i) * ld + k] = vv[i];   // keep the reflector
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dd[n - 2] = As[(n - 2) * ld + n - 2];
      ee[n - 2] = As[(n - 1) * ld + n - 2];
      bet[n - 2] = 0.0f;
    }
    dd[n - 1] = As[(n - 1) * ld + n - 1];
    bet[n - 1] = 0.0f;
  }
  __syncthreads();
  // -- eigenvalues of T: Gershgorin interval, then 9-way multisection on
  //    Sturm counts (eight threads per eigenvalue, one count each) --
  if (warp == 0) {
    float lo = 3.0e38f, hi = -3.0e38f, me2 = 0.0f;
    for (int i = lane; i < n; i += 32) {
      const float el = i > 0 ? fabsf(ee[i - 1]) : 0.0f, er = i < n - 1 ? fabsf(ee[i]) : 0.0f;
      lo = fminf(lo, dd[i] - el - er);
      hi = fmaxf(hi, dd[i] + el + er);
      if (i < n - 1) { e2[i] = ee[i] * ee[i]; me2 = fmaxf(me2, e2[i]); }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      me2 = fmaxf(me2, __shfl_xor_sync(0xffffffffu, me2, o));
    }
    if (lane == 0) {
      s_f[0] = lo; s_f[1] = hi;
      s_f[2] = fmaxf(fabsf(lo), fabsf(hi));
      s_f[3] = 1.0e-30f * fmaxf(1.0f, me2);      // smallest pivot of a Sturm sequence
    }
  }
  __syncthreads();
  const float tn = s_f[2], pivmin = s_f[3];
  {
    // every warp takes part in full (the groups past n repeat the last
    // eigenvalue and store nothing); 9 rounds shrink the interval by 9^9
    const int ev = min(tid >> 3, n - 1), sub = tid & 7, base = lane & ~7;
    float lo = s_f[0], hi = s_f[1];
    for (int it = 0; it < 9; ++it) {
      const float x = lo + (hi - lo) * (float)(sub + 1) * (1.0f / 9.0f);
      int cnt = 0;
      float q = dd[0] - x;
      for (int j = 0;; ++j) {
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.0f;
        if (j == n - 1) break;
        q = (dd[j + 1] - x) - __fdividef(e2[j], q);
      }
      // bit s of grp: point s has at most ev eigenvalues below it; the
      // eigenvalue lies between the highest such point and the next one
      const unsigned grp = (__ballot_sync(0xffffffffu, cnt <= ev) >> base) & 0xffu;
      const int s_lo = grp ? 31 - __clz(grp) : -1;
      const float xlo = __shfl_sync(0xffffffffu, x, base + (s_lo >= 0 ? s_lo : 0));
      const float xhi = __shfl_sync(0xffffffffu, x, base + (s_lo + 1 <= 7 ? s_lo + 1 : 7));
      if (s_lo >= 0) lo = xlo;
      if (s_lo < 7) hi = xhi;
    }
    if (sub == 0 && (tid >> 3) < n) lam[tid >> 3] = 0.5f * (lo + hi);
  }
  __syncthreads();
  // -- eigenvectors of T by inverse iteration; clusters (gaps <= 1e-3 ||T||)
  //    are solved in turn by one thread; batches of kInvBatch cluster starts
  //    keep their pivot rows in shared memory; y lives in Z's column --
  if (tid < n) s_start[tid] = (tid == 0 || lam[tid] - lam[tid - 1] > kInvCluster * tn) ? 1 : 0;
  __syncthreads();
  const float floor = 1.2e-7f * tn;
  for (int b0 = 0; b0 < n; b0 += kInvBatch) {
    const int slot = tid - b0;
    if (slot >= 0 && slot < kInvBatch && tid < n && s_start[tid]) {
      int last = tid;
      while (last + 1 < n && !s_start[last + 1]) ++last;
      float *U0 = Ub + slot, *U1 = U0 + n * kInvBatch, *U2 = U1 + n * kInvBatch;
      float prev = 0.0f;
      for (int mm = tid; mm <= last; ++mm) {
        float *Y = Zs + mm;             // y_j = Y[j * ld]
        // a member equal (to 10 ulps) to the previous one is moved 10 ulps above it
        float lm = lam[mm];
        const float pert = 10.0f * 1.2e-7f * fabsf(lm);
        if (mm > tid && lm < prev + pert) lm = prev + pert;
        prev = lm;
        for (int j = 0; j < n; ++j) Y[j * ld] = (float)((j * 7919 + mm * 104729) % 1000) * 1.0e-3f - 0.5f;
        for (int it = 0; it < 3; ++it) {
          // (T - lm I) y = y: Gaussian elimination with partial pivoting
          float cd = dd[0] - lm, c1 = n > 1 ? ee[0] : 0.0f, c2 = 0.0f;
          float yc = Y[0];
          for (int i = 0; i < n - 1; ++i) {
            const float nd = dd[i + 1] - lm, n1 = i + 1 < n - 1 ? ee[i + 1] : 0.0f, sdn = ee[i];
            const float yn = Y[(i + 1) * ld];
            float p0, p1, p2, py;
            if (fabsf(sdn) > fabsf(cd)) {   // swap: row i+1 is the pivot
              const float m = cd / sdn;
              p0 = sdn; p1 = nd; p2 = n1; py = yn;
              cd = c1 - m * nd; c1 = c2 - m * n1; c2 = 0.0f;
              yc = yc - m * yn;
            } else {
              const float m = cd != 0.0f ? sdn / cd : 0.0f;
              p0 = cd; p1 = c1; p2 = c2; py = yc;
              cd = nd - m * c1; c1 = n1 - m * c2; c2 = 0.0f;
              yc = yn - m * yc;
            }
            U0[i * kInvBatch] = p0; U1[i * kInvBatch] = p1; U2[i * kInvBatch] = p2;
            Y[i * ld] = py;
          }
          U0[(n - 1) * kInvBatch] = cd;
          U1[(n - 1) * kInvBatch] = 0.0f;
          U2[(n - 1) * kInvBatch] = 0.0f;
          Y[(n - 1) * ld] = yc;
          // back substitution (pivots no smaller than floor in magnitude)
          float x1 = 0.0f, x2 = 0.0f;
          for (int i = n - 1; i >= 0; --i) {
            float u0 = U0[i * kInvBatch];
            if (fabsf(u0) < floor) u0 = u0 >= 0.0f ? floor : -floor;
            const float xi = (Y[i * ld] - U1[i * kInvBatch] * x1 - U2[i * kInvBatch] * x2) / u0;
            Y[i * ld] = xi;
            x2 = x1; x1 = xi;
          }
          // orthogonalise against the cluster's earlier vectors, normalise
          for (int q = tid; q < mm; ++q) {
            float d = 0.0f;
            for (int j = 0; j < n; ++j) d += Zs[j * ld + q] * Y[j * ld];
            for (int j = 0; j < n; ++j) Y[j * ld] -= d * Zs[j * ld + q];
          }
          float nrm = 0.0f;
          for (int j = 0; j < n; ++j) nrm += Y[j * ld] * Y[j * ld];
          const float inv = nrm > 0.0f ? rsqrtf(nrm) : 0.0f;
          for (int j = 0; j < n; ++j) Y[j * ld] *= inv;
        }
      }
    }
    __syncthreads();
  }
  // -- back-transform: Z <- H_0 ... H_{n-3} Z --
  for (int k = n - 3; k >= 0; --k) {
    const float beta = bet[k];
    if (beta == 0.0f) continue;
    const int m = n - k - 1;
    {
      const int c = tid >> 3, sub = tid & 7;
      float acc = 0.0f;
      if (c < n)
        for (int i = sub; i < m; i += 8) acc += As[(k + 1 + i) * ld + k] * Zs[(k + 1 + i) * ld + c];
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (c < n && sub == 0) pw[c] = beta * acc;
    }
    __syncthreads();
    for (int i = warp; i < m; i += nt / 32) {
      const float vi = As[(k + 1 + i) * ld + k];
      float *row = Zs + (k + 1 + i) * ld;
      for (int c = lane; c < n; c += 32) row[c] -= vi * pw[c];
    }
    __syncthreads();
  }
  for (int t = tid; t < n * n; t += nt) jb.X[t] = (double)Zs[(t / n) * ld + t % n];
}

// ---- fast route: dense FP64 products C = op(A) B (+ D), many CTAs ----
struct GemmJob {
  int n, transA;
  const double *A, *B, *D;
  double *C;
  const int *state;        // skip unless *state == 0
  // B = E of the refinement step, formed while loading (B unused): from
  // G = X^T X, S = X^T K~ X, lambda (lam) and the cluster bound delta (*dl)
  const double *G, *S, *lam, *dl;
};
struct GemmBatch {
  GemmJob j[6];
};

// 8 x 8 output tile per CTA (64 threads), K in panels of 64: at n = 128 a
// product is 256 CTAs, spread over all SMs (one SM's FP64 rate is low, so
// the products want as many SMs as possible).
constexpr int kGT = 8;
__global__ void __launch_bounds__(64) gemm64_kernel(GemmBatch b) {
  const GemmJob g = b.j[blockIdx.y];
  if (g.n == 0 || *g.state != 0) return;
  const int n = g.n, tpr = (n + kGT - 1) / kGT;
  if ((int)blockIdx.x >= tpr * tpr) return;
  const int ti = blockIdx.x / tpr, tj = blockIdx.x % tpr;
  const int ty = threadIdx.x / kGT, tx = threadIdx.x % kGT;
  constexpr int KP = 64;
  __shared__ double As[kGT][KP + 1], Bs[KP][kGT + 1];
  const int row = ti * kGT + ty, col = tj * kGT + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += KP) {
    for (int t = threadIdx.x; t < kGT * KP; t += kGT * kGT) {
      if (g.transA) {
        const int kk = t / kGT, r = t % kGT, ra = ti * kGT + r, ka = k0 + kk;
        As[r][kk] = (ra < n && ka < n) ? g.A[(size_t)ka * n + ra] : 0.0;
      } else {
        const int r = t / KP, kk = t % KP, ra = ti * kGT + r, ka = k0 + kk;
        As[r][kk] = (ra < n && ka < n) ? g.A[(size_t)ra * n + ka] : 0.0;
      }
      const int kk = t / kGT, c = t % kGT, kb = k0 + kk, cb = tj * kGT + c;
      double bv = 0.0;
      if (kb < n && cb < n) {
        if (!g.G) {
          bv = g.B[(size_t)kb * n + cb];
        } else {
          // E_ii = r_ii / 2; E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)
          // for separated pairs, r_ij / 2 within a cluster (r = I - G)
          const double gv = g.G[(size_t)kb * n + cb];
          if (kb == cb) {
            bv = 0.5 * (1.0 - gv);
          } else {
            const double d = g.lam[cb] - g.lam[kb];
            bv = fabs(d) > *g.dl ? (g.S[(size_t)kb * n + cb] - g.lam[cb] * gv) / d : -0.5 * gv;
          }
        }
      }
      Bs[kk][c] = bv;
    }
    __syncthreads();
#pragma unroll 16
    for (int kk = 0; kk < KP; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (row < n && col < n) g.C[(size_t)row * n + col] = acc + (g.D ? g.D[(size_t)row * n + col] : 0.0);
}

// block-wide max of a non-negative value (result valid in every thread)
__device__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
  __syncthreads();
  return m;
}

// ---- fast route, refinement step: E from G = X^T X and S = X^T K~ X ----
constexpr double kClusterRel = 1e-5;   // pairs closer than this x ||K~||_inf stay clusters

// Refinement step, first half: lambda_i = s_ii / g_ii (into E's first row)
// and the cluster bound delta = 2 (||S - diag(lambda)|| + ||K~|| ||R||)
// (infinity norms bound the 2-norms), at least kClusterRel ||K~||_inf, into
// sc[1]. The correction E itself is formed inside the X + X E product.
__global__ void __launch_bounds__(1024) refine_kernel(EigJob *jobs) {
  EigJob jb = jobs[blockIdx.x];
  if (*jb.state != 0) return;
  const int n = jb.n, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const double *G = jb.G, *S = jb.S;
  double *lam = jb.E;
  __shared__ double lam_s[kFastMaxN];
  __shared__ double sh[32];
  for (int i = tid; i < n; i += nt) {
    lam_s[i] = S[(size_t)i * n + i] / G[(size_t)i * n + i];
    lam[i] = lam_s[i];
  }
  __syncthreads();
  double ns = 0.0, nr = 0.0;
  for (int i = warp; i < n; i += nt / 32) {
    double a = 0.0, b = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double gv = G[(size_t)i * n + j], sv = S[(size_t)i * n + j];
      a += fabs(i == j ? sv - lam_s[i] : sv);
      b += fabs(i == j ? 1.0 - gv : gv);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    ns = fmax(ns, a);
    nr = fmax(nr, b);
  }
  ns = block_max(ns, sh);
  nr = block_max(nr, sh);
  if (tid == 0) jb.sc[1] = fmax(2.0 * (ns + jb.sc[0] * nr), kClusterRel * jb.sc[0]);
}

// ---- fast route: exact 2x2 rotations for nearly degenerate pairs ----
// Pairs with |s_ii - s_jj| <= kClusterRel ||K~||_inf (the refinement's
// clusters) are rotated (four passes over the list, cyclic Jacobi on each
// cluster's block) so that S is diagonal there; X's columns and S's rows and
// columns follow. More than kMaxPairs such pairs: take the FP64 route.
__global__ void __launch_bounds__(1024) cluster_kernel(EigJob *jobs, int parity) {
  EigJob jb = jobs[blockIdx.x];
  if (*jb.state != 0) return;
  constexpr int kMaxPairs = 128;
  const int n = jb.n, tid = threadIdx.x, nt = blockDim.x;
  double *X = parity ? jb.Xn : jb.X;
  double *S = jb.S;
  __shared__ int np_s, pi_s[kMaxPairs], pj_s[kMaxPairs];
  __shared__ double c_sh, s_sh, dg[kFastMaxN];
  for (int i = tid; i < n; i += nt) dg[i] = S[(size_t)i * n + i];
  __syncthreads();
  // the pair list in a fixed order ((i, j) lexicographic: row counts, a
  // prefix sum, then each row writes its own pairs), so results are reproducible
  __shared__ int cnt_s[kFastMaxN], off_s[kFastMaxN];
  const double thr = kClusterRel * jb.sc[0];
  if (tid < n) {
    int c = 0;
    for (int j = tid + 1; j < n; ++j) c += fabs(dg[tid] - dg[j]) <= thr;
    cnt_s[tid] = c;
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int i = 0; i < n; ++i) { off_s[i] = acc; acc += cnt_s[i]; }
    np_s = acc;
  }
  __syncthreads();
  if (tid < n && cnt_s[tid] > 0) {
    int o = off_s[tid];
    for (int j = tid + 1; j < n; ++j)
      if (fabs(dg[tid] - dg[j]) <= thr) {
        if (o < kMaxPairs) { pi_s[o] = tid; pj_s[o] = j; }
        ++o;
      }
  }
  __syncthreads();
  const int npairs = np_s;
  if (npairs > kMaxPairs) {
    if (tid == 0) *jb.state = 1;
    return;
  }
  for (int pass = 0; pass < 4; ++pass) {
    for (int k = 0; k < npairs; ++k) {
      const int p = pi_s[k], q = pj_s[k];
      if (tid == 0) {
        const double apq = S[(size_t)p * n + q];
        double c = 1.0, sn = 0.0;
        if (apq != 0.0) {
          const double tau = (S[(size_t)q * n + q] - S[(size_t)p * n + p]) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          sn = t * c;
        }
        c_sh = c; s_sh = sn;
      }
      __syncthreads();
      const double c = c_sh, sn = s_sh;
      if (sn != 0.0) {
        // rows of S
        for (int j = tid; j < n; j += nt) {
          const double ap = S[(size_t)p * n + j], aq = S[(size_t)q * n + j];
          S[(size_t)p * n + j] = c * ap - sn * aq;
          S[(size_t)q * n + j] = sn * ap + c * aq;
        }
        __syncthreads();
        // columns of S and of X
        for (int i = tid; i < n; i += nt) {
          const double ap = S[(size_t)i * n + p], aq = S[(size_t)i * n + q];
          S[(size_t)i * n + p] = c * ap - sn * aq;
          S[(size_t)i * n + q] = sn * ap + c * aq;
          const double xp = X[(size_t)i * n + p], xq = X[(size_t)i * n + q];
          X[(size_t)i * n + p] = c * xp - sn * xq;
          X[(size_t)i * n + q] = sn * xp + c * xq;
        }
        __syncthreads();
        if (tid == 0) { S[(size_t)p * n + q] = 0.0; S[(size_t)q * n + p] = 0.0; }
      }
      __syncthreads();
    }
  }
}

// ---- fast route: accept, or send the direction to the FP64 route ----
__global__ void __launch_bounds__(1024) check_kernel(EigJob *jobs) {
  EigJob jb = jobs[blockIdx.x];
  if (*jb.state != 0) return;
  const int n = jb.n, tid = threadIdx.x, nt = blockDim.x;
  __shared__ double sh[32];
  double orth = 0.0, off = 0.0, dm = 0.0;
  for (int t = tid; t < n * n; t += nt) {
    const int i = t / n, j = t % n;
    const double g = jb.G[t], sv = jb.S[t];
    const double eo = fabs(i == j ? g - 1.0 : g);
    // fmax drops NaN: a value that is not finite counts as a failure
    orth = fmax(orth, eo < 1e300 ? eo : 1.0);
    if (!(fabs(sv) < 1e300)) off = 1e300;
    else if (i == j) dm = fmax(dm, fabs(sv));
    else off = fmax(off, fabs(sv));
  }
  orth = block_max(orth, sh);
  off = block_max(off, sh);
  dm = block_max(dm, sh);
  if (tid == 0) {
    jb.sc[2] = orth;
    jb.sc[3] = dm > 0.0 ? off / dm : 1.0;
    if (!(orth <= 1e-12) || !(off <= 1e-12 * dm)) *jb.state = 1;
  }
}

// ---- FP64 route: cyclic two-sided Jacobi on A (K~), rotations into V ----
__global__ void __launch_bounds__(1024) jacobi64_kernel(EigJob *jobs, int *err, int max_sweeps) {
  EigJob jb = jobs[blockIdx.x];
  if (*jb.state != 1) return;
  const int n = jb.n;
  double *A = jb.A, *V = jb.V;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double s_red[32];
  __shared__ double c_s[512], s_s[512];
  __shared__ int pp_s[512], qq_s[512];
  for (int t = tid; t < n * n; t += nt) {
    int i = t / n, j = t % n;
    V[t] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int ne = (n + 1) & ~1;   // even player count (player n is a bye if n odd)
  const int npair = ne / 2;
  bool converged = false;
  int settled = 0;   // one extra sweep after the off-diagonal test passes
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    for (int round = 0; round < ne - 1; ++round) {
      for (int k = tid; k < npair; k += nt) {
        int pi, qi;
        tournament_pair(round, k, ne, pi, qi);
        double c = 1.0, s = 0.0;
        if (qi < n) {
          double apq = A[(size_t)pi * n + qi];
          if (apq != 0.0) {
            double app = A[(size_t)pi * n + pi], aqq = A[(size_t)qi * n + qi];
            double tau = (aqq - app) / (2.0 * apq);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        } else {
          qi = -1;
        }
        c_s[k] = c; s_s[k] = s; pp_s[k] = pi; qq_s[k] = qi;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int t = tid; t < npair * n; t += nt) {
        int k = t / n, j = t % n;
        int pi = pp_s[k], qi = qq_s[k];
        if (qi < 0) continue;
        double c = c_s[k], s = s_s[k];
        double ap = A[(size_t)pi * n + j], aq = A[(size_t)qi * n + j];
        A[(size_t)pi * n + j] = c * ap - s * aq;
        A[(size_t)qi * n + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int t = tid; t < npair * n; t += nt) {
        int k = t % npair, i = t / npair;
        int pi = pp_s[k], qi = qq_s[k];
        if (qi < 0) continue;
        double c = c_s[k], s = s_s[k];
        double ap = A[(size_t)i * n + pi], aq = A[(size_t)i * n + qi];
        A[(size_t)i * n + pi] = c * ap - s * aq;
        A[(size_t)i * n + qi] = s * ap + c * aq;
        double vp = V[(size_t)i * n + pi], vq = V[(size_t)i * n + qi];
        V[(size_t)i * n + pi] = c * vp - s * vq;
        V[(size_t)i * n + qi] = s * vp + c * vq;
      }
      __syncthreads();
      for (int k = tid; k < npair; k += nt) {
        int pi = pp_s[k], qi = qq_s[k];
        if (qi >= 0 && s_s[k] != 0.0) {
          A[(size_t)pi * n + qi] = 0.0;
          A[(size_t)qi * n + pi] = 0.0;
        }
      }
      __syncthreads();
    }
    // off-diagonal mass relative to the diagonal
    double off = 0.0, dia = 0.0;
    for (int t = tid; t < n * n; t += nt) {
      int i = t / n, j = t % n;
      double a = A[t];
      if (i == j) dia += a * a; else off += a * a;
    }
    off = block_sum(off, s_red);
    __syncthreads();
    if (tid == 0) s_red[0] = off;
    __syncthreads();
    double offs = s_red[0];
    __syncthreads();
    dia = block_sum(dia, s_red);
    __syncthreads();
    if (tid == 0) s_red[1] = dia;
    __syncthreads();
    double dias = s_red[1];
    __syncthreads();
    if (offs <= 1e-30 * dias) {
      if (settled) converged = true;
      settled = 1;
    }
  }
  if (!converged && tid == 0) {
    atomicExch(err, (int)IGAFD_ERR_EIG);
    *jb.state = 2;
  }
}

// ---- U = L^{-T} (eigenvectors of K~), sort ascending, sign-normalise ----
// Eigenvectors and values come from (X, diag S) on the fast route and from
// (V, diag A) on the FP64 route.
__global__ void __launch_bounds__(1024) finish_kernel(EigJob *jobs, int parity) {
  EigJob jb = jobs[blockIdx.x];
  const int st = *jb.state;
  if (st == 2) return;
  const int n = jb.n, tid = threadIdx.x, nt = blockDim.x;
  const double *Vsrc = st == 0 ? (parity ? jb.Xn : jb.X) : jb.V;
  const double *Lam = st == 0 ? jb.S : jb.A;
  const double *M = jb.M;
  double *K = jb.K, *U = jb.U;
  __shared__ double rdiag[kFastMaxN];
  double *rd = n <= kFastMaxN ? rdiag : jb.E;     // E is free at this point
  for (int i = tid; i < n; i += nt) rd[i] = 1.0 / M[(size_t)i * n + i];
  __syncthreads();
  // U = L^{-T} V (column-parallel backward substitution); w[d] = U[i+1+d][c]
  for (int c = tid; c < n; c += nt) {
    double w[kMaxBand];
#pragma unroll
    for (int d = 0; d < kMaxBand; ++d) w[d] = 0.0;
    for (int i = n - 1; i >= 0; --i) {
      double acc = Vsrc[(size_t)i * n + c];
#pragma unroll
      for (int d = 0; d < kMaxBand; ++d)
        if (d < jb.p && i + 1 + d < n) acc -= M[(size_t)(i + 1 + d) * n + i] * w[d];
      const double x = acc * rd[i];
      K[(size_t)i * n + c] = x;
#pragma unroll
      for (int d = kMaxBand - 1; d > 0; --d) w[d] = w[d - 1];
      w[0] = x;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    double li = Lam[(size_t)i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double lj = Lam[(size_t)j * n + j];
      if (lj < li || (lj == li && j < i)) ++rank;
    }
    int imax = 0;
    double vmax = -1.0;
    for (int r = 0; r < n; ++r) {
      double a = fabs(K[(size_t)r * n + i]);
      if (a > vmax) { vmax = a; imax = r; }
    }
    double sg = K[(size_t)imax * n + i] < 0.0 ? -1.0 : 1.0;
    jb.D[rank] = li;
    for (int r = 0; r < n; ++r) U[(size_t)r * n + rank] = sg * K[(size_t)r * n + i];
  }
}

// inv_lam[i] = 1 / (D_1[i_1] + D_2[i_2] + D_3[i_3])
__global__ void inv_lambda_kernel(const double *D1, const double *D2, const double *D3, int n1,
                                  int n2, long long N, double *inv, float *inv32) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int i1 = (int)(i % n1);
  int i2 = (int)((i / n1) % n2);
  long long i3 = i / ((long long)n1 * n2);
  double lam = D1[i1] + D2[i2] + (D3 ? D3[i3] : 0.0);
  double r = 1.0 / lam;
  inv[i] = r;
  inv32[i] = (float)r;
}

}  // namespace

static GemmJob gemm_job(int n, int transA, const double *A, const double *B, const double *D,
                        double *C, const int *state) {
  GemmJob g{};
  g.n = n; g.transA = transA; g.A = A; g.B = B; g.D = D; g.C = C; g.state = state;
  return g;
}

igafd_status igafd_setup_pencils_eig(igafd_patch *P, cudaStream_t s, const double *const *wK,
                                     const double *const *wM) {
  const int dim = P->dim, p = P->p;
  // scratch for all directions, kept by the patch: 12 n^2 doubles, 4 scalars
  // and a route flag per direction, and the job table
  constexpr int kMats = 12;
  if (!P->eig_work) {
    size_t tot = 0;
    for (int k = 0; k < dim; ++k) tot += kMats * (size_t)P->n[k] * P->n[k] + 8;
    if (cudaMalloc(&P->eig_work, tot * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->eig_jobs, 3 * sizeof(EigJob)) != cudaSuccess) {
      cudaGetLastError();
      return IGAFD_ERR_OOM;
    }
  }
  EigJob hjobs[3];
  size_t off = 0;
  int max_n = 0;
  for (int k = 0; k < dim; ++k) {
    int n = P->n[k];
    max_n = n > max_n ? n : max_n;
    size_t nn = (size_t)n * n;
    EigJob &j = hjobs[k];
    double *w = P->eig_work + off;
    j.n = n; j.p = p;
    j.M = w; j.K = w + nn; j.A = w + 2 * nn; j.V = w + 3 * nn;
    j.X = w + 4 * nn; j.Xn = w + 5 * nn; j.G = w + 6 * nn; j.AX = w + 7 * nn;
    j.S = w + 8 * nn; j.E = w + 9 * nn; j.W = w + 10 * nn;
    j.sc = w + kMats * nn;
    j.state = (int *)(j.sc + 4);
    j.U = P->U[k]; j.D = P->D[k];
    off += kMats * nn + 8;
    IGAFD_CUDA(cudaMemsetAsync(j.M, 0, 2 * nn * sizeof(double), s));
    int th = n * (2 * p + 1);
    pencil_kernel<<<(th + 127) / 128, 128, 0, s>>>(P->dir[k], p, j.K, j.M, wK ? wK[k] : nullptr,
                                                   wM ? wM[k] : nullptr);
    IGAFD_LAUNCHED(1);
  }
  EigJob *djobs = (EigJob *)P->eig_jobs;
  IGAFD_CUDA(cudaMemcpyAsync(djobs, hjobs, sizeof(hjobs), cudaMemcpyHostToDevice, s));
  IGAFD_CUDA(cudaMemsetAsync(P->err_flag, 0, sizeof(int), s));
  cudaEvent_t e0, e1;
  IGAFD_CUDA(cudaEventCreate(&e0));
  IGAFD_CUDA(cudaEventCreate(&e1));
  IGAFD_CUDA(cudaEventRecord(e0, s));
  const int allow_fast = P->eig_route != 1;
  prep_kernel<<<dim, 1024, 0, s>>>(djobs, P->err_flag, allow_fast);
  IGAFD_LAUNCHED(1);
  int parity = 0;
  if (allow_fast && max_n > 0) {
    // fast route for the directions with n <= 128 (the kernels skip the others)
    static bool attr = false;
    const int nmax = kFastMaxN;
    const size_t smem32 = tri32_smem_floats(nmax) * sizeof(float);
    if (!attr) {
      IGAFD_CUDA(cudaFuncSetAttribute(tri32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem32));
      attr = true;
    }
    tri32_kernel<<<dim, 1024, smem32, s>>>(djobs);
    IGAFD_LAUNCHED(1);
    int tiles = 0;
    for (int k = 0; k < dim; ++k) {
      const int t = (P->n[k] + kGT - 1) / kGT;
      tiles = t * t > tiles ? t * t : tiles;
    }
    auto products = [&](bool with_s) -> igafd_status {
      // G = X^T X and AX = K~ X, then S = X^T AX
      GemmBatch b1{}, b2{};
      for (int k = 0; k < dim; ++k) {
        const EigJob &j = hjobs[k];
        const double *X = parity ? j.Xn : j.X;
        b1.j[2 * k] = gemm_job(j.n, 1, X, X, nullptr, j.G, j.state);
        b1.j[2 * k + 1] = gemm_job(j.n, 0, j.A, X, nullptr, j.AX, j.state);
        b2.j[k] = gemm_job(j.n, 1, X, j.AX, nullptr, j.S, j.state);
      }
      gemm64_kernel<<<dim3(tiles, 2 * dim), kGT * kGT, 0, s>>>(b1);
      IGAFD_LAUNCHED(1);
      if (with_s) {
        gemm64_kernel<<<dim3(tiles, dim), kGT * kGT, 0, s>>>(b2);
        IGAFD_LAUNCHED(1);
      }
      IGAFD_CUDA(cudaGetLastError());
      return IGAFD_OK;
    };
    for (int it = 0; it < 4; ++it) {
      IGAFD_TRY(products(true));
      refine_kernel<<<dim, 1024, 0, s>>>(djobs);
      IGAFD_LAUNCHED(1);
      GemmBatch b3{};
      for (int k = 0; k < dim; ++k) {
        const EigJob &j = hjobs[k];
        const double *X = parity ? j.Xn : j.X;
        double *Xnext = parity ? j.X : j.Xn;
        b3.j[k] = gemm_job(j.n, 0, X, nullptr, X, Xnext, j.state);
        b3.j[k].G = j.G; b3.j[k].S = j.S; b3.j[k].lam = j.E; b3.j[k].dl = j.sc + 1;
      }
      gemm64_kernel<<<dim3(tiles, dim), kGT * kGT, 0, s>>>(b3);
      IGAFD_LAUNCHED(1);
      parity ^= 1;
    }
    IGAFD_TRY(products(true));
    cluster_kernel<<<dim, 1024, 0, s>>>(djobs, parity);
    IGAFD_LAUNCHED(1);
    IGAFD_TRY(products(true));
    check_kernel<<<dim, 1024, 0, s>>>(djobs);
    IGAFD_LAUNCHED(1);
  }
  jacobi64_kernel<<<dim, 1024, 0, s>>>(djobs, P->err_flag, 40);
  IGAFD_LAUNCHED(1);
  finish_kernel<<<dim, 1024, 0, s>>>(djobs, parity);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaEventRecord(e1, s));
  long long N = P->N;
  inv_lambda_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
      P->D[0], P->D[1], dim == 3 ? P->D[2] : nullptr, P->n[0], P->n[1], N, P->inv_lam,
      P->inv_lam32);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  // route taken per direction (0 fast, 1 FP64 Jacobi, 2 failed) and the error flag
  int hstate[3] = {0, 0, 0};
  double hsc[3][4] = {};
  int herr = 0;
  for (int k = 0; k < dim; ++k) {
    IGAFD_CUDA(cudaMemcpyAsync(&hstate[k], hjobs[k].state, sizeof(int), cudaMemcpyDeviceToHost, s));
    IGAFD_CUDA(cudaMemcpyAsync(hsc[k], hjobs[k].sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  IGAFD_CUDA(cudaMemcpyAsync(&herr, P->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  igafd_status st = IGAFD_OK;
  cudaError_t ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    fprintf(stderr, "igafd: eigen setup failed: %s\n", cudaGetErrorString(ce));
    st = IGAFD_ERR_CUDA;
  } else if (herr != 0) {
    st = (igafd_status)herr;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  P->eig_ms = ms;
  for (int k = 0; k < dim; ++k) {
    P->eig_used[k] = hstate[k];
    P->eig_check[k][0] = allow_fast && P->n[k] <= kFastMaxN ? hsc[k][2] : 0.0;
    P->eig_check[k][1] = allow_fast && P->n[k] <= kFastMaxN ? hsc[k][3] : 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}
