// 1D pencils and their generalized eigendecompositions (Section 3 and
// Algorithm 1 line 1 / Eq. (eigen3d)), all in FP64 on the device.
//
//   M_k, K_k: (p+1)-point Gauss quadrature of B_i B_j and B_i' B_j'
//   M = L L^T (banded Cholesky), K~ = L^{-1} K L^{-T} (banded triangular
//   solves), K~ = U~ D U~^T by cyclic two-sided Jacobi with a round-robin
//   (tournament) ordering so that n/2 disjoint rotations run in parallel,
//   U = L^{-T} U~ (Section 4.1). Eigenvalues sorted ascending, each
//   eigenvector signed so that its largest-magnitude entry is positive.
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
// K (becomes X = L^{-1} K), A (K~, then Jacobi-reduced), V (rotations),
// U (output eigenvectors).
struct EigJob {
  int n, p;
  double *M, *K, *A, *V, *U, *D;
};

__global__ void __launch_bounds__(1024) geneig_kernel(EigJob *jobs, int *err, int max_sweeps) {
  EigJob jb = jobs[blockIdx.x];
  const int n = jb.n, p = jb.p;
  double *M = jb.M, *K = jb.K, *A = jb.A, *V = jb.V, *U = jb.U;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_fail;
  __shared__ double s_red[32];
  __shared__ double c_s[512], s_s[512];
  __shared__ int pp_s[512], qq_s[512];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // ---- banded Cholesky M = L L^T (L stored in the lower band of M) ----
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = M[(size_t)k * n + k];
      if (!(d > 0.0)) s_fail = 1;
      M[(size_t)k * n + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    double lkk = M[(size_t)k * n + k];
    int hi = min(n, k + p + 1);
    for (int i = k + 1 + tid; i < hi; i += nt) M[(size_t)i * n + k] /= lkk;
    __syncthreads();
    int bw = hi - (k + 1);
    for (int t = tid; t < bw * bw; t += nt) {
      int i = k + 1 + t / bw, j = k + 1 + t % bw;
      if (j <= i) M[(size_t)i * n + j] -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) atomicExch(err, (int)IGAFD_ERR_NOT_SPD);
    return;
  }
  // ---- X = L^{-1} K (column-parallel forward substitution), into K ----
  for (int c = tid; c < n; c += nt) {
    for (int i = 0; i < n; ++i) {
      double acc = K[(size_t)i * n + c];
      for (int j = max(0, i - p); j < i; ++j) acc -= M[(size_t)i * n + j] * K[(size_t)j * n + c];
      K[(size_t)i * n + c] = acc / M[(size_t)i * n + i];
    }
  }
  __syncthreads();
  // ---- K~ = X L^{-T} (row-parallel), into A ----
  for (int r = tid; r < n; r += nt) {
    for (int j = 0; j < n; ++j) {
      double acc = K[(size_t)r * n + j];
      for (int l = max(0, j - p); l < j; ++l) acc -= M[(size_t)j * n + l] * A[(size_t)r * n + l];
      A[(size_t)r * n + j] = acc / M[(size_t)j * n + j];
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
    V[t] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // ---- cyclic Jacobi with tournament ordering ----
  const int ne = (n + 1) & ~1;   // even player count (player n is a bye if n odd)
  const int npair = ne / 2;
  bool converged = false;
  int settled = 0;   // one extra sweep after the off-diagonal test passes
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    for (int round = 0; round < ne - 1; ++round) {
      for (int k = tid; k < npair; k += nt) {
        int a, b;
        if (k == 0) { a = ne - 1; b = round; }
        else { a = (round + k) % (ne - 1); b = (round - k + ne - 1) % (ne - 1); }
        int pi = min(a, b), qi = max(a, b);
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
  if (!converged) {
    if (tid == 0) atomicExch(err, (int)IGAFD_ERR_EIG);
    return;
  }
  // ---- U = L^{-T} V (column-parallel backward substitution), into K ----
  for (int c = tid; c < n; c += nt) {
    for (int i = n - 1; i >= 0; --i) {
      double acc = V[(size_t)i * n + c];
      for (int j = i + 1; j <= min(n - 1, i + p); ++j) acc -= M[(size_t)j * n + i] * K[(size_t)j * n + c];
      K[(size_t)i * n + c] = acc / M[(size_t)i * n + i];
    }
  }
  __syncthreads();
  // ---- sort ascending, sign-normalise, write U and D ----
  for (int i = tid; i < n; i += nt) {
    double li = A[(size_t)i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double lj = A[(size_t)j * n + j];
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

igafd_status igafd_setup_pencils_eig(igafd_patch *P, cudaStream_t s, const double *const *wK,
                                     const double *const *wM) {
  const int dim = P->dim, p = P->p;
  // scratch for all directions
  size_t tot = 0;
  for (int k = 0; k < dim; ++k) tot += 4 * (size_t)P->n[k] * P->n[k];
  double *work = nullptr;
  if (cudaMalloc(&work, tot * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return IGAFD_ERR_OOM;
  }
  EigJob hjobs[3];
  size_t off = 0;
  for (int k = 0; k < dim; ++k) {
    int n = P->n[k];
    size_t nn = (size_t)n * n;
    EigJob &j = hjobs[k];
    j.n = n; j.p = p;
    j.M = work + off; j.K = j.M + nn; j.A = j.K + nn; j.V = j.A + nn;
    j.U = P->U[k]; j.D = P->D[k];
    off += 4 * nn;
    cudaMemsetAsync(j.M, 0, 2 * nn * sizeof(double), s);
    int th = n * (2 * p + 1);
    pencil_kernel<<<(th + 127) / 128, 128, 0, s>>>(P->dir[k], p, j.K, j.M, wK ? wK[k] : nullptr,
                                                   wM ? wM[k] : nullptr);
  }
  EigJob *djobs = nullptr;
  igafd_status st = IGAFD_OK;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  if (cudaMalloc(&djobs, sizeof(hjobs)) != cudaSuccess) { cudaGetLastError(); st = IGAFD_ERR_OOM; }
  if (st == IGAFD_OK) {
    cudaMemcpyAsync(djobs, hjobs, sizeof(hjobs), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(P->err_flag, 0, sizeof(int), s);
    cudaEventRecord(e0, s);
    geneig_kernel<<<dim, 1024, 0, s>>>(djobs, P->err_flag, 40);
    cudaEventRecord(e1, s);
    long long N = P->N;
    inv_lambda_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
        P->D[0], P->D[1], dim == 3 ? P->D[2] : nullptr, P->n[0], P->n[1], N, P->inv_lam,
        P->inv_lam32);
    int herr = 0;
    cudaMemcpyAsync(&herr, P->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
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
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(djobs);
  cudaFree(work);
  return st;
}
