// Conforming multi-patch numbering (Section 6): patches whose shared sides
// carry the same trace space are glued C^0 by identifying the functions of
// the two sides (the side's row of control points, matched in order, with an
// optional reversal or exchange of the tangential directions). Functions on
// sides that are glued to nothing carry the homogeneous Dirichlet condition.
// This is the host-side index map of the multi-patch Schwarz preconditioner:
// the global space, its Dirichlet set, and so the restriction R_i of each
// subdomain.
#include "common.cuh"

#include <cmath>

#include <algorithm>
#include <vector>

namespace {

// union-find with path halving; the smaller index becomes the root, so the
// numbering below does not depend on the order of the glued sides
struct Dsu {
  std::vector<long long> parent;
  explicit Dsu(long long n) : parent(n) {
    for (long long i = 0; i < n; ++i) parent[i] = i;
  }
  long long find(long long x) {
    while (parent[x] != x) {
      parent[x] = parent[parent[x]];
      x = parent[x];
    }
    return x;
  }
  void unite(long long a, long long b) {
    a = find(a);
    b = find(b);
    if (a == b) return;
    if (a < b) parent[b] = a; else parent[a] = b;
  }
};

// local index of the t-th function (tangential coordinates ta, tb) of side s
// of a patch with m[0..dim) functions per direction, direction 1 fastest
long long side_index(int dim, const int *m, int side, int ta, int tb) {
  const int dir = side / 2, hi = side % 2;
  int idx[3] = {0, 0, 0};
  idx[dir] = hi ? m[dir] - 1 : 0;
  int t = 0;
  for (int k = 0; k < dim; ++k) {
    if (k == dir) continue;
    idx[k] = t == 0 ? ta : tb;
    ++t;
  }
  return idx[0] + (long long)m[0] * (idx[1] + (long long)m[1] * idx[2]);
}

// tangential extents of side s (the directions other than s / 2, in order)
void side_extent(int dim, const int *m, int side, int *na, int *nb) {
  const int dir = side / 2;
  int t = 0, e[2] = {1, 1};
  for (int k = 0; k < dim; ++k)
    if (k != dir) e[t++] = m[k];
  *na = e[0];
  *nb = e[1];
}

}  // namespace

extern "C" igafd_status igafd_mp_numbering(int dim, int npatch, const int *m, int nglue, const int *glue,
                                           long long *global, unsigned char *fixed, long long *n_global) {
  if ((dim != 2 && dim != 3) || npatch < 1 || !m || nglue < 0 || (nglue > 0 && !glue) || !global ||
      !fixed || !n_global)
    return IGAFD_ERR_ARG;
  std::vector<long long> off(npatch + 1, 0);
  for (int q = 0; q < npatch; ++q) {
    long long sz = 1;
    for (int k = 0; k < dim; ++k) {
      if (m[q * dim + k] < 2) return IGAFD_ERR_ARG;
      sz *= m[q * dim + k];
    }
    off[q + 1] = off[q] + sz;
  }
  const long long total = off[npatch];
  Dsu dsu(total);
  std::vector<unsigned char> glued((size_t)npatch * 2 * dim, 0);
  for (int g = 0; g < nglue; ++g) {
    const int *e = glue + 5 * g;
    const int qa = e[0], sa = e[1], qb = e[2], sb = e[3], orient = e[4];
    if (qa < 0 || qa >= npatch || qb < 0 || qb >= npatch || sa < 0 || sa >= 2 * dim || sb < 0 ||
        sb >= 2 * dim || orient < 0 || orient > 7 || (qa == qb && sa == sb))
      return IGAFD_ERR_ARG;
    const int *ma = m + qa * dim, *mb = m + qb * dim;
    int na1, na2, nb1, nb2;
    side_extent(dim, ma, sa, &na1, &na2);
    side_extent(dim, mb, sb, &nb1, &nb2);
    const bool swap = (orient & 4) != 0;     // b's tangential directions exchanged
    if ((swap ? nb2 : nb1) != na1 || (swap ? nb1 : nb2) != na2) return IGAFD_ERR_ARG;   // not conforming
    for (int tb2 = 0; tb2 < na2; ++tb2)
      for (int ta1 = 0; ta1 < na1; ++ta1) {
        // a's (ta1, tb2) meets b's (u, v): orientation bit 0 reverses a's first
        // tangential direction on b, bit 1 the second, bit 2 exchanges them
        int u = (orient & 1) ? na1 - 1 - ta1 : ta1;
        int v = (orient & 2) ? na2 - 1 - tb2 : tb2;
        if (swap) { const int t = u; u = v; v = t; }
        dsu.unite(off[qa] + side_index(dim, ma, sa, ta1, tb2), off[qb] + side_index(dim, mb, sb, u, v));
      }
    glued[(size_t)qa * 2 * dim + sa] = 1;
    glued[(size_t)qb * 2 * dim + sb] = 1;
  }
  // global ids in order of first appearance (patches in order, direction 1 fastest)
  std::vector<long long> id_of_root(total, -1);
  long long ng = 0;
  for (long long t = 0; t < total; ++t) {
    const long long r = dsu.find(t);
    if (id_of_root[r] < 0) id_of_root[r] = ng++;
    global[t] = id_of_root[r];
  }
  for (long long g = 0; g < ng; ++g) fixed[g] = 0;
  // Dirichlet: every function of a side that is glued to nothing
  for (int q = 0; q < npatch; ++q) {
    const int *mq = m + q * dim;
    for (int side = 0; side < 2 * dim; ++side) {
      if (glued[(size_t)q * 2 * dim + side]) continue;
      int n1, n2;
      side_extent(dim, mq, side, &n1, &n2);
      for (int b = 0; b < n2; ++b)
        for (int a = 0; a < n1; ++a) fixed[global[off[q] + side_index(dim, mq, side, a, b)]] = 1;
    }
  }
  *n_global = ng;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_mp_subdomain(int dim, int npatch, const int *m, const long long *global,
                                           const unsigned char *fixed, int qa, int qb, int dir,
                                           long long *rows, int *shape) {
  if ((dim != 2 && dim != 3) || !m || !global || !fixed || !rows || !shape || qa < 0 || qa >= npatch ||
      qb < 0 || qb >= npatch || qa == qb || dir < 0 || dir >= dim)
    return IGAFD_ERR_ARG;
  std::vector<long long> off(npatch + 1, 0);
  for (int q = 0; q < npatch; ++q) {
    long long sz = 1;
    for (int k = 0; k < dim; ++k) sz *= m[q * dim + k];
    off[q + 1] = off[q] + sz;
  }
  const int *ma = m + qa * dim, *mb = m + qb * dim;
  for (int k = 0; k < dim; ++k)
    if (k != dir && ma[k] != mb[k]) return IGAFD_ERR_ARG;
  // the merged patch: a's functions, then b's beyond the shared side
  int mm[3] = {1, 1, 1};
  for (int k = 0; k < dim; ++k) mm[k] = k == dir ? ma[k] + mb[k] - 1 : ma[k];
  for (int k = 0; k < dim; ++k) shape[k] = mm[k] - 2;
  long long t = 0;
  const int hi3 = dim == 3 ? mm[2] - 1 : 1, lo3 = dim == 3 ? 1 : 0;
  for (int j3 = lo3; j3 < hi3; ++j3)
    for (int j2 = 1; j2 < mm[1] - 1; ++j2)
      for (int j1 = 1; j1 < mm[0] - 1; ++j1) {
        int j[3] = {j1, j2, j3};
        const bool in_a = j[dir] <= ma[dir] - 1;
        const int *mq = in_a ? ma : mb;
        if (!in_a) j[dir] -= ma[dir] - 1;
        const long long loc = j[0] + (long long)mq[0] * (j[1] + (long long)mq[1] * (dim == 3 ? j[2] : 0));
        const long long gid = global[(in_a ? off[qa] : off[qb]) + loc];
        if (in_a && j[dir] == ma[dir] - 1) {
          // the shared side: a's last functions must be b's first ones
          int jb[3] = {j[0], j[1], j[2]};
          jb[dir] = 0;
          const long long lb = jb[0] + (long long)mb[0] * (jb[1] + (long long)mb[1] * (dim == 3 ? jb[2] : 0));
          if (global[off[qb] + lb] != gid) return IGAFD_ERR_ARG;   // not glued in this order
        }
        if (fixed[gid]) return IGAFD_ERR_ARG;      // an interior function of the subdomain is fixed
        rows[t++] = gid;
      }
  return IGAFD_OK;
}

// ---- additive Schwarz preconditioner P_IAS (Eq. (Pias)) on the device ----

struct igafd_mp {
  int nsub = 0, dev = 0;
  long long n = 0;                          // global (free) functions
  std::vector<igafd_patch *> patches;       // subdomain patches (owned by the caller)
  std::vector<long long *> rows;            // device rows of R_i
  std::vector<long long> len;               // N_i
  double *tr = nullptr, *tz = nullptr;      // subdomain vectors, max N_i each
  // the operator A (igafd_mp_set_operator): full-space patches and the free
  // index of each of their local functions (-1: Dirichlet)
  std::vector<igafd_patch *> ops;
  std::vector<long long *> omap;
  double *ox = nullptr, *oy = nullptr;      // gathered patch vectors, max over the patches
  // PCG workspace: 7 vectors of n, dot slots (device and pinned host), reduction scratch
  double *w = nullptr;
  double *dots = nullptr, *hdots = nullptr, *partial = nullptr;
  unsigned *counter = nullptr;
};

namespace {

// y[t] = x[rows[t]]: R_i x
__global__ void gather_kernel(const double *__restrict__ x, const long long *__restrict__ rows, long long n,
                              double *__restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = x[rows[t]];
}

// z[rows[t]] += y[t]: R_i^T y (the rows of one subdomain are distinct, so
// one launch per subdomain needs no atomics)
__global__ void scatter_add_kernel(const double *__restrict__ y, const long long *__restrict__ rows, long long n,
                                   double *__restrict__ z) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    z[rows[t]] += y[t];
}

void free_operator(igafd_mp *M) {
  for (long long *d : M->omap) cudaFree(d);
  M->omap.clear();
  M->ops.clear();
  cudaFree(M->ox); cudaFree(M->oy); cudaFree(M->w); cudaFree(M->dots); cudaFree(M->partial);
  cudaFree(M->counter);
  if (M->hdots) cudaFreeHost(M->hdots);
  M->ox = M->oy = M->w = M->dots = M->hdots = M->partial = nullptr;
  M->counter = nullptr;
}

void free_mp(igafd_mp *M) {
  if (!M) return;
  for (long long *r : M->rows) cudaFree(r);
  cudaFree(M->tr);
  cudaFree(M->tz);
  free_operator(M);
  delete M;
}

// y[t] = x[map[t]] (0 where map[t] < 0): a global vector on a patch's full
// index box, Dirichlet functions zero
__global__ void gather_full_kernel(const double *__restrict__ x, const long long *__restrict__ map,
                                   long long n, double *__restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long g = map[t];
    y[t] = g >= 0 ? x[g] : 0.0;
  }
}

// z[map[t]] += y[t] where map[t] >= 0 (a patch's functions map to distinct
// global ones; patches are added one launch after the other, no atomics)
__global__ void scatter_add_full_kernel(const double *__restrict__ y, const long long *__restrict__ map,
                                        long long n, double *__restrict__ z) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long g = map[t];
    if (g >= 0) z[g] += y[t];
  }
}

constexpr int kDotBlocks = 296;      // 2 x 148: fixed grid, fixed summation order

// out = (a, b): CTA partial sums, then the last CTA sums them in order
__global__ void __launch_bounds__(256) mp_dot_kernel(const double *__restrict__ a,
                                                     const double *__restrict__ b, long long n,
                                                     double *partial, unsigned *counter, double *out) {
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v = fma(a[i], b[i], v);
  __shared__ double sh32[32];
  __shared__ bool am_last;
  const double bs = block_sum(v, sh32);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!am_last) return;
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += ((volatile double *)partial)[i];
  t = block_sum(t, sh32);
  if (threadIdx.x == 0) {
    *out = t;
    *counter = 0u;
  }
}

// y += alpha x (alpha from the host)
__global__ void mp_axpy_kernel(double alpha, const double *__restrict__ x, double *__restrict__ y,
                               long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(alpha, x[i], y[i]);
}

// p = z + beta p
__global__ void mp_xpby_kernel(const double *__restrict__ z, double beta, double *__restrict__ p,
                               long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// r = b - t
__global__ void mp_sub_kernel(const double *__restrict__ b, const double *__restrict__ t,
                              double *__restrict__ r, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - t[i];
}

}  // namespace

extern "C" igafd_status igafd_mp_create(int nsub, igafd_patch *const *patches, const long long *const *rows,
                                        long long n_global, igafd_mp **out) {
  if (!out) return IGAFD_ERR_ARG;
  *out = nullptr;
  if (nsub < 1 || !patches || !rows || n_global < 1) return IGAFD_ERR_ARG;
  for (int i = 0; i < nsub; ++i) {
    if (!patches[i] || !rows[i] || patches[i]->dev != patches[0]->dev) return IGAFD_ERR_ARG;
    std::vector<unsigned char> seen((size_t)n_global, 0);
    for (long long t = 0; t < patches[i]->N; ++t) {
      const long long g = rows[i][t];
      if (g < 0 || g >= n_global || seen[(size_t)g]) return IGAFD_ERR_ARG;   // in range, distinct
      seen[(size_t)g] = 1;
    }
  }
  IGAFD_CUDA(cudaSetDevice(patches[0]->dev));
  igafd_mp *M = new igafd_mp();
  M->nsub = nsub;
  M->dev = patches[0]->dev;
  M->n = n_global;
  long long nmax = 0;
  for (int i = 0; i < nsub; ++i) {
    const long long n = patches[i]->N;
    long long *d = nullptr;
    if (cudaMalloc(&d, n * sizeof(long long)) != cudaSuccess) {
      cudaGetLastError();
      free_mp(M);
      return IGAFD_ERR_OOM;
    }
    M->rows.push_back(d);
    if (cudaMemcpy(d, rows[i], n * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_mp(M);
      return IGAFD_ERR_CUDA;
    }
    M->patches.push_back(patches[i]);
    M->len.push_back(n);
    nmax = std::max(nmax, n);
  }
  if (cudaMalloc(&M->tr, nmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M->tz, nmax * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    free_mp(M);
    return IGAFD_ERR_OOM;
  }
  *out = M;
  return IGAFD_OK;
}

extern "C" void igafd_mp_destroy(igafd_mp *M) {
  if (!M) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(M->dev);
  free_mp(M);
  if (cur >= 0) cudaSetDevice(cur);
}

extern "C" igafd_status igafd_mp_apply_ias(igafd_mp *M, igafd_dtype dtype, const double *r, double *z,
                                           void *stream) {
  if (!M || !r || !z || r == z) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(M->dev));
  cudaStream_t s = (cudaStream_t)stream;
  IGAFD_CUDA(cudaMemsetAsync(z, 0, M->n * sizeof(double), s));
  for (int i = 0; i < M->nsub; ++i) {
    const long long n = M->len[i];
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 152 * 8);
    gather_kernel<<<grid, 256, 0, s>>>(r, M->rows[i], n, M->tr);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
    IGAFD_TRY(igafd_apply_prec(M->patches[i], dtype, M->tr, M->tz, s));   // P_i^{-1}, fast diagonalization
    scatter_add_kernel<<<grid, 256, 0, s>>>(M->tz, M->rows[i], n, z);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
  }
  return IGAFD_OK;
}

// ---- the multi-patch operator and its PCG ------------------------------------
extern "C" igafd_status igafd_mp_set_operator(igafd_mp *M, int npatch, igafd_patch *const *patches,
                                              const long long *const *free_of_local) {
  if (!M || npatch < 1 || !patches || !free_of_local) return IGAFD_ERR_ARG;
  for (int q = 0; q < npatch; ++q) {
    igafd_patch *P = patches[q];
    if (!P || !free_of_local[q] || P->dev != M->dev || P->dshift != 0 || !P->stencil)
      return IGAFD_ERR_ARG;                  // full-space patches with a stencil
    std::vector<unsigned char> seen((size_t)M->n, 0);
    for (long long t = 0; t < P->N; ++t) {
      const long long g = free_of_local[q][t];
      if (g < -1 || g >= M->n || (g >= 0 && seen[(size_t)g])) return IGAFD_ERR_ARG;
      if (g >= 0) seen[(size_t)g] = 1;
    }
  }
  IGAFD_CUDA(cudaSetDevice(M->dev));
  free_operator(M);
  long long nmax = 0;
  for (int q = 0; q < npatch; ++q) {
    const long long n = patches[q]->N;
    long long *d = nullptr;
    if (cudaMalloc(&d, n * sizeof(long long)) != cudaSuccess) {
      cudaGetLastError();
      free_operator(M);
      return IGAFD_ERR_OOM;
    }
    M->omap.push_back(d);
    if (cudaMemcpy(d, free_of_local[q], n * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_operator(M);
      return IGAFD_ERR_CUDA;
    }
    M->ops.push_back(patches[q]);
    nmax = std::max(nmax, n);
  }
  if (cudaMalloc(&M->ox, nmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M->oy, nmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M->w, 7 * M->n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M->dots, 8 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M->partial, kDotBlocks * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M->counter, sizeof(unsigned)) != cudaSuccess ||
      cudaHostAlloc((void **)&M->hdots, 8 * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    free_operator(M);
    return IGAFD_ERR_OOM;
  }
  IGAFD_CUDA(cudaMemset(M->counter, 0, sizeof(unsigned)));
  return IGAFD_OK;
}

extern "C" igafd_status igafd_mp_apply_A(igafd_mp *M, const double *x, double *y, void *stream) {
  if (!M || !x || !y || x == y || M->ops.empty()) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(M->dev));
  cudaStream_t s = (cudaStream_t)stream;
  IGAFD_CUDA(cudaMemsetAsync(y, 0, M->n * sizeof(double), s));
  for (size_t q = 0; q < M->ops.size(); ++q) {
    igafd_patch *P = M->ops[q];
    const unsigned grid = (unsigned)std::min<long long>((P->N + 255) / 256, 152 * 8);
    gather_full_kernel<<<grid, 256, 0, s>>>(x, M->omap[q], P->N, M->ox);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
    IGAFD_TRY(igafd_apply_A(P, M->ox, M->oy, s));       // the patch's own stencil (Eq. (A))
    scatter_add_full_kernel<<<grid, 256, 0, s>>>(M->oy, M->omap[q], P->N, y);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
  }
  return IGAFD_OK;
}

namespace {

// (a, b) into dot slot k, read back to the host (synchronises the stream)
igafd_status mp_dots(igafd_mp *M, cudaStream_t s, int cnt, const double *const *a,
                     const double *const *b) {
  for (int k = 0; k < cnt; ++k) {
    mp_dot_kernel<<<kDotBlocks, 256, 0, s>>>(a[k], b[k], M->n, M->partial, M->counter, M->dots + k);
    IGAFD_LAUNCHED(1);
  }
  IGAFD_CUDA(cudaGetLastError());
  IGAFD_CUDA(cudaMemcpyAsync(M->hdots, M->dots, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  return IGAFD_OK;
}

}  // namespace

extern "C" igafd_status igafd_mp_pcg_solve(igafd_mp *M, const igafd_pcg_opts *opts, const double *b,
                                           double *x, igafd_pcg_info *info, void *stream) {
  if (!M || !b || !x || b == x || M->ops.empty()) return IGAFD_ERR_ARG;
  igafd_pcg_opts o;
  if (opts) o = *opts; else igafd_pcg_default_opts(&o);
  if (!(o.tol >= 0.0) || o.max_iter < 0 || o.true_every < 0) return IGAFD_ERR_ARG;
  if (o.prec_dtype < IGAFD_FP64 || o.prec_dtype > IGAFD_TF32) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(M->dev));
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = M->n;
  const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 152 * 8);
  double *xs = M->w, *r = M->w + n, *z = M->w + 2 * n, *zn = M->w + 3 * n, *p = M->w + 4 * n,
         *q = M->w + 5 * n, *t = M->w + 6 * n;
  const double *h = M->hdots;
  igafd_pcg_info inf{};
  inf.status = IGAFD_ERR_NOT_CONVERGED;
  auto finish = [&](igafd_status st) -> igafd_status {
    inf.status = st;
    IGAFD_CUDA(cudaMemcpyAsync(x, xs, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    IGAFD_CUDA(cudaStreamSynchronize(s));
    if (info) *info = inf;
    return st;
  };
  const double *bb_args[1] = {b};
  IGAFD_TRY(mp_dots(M, s, 1, bb_args, bb_args));
  const double bb = h[0];
  if (!(bb >= 0.0) || !std::isfinite(bb)) {
    IGAFD_CUDA(cudaMemsetAsync(xs, 0, n * sizeof(double), s));
    return finish(IGAFD_ERR_BREAKDOWN);
  }
  if (bb == 0.0) {
    IGAFD_CUDA(cudaMemsetAsync(xs, 0, n * sizeof(double), s));
    return finish(IGAFD_OK);
  }
  // x0 = 0 or the caller's; r0 = b - A x0; z0 = P_IAS r0; p0 = z0
  if (o.x0_given) {
    IGAFD_CUDA(cudaMemcpyAsync(xs, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    IGAFD_TRY(igafd_mp_apply_A(M, xs, t, s));
    mp_sub_kernel<<<grid, 256, 0, s>>>(b, t, r, n);
    IGAFD_LAUNCHED(1);
  } else {
    IGAFD_CUDA(cudaMemsetAsync(xs, 0, n * sizeof(double), s));
    IGAFD_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  IGAFD_TRY(igafd_mp_apply_ias(M, o.prec_dtype, r, z, s));
  IGAFD_CUDA(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const double *rz_a[1] = {r}, *rz_b[1] = {z};
  IGAFD_TRY(mp_dots(M, s, 1, rz_a, rz_b));
  double rho = h[0];
  const double tol2 = o.tol * o.tol * bb;
  for (int k = 1; k <= o.max_iter; ++k) {
    IGAFD_TRY(igafd_mp_apply_A(M, p, q, s));                          // q = A p
    const double *pq_a[1] = {p}, *pq_b[1] = {q};
    IGAFD_TRY(mp_dots(M, s, 1, pq_a, pq_b));
    const double alpha = rho / h[0];
    if (!(h[0] > 0.0) || !std::isfinite(alpha)) return finish(IGAFD_ERR_BREAKDOWN);
    mp_axpy_kernel<<<grid, 256, 0, s>>>(alpha, p, xs, n);            // x += alpha p
    mp_axpy_kernel<<<grid, 256, 0, s>>>(-alpha, q, r, n);            // r -= alpha q
    IGAFD_LAUNCHED(2);
    IGAFD_TRY(mp_dots(M, s, 1, rz_a, rz_a));
    inf.iterations = k;
    inf.relres = sqrt(h[0] / bb);
    if (!std::isfinite(h[0])) return finish(IGAFD_ERR_BREAKDOWN);
    if (h[0] <= tol2) {                                              // confirm by the true residual
      IGAFD_TRY(igafd_mp_apply_A(M, xs, t, s));
      mp_sub_kernel<<<grid, 256, 0, s>>>(b, t, t, n);
      IGAFD_LAUNCHED(1);
      const double *tt[1] = {t};
      IGAFD_TRY(mp_dots(M, s, 1, tt, tt));
      inf.true_relres = sqrt(h[0] / bb);
      inf.true_checks++;
      if (h[0] <= tol2) return finish(IGAFD_OK);
      IGAFD_CUDA(cudaMemcpyAsync(r, t, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if (o.true_every > 0 && k % o.true_every == 0) {
      IGAFD_TRY(igafd_mp_apply_A(M, xs, t, s));
      mp_sub_kernel<<<grid, 256, 0, s>>>(b, t, r, n);
      IGAFD_LAUNCHED(1);
      inf.true_checks++;
    }
    if (k == o.max_iter) break;
    IGAFD_TRY(igafd_mp_apply_ias(M, o.prec_dtype, r, zn, s));       // z_new = P_IAS r
    const double *a2[2] = {r, r}, *b2[2] = {zn, z};
    IGAFD_TRY(mp_dots(M, s, 2, a2, b2));
    const double rho_new = h[0];
    const double beta = o.flexible ? (h[0] - h[1]) / rho : rho_new / rho;
    if (!(rho_new > 0.0) || !std::isfinite(beta)) return finish(IGAFD_ERR_BREAKDOWN);
    mp_xpby_kernel<<<grid, 256, 0, s>>>(zn, beta, p, n);             // p = z_new + beta p
    IGAFD_LAUNCHED(1);
    std::swap(z, zn);
    rho = rho_new;
  }
  // not converged: the true residual of the last iterate
  IGAFD_TRY(igafd_mp_apply_A(M, xs, t, s));
  mp_sub_kernel<<<grid, 256, 0, s>>>(b, t, t, n);
  IGAFD_LAUNCHED(1);
  const double *tt[1] = {t};
  IGAFD_TRY(mp_dots(M, s, 1, tt, tt));
  inf.true_relres = sqrt(h[0] / bb);
  return finish(IGAFD_ERR_NOT_CONVERGED);
}
