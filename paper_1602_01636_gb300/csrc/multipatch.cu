// Conforming multi-patch numbering (Section 6): patches whose shared sides
// carry the same trace space are glued C^0 by identifying the functions of
// the two sides (the side's row of control points, matched in order, with an
// optional reversal or exchange of the tangential directions). Functions on
// sides that are glued to nothing carry the homogeneous Dirichlet condition.
// This is the host-side index map of the multi-patch Schwarz preconditioner:
// the global space, its Dirichlet set, and so the restriction R_i of each
// subdomain.
#include "common.cuh"

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

void free_mp(igafd_mp *M) {
  if (!M) return;
  for (long long *r : M->rows) cudaFree(r);
  cudaFree(M->tr);
  cudaFree(M->tz);
  delete M;
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
