// Three-variable ADI preconditioner (Section 5.2): the Douglas iteration of
// Eq. (ADI3D) in the mass-scaled form of Eq. (ADI3D2) and Algorithm 4, from
// s_0 = 0, so that J iterations applied to r give P_J^{-1} r (Theorem 1 and
// its 3D analogue). Parameters by the greedy rule of Eqs. (greedy1)-(greedy2)
// over the triples of eigenvalues of M_k^{-1} K_k, stopped at the first J
// with rho_J <= eps.
//
// Every step of an iteration is a set of independent line problems along one
// direction: a banded product with K_k or M_k followed by a banded Cholesky
// solve with K_k + w_j M_k or M_k. One CTA takes kL lines of one direction
// into shared memory with coalesced loads (direction 1: kL whole rows, which
// are contiguous; directions 2 and 3: kL consecutive i_1 at every position
// along the line), forms the products with all its threads, solves with one
// thread per line (forward and backward substitution, p terms each), and
// stores coalesced. Per iteration four such kernels run:
//   dir 2: u_j = (M2^{-1} K2) s_{j-1}
//   dir 1: s*_j = (K1 + w M1)^{-1} (r~ - (K1 - w M1) s_{j-1} - 2 M1 (u_j + v_j))
//   dir 2: b_j = v_j + w (K2 + w M2)^{-1} M2 (u_j + w s*_j)
//   dir 3: s_j = (K3 + w M3)^{-1} M3 b_j,  v_{j+1} = b_j - w s_j
// after r~ = 2 (I (x) M2 (x) M3)^{-1} r (two more line kernels). Arithmetic is
// FP64 (the paper's) or FP32 (an inexact P_J, like the mixed FD).
//
// Two variables (Section 4.2, Algorithm 2): the Peaceman-Rachford iteration of
// Eq. (ADI) in the mass-scaled variables s~, with gamma_j = omega_j (the
// optimal parameters for equal spectral intervals, w_j = b dn((2j-1)K/(2J), k),
// and J from Eq. (ADIits)). Each half step solves along one direction and
// forms the next half step's right-hand side along the same direction, so an
// iteration is two line kernels:
//   dir 1: s~_{j-1/2} = (K1 + w_j M1)^{-1} r_{j-1},  r_{j-1/2} = r - (K1 - w_j M1) s~_{j-1/2}
//   dir 2: s~_j = (K2 + w_j M2)^{-1} r_{j-1/2},      r_j = r - (K2 - w_{j+1} M2) s~_j
// with r_0 = r, and a last dir-1 kernel s_J = M1^{-1} s~_J.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

// device state of a patch's ADI preconditioner (owned by the patch)
struct AdiState {
  int J = 0, fp32 = 0, p = 0, dim = 3, n[3] = {0, 0, 0};
  size_t esz = 8;                  // bytes per element (8 FP64, 4 FP32)
  double *omega = nullptr;         // [J] host copy
  void *band[3] = {nullptr, nullptr, nullptr};   // [2][n][2p+1]: K band, M band
  void *fac[3] = {nullptr, nullptr, nullptr};    // [J+1][n][p+1]: K + w_j M (j < J), M (j = J)
  void *vec = nullptr;             // 6 N-vectors: r~, u, v, s, s*, b
};

namespace {

constexpr int kL = 32;      // lines per CTA (one solving thread each)
constexpr int kT = 128;     // threads per CTA
constexpr int kMaxLen = 256;

enum { ST_PRE2 = 0, ST_PRE3, ST_U, ST_S1, ST_B, ST_S, ST2_A, ST2_B, ST2_F };

// direction (0-based) whose lines a step works on
__host__ __device__ constexpr int step_mode(int st) {
  return (st == ST_S1 || st == ST2_A || st == ST2_F) ? 0 : (st == ST_PRE3 || st == ST_S) ? 2 : 1;
}

template <typename T>
struct LineArgs {
  int n1, n2, n3, p, len, chunks;
  unsigned len_magic;              // floor(e / len) = umulhi(e, len_magic) for e < 2^16 (0: len = 1)
  double w;                        // w_j of this iteration
  double w_next;                   // w_{j+1} (two-variable ADI: the next right-hand side)
  int first, last;                 // first / last iteration of the apply
  const double *r;                 // FP64 input (ST_PRE2)
  double *z;                       // FP64 output (ST_S of the last iteration)
  T *rt, *u, *v, *s, *s1, *b;      // N-vectors
  const T *bK, *bM;                // bands of this direction's pencil [n][2p+1]
  const T *fac;                    // Cholesky factor used by the solve [n][p+1]
  const double *done;              // PCG convergence flag: skip all work while != 0 (or null)
};

// line l of CTA blk, element i along the line: address in the N-vector
template <int MODE>
__device__ __forceinline__ long long elem_addr(int n1, int n2, int chunks, int blk, int l, int i) {
  if (MODE == 0) return ((long long)blk * kL + l) * n1 + i;
  const int c = blk % chunks, q = blk / chunks;
  const long long i1 = (long long)c * kL + l;
  if (MODE == 1) return i1 + (long long)n1 * (i + (long long)n2 * q);   // q = i3
  return i1 + (long long)n1 * (q + (long long)n2 * i);                  // q = i2
}

template <int MODE>
__device__ __forceinline__ int lines_in(int n1, int n2, int n3, int chunks, int blk) {
  const int left = MODE == 0 ? n2 * n3 - blk * kL : n1 - (blk % chunks) * kL;
  return left < kL ? left : kL;
}

// shared-memory tile index of (line l, element i)
template <int MODE>
__device__ __forceinline__ int tix(int len, int l, int i) {
  return MODE == 0 ? l * (len + 1) + i : i * kL + l;
}

// Elements a thread loads (or stores) per batch: the loads of a batch are all
// issued before their values are written to shared memory, so a thread keeps
// kU global loads in flight instead of one (the line kernels run few warps
// per SM, and a load-to-store chain per element left them waiting on memory).
constexpr int kU = 8;
template <typename T>
constexpr int batch_of() { return sizeof(T) == 4 ? 2 * kU : kU; }   // 64 bytes of loads per batch

// (line, element) of the e-th entry of the CTA's tile in load order: lines
// outermost in direction 1 (whole rows), elements outermost otherwise
template <int MODE, typename T>
__device__ __forceinline__ void entry(const LineArgs<T> &a, int e, int &l, int &i) {
  if (MODE == 0) {
    l = a.len_magic ? (int)__umulhi((unsigned)e, a.len_magic) : e;   // magic 0: len = 1
    i = e - l * a.len;
  } else {
    l = e % kL;
    i = e / kL;
  }
}

// tile(l, i) = f(address) for the CTA's lines, coalesced
template <int MODE, typename T, typename F>
__device__ __forceinline__ void load_tile(T *tile, const LineArgs<T> &a, int nv, F f) {
  constexpr int U = batch_of<T>();
  const int len = a.len, total = len * kL;
  for (int e0 = threadIdx.x; e0 < total; e0 += kT * U) {
    T v[U];
    int t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kT;
      int l, i;
      entry<MODE>(a, e, l, i);
      t[u] = (e < total && l < nv) ? tix<MODE>(len, l, i) : -1;
      if (t[u] >= 0) v[u] = f(elem_addr<MODE>(a.n1, a.n2, a.chunks, blockIdx.x, l, i));
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (t[u] >= 0) tile[t[u]] = v[u];
  }
}

// two tiles at once (their loads in flight together)
template <int MODE, typename T, typename F0, typename F1>
__device__ __forceinline__ void load_tiles2(T *tile0, F0 f0, T *tile1, F1 f1, const LineArgs<T> &a,
                                            int nv) {
  constexpr int U = batch_of<T>() / 2;
  const int len = a.len, total = len * kL;
  for (int e0 = threadIdx.x; e0 < total; e0 += kT * U) {
    T v0[U], v1[U];
    int t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kT;
      int l, i;
      entry<MODE>(a, e, l, i);
      t[u] = (e < total && l < nv) ? tix<MODE>(len, l, i) : -1;
      if (t[u] >= 0) {
        const long long g = elem_addr<MODE>(a.n1, a.n2, a.chunks, blockIdx.x, l, i);
        v0[u] = f0(g);
        v1[u] = f1(g);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (t[u] >= 0) {
        tile0[t[u]] = v0[u];
        tile1[t[u]] = v1[u];
      }
  }
}

// g(address, tile(l, i)) for the CTA's lines, coalesced (g only writes)
template <int MODE, typename T, typename G>
__device__ __forceinline__ void store_tile(const T *tile, const LineArgs<T> &a, int nv, G g) {
  const int len = a.len;
  for (int e = threadIdx.x; e < len * kL; e += kT) {
    int l, i;
    entry<MODE>(a, e, l, i);
    if (l < nv) g(elem_addr<MODE>(a.n1, a.n2, a.chunks, blockIdx.x, l, i), tile[tix<MODE>(len, l, i)]);
  }
}

// out(l, i) = base(l, i) + sum_{|o| <= p} coef(i, o) x(l, i + o) over the
// CTA's lines; coef(i, o) reads the staged bands. Terms are added in
// increasing o, those outside the line skipped; P > 0 is the compile-time band
// half-width (an unrolled sum whose skipped terms are predicated off, so the
// lanes of a warp never split between paths), P = 0 the run-time one.
template <int MODE, int P, typename T, typename C, typename B>
__device__ __forceinline__ void band_product_p(const LineArgs<T> &a, T *out, const T *x, int p,
                                               int nv, C coef, B base) {
  const int len = a.len;
  for (int e = threadIdx.x; e < len * kL; e += kT) {
    int l, i;
    entry<MODE>(a, e, l, i);
    if (l >= nv) continue;
    T acc = base(l, i);
    if (P > 0) {
#pragma unroll
      for (int o = -P; o <= P; ++o) {
        const int j = i + o;
        if (j >= 0 && j < len) acc += coef(i, o) * x[tix<MODE>(len, l, j)];
      }
    } else {
      const int olo = i - p < 0 ? -i : -p, ohi = i + p >= len ? len - 1 - i : p;
      for (int o = olo; o <= ohi; ++o) acc += coef(i, o) * x[tix<MODE>(len, l, i + o)];
    }
    out[tix<MODE>(len, l, i)] = acc;
  }
}

template <int MODE, typename T, typename C, typename B>
__device__ __forceinline__ void band_product(const LineArgs<T> &a, T *out, const T *x, int p, int nv,
                                             C coef, B base) {
  switch (p) {
    case 1: band_product_p<MODE, 1>(a, out, x, p, nv, coef, base); break;
    case 2: band_product_p<MODE, 2>(a, out, x, p, nv, coef, base); break;
    case 3: band_product_p<MODE, 3>(a, out, x, p, nv, coef, base); break;
    case 4: band_product_p<MODE, 4>(a, out, x, p, nv, coef, base); break;
    default: band_product_p<MODE, 0>(a, out, x, p, nv, coef, base);
  }
}

// (L L^T) y = t in place on line l; F[i][t] = L[i][i-p+t] for t < p, F[i][p] = 1 / L[i][i]
template <int MODE, typename T>
__device__ __forceinline__ void chol_solve(T *tile, const T *F, int len, int p, int l) {
  const int W = p + 1;
  for (int i = 0; i < len; ++i) {
    T acc = tile[tix<MODE>(len, l, i)];
    const int kmax = i < p ? i : p;
    for (int k = kmax; k >= 1; --k) acc -= F[i * W + p - k] * tile[tix<MODE>(len, l, i - k)];
    tile[tix<MODE>(len, l, i)] = acc * F[i * W + p];
  }
  for (int i = len - 1; i >= 0; --i) {
    T acc = tile[tix<MODE>(len, l, i)];
    const int kmax = len - 1 - i < p ? len - 1 - i : p;
    for (int k = kmax; k >= 1; --k) acc -= F[(i + k) * W + p - k] * tile[tix<MODE>(len, l, i + k)];
    tile[tix<MODE>(len, l, i)] = acc * F[i * W + p];
  }
}

// The same two substitutions with the last P solved values of the line kept
// in registers, so each step's dependency runs from register to register
// (the tile supplies only the right-hand side and takes the result); the
// products are summed in the order of chol_solve. The factor's slots left of
// the band in the first P rows are never read.
template <int MODE, typename T, int P>
__device__ __forceinline__ void chol_solve_reg(T *tile, const T *F, int len, int l) {
  constexpr int W = P + 1;
  T win[P];                               // win[k - 1] = x[i - k] (forward), x[i + k] (backward)
#pragma unroll
  for (int k = 0; k < P; ++k) win[k] = (T)0;
#pragma unroll 2
  for (int i = 0; i < len; ++i) {
    T acc = tile[tix<MODE>(len, l, i)];
#pragma unroll
    for (int k = P; k >= 1; --k)
      if (k <= i) acc -= F[i * W + P - k] * win[k - 1];
    const T x = acc * F[i * W + P];
    tile[tix<MODE>(len, l, i)] = x;
#pragma unroll
    for (int k = P - 1; k >= 1; --k) win[k] = win[k - 1];
    win[0] = x;
  }
#pragma unroll
  for (int k = 0; k < P; ++k) win[k] = (T)0;
#pragma unroll 2
  for (int i = len - 1; i >= 0; --i) {
    T acc = tile[tix<MODE>(len, l, i)];
#pragma unroll
    for (int k = P; k >= 1; --k)
      if (k <= len - 1 - i) acc -= F[(i + k) * W + P - k] * win[k - 1];
    const T x = acc * F[i * W + P];
    tile[tix<MODE>(len, l, i)] = x;
#pragma unroll
    for (int k = P - 1; k >= 1; --k) win[k] = win[k - 1];
    win[0] = x;
  }
}

template <int MODE, typename T>
__device__ __forceinline__ void chol_solve_line(T *tile, const T *F, int len, int p, int l) {
  switch (p) {
    case 1: chol_solve_reg<MODE, T, 1>(tile, F, len, l); break;
    case 2: chol_solve_reg<MODE, T, 2>(tile, F, len, l); break;
    case 3: chol_solve_reg<MODE, T, 3>(tile, F, len, l); break;
    case 4: chol_solve_reg<MODE, T, 4>(tile, F, len, l); break;
    case 5: chol_solve_reg<MODE, T, 5>(tile, F, len, l); break;
    case 6: chol_solve_reg<MODE, T, 6>(tile, F, len, l); break;
    case 7: chol_solve_reg<MODE, T, 7>(tile, F, len, l); break;
    default: chol_solve<MODE>(tile, F, len, p, l);
  }
}

// dynamic shared memory: two tiles, two bands (the ones the step's products
// use, formed from K and M when staged) and one factor
template <typename T>
__host__ __device__ size_t line_smem(int len, int p) {
  return ((size_t)2 * kL * (len + 1) + (size_t)2 * len * (2 * p + 1) + (size_t)len * (p + 1)) * sizeof(T);
}

template <typename T, int STEP>
__global__ void __launch_bounds__(kT) adi_line_kernel(LineArgs<T> a) {
  constexpr int MODE = step_mode(STEP);
  if (a.done && *a.done != 0.0) return;      // the whole CTA leaves (uniform)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *t0 = reinterpret_cast<T *>(smem_raw);
  T *t1 = t0 + kL * (a.len + 1);
  T *sK = t1 + kL * (a.len + 1);
  const int len = a.len, p = a.p, BW = 2 * p + 1;
  // the step's bands: K (ST_U); M (ST_B, ST_S); -(K - w M) and -2 M (ST_S1);
  // -(K - w M) with w of this half step (ST2_A) or the next (ST2_B)
  T *sX = sK, *sY = sK + len * BW;
  T *sF = sY + len * BW;
  const int nv = lines_in<MODE>(a.n1, a.n2, a.n3, a.chunks, blockIdx.x);
  const T w = (T)a.w;
  const T wc = STEP == ST2_B ? (T)a.w_next : w;
  // bands and factor, kU loads in flight per thread
  const int nb = len * BW, nf = len * (p + 1);
  for (int e0 = threadIdx.x; e0 < nb; e0 += kT * kU) {
    T k[kU], m[kU];   // two loads per entry
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * kT;
      if (e < nb) {
        k[u] = STEP == ST_B || STEP == ST_S ? (T)0 : a.bK[e];
        m[u] = STEP == ST_U ? (T)0 : a.bM[e];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * kT;
      if (e >= nb) continue;
      if (STEP == ST_U) {
        sX[e] = k[u];
      } else if (STEP == ST_B || STEP == ST_S) {
        sX[e] = m[u];
      } else if (STEP == ST_S1 || STEP == ST2_A || STEP == ST2_B) {
        sX[e] = -(k[u] - wc * m[u]);
        sY[e] = (T)-2 * m[u];
      }
    }
  }
  for (int e0 = threadIdx.x; e0 < nf; e0 += kT * kU) {
    T f[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (e0 + u * kT < nf) f[u] = a.fac[e0 + u * kT];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (e0 + u * kT < nf) sF[e0 + u * kT] = f[u];
  }
  auto Kc = [&](int i, int o) { return sX[i * BW + o + p]; };
  auto Mc = [&](int i, int o) { return sX[i * BW + o + p]; };
  auto Cc = [&](int i, int o) { return sX[i * BW + o + p]; };
  auto Dc = [&](int i, int o) { return sY[i * BW + o + p]; };
  auto zero = [&](int, int) { return (T)0; };
  auto same = [&](T *t) { return [t, len](int l, int i) { return t[tix<MODE>(len, l, i)]; }; };
  T *res = t1;                     // the tile the solve works on
  if (STEP == ST_PRE2) {
    load_tile<MODE>(t1, a, nv, [&](long long g) { return (T)a.r[g]; });
  } else if (STEP == ST_PRE3) {
    load_tile<MODE>(t1, a, nv, [&](long long g) { return a.b[g]; });
  } else if (STEP == ST_U) {
    load_tile<MODE>(t0, a, nv, [&](long long g) { return a.s[g]; });
    __syncthreads();
    band_product<MODE>(a, t1, t0, p, nv, Kc, zero);                       // K2 s
  } else if (STEP == ST_S1) {
    if (a.first) {
      load_tile<MODE>(t1, a, nv, [&](long long g) { return a.rt[g]; });      // s = u = v = 0
    } else {
      load_tiles2<MODE>(t0, [&](long long g) { return a.s[g]; }, t1,
                        [&](long long g) { return a.rt[g]; }, a, nv);
      __syncthreads();
      band_product<MODE>(a, t1, t0, p, nv, Cc, same(t1));                  // r~ - (K1 - w M1) s
      __syncthreads();
      load_tile<MODE>(t0, a, nv, [&](long long g) { return a.u[g] + a.v[g]; });
      __syncthreads();
      band_product<MODE>(a, t1, t0, p, nv, Dc, same(t1));                  // - 2 M1 (u + v)
    }
  } else if (STEP == ST_B) {
    if (a.first)
      load_tile<MODE>(t0, a, nv, [&](long long g) { return w * a.s1[g]; });
    else
      load_tile<MODE>(t0, a, nv, [&](long long g) { return a.u[g] + w * a.s1[g]; });
    __syncthreads();
    band_product<MODE>(a, t1, t0, p, nv, Mc, zero);                       // M2 (u + w s*)
  } else if (STEP == ST_S) {
    load_tile<MODE>(t0, a, nv, [&](long long g) { return a.b[g]; });
    __syncthreads();
    band_product<MODE>(a, t1, t0, p, nv, Mc, zero);                       // M3 b
  } else if (STEP == ST2_A) {
    if (a.first)
      load_tile<MODE>(t1, a, nv, [&](long long g) { return (T)a.r[g]; });  // r_0 = r
    else
      load_tile<MODE>(t1, a, nv, [&](long long g) { return a.u[g]; });     // r_{j-1}
  } else if (STEP == ST2_B) {
    load_tile<MODE>(t1, a, nv, [&](long long g) { return a.v[g]; });       // r_{j-1/2}
  } else {                                                                  // ST2_F
    load_tile<MODE>(t1, a, nv, [&](long long g) { return a.s[g]; });       // s~_J
  }
  __syncthreads();
  if ((int)threadIdx.x < nv) chol_solve_line<MODE>(res, sF, len, p, threadIdx.x);
  __syncthreads();
  if (STEP == ST_PRE2) {
    store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.b[g] = x; });               // M2^{-1} r
  } else if (STEP == ST_PRE3) {
    store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.rt[g] = (T)2 * x; });      // r~
  } else if (STEP == ST_U) {
    store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.u[g] = x; });
  } else if (STEP == ST_S1) {
    store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.s1[g] = x; });
  } else if (STEP == ST_B) {
    if (a.first) {
      store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.b[g] = w * x; });
    } else {
      load_tile<MODE>(t0, a, nv, [&](long long g) { return a.v[g]; });       // t0 is free
      __syncthreads();
      const int len_ = len;
      for (int e = threadIdx.x; e < len_ * kL; e += kT) {
        int l, i;
        entry<MODE>(a, e, l, i);
        if (l >= nv) continue;
        const int t = tix<MODE>(len_, l, i);
        a.b[elem_addr<MODE>(a.n1, a.n2, a.chunks, blockIdx.x, l, i)] = t0[t] + w * t1[t];
      }
    }
  } else if (STEP == ST2_A || (STEP == ST2_B && !a.last)) {
    // the next half step's right-hand side r - (K - w M) s~ along the same lines
    load_tile<MODE>(t0, a, nv, [&](long long g) { return (T)a.r[g]; });      // t0 is free
    __syncthreads();
    band_product<MODE>(a, t0, t1, p, nv, Cc, same(t0));
    __syncthreads();
    if (STEP == ST2_A)
      store_tile<MODE>(t0, a, nv, [&](long long g, T x) { a.v[g] = x; });  // r_{j-1/2}
    else
      store_tile<MODE>(t0, a, nv, [&](long long g, T x) { a.u[g] = x; });  // r_j
  } else if (STEP == ST2_B) {
    store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.s[g] = x; });    // s~_J
  } else if (STEP == ST2_F) {
    store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.z[g] = (double)x; });
  } else {
    if (a.last) {
      store_tile<MODE>(t1, a, nv, [&](long long g, T x) { a.z[g] = (double)x; });
    } else {
      const int len_ = len;
      for (int e = threadIdx.x; e < len_ * kL; e += kT) {               // s_j and v_{j+1} = b_j - w s_j
        int l, i;
        entry<MODE>(a, e, l, i);
        if (l >= nv) continue;
        const long long g = elem_addr<MODE>(a.n1, a.n2, a.chunks, blockIdx.x, l, i);
        const T x = t1[tix<MODE>(len_, l, i)];
        a.s[g] = x;
        a.v[g] = t0[tix<MODE>(len_, l, i)] - w * x;
      }
    }
  }
}

// bands of the dense pencil: B[i][o + p] = A[i][i + o] (0 outside the matrix)
template <typename T>
__global__ void band_kernel(const double *K, const double *M, int n, int p, T *bK, T *bM) {
  const int BW = 2 * p + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * BW) return;
  const int i = t / BW, j = i + t % BW - p;
  const bool in = j >= 0 && j < n;
  bK[t] = in ? (T)K[(size_t)i * n + j] : (T)0;
  bM[t] = in ? (T)M[(size_t)i * n + j] : (T)0;
}

// banded Cholesky of K + w_j M (j < J) and of M (j = J), one thread each, in
// FP64; F[j][i][t] = L[i][i-p+t] (t < p), F[j][i][p] = 1 / L[i][i]
template <typename T>
__global__ void factor_kernel(const double *K, const double *M, int n, int p, const double *omega,
                              int J, T *F, double *work, int *err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > J) return;
  const int W = p + 1;
  const double ck = j < J ? 1.0 : 0.0;           // K + w_j M, or M
  const double cm = j < J ? omega[j] : 1.0;
  double *L = work + (size_t)j * n * W;          // FP64 factor, same layout
  for (int i = 0; i < n; ++i) {
    const int j0 = i - p < 0 ? 0 : i - p;
    for (int c = j0; c <= i; ++c) {
      double sum = ck * K[(size_t)i * n + c] + cm * M[(size_t)i * n + c];
      const int m0 = j0;                         // L[i][m] L[c][m] != 0 needs m >= i - p (c <= i)
      for (int m = m0; m < c; ++m) sum -= L[i * W + m - i + p] * L[c * W + m - c + p];
      if (c == i) {
        if (!(sum > 0.0)) {
          atomicExch(err, 1);
          return;
        }
        L[i * W + p] = sqrt(sum);
      } else {
        L[i * W + c - i + p] = sum / L[c * W + p];
      }
    }
  }
  T *out = F + (size_t)j * n * W;
  for (int i = 0; i < n; ++i) {
    for (int t = 0; t < p; ++t) out[i * W + t] = (T)L[i * W + t];
    out[i * W + p] = (T)(1.0 / L[i * W + p]);
  }
}

void free_state(AdiState *A) {
  if (!A) return;
  for (int k = 0; k < 3; ++k) {
    cudaFree(A->band[k]);
    cudaFree(A->fac[k]);
  }
  cudaFree(A->vec);
  delete[] A->omega;
  delete A;
}

template <typename T, int STEP>
igafd_status launch_step(const AdiState &S, const LineArgs<T> &base, int dir, int fac_index,
                         cudaStream_t s) {
  LineArgs<T> a = base;
  const int n2 = S.n[1], n3 = S.n[2], p = S.p;
  a.len = S.n[dir];
  a.len_magic = a.len > 1 ? 0xffffffffu / (unsigned)a.len + 1u : 0u;
  a.bK = (const T *)S.band[dir];
  a.bM = (const T *)S.band[dir] + (size_t)S.n[dir] * (2 * p + 1);
  a.fac = (const T *)S.fac[dir] + (size_t)fac_index * S.n[dir] * (p + 1);
  constexpr int MODE = step_mode(STEP);
  const long long grid = MODE == 0 ? ((long long)n2 * n3 + kL - 1) / kL
                                   : (long long)a.chunks * (MODE == 1 ? n3 : n2);
  const size_t smem = line_smem<T>(a.len, p);
  auto kern = adi_line_kernel<T, STEP>;
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  IGAFD_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_set.load() & bit)) {
    int optin = 0;
    IGAFD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    IGAFD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    attr_set.fetch_or(bit);
  }
  kern<<<(unsigned)grid, kT, smem, s>>>(a);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

template <typename T>
igafd_status apply(igafd_patch *P, const double *r, double *z, cudaStream_t s, const double *done) {
  const AdiState &S = *(const AdiState *)P->adi;
  const long long N = P->N;
  LineArgs<T> a{};
  a.done = done;
  a.n1 = S.n[0]; a.n2 = S.n[1]; a.n3 = S.n[2]; a.p = S.p;
  a.chunks = (S.n[0] + kL - 1) / kL;
  a.r = r; a.z = z;
  T *v0 = (T *)S.vec;
  a.rt = v0; a.u = v0 + N; a.v = v0 + 2 * N; a.s = v0 + 3 * N; a.s1 = v0 + 4 * N; a.b = v0 + 5 * N;
  const int J = S.J;
  if (S.dim == 2) {
    for (int j = 0; j < J; ++j) {
      a.w = S.omega[j];
      a.w_next = j + 1 < J ? S.omega[j + 1] : 0.0;
      a.first = j == 0;
      a.last = j == J - 1;
      IGAFD_TRY((launch_step<T, ST2_A>(S, a, 0, j, s)));
      IGAFD_TRY((launch_step<T, ST2_B>(S, a, 1, j, s)));
    }
    return launch_step<T, ST2_F>(S, a, 0, J, s);               // s_J = M1^{-1} s~_J
  }
  IGAFD_TRY((launch_step<T, ST_PRE2>(S, a, 1, J, s)));        // M2^{-1} r
  IGAFD_TRY((launch_step<T, ST_PRE3>(S, a, 2, J, s)));        // r~ = 2 M3^{-1} (M2^{-1} r)
  for (int j = 0; j < J; ++j) {
    a.w = S.omega[j];
    a.first = j == 0;
    a.last = j == J - 1;
    if (j > 0) IGAFD_TRY((launch_step<T, ST_U>(S, a, 1, J, s)));   // u_j (0 at j = 1)
    IGAFD_TRY((launch_step<T, ST_S1>(S, a, 0, j, s)));
    IGAFD_TRY((launch_step<T, ST_B>(S, a, 1, j, s)));
    IGAFD_TRY((launch_step<T, ST_S>(S, a, 2, j, s)));
  }
  return IGAFD_OK;
}

// Douglas factor of one triple, in the oracle's evaluation order
inline double douglas(double w, double l1, double l2, double l3) {
  return 1.0 - 2.0 * w * w * (l1 + l2 + l3) / ((w + l1) * (w + l2) * (w + l3));
}

// positive root of w^3 - e2 w - 2 e3 (one sign change: exactly one), by
// Newton from the right, where the cubic is increasing and convex
double stationary_root(double e2, double e3) {
  double w = std::sqrt(e2) + std::cbrt(2.0 * e3) + 1e-300;
  for (int it = 0; it < 200; ++it) {
    const double f = w * w * w - e2 * w - 2.0 * e3;
    const double d = 3.0 * w * w - e2;
    const double nw = w - f / d;
    if (!(nw < w)) break;
    w = nw;
  }
  return w;
}

// root of h(w) = w^3 - S w^2 + e2 w + e3 in [lo, hi] with h(lo), h(hi) of
// opposite signs, by bisection
double bisect_root(double S, double e2, double e3, double lo, double hi) {
  auto h = [&](double w) { return ((w - S) * w + e2) * w + e3; };
  const double hlo = h(lo);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if ((h(mid) > 0.0) == (hlo > 0.0)) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

void igafd_adi_free(igafd_patch *P) {
  if (P && P->adi) {
    free_state((AdiState *)P->adi);
    P->adi = nullptr;
    // a captured PCG loop may hold this state's buffers in its kernel
    // arguments: make the next solve capture it again
    memset(P->loop_key, 0, sizeof(P->loop_key));
  }
}

igafd_status igafd_adi_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                             double *done) {
  if (!P || !P->adi || !r || !z || r == z) return IGAFD_ERR_ARG;
  const AdiState *S = (const AdiState *)P->adi;
  return S->fp32 ? apply<float>(P, r, z, s, done) : apply<double>(P, r, z, s, done);
}

namespace {

// f(chunk, lo, hi) over [0, NT) split into nthr contiguous chunks, one thread each
template <typename F>
void for_chunks(size_t NT, int nthr, F f) {
  if (nthr <= 1) {
    f(0, (size_t)0, NT);
    return;
  }
  std::vector<std::thread> th;
  const size_t per = (NT + nthr - 1) / nthr;
  for (int c = 0; c < nthr; ++c) {
    const size_t lo = (size_t)c * per, hi = std::min(NT, lo + per);
    if (lo < hi) th.emplace_back(f, c, lo, hi);
  }
  for (auto &t : th) t.join();
}

}  // namespace

extern "C" igafd_status igafd_adi_greedy(const double *L1, int n1, const double *L2, int n2,
                                         const double *L3, int n3, double eps, int max_J,
                                         double *omega, int *J_out) {
  if (!L1 || !L2 || !L3 || n1 < 1 || n2 < 1 || n3 < 1 || !omega || !J_out || max_J < 1 ||
      !(eps > 0.0) || !(eps < 1.0))
    return IGAFD_ERR_ARG;
  const size_t NT = (size_t)n1 * n2 * n3;
  for (int i = 0; i < n1; ++i) if (!(L1[i] > 0.0)) return IGAFD_ERR_ARG;
  for (int i = 0; i < n2; ++i) if (!(L2[i] > 0.0)) return IGAFD_ERR_ARG;
  for (int i = 0; i < n3; ++i) if (!(L3[i] > 0.0)) return IGAFD_ERR_ARG;
  std::vector<double> prod(NT, 1.0);
  const unsigned hc = std::thread::hardware_concurrency();
  const int nthr = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>(hc ? hc : 1, 16), NT / 65536));
  std::vector<double> cmax(2 * 16), amax(16);
  std::vector<size_t> aarg(16);
  // visit the triples of [lo, hi) in (i3, i2, i1) order: fn(t, l1, l2, l3)
  auto sweep = [&](size_t lo, size_t hi, auto fn) {
    size_t i1 = lo % n1, i2 = (lo / n1) % n2, i3 = lo / ((size_t)n1 * n2);
    for (size_t t = lo; t < hi; ++t) {
      fn(t, L1[i1], L2[i2], L3[i3]);
      if (++i1 == (size_t)n1) {
        i1 = 0;
        if (++i2 == (size_t)n2) { i2 = 0; ++i3; }
      }
    }
  };
  // greedy start: the triple of smallest eigenvalues (the empty product is 1 everywhere)
  double st1 = L1[0], st2 = L2[0], st3 = L3[0];
  int J = 0;
  bool met = false;
  while (J < max_J) {
    const double S = st1 + st2 + st3;
    const double e2 = st1 * st2 + st1 * st3 + st2 * st3, e3 = st1 * st2 * st3;
    double cand[2] = {0.0, 0.0};
    int nc = 1;
    cand[0] = stationary_root(e2, e3);
    if (douglas(cand[0], st1, st2, st3) < 0.0) {           // |g| = 0 at the two zeros of g
      const double ws = cand[0];
      cand[0] = bisect_root(S, e2, e3, 0.0, ws);
      cand[1] = bisect_root(S, e2, e3, ws, 2.0 * S);
      nc = 2;
    }
    int best = 0;
    if (nc == 2) {   // the zero whose use gives the smaller max |prod * g(w)|
      std::fill(cmax.begin(), cmax.end(), 0.0);
      for_chunks(NT, nthr, [&](int c, size_t lo, size_t hi) {
        double m0 = 0.0, m1 = 0.0;
        sweep(lo, hi, [&](size_t t, double l1, double l2, double l3) {
          const double v0 = std::fabs(prod[t] * douglas(cand[0], l1, l2, l3));
          const double v1 = std::fabs(prod[t] * douglas(cand[1], l1, l2, l3));
          m0 = v0 > m0 ? v0 : m0;
          m1 = v1 > m1 ? v1 : m1;
        });
        cmax[2 * c] = m0;
        cmax[2 * c + 1] = m1;
      });
      double m0 = 0.0, m1 = 0.0;
      for (int c = 0; c < nthr; ++c) {
        m0 = std::max(m0, cmax[2 * c]);
        m1 = std::max(m1, cmax[2 * c + 1]);
      }
      best = m1 < m0 ? 1 : 0;
    }
    const double w = cand[best];
    omega[J++] = w;
    // apply it, and find the next worst triple (first maximum in i3, i2, i1 order)
    std::fill(amax.begin(), amax.end(), -1.0);
    for_chunks(NT, nthr, [&](int c, size_t lo, size_t hi) {
      double mx = -1.0;
      size_t arg = lo;
      sweep(lo, hi, [&](size_t t, double l1, double l2, double l3) {
        prod[t] = prod[t] * douglas(w, l1, l2, l3);
        const double v = std::fabs(prod[t]);
        if (v > mx) {
          mx = v;
          arg = t;
        }
      });
      amax[c] = mx;
      aarg[c] = arg;
    });
    double mx = -1.0;
    size_t arg = 0;
    for (int c = 0; c < nthr; ++c)
      if (amax[c] > mx) {        // strict: the earlier chunk keeps a tie
        mx = amax[c];
        arg = aarg[c];
      }
    if (mx <= eps) {
      met = true;
      break;
    }
    const size_t i1 = arg % n1, i2 = (arg / n1) % n2, i3 = arg / ((size_t)n1 * n2);
    st1 = L1[i1]; st2 = L2[i2]; st3 = L3[i3];
  }
  *J_out = J;
  return met ? IGAFD_OK : IGAFD_ERR_NOT_CONVERGED;
}

namespace {

// complete elliptic integral K(k), k^2 = 1 - kp^2, by the arithmetic-geometric
// mean of 1 and kp (Abramowitz and Stegun 17.6: K = pi / (2 AGM(1, k')))
double agm_K(double kp) {
  double a = 1.0, b = kp;
  for (int it = 0; it < 64 && std::fabs(a - b) > 1e-16 * a; ++it) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return 3.14159265358979323846 / (2.0 * a);
}

// Jacobi dn(u, k), k^2 = 1 - kp^2, by the AGM method (Abramowitz and Stegun
// 16.4) started from kp itself: a_0 = 1, b_0 = k', c_0 = k, c_{n+1} =
// c_n^2 / (4 a_{n+1}) until c_N is negligible; phi_N = 2^N a_N u, then
// phi_{n-1} = (phi_n + asin((c_n / a_n) sin phi_n)) / 2, and
// dn = cos(phi_0) / cos(phi_1 - phi_0)
double agm_dn(double u, double kp) {
  double a[64], c[64];
  a[0] = 1.0;
  c[0] = std::sqrt((1.0 - kp) * (1.0 + kp));
  double b = kp;
  int N = 0;
  while (c[N] > 1e-16 * a[N] && N < 63) {
    a[N + 1] = 0.5 * (a[N] + b);
    c[N + 1] = c[N] * c[N] / (4.0 * a[N + 1]);
    b = std::sqrt(a[N] * b);
    ++N;
  }
  if (N == 0) return 1.0;
  double phi = std::ldexp(a[N] * u, N);
  double prev = phi;
  for (int n = N; n >= 1; --n) {
    prev = phi;
    phi = 0.5 * (phi + std::asin(c[n] / a[n] * std::sin(phi)));
  }
  return std::cos(phi) / std::cos(prev - phi);
}

}  // namespace

extern "C" igafd_status igafd_adi_wachspress(double a, double b, double eps, int max_J,
                                             double *omega, int *J_out) {
  if (!omega || !J_out || max_J < 1 || !(a > 0.0) || !(b >= a) || !std::isfinite(b) ||
      !(eps > 0.0) || !(eps < 1.0))
    return IGAFD_ERR_ARG;
  // Eq. (ADIits)
  const double pi = 3.14159265358979323846;
  const double Jr = std::ceil(std::log(4.0 * b / a) * std::log(4.0 / eps) / (pi * pi));
  const int J = Jr < 1.0 ? 1 : (int)Jr;
  if (J > max_J) {
    *J_out = max_J;
    return IGAFD_ERR_NOT_CONVERGED;
  }
  if (a == b) {
    for (int j = 0; j < J; ++j) omega[j] = a;
  } else {
    const double kp = a / b, K = agm_K(kp);
    for (int j = 1; j <= J; ++j) {
      const double u = (2 * j - 1) * K / (2.0 * J);
      // dn(K - u) = k' / dn(u): evaluate dn only for u <= K / 2
      omega[j - 1] = (2 * j - 1 <= J) ? b * agm_dn(u, kp) : a / agm_dn(K - u, kp);
    }
  }
  *J_out = J;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_adi_parameters(igafd_patch *P, double eps, int max_J, double *omega,
                                             int *J_out) {
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // a full-space patch has no preconditioner
  if (!P || (P->dim != 2 && P->dim != 3) || !omega || !J_out || max_J < 1 || !(eps > 0.0) ||
      !(eps < 1.0))
    return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  std::vector<double> L1(n1), L2(n2), L3(n3);
  IGAFD_CUDA(cudaDeviceSynchronize());
  IGAFD_CUDA(cudaMemcpy(L1.data(), P->D[0], n1 * sizeof(double), cudaMemcpyDeviceToHost));
  IGAFD_CUDA(cudaMemcpy(L2.data(), P->D[1], n2 * sizeof(double), cudaMemcpyDeviceToHost));
  if (P->dim == 2) {
    // the hull of the two spectra (Eq. (ADIits) assumes equal intervals)
    const double a = std::min(L1[0], L2[0]), b = std::max(L1[n1 - 1], L2[n2 - 1]);
    return igafd_adi_wachspress(a, b, eps, max_J, omega, J_out);
  }
  IGAFD_CUDA(cudaMemcpy(L3.data(), P->D[2], n3 * sizeof(double), cudaMemcpyDeviceToHost));
  return igafd_adi_greedy(L1.data(), n1, L2.data(), n2, L3.data(), n3, eps, max_J, omega, J_out);
}

extern "C" igafd_status igafd_adi_setup(igafd_patch *P, const double *omega, int J, igafd_dtype dtype,
                                        void *stream) {
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // a full-space patch has no preconditioner
  if (!P || (P->dim != 2 && P->dim != 3) || !omega || J < 1 || J > 100000 ||
      (dtype != IGAFD_FP64 && dtype != IGAFD_FP32))
    return IGAFD_ERR_ARG;
  for (int j = 0; j < J; ++j)
    if (!(omega[j] > 0.0) || !std::isfinite(omega[j])) return IGAFD_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (P->n[k] < 1 || P->n[k] > kMaxLen) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  cudaStream_t s = (cudaStream_t)stream;
  igafd_adi_free(P);
  AdiState *S = new AdiState();
  S->J = J;
  S->fp32 = dtype == IGAFD_FP32;
  S->esz = S->fp32 ? sizeof(float) : sizeof(double);
  S->p = P->p;
  S->dim = P->dim;
  for (int k = 0; k < 3; ++k) S->n[k] = P->n[k];
  S->omega = new double[J];
  std::copy(omega, omega + J, S->omega);
  const int p = P->p;
  int nmax = 0;
  for (int k = 0; k < 3; ++k) nmax = std::max(nmax, P->n[k]);
  double *dense = nullptr, *work = nullptr, *dom = nullptr;
  int *err = nullptr;
  igafd_status st = IGAFD_OK;
  auto fail = [&](igafd_status e) {
    cudaGetLastError();
    cudaFree(dense); cudaFree(work); cudaFree(dom); cudaFree(err);
    free_state(S);
    return e;
  };
  if (cudaMalloc(&S->vec, 6 * (size_t)P->N * S->esz) != cudaSuccess ||
      cudaMalloc(&dense, 2 * (size_t)nmax * nmax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&work, (size_t)(J + 1) * nmax * (p + 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dom, J * sizeof(double)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess)
    return fail(IGAFD_ERR_OOM);
  for (int k = 0; k < P->dim; ++k) {
    const int n = P->n[k];
    if (cudaMalloc(&S->band[k], 2 * (size_t)n * (2 * p + 1) * S->esz) != cudaSuccess ||
        cudaMalloc(&S->fac[k], (size_t)(J + 1) * n * (p + 1) * S->esz) != cudaSuccess)
      return fail(IGAFD_ERR_OOM);
  }
  if (cudaMemcpyAsync(dom, omega, J * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess)
    return fail(IGAFD_ERR_CUDA);
  for (int k = 0; k < P->dim; ++k) {
    const int n = P->n[k];
    double *K = dense, *M = dense + (size_t)n * n;
    st = igafd_pencils_dense(P, k, K, M, s);
    if (st != IGAFD_OK) return fail(st);
    const int nb = n * (2 * p + 1);
    if (S->fp32) {
      band_kernel<float><<<(nb + 127) / 128, 128, 0, s>>>(K, M, n, p, (float *)S->band[k],
                                                          (float *)S->band[k] + nb);
      factor_kernel<float><<<(J + 1 + 63) / 64, 64, 0, s>>>(K, M, n, p, dom, J, (float *)S->fac[k], work, err);
    } else {
      band_kernel<double><<<(nb + 127) / 128, 128, 0, s>>>(K, M, n, p, (double *)S->band[k],
                                                           (double *)S->band[k] + nb);
      factor_kernel<double><<<(J + 1 + 63) / 64, 64, 0, s>>>(K, M, n, p, dom, J, (double *)S->fac[k], work, err);
    }
    IGAFD_LAUNCHED(2);
    if (cudaGetLastError() != cudaSuccess) return fail(IGAFD_ERR_CUDA);
    // (the dense pencils and the FP64 factors are reused, in stream order, by
    // the next direction)
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(IGAFD_ERR_CUDA);
  int herr = 0;
  if (cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(IGAFD_ERR_CUDA);
  if (herr) return fail(IGAFD_ERR_NOT_SPD);
  cudaFree(dense); cudaFree(work); cudaFree(dom); cudaFree(err);
  P->adi = S;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_apply_prec_adi(igafd_patch *P, const double *r, double *z, void *stream) {
  if (!P || !P->adi || !r || !z || r == z) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  return igafd_adi_apply(P, r, z, (cudaStream_t)stream, nullptr);
}
