// y = A x with A stored as a (2p+1)^d-point FP64 stencil, offset-major:
// S[o][row], o = sum_k (delta_k + p)(2p+1)^(k-1) (Section 2.1: an interior
// row of A couples to (2p+1)^d columns). Also r = b - A x (true residual).
//
// One thread per row (grid-stride over a fixed grid that is a multiple of the
// SM count); coefficients are streamed once (evict-first loads), x is read
// through the read-only cache (it stays resident in L2). Couplings that leave
// the index box are skipped, so x is never read out of bounds. Optional
// fused partial dot products with a deterministic last-block reduction.
#include "common.cuh"

namespace {

__device__ __forceinline__ double ld_stream(const double *p) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// Last block of a grid-stride reduction: returns true in every thread of the
// block that finished last (all partials visible), resets the counter.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return am_last;
}

__device__ double sum_partials(const double *part, int n, double *sh32) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += ((volatile const double *)part)[i];
  return block_sum(v, sh32);
}

// mode 0: y = A x, partial (x, y) -> alpha = rho / (x, y) (PCG step) when
//         scal != null; mode 1: y = b - A x, partial (y, y) -> true (r, r).
template <int DIM, int P, int MODE>
__global__ void __launch_bounds__(256) stencil_kernel(const double *__restrict__ S,
                                                      const double *__restrict__ x,
                                                      double *__restrict__ y,
                                                      const double *__restrict__ b, int n1, int n2,
                                                      int n3, long long N, double *partial,
                                                      unsigned int *counter, double *scal,
                                                      int pcg, const double *done) {
  if (done && *done != 0.0) return;
  constexpr int W = 2 * P + 1;
  const long long n12 = (long long)n1 * n2;
  double dot = 0.0;
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < N;
       row += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(row % n1);
    const int i2 = (int)((row / n1) % n2);
    const int i3 = DIM == 3 ? (int)(row / n12) : 0;
    double acc0 = 0.0, acc1 = 0.0;
    const int lo1 = max(-P, -i1), hi1 = min(P, n1 - 1 - i1);
#pragma unroll 1
    for (int d3 = (DIM == 3 ? -P : 0); d3 <= (DIM == 3 ? P : 0); ++d3) {
      if (DIM == 3 && (i3 + d3 < 0 || i3 + d3 >= n3)) continue;
#pragma unroll 1
      for (int d2 = -P; d2 <= P; ++d2) {
        if (i2 + d2 < 0 || i2 + d2 >= n2) continue;
        const long long base = row + (long long)d3 * n12 + (long long)d2 * n1;
        const int ob = (DIM == 3 ? (d3 + P) * W * W : 0) + (d2 + P) * W + P;
        const double *Srow = S + (long long)ob * N + row;
        if (lo1 == -P && hi1 == P) {
#pragma unroll
          for (int d1 = -P; d1 <= P; ++d1) {
            double a = ld_stream(Srow + (long long)d1 * N);
            double v = __ldg(x + base + d1);
            if (d1 & 1) acc1 = fma(a, v, acc1); else acc0 = fma(a, v, acc0);
          }
        } else {
          for (int d1 = lo1; d1 <= hi1; ++d1) {
            double a = ld_stream(Srow + (long long)d1 * N);
            double v = __ldg(x + base + d1);
            acc0 = fma(a, v, acc0);
          }
        }
      }
    }
    double ax = acc0 + acc1;
    if (MODE == 0) {
      y[row] = ax;
      dot = fma(x[row], ax, dot);
    } else {
      double rr = b[row] - ax;
      y[row] = rr;
      dot = fma(rr, rr, dot);
    }
  }
  if (!partial) return;
  __shared__ double sh32[32];
  double bs = block_sum(dot, sh32);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
  if (!last_block(counter)) return;
  double tot = sum_partials(partial, gridDim.x, sh32);
  if (threadIdx.x == 0) {
    *counter = 0u;
    if (pcg) {
      if (MODE == 0) {
        scal[S_PQ] = tot;
        double alpha = scal[S_RHO] / tot;
        if (!(tot > 0.0) || !isfinite(alpha)) {
          scal[S_STATUS] = (double)IGAFD_ERR_BREAKDOWN;
          scal[S_DONE] = 1.0;
        }
        scal[S_ALPHA] = alpha;
      } else {
        scal[S_TRUE_RR] = tot;
        scal[S_RR] = tot;
      }
    }
  }
}

template <int DIM, int MODE>
igafd_status launch_p(int p, dim3 grid, cudaStream_t s, const double *S, const double *x, double *y,
                      const double *b, const int *n, long long N, double *partial, unsigned *counter,
                      double *scal, int pcg, const double *done) {
#define IGAFD_CASE(PP)                                                                   \
  case PP:                                                                               \
    stencil_kernel<DIM, PP, MODE><<<grid, 256, 0, s>>>(S, x, y, b, n[0], n[1], n[2], N,  \
                                                        partial, counter, scal, pcg, done); \
    IGAFD_LAUNCHED(1);                                                                   \
    break;
  switch (p) {
    IGAFD_CASE(1)
    IGAFD_CASE(2)
    IGAFD_CASE(3)
    IGAFD_CASE(4)
    IGAFD_CASE(5)
    IGAFD_CASE(6)
    IGAFD_CASE(7)
    default:
      return IGAFD_ERR_ARG;
  }
#undef IGAFD_CASE
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

}  // namespace

// Internal: y = A x (b == null) or y = b - A x. With pcg != 0 the fused dot
// feeds the PCG scalars; with skip_done != 0 the kernel does nothing once the
// PCG convergence flag is set.
igafd_status igafd_stencil_launch(igafd_patch *P, const double *x, double *y, const double *b,
                                  int pcg, int skip_done, cudaStream_t s) {
  dim3 grid(IGAFD_RED_BLOCKS);
  double *partial = pcg ? P->partial : nullptr;
  double *scal = pcg ? P->scal : nullptr;
  const double *done = skip_done ? P->scal + S_DONE : nullptr;
  unsigned *counter = P->counter;
  if (P->dim == 3) {
    if (b) return launch_p<3, 1>(P->p, grid, s, P->stencil, x, y, b, P->n, P->N, partial, counter, scal, pcg, done);
    return launch_p<3, 0>(P->p, grid, s, P->stencil, x, y, b, P->n, P->N, partial, counter, scal, pcg, done);
  }
  if (b) return launch_p<2, 1>(P->p, grid, s, P->stencil, x, y, b, P->n, P->N, partial, counter, scal, pcg, done);
  return launch_p<2, 0>(P->p, grid, s, P->stencil, x, y, b, P->n, P->N, partial, counter, scal, pcg, done);
}
