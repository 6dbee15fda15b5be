// Preconditioned conjugate gradients for A x = b with P^{-1} applied by
// fast diagonalization (Section 3: CG preconditioned by P).
//
// Readings (the paper prints neither the algorithm nor its stopping rule):
// stop when ||r_k|| <= tol ||b|| by the recurrence residual, confirmed by the
// true residual b - A x_k (which replaces r when it does not confirm); the
// true residual is also recomputed every `true_every` iterations; the
// iteration count is the number of products with A inside the loop; beta is
// Fletcher-Reeves or, for an inexact preconditioner, the flexible
// (r_{k+1}, z_{k+1} - z_k) / (r_k, z_k).
//
// All scalars live on the device; every kernel of an iteration returns at
// once when the device convergence flag is set, so the host can enqueue
// several iterations ahead and poll the flag rarely. Reductions use a fixed
// grid and a last-block sum in fixed order (bitwise reproducible).
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

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

// x += alpha p, r -= alpha q; partials (r, r) and (r, z_old).
__global__ void __launch_bounds__(256) update_xr_kernel(double *__restrict__ x, double *__restrict__ r,
                                                        const double *__restrict__ p,
                                                        const double *__restrict__ q,
                                                        const double *__restrict__ z, long long N,
                                                        double *scal, double *partial,
                                                        unsigned *counter, int flexible,
                                                        double *coef) {
  pdl_wait();
  pdl_trigger();
  if (scal[S_DONE] != 0.0) return;
  const double alpha = scal[S_ALPHA];
  double rr = 0.0, rz = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
    if (flexible) rz = fma(ri, z[i], rz);
  }
  __shared__ double sh32[32];
  double a = block_sum(rr, sh32);
  double b = flexible ? block_sum(rz, sh32) : 0.0;
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = a;
    partial[gridDim.x + blockIdx.x] = b;
  }
  if (!last_block(counter)) return;
  double trr = sum_partials(partial, gridDim.x, sh32);
  double trz = flexible ? sum_partials(partial + gridDim.x, gridDim.x, sh32) : 0.0;
  if (threadIdx.x == 0) {
    *counter = 0u;
    scal[S_RR] = trr;
    scal[S_RZOLD] = trz;
    const int k = (int)scal[S_ITER];
    if (k < IGAFD_COEF_CAP) coef[2 * k] = scal[S_ALPHA];     // alpha_k (Lanczos relation)
    scal[S_ITER] += 1.0;
    if (!isfinite(trr)) {
      scal[S_STATUS] = (double)IGAFD_ERR_BREAKDOWN;
      scal[S_DONE] = 1.0;
    } else if (trr <= scal[S_TOL2] * scal[S_BB]) {
      scal[S_DONE] = 1.0;   // converged by the recurrence; the host confirms
    } else if (scal[S_ITER] >= scal[S_MAXIT]) {
      scal[S_STATUS] = (double)IGAFD_ERR_NOT_CONVERGED;
      scal[S_DONE] = 1.0;   // iteration cap
    }
  }
}

// (r, z) -> rho (init) or beta and rho (iteration).
__global__ void __launch_bounds__(256) dot_rz_kernel(const double *__restrict__ r,
                                                     const double *__restrict__ z, long long N,
                                                     double *scal, double *partial,
                                                     unsigned *counter, int init, int flexible,
                                                     int skip_done, double *coef) {
  pdl_wait();
  pdl_trigger();
  if (skip_done && scal[S_DONE] != 0.0) return;
  double rz = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    rz = fma(r[i], z[i], rz);
  __shared__ double sh32[32];
  double a = block_sum(rz, sh32);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
  if (!last_block(counter)) return;
  double t = sum_partials(partial, gridDim.x, sh32);
  if (threadIdx.x == 0) {
    *counter = 0u;
    if (!(t > 0.0) || !isfinite(t)) {
      scal[S_STATUS] = (double)IGAFD_ERR_BREAKDOWN;
      scal[S_DONE] = 1.0;
    }
    if (init) {
      scal[S_BETA] = 0.0;
    } else {
      double rho = scal[S_RHO];
      scal[S_BETA] = flexible ? (t - scal[S_RZOLD]) / rho : t / rho;
      const int k = (int)scal[S_ITER] - 1;                   // beta_k, after step k
      if (k >= 0 && k < IGAFD_COEF_CAP) coef[2 * k + 1] = scal[S_BETA];
    }
    scal[S_RHO] = t;
  }
}

// p = z + beta p
__global__ void __launch_bounds__(256) update_p_kernel(double *__restrict__ p,
                                                       const double *__restrict__ z, long long N,
                                                       const double *scal, int skip_done) {
  pdl_wait();
  pdl_trigger();
  if (skip_done && scal[S_DONE] != 0.0) return;
  const double beta = scal[S_BETA];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// (v, v) -> scal[slot]
__global__ void __launch_bounds__(256) norm2_kernel(const double *__restrict__ v, long long N,
                                                    double *scal, int slot, double *partial,
                                                    unsigned *counter) {
  pdl_wait();
  pdl_trigger();
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    s = fma(v[i], v[i], s);
  __shared__ double sh32[32];
  double a = block_sum(s, sh32);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
  if (!last_block(counter)) return;
  double t = sum_partials(partial, gridDim.x, sh32);
  if (threadIdx.x == 0) {
    *counter = 0u;
    scal[slot] = t;
  }
}

__global__ void init_scalars_kernel(double *scal, double tol2, double maxit) {
  if (threadIdx.x == 0) {
    scal[S_DONE] = maxit > 0.0 ? 0.0 : 1.0;
    scal[S_ITER] = 0.0;
    scal[S_STATUS] = maxit > 0.0 ? 0.0 : (double)IGAFD_ERR_NOT_CONVERGED;
    scal[S_BETA] = 0.0;
    scal[S_RZOLD] = 0.0;
    scal[S_TRUE_RR] = -1.0;
    scal[S_TOL2] = tol2;
    scal[S_MAXIT] = maxit;
  }
}

__global__ void set_scalar_kernel(double *scal, int slot, double v) {
  if (threadIdx.x == 0) scal[slot] = v;
}

}  // namespace

static igafd_status fd_apply(igafd_patch *P, igafd_dtype dt, const double *r, double *z,
                             cudaStream_t s, double *done) {
  switch (dt) {
    case IGAFD_FP64: return igafd_fd64_apply(P, r, z, s, done);
    case IGAFD_FP32: return igafd_fd32_apply(P, r, z, s, done);
    case IGAFD_BF16:
    case IGAFD_FP16:
    case IGAFD_TF32: return igafd_fd_tc_apply(P, dt, r, z, s, done);
    case IGAFD_ADI: return igafd_adi_apply(P, r, z, s, done);
    default: return IGAFD_ERR_ARG;
  }
}

extern "C" igafd_status igafd_apply_prec(igafd_patch *P, igafd_dtype dt, const double *r,
                                         double *z, void *stream) {
  if (!P || !r || !z || r == z) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  return fd_apply(P, dt, r, z, (cudaStream_t)stream, nullptr);
}

extern "C" igafd_status igafd_apply_A(igafd_patch *P, const double *x, double *y, void *stream) {
  if (!P || !x || !y || x == y || !P->stencil) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  return igafd_stencil_launch(P, x, y, nullptr, 0, 0, (cudaStream_t)stream);
}

extern "C" void igafd_pcg_default_opts(igafd_pcg_opts *o) {
  if (!o) return;
  o->tol = 1e-8;
  o->max_iter = 1000;
  o->true_every = 50;
  o->prec_dtype = IGAFD_FP64;
  o->flexible = 0;
  o->x0_given = 0;
  o->check_every = 4;
  o->timing = 0;
}

std::atomic<long long> g_igafd_launches{0};

extern "C" long long igafd_kernel_launches(void) { return g_igafd_launches.load(); }

static igafd_status read_scalars(igafd_patch *P, cudaStream_t s) {
  IGAFD_CUDA(cudaMemcpyAsync(P->host_scal, P->scal, S_COUNT * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  return IGAFD_OK;
}

// One PCG iteration on patch-internal buffers only (so it can be captured
// once and replayed): q = A p, alpha, x += alpha p, r -= alpha q, stopping
// test and cap, periodic true residual, z = P^{-1} r, beta, p = z + beta p.
// Every kernel returns at once when the device flag S_DONE is set.
static igafd_status enqueue_iteration(igafd_patch *P, igafd_dtype dt, int flex, int true_every,
                                      cudaStream_t s, bool timed) {
  const dim3 G(IGAFD_RED_BLOCKS), B(256);
  double *scal = P->scal, *done = P->scal + S_DONE;
  const long long N = P->N;
  IGAFD_TRY(igafd_stencil_launch(P, P->pv, P->q, nullptr, 1, 1, s, 0, timed ? P->tstat : nullptr));
  IGAFD_CUDA(igafd_launch(update_xr_kernel, G, B, 0, s, P->xs, P->r, P->pv, P->q, P->z, N, scal, P->partial,
                                   P->counter, flex, P->coef));
  IGAFD_LAUNCHED(1);
  if (true_every > 0)
    IGAFD_TRY(igafd_stencil_launch(P, P->xs, P->r, P->bint, 1, 1, s, true_every, nullptr,
                                   flex ? P->z : nullptr));
  IGAFD_TRY(fd_apply(P, dt, P->r, P->z, s, done));
  IGAFD_CUDA(igafd_launch(dot_rz_kernel, G, B, 0, s, P->r, P->z, N, scal, P->partial, P->counter, 0, flex, 1, P->coef));
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(igafd_launch(update_p_kernel, G, B, 0, s, P->pv, P->z, N, scal, 1));
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

// The captured chunk: `chunk` iterations followed by a copy of the device
// scalars to pinned host memory; with timing, the stencil launches stamp
// their own start and end on the device clock (CUDA events recorded between
// the nodes of a captured graph give no elapsed times). Rebuilt when its
// parameters change; the un-instantiated graph is kept for batched solves.
static igafd_status loop_graph(igafd_patch *P, igafd_dtype dt, int flex, int true_every, int chunk,
                               int timing) {
  // everything that selects the captured kernels: the FD form and the stencil
  // pipeline too (set by the autotuner or explicitly between solves)
  const int op = dt == IGAFD_TF32 ? 0 : dt == IGAFD_BF16 ? 1 : 2;
  const int key[9] = {(int)dt, flex, true_every, chunk, 1 + timing, P->fd_fused,
                      P->fd_fused_op[op], P->stencil_stages, P->stencil_rows};
  if (P->loop_exec && memcmp(key, P->loop_key, sizeof(key)) == 0) return IGAFD_OK;
  if (P->loop_exec) {
    cudaGraphExecDestroy(P->loop_exec);
    P->loop_exec = nullptr;
  }
  if (P->loop_graph) {
    cudaGraphDestroy(P->loop_graph);
    P->loop_graph = nullptr;
  }
  cudaStream_t cs = P->cap_stream;
  const long long l0 = g_igafd_launches.load();
  IGAFD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  igafd_status st = IGAFD_OK;
  for (int c = 0; c < chunk && st == IGAFD_OK; ++c)
    st = enqueue_iteration(P, dt, flex, true_every, cs, timing != 0);
  if (st == IGAFD_OK && cudaMemcpyAsync(P->host_scal, P->scal, S_COUNT * sizeof(double),
                                        cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    st = IGAFD_ERR_CUDA;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  const long long nodes = g_igafd_launches.load() - l0;
  g_igafd_launches.fetch_sub(nodes);     // captured, not executed
  if (st != IGAFD_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != IGAFD_OK ? st : IGAFD_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&P->loop_exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    P->loop_exec = nullptr;
    cudaGetLastError();
    return IGAFD_ERR_CUDA;
  }
  P->loop_graph = g;
  P->loop_nodes = nodes;
  memcpy(P->loop_key, key, sizeof(key));
  return IGAFD_OK;
}

// Per-solve state of one problem (shared by the single and batched solves).
struct SolveState {
  igafd_pcg_opts o;
  int flex;
  double bb;
  int k;                 // iterations enqueued
  double rec_rr;         // recurrence (r, r) when the flag was raised
  igafd_status status;
  bool finished;
  bool timing;
  bool graphed;
  double *x;
  igafd_pcg_info inf;
};

// Set-up on patch-internal copies of b and x: r0 = b - A x0, z0 = P^{-1} r0,
// rho0 = (r0, z0), p0 = z0. Synchronises once (to read (b, b)).
static igafd_status solve_begin(igafd_patch *P, const igafd_pcg_opts *opts, const double *b,
                                double *x, cudaStream_t s, SolveState &S) {
  if (!P || !b || !x || b == x || !P->stencil) return IGAFD_ERR_ARG;
  igafd_pcg_opts o;
  if (opts) o = *opts; else igafd_pcg_default_opts(&o);
  if (!(o.tol >= 0.0) || o.max_iter < 0 || o.check_every < 1 || o.true_every < 0)
    return IGAFD_ERR_ARG;
  if (o.prec_dtype < IGAFD_FP64 || o.prec_dtype > IGAFD_ADI) return IGAFD_ERR_ARG;
  if (o.prec_dtype == IGAFD_ADI && !P->adi) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  S = SolveState{};
  S.timing = o.timing != 0;
  if (S.timing && o.check_every > 32) o.check_every = 32;
  S.o = o;
  S.flex = o.flexible ? 1 : 0;
  S.x = x;
  S.rec_rr = -1.0;
  S.status = IGAFD_ERR_NOT_CONVERGED;
  const long long N = P->N;
  const dim3 G(IGAFD_RED_BLOCKS), B(256);
  double *scal = P->scal;
  if (S.timing) {
    IGAFD_CUDA(cudaEventRecord(P->ev[IGAFD_NEV - 2], s));
    const unsigned long long init[3] = {~0ull, 0ull, 0ull};
    IGAFD_CUDA(cudaMemcpyAsync(P->tstat, init, sizeof(init), cudaMemcpyHostToDevice, s));
    IGAFD_CUDA(cudaStreamSynchronize(s));
  }
  IGAFD_CUDA(cudaMemsetAsync(P->err_flag, 0, sizeof(int), s));
  init_scalars_kernel<<<1, 32, 0, s>>>(scal, o.tol * o.tol, (double)o.max_iter);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaMemcpyAsync(P->bint, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  IGAFD_CUDA(igafd_launch(norm2_kernel, G, B, 0, s, P->bint, N, scal, S_BB, P->partial, P->counter));
  IGAFD_LAUNCHED(1);
  if (o.x0_given) {
    IGAFD_CUDA(cudaMemcpyAsync(P->xs, x, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    IGAFD_TRY(igafd_stencil_launch(P, P->xs, P->r, P->bint, 1, 0, s));   // r0 = b - A x0
  } else {
    IGAFD_CUDA(cudaMemsetAsync(P->xs, 0, N * sizeof(double), s));
    IGAFD_CUDA(cudaMemcpyAsync(P->r, P->bint, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  IGAFD_TRY(read_scalars(P, s));
  S.bb = P->host_scal[S_BB];
  if (!(S.bb > 0.0)) {
    // b == 0: x = 0 is the solution; non-finite b: breakdown
    S.status = S.bb == 0.0 ? IGAFD_OK : IGAFD_ERR_BREAKDOWN;
    if (S.bb == 0.0) IGAFD_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    S.finished = true;
    return IGAFD_OK;
  }
  IGAFD_TRY(fd_apply(P, o.prec_dtype, P->r, P->z, s, nullptr));
  IGAFD_CUDA(igafd_launch(dot_rz_kernel, G, B, 0, s, P->r, P->z, N, scal, P->partial, P->counter, 1, S.flex, 0, P->coef));
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaMemcpyAsync(P->pv, P->z, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  IGAFD_CUDA(cudaGetLastError());
  S.finished = o.max_iter == 0;
  S.graphed = loop_graph(P, o.prec_dtype, S.flex, o.true_every, o.check_every, S.timing ? 1 : 0) ==
              IGAFD_OK;
  return IGAFD_OK;
}

// A chunk of iterations without a graph (fallback), polled like the graph.
static igafd_status run_chunk_direct(igafd_patch *P, cudaStream_t s, SolveState &S) {
  const dim3 G(IGAFD_RED_BLOCKS), B(256);
  const long long N = P->N;
  double *scal = P->scal;
  cudaEvent_t *ev = P->ev;
  const int chunk = S.o.check_every;
  for (int c = 0; c < chunk; ++c) {
    if (S.timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c], s));
    IGAFD_TRY(igafd_stencil_launch(P, P->pv, P->q, nullptr, 1, 1, s));
    if (S.timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c + 1], s));
    IGAFD_CUDA(igafd_launch(update_xr_kernel, G, B, 0, s, P->xs, P->r, P->pv, P->q, P->z, N, scal, P->partial,
                                     P->counter, S.flex, P->coef));
    IGAFD_LAUNCHED(1);
    if (S.o.true_every > 0)
      IGAFD_TRY(igafd_stencil_launch(P, P->xs, P->r, P->bint, 1, 1, s, S.o.true_every, nullptr,
                                     S.flex ? P->z : nullptr));
    if (S.timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c + 2], s));
    IGAFD_TRY(fd_apply(P, S.o.prec_dtype, P->r, P->z, s, P->scal + S_DONE));
    if (S.timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c + 3], s));
    IGAFD_CUDA(igafd_launch(dot_rz_kernel, G, B, 0, s, P->r, P->z, N, scal, P->partial, P->counter, 0, S.flex, 1, P->coef));
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(igafd_launch(update_p_kernel, G, B, 0, s, P->pv, P->z, N, scal, 1));
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
  }
  IGAFD_TRY(read_scalars(P, s));
  if (S.timing) {
    for (int c = 0; c < chunk; ++c) {
      float a = 0.f, b2 = 0.f;
      cudaEventElapsedTime(&a, ev[4 * c], ev[4 * c + 1]);
      cudaEventElapsedTime(&b2, ev[4 * c + 2], ev[4 * c + 3]);
      S.inf.stencil_ms += a;
      S.inf.prec_ms += b2;
    }
  }
  return IGAFD_OK;
}

// After a chunk (its scalars are in P->host_scal): stopping decisions and,
// when the recurrence says converged, the true-residual confirmation.
static igafd_status solve_after_chunk(igafd_patch *P, cudaStream_t s, SolveState &S) {
  const dim3 G(IGAFD_RED_BLOCKS), B(256);
  const long long N = P->N;
  double *scal = P->scal;
  S.k += S.o.check_every;
  const double *h = P->host_scal;
  if (h[S_DONE] != 0.0) {
    S.rec_rr = h[S_RR];
    if (h[S_STATUS] != 0.0) {
      S.status = (igafd_status)(int)h[S_STATUS];
      S.finished = true;
      return IGAFD_OK;
    }
    IGAFD_TRY(igafd_stencil_launch(P, P->xs, P->r, P->bint, 1, 0, s, 0, nullptr,
                                   S.flex ? P->z : nullptr));
    IGAFD_TRY(read_scalars(P, s));
    if (h[S_TRUE_RR] <= S.o.tol * S.o.tol * S.bb) {
      S.status = IGAFD_OK;
      S.finished = true;
      return IGAFD_OK;
    }
    // not confirmed: continue from the true residual
    if ((int)h[S_ITER] >= S.o.max_iter) {
      S.finished = true;
      return IGAFD_OK;
    }
    set_scalar_kernel<<<1, 32, 0, s>>>(scal, S_DONE, 0.0);
    IGAFD_LAUNCHED(1);
    IGAFD_TRY(fd_apply(P, S.o.prec_dtype, P->r, P->z, s, nullptr));
    IGAFD_CUDA(igafd_launch(dot_rz_kernel, G, B, 0, s, P->r, P->z, N, scal, P->partial, P->counter, 0, S.flex, 0, P->coef));
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(igafd_launch(update_p_kernel, G, B, 0, s, P->pv, P->z, N, scal, 0));
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
    S.k = (int)h[S_ITER];
  }
  if (S.k >= S.o.max_iter) S.finished = true;
  return IGAFD_OK;
}

static igafd_status solve_end(igafd_patch *P, cudaStream_t s, SolveState &S) {
  igafd_pcg_info &inf = S.inf;
  if (!(S.bb > 0.0)) {
    inf.status = S.status;
    IGAFD_CUDA(cudaStreamSynchronize(s));
    return S.status;
  }
  IGAFD_TRY(read_scalars(P, s));
  inf.iterations = (int)P->host_scal[S_ITER];
  inf.relres = sqrt((S.rec_rr >= 0.0 && S.status == IGAFD_OK ? S.rec_rr : P->host_scal[S_RR]) / S.bb);
  if (P->host_scal[S_TRUE_RR] < 0.0 || S.status != IGAFD_OK) {
    // true residual of the returned iterate (into the scratch vector)
    IGAFD_TRY(igafd_stencil_launch(P, P->xs, P->xt, P->bint, 1, 0, s));
    IGAFD_TRY(read_scalars(P, s));
  }
  inf.true_relres = sqrt(P->host_scal[S_TRUE_RR] / S.bb);
  IGAFD_CUDA(cudaMemcpyAsync(S.x, P->xs, P->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int herr = 0;
  IGAFD_CUDA(cudaMemcpyAsync(&herr, P->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  if (herr != 0 && S.status == IGAFD_OK) S.status = (igafd_status)herr;
  inf.status = S.status;
  if (S.timing) {
    cudaEvent_t *ev = P->ev;
    IGAFD_CUDA(cudaEventRecord(ev[IGAFD_NEV - 1], s));
    IGAFD_CUDA(cudaEventSynchronize(ev[IGAFD_NEV - 1]));
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[IGAFD_NEV - 2], ev[IGAFD_NEV - 1]);
    inf.solve_ms = t;
    if (S.graphed) {   // in-loop stencil launches timed on the device clock
      unsigned long long h[3];
      IGAFD_CUDA(cudaMemcpy(h, P->tstat, sizeof(h), cudaMemcpyDeviceToHost));
      inf.stencil_ms = h[1] * 1e-6;
      inf.prec_ms = -1.0;   // FD applies are not individually timed inside the graph
    }
  }
  return S.status;
}

extern "C" igafd_status igafd_pcg_solve(igafd_patch *P, const igafd_pcg_opts *opts,
                                        const double *b, double *x, igafd_pcg_info *info,
                                        void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  SolveState S;
  IGAFD_TRY(solve_begin(P, opts, b, x, s, S));
  while (!S.finished) {
    if (S.graphed) {
      IGAFD_CUDA(cudaGraphLaunch(P->loop_exec, s));
      IGAFD_LAUNCHED(P->loop_nodes);
      IGAFD_CUDA(cudaStreamSynchronize(s));
    } else {
      IGAFD_TRY(run_chunk_direct(P, s, S));
    }
    IGAFD_TRY(solve_after_chunk(P, s, S));
  }
  const igafd_status st = solve_end(P, s, S);
  if (info) *info = S.inf;
  return st;
}

// ---- batched solve -----------------------------------------------------------
// Every problem keeps its own captured chunk graph; one parent graph holds
// them as independent child nodes, so a single graph launch advances all
// unfinished problems concurrently. Problems that have finished are dropped
// from the parent graph when at least half of its members are done.
static igafd_status build_parent(igafd_patch *const *ps, const std::vector<int> &active,
                                 cudaGraphExec_t *exec, long long *nodes) {
  cudaGraph_t parent = nullptr;
  IGAFD_CUDA(cudaGraphCreate(&parent, 0));
  long long n = 0;
  for (int i : active) {
    cudaGraphNode_t node;
    if (cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, ps[i]->loop_graph) != cudaSuccess) {
      cudaGraphDestroy(parent);
      cudaGetLastError();
      return IGAFD_ERR_CUDA;
    }
    n += ps[i]->loop_nodes;
  }
  cudaError_t e = cudaGraphInstantiate(exec, parent, 0);
  cudaGraphDestroy(parent);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IGAFD_ERR_CUDA;
  }
  *nodes = n;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_batch_pcg_solve(igafd_patch *const *patches, int count,
                                              const double *const *b, double *const *x,
                                              const igafd_pcg_opts *opts, igafd_pcg_info *infos,
                                              void *stream) {
  if (!patches || count < 1 || !b || !x) return IGAFD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  igafd_pcg_opts o;
  if (opts) o = *opts; else igafd_pcg_default_opts(&o);
  o.timing = 0;   // per-problem timing is not available inside the batch graph
  for (int i = 0; i < count; ++i) {
    if (!patches[i]) return IGAFD_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (patches[j] == patches[i]) return IGAFD_ERR_ARG;   // one problem per patch
    if (patches[i]->dev != patches[0]->dev) return IGAFD_ERR_ARG;
  }
  std::vector<SolveState> S(count);
  std::vector<int> active;
  for (int i = 0; i < count; ++i) {
    IGAFD_TRY(solve_begin(patches[i], &o, b[i], x[i], s, S[i]));
    if (!S[i].finished) {
      if (!S[i].graphed) return IGAFD_ERR_CUDA;
      active.push_back(i);
    }
  }
  cudaGraphExec_t exec = nullptr;
  long long nodes = 0;
  size_t built_for = 0;
  igafd_status st = IGAFD_OK;
  while (!active.empty() && st == IGAFD_OK) {
    if (!exec || active.size() * 2 <= built_for) {
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      st = build_parent(patches, active, &exec, &nodes);
      if (st != IGAFD_OK) break;
      built_for = active.size();
    }
    if (cudaGraphLaunch(exec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      st = IGAFD_ERR_CUDA;
      break;
    }
    IGAFD_LAUNCHED(nodes);
    std::vector<int> still;
    for (int i : active) {
      // problems already finished but still in the parent graph only ran no-op kernels
      st = solve_after_chunk(patches[i], s, S[i]);
      if (st != IGAFD_OK) break;
      if (!S[i].finished) still.push_back(i);
    }
    active.swap(still);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (st != IGAFD_OK) return st;
  igafd_status worst = IGAFD_OK;
  for (int i = 0; i < count; ++i) {
    const igafd_status e = solve_end(patches[i], s, S[i]);
    if (infos) infos[i] = S[i].inf;
    if (e != IGAFD_OK && worst == IGAFD_OK) worst = e;
  }
  return worst;
}

// ---- condition estimate from the CG-Lanczos relation (host arithmetic) ----
// Sturm count of the tridiagonal T (diagonal d, squared off-diagonal e2):
// the number of eigenvalues below x, from the pivots of T - x I = L D L^T.
static int sturm_count(const std::vector<double> &d, const std::vector<double> &e2, double x) {
  const int m = (int)d.size();
  int c = 0;
  double q = d[0] - x;
  for (int j = 0;; ++j) {
    if (fabs(q) < 1e-300) q = -1e-300;
    c += q < 0.0;
    if (j == m - 1) break;
    q = (d[j + 1] - x) - e2[j] / q;
  }
  return c;
}

static double tridiag_eig(const std::vector<double> &d, const std::vector<double> &e2, int idx,
                          double lo, double hi) {
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(hi - lo > 1e-15 * fmax(fabs(lo), fabs(hi)))) break;
    if (sturm_count(d, e2, mid) > idx) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

extern "C" igafd_status igafd_lanczos_extremes(const double *alpha, const double *beta, int m,
                                               double *lmin, double *lmax) {
  if (!alpha || m < 1 || (m > 1 && !beta) || !lmin || !lmax) return IGAFD_ERR_ARG;
  std::vector<double> d(m), e2(m > 1 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) {
    if (!(alpha[j] > 0.0) || !std::isfinite(alpha[j])) return IGAFD_ERR_ARG;
    if (j > 0 && (!(beta[j - 1] >= 0.0) || !std::isfinite(beta[j - 1]))) return IGAFD_ERR_ARG;
    d[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j < m - 1) e2[j] = beta[j] / (alpha[j] * alpha[j]);
  }
  double lo = 1e308, hi = -1e308;
  for (int j = 0; j < m; ++j) {
    const double r = (j > 0 ? sqrt(e2[j - 1]) : 0.0) + (j < m - 1 ? sqrt(e2[j]) : 0.0);
    lo = fmin(lo, d[j] - r);
    hi = fmax(hi, d[j] + r);
  }
  *lmin = tridiag_eig(d, e2, 0, lo, hi);
  *lmax = tridiag_eig(d, e2, m - 1, lo, hi);
  return IGAFD_OK;
}

extern "C" igafd_status igafd_pcg_condition_estimate(igafd_patch *P, int steps, double *kappa,
                                                     double *lmin, double *lmax) {
  if (!P || !kappa || !lmin || !lmax || !P->host_scal) return IGAFD_ERR_ARG;
  int m = (int)P->host_scal[S_ITER];
  if (steps > 0 && steps < m) m = steps;
  if (m > IGAFD_COEF_CAP) m = IGAFD_COEF_CAP;
  if (m < 1) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  std::vector<double> c(2 * (size_t)m), a(m), b(m);
  IGAFD_CUDA(cudaMemcpy(c.data(), P->coef, c.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int j = 0; j < m; ++j) { a[j] = c[2 * j]; b[j] = c[2 * j + 1]; }
  IGAFD_TRY(igafd_lanczos_extremes(a.data(), b.data(), m, lmin, lmax));
  *kappa = *lmax / *lmin;
  return IGAFD_OK;
}
