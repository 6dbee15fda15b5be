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
                                                        unsigned *counter, double tol2, int flexible) {
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
    scal[S_ITER] += 1.0;
    if (!isfinite(trr)) {
      scal[S_STATUS] = (double)IGAFD_ERR_BREAKDOWN;
      scal[S_DONE] = 1.0;
    } else if (trr <= tol2 * scal[S_BB]) {
      scal[S_DONE] = 1.0;   // converged by the recurrence; the host confirms
    }
  }
}

// (r, z) -> rho (init) or beta and rho (iteration).
__global__ void __launch_bounds__(256) dot_rz_kernel(const double *__restrict__ r,
                                                     const double *__restrict__ z, long long N,
                                                     double *scal, double *partial,
                                                     unsigned *counter, int init, int flexible,
                                                     int skip_done) {
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
    }
    scal[S_RHO] = t;
  }
}

// p = z + beta p
__global__ void __launch_bounds__(256) update_p_kernel(double *__restrict__ p,
                                                       const double *__restrict__ z, long long N,
                                                       const double *scal, int skip_done) {
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

__global__ void init_scalars_kernel(double *scal) {
  if (threadIdx.x == 0) {
    scal[S_DONE] = 0.0;
    scal[S_ITER] = 0.0;
    scal[S_STATUS] = 0.0;
    scal[S_BETA] = 0.0;
    scal[S_RZOLD] = 0.0;
    scal[S_TRUE_RR] = -1.0;
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
  if (!P || !x || !y || x == y) return IGAFD_ERR_ARG;
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

extern "C" igafd_status igafd_pcg_solve(igafd_patch *P, const igafd_pcg_opts *opts,
                                        const double *b, double *x, igafd_pcg_info *info,
                                        void *stream) {
  if (!P || !b || !x || b == x) return IGAFD_ERR_ARG;
  igafd_pcg_opts o;
  if (opts) o = *opts; else igafd_pcg_default_opts(&o);
  if (!(o.tol >= 0.0) || o.max_iter < 0 || o.check_every < 1 || o.true_every < 0)
    return IGAFD_ERR_ARG;
  if (o.prec_dtype < IGAFD_FP64 || o.prec_dtype > IGAFD_TF32) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = P->N;
  const dim3 G(IGAFD_RED_BLOCKS), B(256);
  double *scal = P->scal, *done = P->scal + S_DONE;
  const double tol2 = o.tol * o.tol;
  const int flex = o.flexible ? 1 : 0;
  igafd_pcg_info inf{};
  const bool timing = o.timing != 0;
  if (timing && o.check_every > 32) o.check_every = 32;
  cudaEvent_t *ev = P->ev;
  if (timing) IGAFD_CUDA(cudaEventRecord(ev[IGAFD_NEV - 2], s));

  init_scalars_kernel<<<1, 32, 0, s>>>(scal);
  IGAFD_LAUNCHED(1);
  norm2_kernel<<<G, B, 0, s>>>(b, N, scal, S_BB, P->partial, P->counter);
  IGAFD_LAUNCHED(1);
  // r0 = b - A x0
  if (o.x0_given) {
    IGAFD_TRY(igafd_stencil_launch(P, x, P->r, b, 1, 0, s));
  } else {
    IGAFD_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    IGAFD_CUDA(cudaMemcpyAsync(P->r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  IGAFD_TRY(read_scalars(P, s));
  const double bb = P->host_scal[S_BB];
  if (!(bb > 0.0)) {
    // b == 0 (or non-finite b): x = 0 is the solution when b == 0
    if (bb == 0.0) {
      IGAFD_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
      IGAFD_CUDA(cudaStreamSynchronize(s));
      inf.status = IGAFD_OK;
      if (info) *info = inf;
      return IGAFD_OK;
    }
    inf.status = IGAFD_ERR_BREAKDOWN;
    if (info) *info = inf;
    return IGAFD_ERR_BREAKDOWN;
  }
  // z0 = P^{-1} r0, rho0 = (r0, z0), p0 = z0
  IGAFD_TRY(fd_apply(P, o.prec_dtype, P->r, P->z, s, nullptr));
  dot_rz_kernel<<<G, B, 0, s>>>(P->r, P->z, N, scal, P->partial, P->counter, 1, flex, 0);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaMemcpyAsync(P->pv, P->z, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  IGAFD_CUDA(cudaGetLastError());

  int k = 0;               // iterations enqueued
  double rec_rr = -1.0;    // recurrence (r, r) when the flag was raised
  igafd_status status = IGAFD_ERR_NOT_CONVERGED;
  bool finished = false;
  while (!finished) {
    const int chunk = (o.max_iter - k) < o.check_every ? (o.max_iter - k) : o.check_every;
    for (int c = 0; c < chunk; ++c) {
      ++k;
      // q = A p, alpha = rho / (p, q)
      if (timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c], s));
      IGAFD_TRY(igafd_stencil_launch(P, P->pv, P->q, nullptr, 1, 1, s));
      if (timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c + 1], s));
      update_xr_kernel<<<G, B, 0, s>>>(x, P->r, P->pv, P->q, P->z, N, scal, P->partial,
                                       P->counter, tol2, flex);
  IGAFD_LAUNCHED(1);
      if (o.true_every > 0 && k % o.true_every == 0) {
        IGAFD_TRY(igafd_stencil_launch(P, x, P->r, b, 1, 1, s));
        ++inf.true_checks;
      }
      if (timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c + 2], s));
      IGAFD_TRY(fd_apply(P, o.prec_dtype, P->r, P->z, s, done));
      if (timing) IGAFD_CUDA(cudaEventRecord(ev[4 * c + 3], s));
      dot_rz_kernel<<<G, B, 0, s>>>(P->r, P->z, N, scal, P->partial, P->counter, 0, flex, 1);
  IGAFD_LAUNCHED(1);
      update_p_kernel<<<G, B, 0, s>>>(P->pv, P->z, N, scal, 1);
  IGAFD_LAUNCHED(1);
      IGAFD_CUDA(cudaGetLastError());
    }
    IGAFD_TRY(read_scalars(P, s));
    if (timing) {
      for (int c = 0; c < chunk; ++c) {
        float a = 0.f, b2 = 0.f;
        cudaEventElapsedTime(&a, ev[4 * c], ev[4 * c + 1]);
        cudaEventElapsedTime(&b2, ev[4 * c + 2], ev[4 * c + 3]);
        inf.stencil_ms += a;
        inf.prec_ms += b2;
      }
    }
    const double *h = P->host_scal;
    if (h[S_DONE] != 0.0) {
      rec_rr = h[S_RR];
      if (h[S_STATUS] != 0.0) {
        status = (igafd_status)(int)h[S_STATUS];
        finished = true;
        break;
      }
      // confirm with the true residual
      IGAFD_TRY(igafd_stencil_launch(P, x, P->r, b, 1, 0, s));
      IGAFD_TRY(read_scalars(P, s));
      if (h[S_TRUE_RR] <= tol2 * bb) {
        status = IGAFD_OK;
        finished = true;
        break;
      }
      // not confirmed: continue from the true residual
      if ((int)h[S_ITER] >= o.max_iter) { finished = true; break; }
      set_scalar_kernel<<<1, 32, 0, s>>>(scal, S_DONE, 0.0);
  IGAFD_LAUNCHED(1);
      IGAFD_TRY(fd_apply(P, o.prec_dtype, P->r, P->z, s, nullptr));
      dot_rz_kernel<<<G, B, 0, s>>>(P->r, P->z, N, scal, P->partial, P->counter, 0, flex, 0);
  IGAFD_LAUNCHED(1);
      update_p_kernel<<<G, B, 0, s>>>(P->pv, P->z, N, scal, 0);
  IGAFD_LAUNCHED(1);
      IGAFD_CUDA(cudaGetLastError());
      k = (int)h[S_ITER];
    }
    if (k >= o.max_iter) finished = true;
  }
  IGAFD_TRY(read_scalars(P, s));
  inf.iterations = (int)P->host_scal[S_ITER];
  inf.relres = sqrt((rec_rr >= 0.0 && status == IGAFD_OK ? rec_rr : P->host_scal[S_RR]) / bb);
  if (P->host_scal[S_TRUE_RR] < 0.0 || status != IGAFD_OK) {
    // final true residual of the returned iterate (into the scratch vector)
    IGAFD_TRY(igafd_stencil_launch(P, x, P->xt, b, 1, 0, s));
    IGAFD_TRY(read_scalars(P, s));
  }
  inf.true_relres = sqrt(P->host_scal[S_TRUE_RR] / bb);
  inf.status = status;
  if (timing) {
    IGAFD_CUDA(cudaEventRecord(ev[IGAFD_NEV - 1], s));
    IGAFD_CUDA(cudaEventSynchronize(ev[IGAFD_NEV - 1]));
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[IGAFD_NEV - 2], ev[IGAFD_NEV - 1]);
    inf.solve_ms = t;
  }
  if (info) *info = inf;
  return status;
}
