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

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace {

__device__ __forceinline__ bool last_block(unsigned int *counter, unsigned blocks) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == blocks - 1);
  }
  __syncthreads();
  return am_last;
}

__device__ double sum_partials(const double *part, int n, double *sh32) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += ((volatile const double *)part)[i];
  return block_sum(v, sh32);
}

// The vector kernels below are written per CTA vb of a grid of vg CTAs, so
// that a single problem's launch (vb = blockIdx.x, vg = gridDim.x) and a
// batched launch (one work item per (problem, vb)) reduce in the same order.

// x += alpha p, r -= alpha q; partials (r, r) and (r, z_old).
__device__ __forceinline__ void update_xr_cta(double *__restrict__ x, double *__restrict__ r,
                                              const double *__restrict__ p,
                                              const double *__restrict__ q,
                                              const double *__restrict__ z, long long N,
                                              double *scal, double *partial, unsigned *counter,
                                              int flexible, double *coef, long long vb,
                                              long long vg) {
  const double alpha = scal[S_ALPHA];
  double rr = 0.0, rz = 0.0;
  for (long long i = vb * (long long)blockDim.x + threadIdx.x; i < N; i += vg * blockDim.x) {
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
    partial[vb] = a;
    partial[vg + vb] = b;
  }
  if (!last_block(counter, (unsigned)vg)) return;
  double trr = sum_partials(partial, (int)vg, sh32);
  double trz = flexible ? sum_partials(partial + vg, (int)vg, sh32) : 0.0;
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
      scal[S_DONE] = 1.0;   // converged by the recurrence; the true residual confirms
      scal[S_REC_RR] = trr;
    } else if (scal[S_ITER] >= scal[S_MAXIT]) {
      scal[S_STATUS] = (double)IGAFD_ERR_NOT_CONVERGED;
      scal[S_DONE] = 1.0;   // iteration cap
    }
  }
}

// (r, z) -> rho (init) or beta and rho (iteration).
__device__ __forceinline__ void dot_rz_cta(const double *__restrict__ r,
                                           const double *__restrict__ z, long long N, double *scal,
                                           double *partial, unsigned *counter, int init,
                                           int flexible, double *coef, long long vb, long long vg) {
  double rz = 0.0;
  for (long long i = vb * (long long)blockDim.x + threadIdx.x; i < N; i += vg * blockDim.x)
    rz = fma(r[i], z[i], rz);
  __shared__ double sh32[32];
  double a = block_sum(rz, sh32);
  if (threadIdx.x == 0) partial[vb] = a;
  if (!last_block(counter, (unsigned)vg)) return;
  double t = sum_partials(partial, (int)vg, sh32);
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
__device__ __forceinline__ void update_p_cta(double *__restrict__ p, const double *__restrict__ z,
                                             long long N, const double *scal, long long vb,
                                             long long vg) {
  const double beta = scal[S_BETA];
  for (long long i = vb * (long long)blockDim.x + threadIdx.x; i < N; i += vg * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

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
  update_xr_cta(x, r, p, q, z, N, scal, partial, counter, flexible, coef, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) dot_rz_kernel(const double *__restrict__ r,
                                                     const double *__restrict__ z, long long N,
                                                     double *scal, double *partial,
                                                     unsigned *counter, int init, int flexible,
                                                     int skip_done, double *coef) {
  pdl_wait();
  pdl_trigger();
  if (skip_done && scal[S_DONE] != 0.0) return;
  dot_rz_cta(r, z, N, scal, partial, counter, init, flexible, coef, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) update_p_kernel(double *__restrict__ p,
                                                       const double *__restrict__ z, long long N,
                                                       const double *scal, int skip_done) {
  pdl_wait();
  pdl_trigger();
  if (skip_done && scal[S_DONE] != 0.0) return;
  update_p_cta(p, z, N, scal, blockIdx.x, gridDim.x);
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
  if (!last_block(counter, gridDim.x)) return;
  double t = sum_partials(partial, gridDim.x, sh32);
  if (threadIdx.x == 0) {
    *counter = 0u;
    scal[slot] = t;
  }
}

// ---- batched solve: kernels over many problems --------------------------------
struct VecArgs {             // one problem's PCG vectors and reduction state
  double *x, *r, *p, *q, *z;
  double *scal, *partial, *coef;
  unsigned *counter;
  long long N;
  int flexible;
};

// One launch runs a PCG vector step of every listed (unfinished) problem:
// work item (listed problem k, CTA v of its own grid), items taken in a fixed
// stride by a persistent grid; act[k] is the problem, act_start[k] ..
// act_start[k + 1] its items (the pass's compaction kernel writes the list).
// op 0: update_xr, 1: dot_rz of the iteration, 2: update_p.
constexpr int kVecCache = 128;
__global__ void __launch_bounds__(256) vec_batch_kernel(const VecArgs *args, const int *act,
                                                        const long long *act_start,
                                                        const int *act_count, int op) {
  __shared__ long long s_start[kVecCache + 1];
  __shared__ int s_act[kVecCache];
  __shared__ VecArgs s_a;
  const int n = *act_count;
  const bool cached = n <= kVecCache;
  if (cached) {
    for (int k = threadIdx.x; k <= n; k += blockDim.x) s_start[k] = act_start[k];
    for (int k = threadIdx.x; k < n; k += blockDim.x) s_act[k] = act[k];
  }
  __syncthreads();
  const long long *st = cached ? s_start : act_start;
  const int *ax = cached ? s_act : act;
  const long long total = n > 0 ? st[n] : 0;
  int cur = -1;                      // listed problem whose arguments s_a holds
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    int lo = 0, hi = n - 1;          // every thread searches the (shared) list
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (st[mid] <= it) lo = mid; else hi = mid - 1;
    }
    if (lo != cur) {
      __syncthreads();
      if (threadIdx.x < 32) {
        const unsigned *src = reinterpret_cast<const unsigned *>(&args[ax[lo]]);
        unsigned *dst = reinterpret_cast<unsigned *>(&s_a);
        for (int w = threadIdx.x; w < (int)(sizeof(VecArgs) / 4); w += 32) dst[w] = src[w];
      }
      __syncthreads();
      cur = lo;
    }
    const VecArgs &a = s_a;
    const long long vb = it - st[lo], vg = st[lo + 1] - st[lo];
    if (a.scal[S_DONE] != 0.0) continue;   // uniform over the CTA
    if (op == 0)
      update_xr_cta(a.x, a.r, a.p, a.q, a.z, a.N, a.scal, a.partial, a.counter, a.flexible, a.coef,
                    vb, vg);
    else if (op == 1)
      dot_rz_cta(a.r, a.z, a.N, a.scal, a.partial, a.counter, 0, a.flexible, a.coef, vb, vg);
    else
      update_p_cta(a.p, a.z, a.N, a.scal, vb, vg);
  }
}

// The lists of one stencil class for a pass (device pointers).
struct ClassTab {
  int nmem;
  const int *prob;                  // problem of each member (the class's order)
  const long long *vg[3];           // its CTAs (work items) per stencil mode
  int *act_idx;                     // out: members of the unfinished problems, in order
  long long *act_start[3];          // out: their item prefix per mode
  int *act_count;
};

struct FusedTab {
  int nmem;
  const int *prob;                  // problem of each fused member
  const int *blocks[3];             // its CTAs per fused kernel kind
  int *act;                         // out: the members of the unfinished problems
  int *act_start[3];                // out: their CTA prefix per kind
  int *act_count;
  unsigned *queue;                  // out: the kinds' work-queue counters, zeroed
};

struct VecTab {
  int n;
  const long long *vg;              // CTAs of the vector kernels per problem
  int *act;                         // out: unfinished problems
  long long *act_start;             // out: their item prefix
  int *act_count;
};

// Device-clock record of one pass of the batched loop.
struct PassLog {
  unsigned long long t0, t1;        // globaltimer (ns) at the pass's start and end
  int active;                       // unfinished problems at its start
  int pad;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Start of a pass: the unfinished problems of every stencil class and of the
// vector kernels, with their work-item prefixes (one thread per list).
__global__ void batch_compact_kernel(const ClassTab *tabs, int nclass, VecTab vt, FusedTab ft,
                                     double *const *scal, PassLog *log, const unsigned *passes,
                                     unsigned log_cap) {
  const int t = threadIdx.x;
  const unsigned long long t0 = global_ns();
  if (t < nclass) {
    const ClassTab c = tabs[t];
    int k = 0;
    long long acc[3] = {0, 0, 0};
    for (int m = 0; m < c.nmem; ++m) {
      if (scal[c.prob[m]][S_FIN] != 0.0) continue;
      c.act_idx[k] = m;
      for (int sel = 0; sel < 3; ++sel) {
        c.act_start[sel][k] = acc[sel];
        acc[sel] += c.vg[sel][m];
      }
      ++k;
    }
    for (int sel = 0; sel < 3; ++sel) c.act_start[sel][k] = acc[sel];
    *c.act_count = k;
  } else if (t == nclass) {
    int k = 0;
    long long acc = 0;
    for (int i = 0; i < vt.n; ++i) {
      if (scal[i][S_FIN] != 0.0) continue;
      vt.act[k] = i;
      vt.act_start[k] = acc;
      acc += vt.vg[i];
      ++k;
    }
    vt.act_start[k] = acc;
    *vt.act_count = k;
    const unsigned n = *passes;
    if (n < log_cap) {
      log[n].t0 = t0;
      log[n].active = k;
    }
  } else if (t == nclass + 1 && ft.nmem > 0) {
    int k = 0, acc[3] = {0, 0, 0};
    for (int m = 0; m < ft.nmem; ++m) {
      if (scal[ft.prob[m]][S_FIN] != 0.0) continue;
      ft.act[k] = m;
      for (int kind = 0; kind < 3; ++kind) {
        ft.act_start[kind][k] = acc[kind];
        acc[kind] += ft.blocks[kind][m];
      }
      ++k;
    }
    for (int kind = 0; kind < 3; ++kind) {
      ft.act_start[kind][k] = acc[kind];
      ft.queue[kind] = 0u;
    }
    *ft.act_count = k;
  }
}

// After the convergence confirmation (true residual computed for every
// problem the recurrence called converged): confirmed -> finished; not
// confirmed at the iteration cap -> finished, not converged; otherwise the
// iteration continues from the recomputed residual (done flag cleared, as
// the single solve's restart does). Problems stopped by breakdown or the cap
// are finished.
__global__ void batch_decide_kernel(double *const *scal, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  double *sc = scal[i];
  if (sc[S_FIN] != 0.0 || sc[S_DONE] == 0.0) return;
  if (sc[S_STATUS] != 0.0) {
    sc[S_FIN] = 1.0;
  } else if (sc[S_TRUE_RR] <= sc[S_TOL2] * sc[S_BB]) {
    sc[S_FIN] = 1.0;
  } else if (sc[S_ITER] >= sc[S_MAXIT]) {
    sc[S_STATUS] = (double)IGAFD_ERR_NOT_CONVERGED;
    sc[S_FIN] = 1.0;
  } else {
    sc[S_DONE] = 0.0;
  }
}

// Loop condition of a group's loop: another pass while any member is
// unfinished, bounded by `guard` passes in the solve (every problem finishes
// within its iteration cap plus its confirmation restarts) and by `chunk`
// passes per launch of the loop's graph (0: no bound); *more (host-mapped)
// tells the host whether the group needs another launch.
__global__ void batch_cond_kernel(cudaGraphConditionalHandle h, double *const *scal, int nprob,
                                  unsigned *passes, unsigned *lpasses, unsigned guard,
                                  unsigned chunk, PassLog *log, unsigned log_cap,
                                  volatile int *more_host) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool more = false;
  for (int i = 0; i < nprob && !more; ++i) more = scal[i][S_FIN] == 0.0;
  if (*passes < log_cap) log[*passes].t1 = global_ns();
  const unsigned n = ++*passes, ln = ++*lpasses;
  const bool again = more && n < guard;
  cudaGraphSetConditional(h, (again && (chunk == 0 || ln < chunk)) ? 1u : 0u);
  if (!(again && (chunk == 0 || ln < chunk))) *more_host = again ? 1 : 0;
}

// Start of a launch of a group's loop graph: its per-launch pass count.
__global__ void batch_reset_kernel(unsigned *lpasses) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *lpasses = 0u;
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
    scal[S_FIN] = 0.0;
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
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // a full-space patch has no preconditioner
  if (!P || !r || !z || r == z) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  return fd_apply(P, dt, r, z, (cudaStream_t)stream, nullptr);
}

extern "C" igafd_status igafd_apply_A(igafd_patch *P, const double *x, double *y, void *stream) {
  if (!P || !x || !y || x == y || !P->stencil) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  return igafd_stencil_launch(P, x, y, nullptr, 0, 0, (cudaStream_t)stream);
}

// CTAs of the PCG vector kernels: about 1024 elements per CTA (four per
// thread), at most IGAFD_RED_BLOCKS (the partial-sum slots).
int igafd_red_blocks(long long N) {
  const long long b = (N + 1023) / 1024;
  return (int)(b < 1 ? 1 : b > IGAFD_RED_BLOCKS ? IGAFD_RED_BLOCKS : b);
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
thread_local bool g_igafd_plain_launch = false;

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
  const dim3 G(igafd_red_blocks(P->N)), B(256);
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
  const int key[13] = {(int)dt, flex, true_every, chunk, 1 + timing, P->fd_fused,
                       P->fd_fused_op[op], P->stencil_stages, P->stencil_rows, P->fd_tile[op][0],
                       P->fd_tile[op][1], P->fd_tile[op][2], P->fd_tile[op][3]};
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

// Set-up on patch-internal copies of b and x, first part (no synchronisation):
// scalars, b and x copied in, (b, b) and r0 = b - A x0 enqueued.
static igafd_status solve_begin_enqueue(igafd_patch *P, const igafd_pcg_opts *opts, const double *b,
                                        double *x, cudaStream_t s, SolveState &S) {
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // a full-space patch has no preconditioner
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
  const dim3 G(igafd_red_blocks(P->N)), B(256);
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
  return IGAFD_OK;
}

// Second part, with (b, b) in P->host_scal: z0 = P^{-1} r0, rho0 = (r0, z0),
// p0 = z0, and (graph) the captured iteration chunk of the single solve.
static igafd_status solve_begin_finish(igafd_patch *P, cudaStream_t s, SolveState &S, bool graph) {
  const igafd_pcg_opts &o = S.o;
  const long long N = P->N;
  const dim3 G(igafd_red_blocks(P->N)), B(256);
  double *scal = P->scal;
  double *x = S.x;
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
  if (graph)
    S.graphed = loop_graph(P, o.prec_dtype, S.flex, o.true_every, o.check_every,
                           S.timing ? 1 : 0) == IGAFD_OK;
  return IGAFD_OK;
}

// r0 = b - A x0, z0 = P^{-1} r0, rho0 = (r0, z0), p0 = z0. Synchronises once
// (to read (b, b)).
static igafd_status solve_begin(igafd_patch *P, const igafd_pcg_opts *opts, const double *b,
                                double *x, cudaStream_t s, SolveState &S) {
  IGAFD_TRY(solve_begin_enqueue(P, opts, b, x, s, S));
  IGAFD_TRY(read_scalars(P, s));
  return solve_begin_finish(P, s, S, true);
}

// A chunk of iterations without a graph (fallback), polled like the graph.
static igafd_status run_chunk_direct(igafd_patch *P, cudaStream_t s, SolveState &S) {
  const dim3 G(igafd_red_blocks(P->N)), B(256);
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
  const dim3 G(igafd_red_blocks(P->N)), B(256);
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
// Many problems advance on the device, in groups of like size. A group's loop
// is a CUDA graph holding a conditional while-node whose body is one pass: a
// PCG iteration of every unfinished member, as a few launches over all of
// them -- a compaction that lists the unfinished members, the stencil q = A p
// (one launch per (dim, p, ring stages, rows) class: persistent and
// queue-fed in a group of several problems, the single solve's grid in a
// group of one), x/r update, periodic true residual, convergence
// confirmation and its decision, the FD (one launch per fused kind for
// problems on the generic tensor-core FD, the problem's own FD launches
// otherwise), (r, z) and p update -- and a kernel that keeps the loop going
// while any member is unfinished. The groups' graphs run concurrently, each
// on its own stream. Every problem's work items are CTAs of its own
// single-problem grids, so the iterates are bitwise those of
// igafd_pcg_solve. The host synchronises once before the loops (to read
// every (b, b)) and once after them, and in between only polls completion
// events when a loop's launch is bounded to a number of passes.

struct BatchClass {             // problems whose stencil shares (dim, p, ring stages, rows)
  int dim, p, stages, rows;
  std::vector<int> members;     // largest work item first (shorter tails of the queue)
  void *args[3];                // StencilArgs per member, for sel 0, 1, 2 (device)
  int *act_idx;                 // the pass's list of unfinished members (device)
  long long *act_start[3];      // and their item prefix per sel (device)
  long long items[3];           // work items of all members per sel
  int *act_count;
  unsigned long long *queue;    // the class's work-queue counter (device)
  cudaStream_t side;            // capture stream of its branch (classes run concurrently)
  cudaEvent_t done;
};

// One group of a batch: problems that advance together, one pass (an
// iteration of each unfinished member) per turn of the group's own
// device-driven loop.
struct BatchGroup {
  int count, dev, num_sms;
  igafd_pcg_opts o;
  int flex;
  std::vector<igafd_patch *> ps;
  std::vector<BatchClass> classes;
  std::vector<int> other_fd;    // problems whose FD is launched on its own
  int nfused;
  void *fused_args[3];          // FusedArgs per fused problem and kind (device)
  int fused_total[3];           // CTAs per kind over all fused problems
  FusedTab ftab;                // the fused problems' list tables (device)
  size_t fused_smem;
  VecArgs *vec_args;            // per problem (device)
  int *vec_act;                 // the pass's list of unfinished problems (device)
  long long *vec_act_start;
  int *vec_act_count;
  long long vec_total;          // items of the vector kernels over all problems
  ClassTab *tabs;               // the classes' list tables (device)
  VecTab vtab;
  double **scal_ptrs;           // per problem (device)
  unsigned *passes;             // loop passes in the solve (device)
  unsigned *lpasses;            // loop passes in the current launch of the graph (device)
  unsigned chunk;               // passes per launch (0: the whole solve in one launch)
  int *more_host;               // pinned, mapped: the group needs another launch
  int *more_dev;                // its device address
  PassLog *pass_log;            // one record per pass of the last solve (device)
  unsigned guard;               // pass bound of the loop
  unsigned log_cap;             // records in pass_log (the first passes)
  cudaEvent_t fork;             // start of a forked stencil phase
  std::vector<void *> allocs;
  long long body_launches;      // launches of one pass (captured body)
  bool persistent;              // stencil and FD as persistent work-queue launches
  cudaGraph_t graph;            // the group's loop: reset, then while (unfinished) { pass }
  cudaGraphExec_t exec;
  cudaStream_t stream;          // the loop's stream (groups run concurrently)
  cudaEvent_t done;
};

// The batch: its groups' loops run concurrently, each its own graph launched
// on its own stream (a group whose problems need few iterations does not wait
// for the others).
struct igafd_batch {
  int count, dev, num_sms;
  igafd_pcg_opts o;
  std::vector<igafd_patch *> ps;
  std::vector<BatchGroup *> groups;
  std::vector<int> group_of;    // group of each problem
  cudaStream_t cap;
  cudaEvent_t fork;             // the caller's stream, before the loops
};

template <typename T>
static igafd_status batch_upload(BatchGroup *B, const std::vector<T> &v, T **out) {
  void *p = nullptr;
  if (cudaMalloc(&p, (v.empty() ? 1 : v.size()) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return IGAFD_ERR_OOM;
  }
  B->allocs.push_back(p);
  if (!v.empty()) IGAFD_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = (T *)p;
  return IGAFD_OK;
}

// One PCG iteration of every problem (the while-node's body), enqueued on s.
static igafd_status batch_body(BatchGroup *B, cudaStream_t s, cudaGraphConditionalHandle h) {
  const int nvb = B->num_sms * 8;
  auto vec = [&](int op) -> igafd_status {
    const long long want = B->vec_total < nvb ? B->vec_total : nvb;
    vec_batch_kernel<<<(unsigned)(want > 0 ? want : 1), 256, 0, s>>>(
        B->vec_args, B->vec_act, B->vec_act_start, B->vec_act_count, op);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
    return IGAFD_OK;
  };
  // the classes' launches are independent: each on its own branch of the
  // graph (forked from and joined back to s), so their queues drain together
  auto stencil = [&](int sel) -> igafd_status {
    IGAFD_CUDA(cudaEventRecord(B->fork, s));
    for (size_t i = 0; i < B->classes.size(); ++i) {
      BatchClass &c = B->classes[i];
      cudaStream_t cs = i == 0 ? s : c.side;
      if (i > 0) IGAFD_CUDA(cudaStreamWaitEvent(cs, B->fork, 0));
      IGAFD_TRY(igafd_stencil_batch_launch(c.dim, c.p, c.stages, c.rows, sel, c.args[sel], c.act_idx,
                                           c.act_start[sel], c.act_count, c.queue,
                                           B->persistent ? 0 : c.items[sel], B->num_sms, cs));
      if (i > 0) IGAFD_CUDA(cudaEventRecord(c.done, cs));
    }
    for (size_t i = 1; i < B->classes.size(); ++i)
      IGAFD_CUDA(cudaStreamWaitEvent(s, B->classes[i].done, 0));
    return IGAFD_OK;
  };
  const int ct = ((int)B->classes.size() + 2 + 31) / 32 * 32;   // a thread per list
  batch_compact_kernel<<<1, ct, 0, s>>>(B->tabs, (int)B->classes.size(), B->vtab, B->ftab,
                                        B->scal_ptrs, B->pass_log, B->passes, B->log_cap);
  IGAFD_LAUNCHED(1);                                        // the pass's unfinished problems
  IGAFD_TRY(stencil(0));                                    // q = A p, alpha
  IGAFD_TRY(vec(0));                                        // x, r, (r, r), stopping test
  if (B->o.true_every > 0) IGAFD_TRY(stencil(1));           // periodic true residual
  IGAFD_TRY(stencil(2));                                    // confirm a recurrence convergence
  batch_decide_kernel<<<(B->count + 127) / 128, 128, 0, s>>>(B->scal_ptrs, B->count);
  IGAFD_LAUNCHED(1);
  for (int k = 0; k < 3; ++k)                               // z = P^{-1} r (fused FD)
    IGAFD_TRY(igafd_fd_fused_batch_launch(B->o.prec_dtype, k, B->fused_args[k], B->ftab.act,
                                          B->ftab.act_start[k], B->ftab.act_count,
                                          B->persistent ? B->ftab.queue + k : nullptr,
                                          B->fused_total[k], B->fused_smem, B->num_sms, s));
  for (int i : B->other_fd)                                 // z = P^{-1} r (own launches)
    IGAFD_TRY(fd_apply(B->ps[i], B->o.prec_dtype, B->ps[i]->r, B->ps[i]->z, s,
                       B->ps[i]->scal + S_DONE));
  IGAFD_TRY(vec(1));                                        // (r, z), beta
  IGAFD_TRY(vec(2));                                        // p = z + beta p
  batch_cond_kernel<<<1, 32, 0, s>>>(h, B->scal_ptrs, B->count, B->passes, B->lpasses, B->guard,
                                     B->chunk, B->pass_log, B->log_cap, B->more_dev);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

static void group_destroy(BatchGroup *B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->stream) cudaStreamDestroy(B->stream);
  if (B->done) cudaEventDestroy(B->done);
  if (B->more_host) cudaFreeHost(B->more_host);
  for (BatchClass &c : B->classes) {
    if (c.side) cudaStreamDestroy(c.side);
    if (c.done) cudaEventDestroy(c.done);
  }
  if (B->fork) cudaEventDestroy(B->fork);
  for (void *p : B->allocs) cudaFree(p);
  delete B;
}

extern "C" void igafd_batch_destroy(igafd_batch *B) {
  if (!B) return;
  cudaSetDevice(B->dev);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->fork) cudaEventDestroy(B->fork);
  for (BatchGroup *g : B->groups) group_destroy(g);
  delete B;
}

// A group's device tables (options already checked; o.check_every = 1).
static igafd_status group_create(igafd_patch *const *patches, int count, const igafd_pcg_opts &o,
                                 BatchGroup **out) {
  *out = nullptr;
  BatchGroup *B = new BatchGroup{};
  B->count = count;
  B->dev = patches[0]->dev;
  B->num_sms = patches[0]->num_sms;
  B->o = o;
  B->flex = o.flexible ? 1 : 0;
  B->ps.assign(patches, patches + count);
  // a group of one problem launches the grids of its single solve (a CTA per
  // item): CTAs then end after one item, so the concurrent groups' kernels
  // interleave on the SMs instead of waiting for persistent CTAs to drain
  B->persistent = count > 1;
  igafd_status st = IGAFD_OK;
  auto fail = [&](igafd_status e) {
    group_destroy(B);
    return e;
  };
  // stencil classes and their work items
  const size_t sab = igafd_stencil_args_bytes();
  for (int i = 0; i < count; ++i) {
    igafd_patch *P = B->ps[i];
    const int rows = P->dim == 3 && P->stencil_rows == 2 ? 2 : 1;
    const int stages = igafd_stencil_batch_stages(P);
    BatchClass *c = nullptr;
    for (BatchClass &q : B->classes)
      if (q.dim == P->dim && q.p == P->p && q.stages == stages && q.rows == rows) c = &q;
    if (!c) {
      B->classes.push_back(BatchClass{});
      c = &B->classes.back();
      c->dim = P->dim; c->p = P->p; c->stages = stages; c->rows = rows;
    }
    c->members.push_back(i);
  }
  std::vector<unsigned char> tmp_args(sab);
  std::vector<ClassTab> ctabs;
  for (BatchClass &c : B->classes) {
    // largest item (tiles per CTA of the problem's own grid) first
    std::vector<std::pair<double, int>> order;
    for (int i : c.members) {
      long long vg = 1;
      if ((st = igafd_stencil_batch_args(B->ps[i], 0, B->flex, o.true_every, tmp_args.data(), &vg)) !=
          IGAFD_OK)
        return fail(st);
      const double tiles = (double)((B->ps[i]->N + 255) / 256);
      order.push_back({-tiles / (double)(vg > 0 ? vg : 1), i});
    }
    std::stable_sort(order.begin(), order.end());
    for (size_t m = 0; m < order.size(); ++m) c.members[m] = order[m].second;
    std::vector<unsigned long long> q0(1, 0);
    if ((st = batch_upload(B, q0, &c.queue)) != IGAFD_OK) return fail(st);
    if (cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess)
      return fail(IGAFD_ERR_CUDA);
    ClassTab tab{};
    tab.nmem = (int)c.members.size();
    for (int sel = 0; sel < 3; ++sel) {
      std::vector<unsigned char> args(sab * c.members.size());
      std::vector<long long> vgs(c.members.size(), 0);
      for (size_t m = 0; m < c.members.size(); ++m) {
        st = igafd_stencil_batch_args(B->ps[c.members[m]], sel, B->flex, o.true_every,
                                      args.data() + m * sab, &vgs[m]);
        if (st != IGAFD_OK) return fail(st);
      }
      unsigned char *ad = nullptr;
      if ((st = batch_upload(B, args, &ad)) != IGAFD_OK) return fail(st);
      c.args[sel] = ad;
      c.items[sel] = 0;
      for (long long v : vgs) c.items[sel] += v;
      long long *vgd = nullptr;
      if ((st = batch_upload(B, vgs, &vgd)) != IGAFD_OK) return fail(st);
      tab.vg[sel] = vgd;
      std::vector<long long> zero(c.members.size() + 1, 0);
      if ((st = batch_upload(B, zero, &c.act_start[sel])) != IGAFD_OK) return fail(st);
      tab.act_start[sel] = c.act_start[sel];
    }
    std::vector<int> prob(c.members.begin(), c.members.end()), zi(c.members.size(), 0), z1(1, 0);
    int *pd = nullptr;
    if ((st = batch_upload(B, prob, &pd)) != IGAFD_OK) return fail(st);
    tab.prob = pd;
    if ((st = batch_upload(B, zi, &c.act_idx)) != IGAFD_OK) return fail(st);
    if ((st = batch_upload(B, z1, &c.act_count)) != IGAFD_OK) return fail(st);
    tab.act_idx = c.act_idx;
    tab.act_count = c.act_count;
    ctabs.push_back(tab);
  }
  if ((st = batch_upload(B, ctabs, &B->tabs)) != IGAFD_OK) return fail(st);
  // FD: problems on the generic fused tensor-core kernels run batched
  const size_t fab = igafd_fd_fused_args_bytes();
  std::vector<unsigned char> fargs[3];
  std::vector<int> fblocks[3], fprob;
  B->nfused = 0;
  B->fused_smem = 0;
  struct FusedMember {
    int i;
    std::vector<unsigned char> a3;
    int blocks[3];
    size_t smem;
  };
  std::vector<FusedMember> fm;
  for (int i = 0; i < count; ++i) {
    igafd_patch *P = B->ps[i];
    if (!igafd_fd_tc_fused_generic(P, o.prec_dtype)) {
      B->other_fd.push_back(i);
      continue;
    }
    FusedMember m{i, std::vector<unsigned char>(3 * fab), {0, 0, 0}, 0};
    if ((st = igafd_fd_fused_batch_args(P, o.prec_dtype, m.a3.data(), m.blocks, &m.smem)) !=
        IGAFD_OK)
      return fail(st);
    fm.push_back(std::move(m));
  }
  // longest CTAs first (their K, which sizes the shared memory), so that the
  // queue's last items are short
  std::stable_sort(fm.begin(), fm.end(), [&](const FusedMember &a, const FusedMember &b) {
    if (a.smem != b.smem) return a.smem > b.smem;
    return B->ps[a.i]->N > B->ps[b.i]->N;
  });
  for (const FusedMember &m : fm) {
    for (int k = 0; k < 3; ++k) {
      fargs[k].insert(fargs[k].end(), m.a3.begin() + k * fab, m.a3.begin() + (k + 1) * fab);
      fblocks[k].push_back(m.blocks[k]);
    }
    fprob.push_back(m.i);
    if (m.smem > B->fused_smem) B->fused_smem = m.smem;
    ++B->nfused;
  }
  B->ftab = FusedTab{};
  B->ftab.nmem = B->nfused;
  {
    std::vector<int> zi(B->nfused + 1, 0), z1(1, 0);
    int *pd = nullptr;
    if ((st = batch_upload(B, fprob, &pd)) != IGAFD_OK) return fail(st);
    B->ftab.prob = pd;
    if ((st = batch_upload(B, zi, &B->ftab.act)) != IGAFD_OK) return fail(st);
    if ((st = batch_upload(B, z1, &B->ftab.act_count)) != IGAFD_OK) return fail(st);
    std::vector<unsigned> zq(3, 0u);
    if ((st = batch_upload(B, zq, &B->ftab.queue)) != IGAFD_OK) return fail(st);
    for (int k = 0; k < 3; ++k) {
      unsigned char *ad = nullptr;
      if ((st = batch_upload(B, fargs[k], &ad)) != IGAFD_OK) return fail(st);
      B->fused_args[k] = ad;
      int *bd = nullptr;
      if ((st = batch_upload(B, fblocks[k], &bd)) != IGAFD_OK) return fail(st);
      B->ftab.blocks[k] = bd;
      if ((st = batch_upload(B, zi, &B->ftab.act_start[k])) != IGAFD_OK) return fail(st);
      B->fused_total[k] = 0;
      for (int b : fblocks[k]) B->fused_total[k] += b;
    }
  }
  // vector kernels, scalars, queue, pass counter
  std::vector<VecArgs> va(count);
  std::vector<long long> vgv(count, 0), vzero(count + 1, 0);
  std::vector<int> izero(count, 0), i1(1, 0);
  std::vector<double *> sp(count);
  B->vec_total = 0;
  for (int i = 0; i < count; ++i) {
    igafd_patch *P = B->ps[i];
    va[i] = VecArgs{P->xs, P->r, P->pv, P->q, P->z, P->scal, P->partial, P->coef, P->counter,
                    P->N, B->flex};
    vgv[i] = igafd_red_blocks(P->N);
    B->vec_total += vgv[i];
    sp[i] = P->scal;
  }
  if ((st = batch_upload(B, va, &B->vec_args)) != IGAFD_OK) return fail(st);
  long long *vgd = nullptr;
  if ((st = batch_upload(B, vgv, &vgd)) != IGAFD_OK) return fail(st);
  if ((st = batch_upload(B, izero, &B->vec_act)) != IGAFD_OK) return fail(st);
  if ((st = batch_upload(B, vzero, &B->vec_act_start)) != IGAFD_OK) return fail(st);
  if ((st = batch_upload(B, i1, &B->vec_act_count)) != IGAFD_OK) return fail(st);
  B->vtab = VecTab{count, vgd, B->vec_act, B->vec_act_start, B->vec_act_count};
  if ((st = batch_upload(B, sp, &B->scal_ptrs)) != IGAFD_OK) return fail(st);
  if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(IGAFD_ERR_CUDA);
  std::vector<unsigned> p1(1, 0);
  if ((st = batch_upload(B, p1, &B->passes)) != IGAFD_OK) return fail(st);
  if ((st = batch_upload(B, p1, &B->lpasses)) != IGAFD_OK) return fail(st);
  if (cudaHostAlloc(&B->more_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
    B->more_host = nullptr;
    cudaGetLastError();
    return fail(IGAFD_ERR_OOM);
  }
  *B->more_host = 0;
  if (cudaHostGetDevicePointer((void **)&B->more_dev, B->more_host, 0) != cudaSuccess)
    return fail(IGAFD_ERR_CUDA);
  B->guard = (unsigned)(2 * B->o.max_iter + 16);   // bounded: every problem stops at its cap;
  {                                                // a failed confirmation costs one pass
    B->log_cap = B->guard < 65536u ? B->guard : 65536u;
    std::vector<PassLog> zl(B->log_cap, PassLog{0, 0, 0, 0});
    if ((st = batch_upload(B, zl, &B->pass_log)) != IGAFD_OK) return fail(st);
  }
  *out = B;
  return IGAFD_OK;
}

// A group's loop graph: reset its pass counter, then while (any member
// unfinished) { one pass }, the body captured from batch_body; instantiated,
// with its stream and completion event.
static igafd_status group_loop(igafd_batch *B, BatchGroup *G, int priority) {
  if (cudaStreamCreateWithPriority(&G->stream, cudaStreamNonBlocking, priority) != cudaSuccess ||
      cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaGraphCreate(&G->graph, 0) != cudaSuccess)
    return IGAFD_ERR_CUDA;
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, G->graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return IGAFD_ERR_CUDA;
  cudaGraphNode_t reset_node, while_node;
  {
    cudaKernelNodeParams kp = {};
    void *kargs[1] = {&G->lpasses};
    kp.func = (void *)batch_reset_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = kargs;
    if (cudaGraphAddKernelNode(&reset_node, G->graph, nullptr, 0, &kp) != cudaSuccess)
      return IGAFD_ERR_CUDA;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (cudaGraphAddNode(&while_node, G->graph, &reset_node, nullptr, 1, &cp) != cudaSuccess)
    return IGAFD_ERR_CUDA;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(B->cap, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return IGAFD_ERR_CUDA;
  const long long l0 = g_igafd_launches.load();
  g_igafd_plain_launch = true;
  const igafd_status st = batch_body(G, B->cap, h);
  g_igafd_plain_launch = false;
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(B->cap, &captured);
  G->body_launches = g_igafd_launches.load() - l0;
  g_igafd_launches.fetch_sub(G->body_launches);              // captured, not executed
  if (st != IGAFD_OK || e != cudaSuccess) {
    cudaGetLastError();
    return st != IGAFD_OK ? st : IGAFD_ERR_CUDA;
  }
  // the group's scheduling priority on every kernel of its pass
  size_t nn = 0;
  if (cudaGraphGetNodes(body, nullptr, &nn) != cudaSuccess) return IGAFD_ERR_CUDA;
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn && cudaGraphGetNodes(body, nodes.data(), &nn) != cudaSuccess) return IGAFD_ERR_CUDA;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess) return IGAFD_ERR_CUDA;
    if (t != cudaGraphNodeTypeKernel) continue;
    cudaLaunchAttributeValue v = {};
    v.priority = priority;
    if (cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v) != cudaSuccess)
      return IGAFD_ERR_CUDA;
  }
  if (cudaGraphInstantiate(&G->exec, G->graph, 0) != cudaSuccess) {
    cudaGetLastError();
    return IGAFD_ERR_CUDA;
  }
  return IGAFD_OK;
}

extern "C" igafd_status igafd_batch_create_grouped(igafd_patch *const *patches, int count,
                                                   const igafd_pcg_opts *opts, int groups,
                                                   int passes_per_launch, igafd_batch **out) {
  if (!out) return IGAFD_ERR_ARG;
  *out = nullptr;
  if (!patches || count < 1 || groups < 0 || passes_per_launch < 0) return IGAFD_ERR_ARG;
  igafd_pcg_opts o;
  if (opts) o = *opts; else igafd_pcg_default_opts(&o);
  if (!(o.tol >= 0.0) || o.max_iter < 0 || o.true_every < 0) return IGAFD_ERR_ARG;
  if (o.prec_dtype < IGAFD_FP64 || o.prec_dtype > IGAFD_ADI) return IGAFD_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    igafd_patch *P = patches[i];
    if (!P || !P->stencil || P->dev != patches[0]->dev) return IGAFD_ERR_ARG;
    if (o.prec_dtype == IGAFD_ADI && !P->adi) return IGAFD_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (patches[j] == P) return IGAFD_ERR_ARG;            // one problem per patch
  }
  IGAFD_CUDA(cudaSetDevice(patches[0]->dev));
  if (groups == 0 || groups > count) groups = count;       // 0: one loop per problem
  o.timing = 0;
  o.check_every = 1;            // the loops run on the device; nothing is polled
  igafd_batch *B = new igafd_batch{};
  B->count = count;
  B->dev = patches[0]->dev;
  B->num_sms = patches[0]->num_sms;
  B->o = o;
  B->ps.assign(patches, patches + count);
  auto fail = [&](igafd_status e) {
    igafd_batch_destroy(B);
    return e;
  };
  // groups of problems with similar work per iteration (stencil FMAs):
  // consecutive runs of the problems ordered by it, of near-equal total work.
  // A group's passes move at the pace of its heaviest member, so problems of
  // like size share one, and light groups loop fast.
  std::vector<std::pair<double, int>> order;
  double total = 0.0;
  for (int i = 0; i < count; ++i) {
    const igafd_patch *P = patches[i];
    double pts = 1.0;
    for (int d = 0; d < P->dim; ++d) pts *= 2.0 * P->p + 1.0;
    order.push_back({-(double)P->N * pts, i});
    total += (double)P->N * pts;
  }
  std::stable_sort(order.begin(), order.end());
  std::vector<double> load(groups, 0.0);
  std::vector<std::vector<int>> members(groups);
  B->group_of.assign(count, 0);
  {
    int g = 0;
    double acc = 0.0;
    for (size_t r = 0; r < order.size(); ++r) {
      const int left = (int)(order.size() - r);           // every group gets a problem
      if (g < groups - 1 && !members[g].empty() &&
          (acc >= total * (g + 1) / groups || left <= groups - 1 - g))
        ++g;
      acc += -order[r].first;
      load[g] += -order[r].first;
      members[g].push_back(order[r].second);
    }
  }
  for (int g = 0; g < groups; ++g) {
    std::sort(members[g].begin(), members[g].end());       // the caller's order within a group
    for (int i : members[g]) B->group_of[i] = g;
    std::vector<igafd_patch *> gp;
    for (int i : members[g]) gp.push_back(patches[i]);
    BatchGroup *G = nullptr;
    const igafd_status st = group_create(gp.data(), (int)gp.size(), o, &G);
    if (st != IGAFD_OK) return fail(st);
    G->chunk = (unsigned)passes_per_launch;
    B->groups.push_back(G);
  }
  // the groups' loop graphs
  if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(IGAFD_ERR_CUDA);
  // priorities: the group of the lightest problems first. Its passes are
  // short chains of small launches whose length is set by latency, so they
  // run ahead of the throughput-bound passes of large problems instead of
  // queueing behind their CTAs, at little cost to those.
  int least = 0, greatest = 0;
  IGAFD_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  const int levels = least - greatest + 1;
  std::vector<std::pair<double, int>> by_load;
  for (int g = 0; g < groups; ++g) by_load.push_back({load[g] / (double)members[g].size(), g});
  std::stable_sort(by_load.begin(), by_load.end());
  std::vector<int> prio(groups, least);
  for (int r = 0; r < groups && groups > 1; ++r)
    prio[by_load[r].second] = greatest + (int)((long long)r * levels / groups);
  for (int g = 0; g < groups; ++g) {
    const igafd_status st = group_loop(B, B->groups[g], prio[g]);
    if (st != IGAFD_OK) return fail(st);
  }
  *out = B;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_batch_create(igafd_patch *const *patches, int count,
                                           const igafd_pcg_opts *opts, igafd_batch **out) {
  // one loop per problem (up to 64 loops; then groups of like size)
  return igafd_batch_create_grouped(patches, count, opts, count <= 64 ? 0 : 64, 0, out);
}

extern "C" igafd_status igafd_batch_groups(const igafd_batch *B, int *groups, int *group_of) {
  if (!B || !groups) return IGAFD_ERR_ARG;
  *groups = (int)B->groups.size();
  if (group_of)
    for (int i = 0; i < B->count; ++i) group_of[i] = B->group_of[i];
  return IGAFD_OK;
}

extern "C" igafd_status igafd_batch_solve(igafd_batch *B, const double *const *b,
                                          double *const *x, igafd_pcg_info *infos, void *stream) {
  if (!B || !b || !x) return IGAFD_ERR_ARG;
  for (int i = 0; i < B->count; ++i)
    if (!b[i] || !x[i] || b[i] == x[i]) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(B->dev));
  cudaStream_t s = (cudaStream_t)stream;
  const int n = B->count;
  std::vector<SolveState> S(n);
  for (int i = 0; i < n; ++i) IGAFD_TRY(solve_begin_enqueue(B->ps[i], &B->o, b[i], x[i], s, S[i]));
  for (int i = 0; i < n; ++i)
    IGAFD_CUDA(cudaMemcpyAsync(B->ps[i]->host_scal, B->ps[i]->scal, S_COUNT * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {
    igafd_patch *P = B->ps[i];
    IGAFD_TRY(solve_begin_finish(P, s, S[i], false));
    if (S[i].finished) {                 // b == 0, non-finite b or no iterations
      set_scalar_kernel<<<1, 32, 0, s>>>(P->scal, S_DONE, 1.0);
      set_scalar_kernel<<<1, 32, 0, s>>>(P->scal, S_FIN, 1.0);
      IGAFD_LAUNCHED(2);
    }
  }
  // the groups' loops, concurrently, between the caller's stream's work; a
  // group whose launch ended at its pass bound with members unfinished is
  // launched again (the host polls the launches' completion events)
  IGAFD_CUDA(cudaEventRecord(B->fork, s));
  std::vector<BatchGroup *> running;
  for (BatchGroup *G : B->groups) {
    IGAFD_CUDA(cudaStreamWaitEvent(G->stream, B->fork, 0));
    IGAFD_CUDA(cudaMemsetAsync(G->passes, 0, sizeof(unsigned), G->stream));
    *G->more_host = 0;
    IGAFD_CUDA(cudaGraphLaunch(G->exec, G->stream));
    IGAFD_CUDA(cudaEventRecord(G->done, G->stream));
    if (G->chunk > 0) running.push_back(G);
  }
  while (!running.empty()) {
    bool progressed = false;
    for (size_t k = 0; k < running.size();) {
      BatchGroup *G = running[k];
      const cudaError_t q = cudaEventQuery(G->done);
      if (q == cudaErrorNotReady) {
        ++k;
        continue;
      }
      IGAFD_CUDA(q);
      progressed = true;
      if (*(volatile int *)G->more_host) {
        *G->more_host = 0;
        IGAFD_CUDA(cudaGraphLaunch(G->exec, G->stream));
        IGAFD_CUDA(cudaEventRecord(G->done, G->stream));
        ++k;
      } else {
        running[k] = running.back();
        running.pop_back();
      }
    }
    if (!progressed) std::this_thread::yield();
  }
  for (BatchGroup *G : B->groups) IGAFD_CUDA(cudaStreamWaitEvent(s, G->done, 0));
  for (int i = 0; i < n; ++i)
    IGAFD_CUDA(cudaMemcpyAsync(B->ps[i]->host_scal, B->ps[i]->scal, S_COUNT * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  for (BatchGroup *G : B->groups) {
    unsigned passes = 0;
    IGAFD_CUDA(cudaMemcpy(&passes, G->passes, sizeof(passes), cudaMemcpyDeviceToHost));
    IGAFD_LAUNCHED((long long)passes * G->body_launches);
  }
  igafd_status worst = IGAFD_OK;
  for (int i = 0; i < n; ++i) {
    igafd_patch *P = B->ps[i];
    const double *h = P->host_scal;
    if (S[i].bb > 0.0 && !S[i].finished) {
      const bool fin = h[S_FIN] != 0.0;
      S[i].status = !fin ? IGAFD_ERR_TIMEOUT
                         : h[S_STATUS] != 0.0 ? (igafd_status)(int)h[S_STATUS] : IGAFD_OK;
      S[i].rec_rr = h[S_REC_RR];
    } else if (S[i].bb > 0.0 && S[i].o.max_iter == 0) {
      S[i].status = IGAFD_ERR_NOT_CONVERGED;
    }
    const igafd_status e = solve_end(P, s, S[i]);
    if (infos) infos[i] = S[i].inf;
    if (e != IGAFD_OK && worst == IGAFD_OK) worst = e;
  }
  return worst;
}

extern "C" igafd_status igafd_batch_pass_log(const igafd_batch *B, int group, int cap,
                                             double *start_us, double *dur_us, int *active,
                                             int *npasses) {
  if (!B || !npasses || cap < 0 || (cap > 0 && (!start_us || !dur_us || !active)))
    return IGAFD_ERR_ARG;
  if (group < 0 || group >= (int)B->groups.size()) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(B->dev));
  // the origin: the earliest pass start over the groups
  unsigned long long t_origin = ~0ull;
  for (const BatchGroup *G : B->groups) {
    unsigned gp = 0;
    IGAFD_CUDA(cudaMemcpy(&gp, G->passes, sizeof(gp), cudaMemcpyDeviceToHost));
    if (gp == 0 || G->log_cap == 0) continue;
    PassLog first;
    IGAFD_CUDA(cudaMemcpy(&first, G->pass_log, sizeof(first), cudaMemcpyDeviceToHost));
    if (first.t0 < t_origin) t_origin = first.t0;
  }
  const BatchGroup *G = B->groups[group];
  unsigned passes = 0;
  IGAFD_CUDA(cudaMemcpy(&passes, G->passes, sizeof(passes), cudaMemcpyDeviceToHost));
  const unsigned n = passes < G->log_cap ? passes : G->log_cap;
  *npasses = (int)n;
  const unsigned m = n < (unsigned)cap ? n : (unsigned)cap;
  if (m == 0) return IGAFD_OK;
  std::vector<PassLog> h(m);
  IGAFD_CUDA(cudaMemcpy(h.data(), G->pass_log, m * sizeof(PassLog), cudaMemcpyDeviceToHost));
  for (unsigned k = 0; k < m; ++k) {
    start_us[k] = (double)(long long)(h[k].t0 - t_origin) * 1e-3;
    dur_us[k] = (double)(long long)(h[k].t1 - h[k].t0) * 1e-3;
    active[k] = h[k].active;
  }
  return IGAFD_OK;
}

extern "C" igafd_status igafd_batch_pcg_solve(igafd_patch *const *patches, int count,
                                              const double *const *b, double *const *x,
                                              const igafd_pcg_opts *opts, igafd_pcg_info *infos,
                                              void *stream) {
  if (!b || !x) return IGAFD_ERR_ARG;
  igafd_batch *B = nullptr;
  IGAFD_TRY(igafd_batch_create(patches, count, opts, &B));
  const igafd_status st = igafd_batch_solve(B, b, x, infos, stream);
  igafd_batch_destroy(B);
  return st;
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
