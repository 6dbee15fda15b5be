// Internal definitions shared by the igafd CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>

#include "../../include/igafd.h"

#define IGAFD_MAXP 7
#define IGAFD_COEF_CAP 2048   // PCG alpha/beta recorded per solve (Lanczos relation)
#define IGAFD_MAXDIM 3
#define IGAFD_NEV 130   // 4 per iteration for 32 iterations + 2

// Return IGAFD_ERR_CUDA from the enclosing function when a runtime call fails.
#define IGAFD_CUDA(call)                                                   \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      fprintf(stderr, "igafd: %s failed: %s (%s:%d)\n", #call,             \
              cudaGetErrorString(e_), __FILE__, __LINE__);                 \
      return IGAFD_ERR_CUDA;                                               \
    }                                                                      \
  } while (0)

#define IGAFD_TRY(expr)                         \
  do {                                          \
    igafd_status s_ = (expr);                   \
    if (s_ != IGAFD_OK) return s_;              \
  } while (0)

// Per-direction quadrature tables (device), nq = p + 1 Gauss points per
// element: index t = e * nq + g runs over the 1D quadrature points.
struct Dir1D {
  int n;          // dofs (Dirichlet-reduced)
  int m;          // B-splines of the discretisation
  int nel;        // non-empty knot spans
  int gm;         // B-splines of the geometry map
  double *knots;  // [m + p + 1]
  double *gknots; // [gm + geo_p + 1]
  int *span;      // [nel] knot-span index s of each element (locals s-p..s)
  double *z, *w;  // [nel*nq] Gauss points and weights
  double *bv, *bd;  // [nel*nq*(p+1)] local basis values / derivatives
  int *gspan;       // [nel*nq] geometry span at each point
  double *gv, *gd;  // [nel*nq*(geo_p+1)] geometry basis values / derivatives
  // coefficient spline (optional)
  int km;           // B-splines of the coefficient field
  double *kknots;   // [km + kappa_p + 1]
  int *kspan;       // [nel*nq]
  double *kv;       // [nel*nq*(kappa_p+1)]
};

// Scalars of the PCG recurrence kept on the device.
enum {
  S_RHO = 0,      // (r, z)
  S_PQ,           // (p, A p)
  S_ALPHA,
  S_BETA,
  S_RR,           // (r, r)
  S_RZOLD,        // (r_{k+1}, z_k) for the flexible beta
  S_BB,           // (b, b)
  S_DONE,         // 1.0 once converged / broken down
  S_ITER,         // iterations executed
  S_STATUS,       // 0 ok, -6 breakdown
  S_TRUE_RR,      // last true residual (r, r)
  S_TOL2,         // tol^2
  S_MAXIT,        // iteration cap
  S_FIN,          // batched solve: 1.0 once the problem is finished (confirmed, capped or broken)
  S_REC_RR,       // the recurrence (r, r) when it first met the tolerance
  S_COUNT
};

struct FDMixed;   // mixed-precision FD workspace (fd_mixed.cu)

struct igafd_patch {
  int dev;
  int dim, p, geo_p, kappa_p;
  int n[3], nel[3];
  int dshift;                   // 1: Dirichlet functions removed (n_k = m_k - 2); 0: full space
  long long N;
  int n_off;
  double kappa;
  Dir1D dir[3];
  int twin[3];                  // smallest direction with the same knot vector (same 1D pencils)
  double *ctrl;                 // [dim][gm_d]..[gm_1]
  double *kctrl;                // coefficient control values [km_d]..[km_1] or null
  // generalized eigenpairs: U[k][i*n + j], D[k][j]; inv_lam[N] = 1/(D1+D2+D3)
  double *U[3], *D[3];
  float *U32[3];
  double *inv_lam;
  float *inv_lam32;
  // stiffness stencil [n_off][Np], Np = N rounded up to the stencil tile; with
  // stencil_half, [(n_off + 1) / 2][sh_ld]: offsets from the centre up, row
  // i at sh_H + i (zero halos of sh_H rows on both ends, sh_ld = Np + 2 sh_H)
  double *stencil;
  long long Np;
  int stencil_half;
  long long sh_H, sh_ld;
  int num_sms;
  int stencil_stages;           // ring depth of the stencil pipeline (0: default; autotuned)
  int stencil_rows;             // rows per compute thread of the stencil (1 or 2 in 3D; autotuned)
  // FD workspace
  double *fd_a, *fd_b;          // N each
  // PCG workspace
  double *r, *z, *q, *xt;       // N each (xt: true-residual scratch)
  // zero-padded vectors read by the stencil (halo elements on both ends):
  // pv = PCG search direction, xpad = copy of a caller's x
  double *pv, *xpad, *pv_base, *xpad_base;
  double *xs, *xs_base;         // PCG iterate (padded), copied to the caller's x at the end
  double *bint;                 // copy of the caller's b for the duration of a solve
  long long halo;
  // captured PCG iteration chunk (replayed by cudaGraphLaunch)
  cudaStream_t cap_stream;
  cudaGraphExec_t loop_exec;
  cudaGraph_t loop_graph;       // the captured chunk (child of batched parent graphs)
  long long loop_nodes;         // kernels per replay
  unsigned long long *tstat;    // stencil timing on the device: [0] earliest block start
                                // of the running launch, [1] summed ns, [2] launches
  int loop_key[13];             // dtype, flexible, true_every, chunk, valid, FD form (2),
                                // stencil depth, stencil rows, FD tile shape (4)
  double *partial;              // [PARTIAL_SLOTS][MAX_BLOCKS]
  unsigned int *counter;        // last-block counters
  double *scal;                 // [S_COUNT]
  double *coef;                 // [2 * IGAFD_COEF_CAP]: alpha_k, beta_k of the last solve
  double *host_scal;            // pinned mirror of scal
  FDMixed *mixed;
  double *wK[3], *wM[3];        // span scalings of the pencils (device, null = unscaled)
  int fd_fused;                 // 1: fused tensor-core FD (3 kernels) when n_k <= 128
  int fd_fused_op[3];           // the same per operand type (TF32, BF16, FP16), set by the autotuner
  int fd_tile[3][4];            // per operand type: per-mode kernel's rows per CTA (64 or 128; 0 =
                                // 128), column split (2 = two column tiles, else one), K stages (3,
                                // else 2); pencil kernel's columns per CTA (64 or 128; 0 = 128)
  int eig_route;                // 0: FP32 Jacobi + FP64 refinement where n_k <= 128; 1: FP64 Jacobi
  int eig_used[3];              // route each direction took: 0 refined, 1 FP64 Jacobi
  double eig_check[3][2];       // refined route's final check (orthogonality, off-diagonal)
  double *eig_work;             // eigen-setup scratch (kept for re-setups)
  void *eig_jobs;
  int scaled;
  float *lfeat;                 // learned scalings: per-span features [rows][6] (kept after the first request)
  double *lybar;                // and slab means of log Q_jj [dim][rows]
  int lstats_valid;
  cudaEvent_t ev[IGAFD_NEV];    // phase-timing events (PCG with timing on)
  // diagnostics
  double min_detJ, q_bound, setup_ms, eig_ms;
  int *err_flag;                // device error flags from setup kernels
  void *adi;                    // three-variable ADI preconditioner state (adi.cu), or null
};

// Reductions: fixed-size partial arrays, deterministic order.
#define IGAFD_RED_BLOCKS 1184   // 152 SMs * 8 (multiple of the SM count)
#define IGAFD_PARTIAL_SLOTS 4

// ---- internal entry points (implemented in the .cu files) ----------------
igafd_status igafd_setup_tables(igafd_patch *P, const igafd_patch_desc *d, cudaStream_t s);
// pencils (optionally span-scaled: wK[k], wM[k] device arrays of nel[k]
// weights, null = unscaled), eigendecompositions, 1/(D1 + D2 + D3)
igafd_status igafd_build_prec(igafd_patch *P, cudaStream_t s);
igafd_status igafd_setup_pencils_eig(igafd_patch *P, cudaStream_t s, const double *const *wK = nullptr,
                                     const double *const *wM = nullptr);
igafd_status igafd_setup_stencil(igafd_patch *P, cudaStream_t s);
// a half-stored stencil written out in the full layout [n_off][N] (setup.cu)
igafd_status igafd_stencil_expand(const igafd_patch *P, double *dst, cudaStream_t s);
// dense (Dirichlet-reduced) pencils K_k, M_k of direction k into K, M (n_k x
// n_k each, device), span-scaled when the patch carries scalings
igafd_status igafd_pencils_dense(igafd_patch *P, int k, double *K, double *M, cudaStream_t s);
void igafd_adi_free(igafd_patch *P);   // releases the ADI state (adi.cu)
// z = P_J^{-1} r by the ADI set up on the patch; kernels do nothing while
// *done_flag != 0 (done_flag may be null)
igafd_status igafd_adi_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                             double *done_flag);
// FD apply; kernels do nothing while *done_flag != 0 (done_flag may be null)
igafd_status igafd_fd64_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                              double *done_flag);
igafd_status igafd_fd32_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                              double *done_flag);
igafd_status igafd_fd_tc_apply(igafd_patch *P, igafd_dtype dt, const double *r, double *z,
                               cudaStream_t s, double *done_flag);
igafd_status igafd_fd_tc_init(igafd_patch *P, cudaStream_t s);
void igafd_fd_tc_free(igafd_patch *P);
// y = A x (b == null) or y = b - A x; see stencil.cu
// every > 0: the kernel only runs when the device iteration counter is a
// multiple of `every` (periodic true residual inside a captured loop);
// z (with b and pcg): the true residual also gives (r, z) to the flexible beta
igafd_status igafd_stencil_launch(igafd_patch *P, const double *x, double *y, const double *b,
                                  int pcg, int skip_done, cudaStream_t s, int every = 0,
                                  unsigned long long *tstat = nullptr,
                                  const double *z = nullptr);
long long igafd_stencil_row_stride(long long N);   // Np for a given N
// batched solve (stencil.cu): the PCG stencil launches of a patch as
// StencilArgs bytes (sel 0: q = A p; 1: periodic r = b - A x every `every`
// iterations; 2: the convergence confirmation) with the single launch's grid,
// and one persistent launch over many problems of one (dim, p, rows) class
size_t igafd_stencil_args_bytes();
igafd_status igafd_stencil_batch_args(igafd_patch *P, int sel, int flexible, int every, void *out,
                                      long long *vgrid);
igafd_status igafd_stencil_batch_launch(int dim, int p, int stages, int rows, int sel,
                                        const void *args_dev, const int *act_idx,
                                        const long long *act_start, const int *act_count,
                                        unsigned long long *queue, long long items, int num_sms,
                                        cudaStream_t s);
int igafd_stencil_batch_stages(const igafd_patch *P);
// batched solve (fd_tc.cu): true when the patch's tensor-core FD of operand
// type dt runs as the generic fused kernels (so a batched launch can run it);
// then the per-kind kernel arguments (FusedArgs bytes) and CTA counts
bool igafd_fd_tc_fused_generic(const igafd_patch *P, igafd_dtype dt);
size_t igafd_fd_fused_args_bytes();
igafd_status igafd_fd_fused_batch_args(igafd_patch *P, igafd_dtype dt, void *args3, int *blocks3,
                                       size_t *smem);
// one batched launch of fused kind (0 slab forward, 1 pencil, 2 slab
// backward) over the listed problems: act (indices into the args), their CTA
// prefix act_start for this kind, *act_count and the zeroed work-queue counter
// (device; persistent CTAs) or null (one CTA per item); total_blocks bounds
// the items
igafd_status igafd_fd_fused_batch_launch(igafd_dtype dt, int kind, const void *args_dev,
                                         const int *act, const int *act_start,
                                         const int *act_count, unsigned *queue, int total_blocks,
                                         size_t smem, int num_sms, cudaStream_t s);
// dense tensor-core FLOP/s for TF32 (op 0) or BF16 (op 1) operands (fd_tc.cu);
// a bounded wait that runs out sets *err_dev to IGAFD_ERR_TIMEOUT
igafd_status igafd_tc_probe(int op, int num_sms, int rounds, int *err_dev, double *flop_per_s);
// number of CTAs of the PCG vector kernels for N dofs (the same in single and
// batched solves, so their reductions agree bitwise)
int igafd_red_blocks(long long N);
long long igafd_stencil_halo(int p, const int *n);   // zero halo of padded vectors
void igafd_tune_lookup(igafd_patch *P);              // apply a cached autotune choice

// Programmatic dependent launch. Kernels of the PCG iteration and of the FD
// are launched with igafd_launch, which lets a kernel start while its
// predecessor on the stream is still finishing (its launch, barrier set-up,
// TMEM allocation and constant-table fetches overlap the predecessor's tail).
// Every such kernel calls pdl_wait() in all threads before reading anything
// an earlier kernel wrote (the wait returns once the predecessor grid has
// completed and its writes are visible, so a chain of such kernels stays
// ordered), then pdl_trigger(), which lets the next kernel launch as soon as
// all of this grid's blocks have started. Outside a programmatic dependency
// both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// While set (on this thread), igafd_launch issues ordinary launches: the
// batched solve captures its loop body that way.
extern thread_local bool g_igafd_plain_launch;
template <typename... KArgs, typename... Args>
inline cudaError_t igafd_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_igafd_plain_launch ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Kernels enqueued by this library (process-wide), for launch accounting.
extern std::atomic<long long> g_igafd_launches;
#define IGAFD_LAUNCHED(n) g_igafd_launches.fetch_add((n), std::memory_order_relaxed)

// ---- device helpers ---------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh32) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh32[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    t = lane < nw ? sh32[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}
