// y = A x and r = b - A x as one launch per product (the single-problem
// kernel); the batched launches over many problems are in stencil_batch.cu.
#include "stencil_dev.cuh"

namespace {

// One launch of the product: CTA b of the grid runs stencil_cta as CTA b of
// gridDim.x CTAs.
//
// MODE 0: y = A x, dot (x, y) -> alpha = rho / (x, y) when pcg.
// MODE 1: y = b - A x, dot (y, y) -> true (r, r) when pcg; with z given also
// (y, z) -> (r, z_old) of the flexible beta, so that a recomputed residual
// replaces the recurrence one in every scalar that uses it.
template <int DIM, int P, int MODE, int kStages, int R, bool HALF>
__global__ void __launch_bounds__(kTile / R + 32) stencil_tma_kernel(StencilArgs a) {
  pdl_wait();
  pdl_trigger();
  if (a.done && *a.done != 0.0) return;
  if (a.every > 0 && ((long long)a.scal[S_ITER]) % a.every != 0) return;
  if (a.tstat && threadIdx.x == 0) atomicMin(&a.tstat[0], global_ns());
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *ring = reinterpret_cast<double *>(smem_raw);              // [kStages][STAGE]
  uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStages * Geom<P, HALF>::STAGE);
  uint64_t *empty = full + kStages;
  __shared__ volatile int s_abort;
  if (threadIdx.x == 0) {
    ring_init<kStages, kTile / R>(full, empty);
    s_abort = 0;
  }
  __syncthreads();
  long long gstage = 0;
  stencil_cta<DIM, P, MODE, kStages, R, HALF>(a, blockIdx.x, gridDim.x, ring, full, empty, gstage,
                                              &s_abort);
}

// One launch of the single-problem kernel, or with grid_out only its grid
// (the resident CTAs of every SM, at most grid_cap).
template <int DIM, int P, int MODE, int kStages, int R, bool HALF = false>
igafd_status launch_one(const StencilArgs &a, long long grid_cap, int num_sms, cudaStream_t s,
                        long long *grid_out) {
  const size_t smem =
      (size_t)kStages * Geom<P, HALF>::STAGE * sizeof(double) + 2 * kStages * sizeof(uint64_t);
  constexpr int kBlock = kTile / R + 32;
  auto kern = stencil_tma_kernel<DIM, P, MODE, kStages, R, HALF>;
  static std::atomic<unsigned long long> attr_set{0};
  static std::atomic<int> per_sm_tab[64];
  int per_sm = 1;
  IGAFD_TRY(per_sm_of(kern, kBlock, smem, attr_set, per_sm_tab, &per_sm));
  long long grid = (long long)num_sms * per_sm;
  if (grid > grid_cap) grid = grid_cap;
  if (grid < 1) grid = 1;
  if (grid_out) {
    *grid_out = grid;
    return IGAFD_OK;
  }
  IGAFD_CUDA(igafd_launch(kern, dim3((unsigned)grid), dim3(kBlock), smem, s, a));
  IGAFD_LAUNCHED(1);
  return IGAFD_OK;
}

// two rows per thread are built for 3D only (2D patches are small)
template <int DIM, int P, int MODE, int kStages>
igafd_status launch_rows(int rows, const StencilArgs &a, long long cap, int sms, cudaStream_t s,
                         long long *grid_out) {
  if constexpr (DIM == 3)
    if (rows == 2) return launch_one<DIM, P, MODE, kStages, 2>(a, cap, sms, s, grid_out);
  return launch_one<DIM, P, MODE, kStages, 1>(a, cap, sms, s, grid_out);
}

// a half-stored stencil runs at the default ring depth
template <int DIM, int P, int MODE>
igafd_status launch_half(int rows, const StencilArgs &a, long long cap, int sms, cudaStream_t s,
                         long long *grid_out) {
  if constexpr (DIM == 3)
    if (rows == 2) return launch_one<DIM, P, MODE, kStagesDefault, 2, true>(a, cap, sms, s, grid_out);
  return launch_one<DIM, P, MODE, kStagesDefault, 1, true>(a, cap, sms, s, grid_out);
}

template <int DIM, int P, int MODE>
igafd_status launch_stages(int stages, int rows, const StencilArgs &a, long long cap, int sms,
                           cudaStream_t s, long long *grid_out) {
  if (stages < 0) return launch_half<DIM, P, MODE>(rows, a, cap, sms, s, grid_out);
  switch (stages) {
    case 3: return launch_rows<DIM, P, MODE, 3>(rows, a, cap, sms, s, grid_out);
    case 6: return launch_rows<DIM, P, MODE, 6>(rows, a, cap, sms, s, grid_out);
    default: return launch_rows<DIM, P, MODE, 4>(rows, a, cap, sms, s, grid_out);
  }
}

template <int DIM, int MODE>
igafd_status launch_p(int p, int stages, int rows, const StencilArgs &a, long long cap, int sms,
                      cudaStream_t s, long long *grid_out = nullptr) {
  switch (p) {
    case 1: return launch_stages<DIM, 1, MODE>(stages, rows, a, cap, sms, s, grid_out);
    case 2: return launch_stages<DIM, 2, MODE>(stages, rows, a, cap, sms, s, grid_out);
    case 3: return launch_stages<DIM, 3, MODE>(stages, rows, a, cap, sms, s, grid_out);
    case 4: return launch_stages<DIM, 4, MODE>(stages, rows, a, cap, sms, s, grid_out);
    case 5: return launch_stages<DIM, 5, MODE>(stages, rows, a, cap, sms, s, grid_out);
    case 6: return launch_stages<DIM, 6, MODE>(stages, rows, a, cap, sms, s, grid_out);
    case 7: return launch_stages<DIM, 7, MODE>(stages, rows, a, cap, sms, s, grid_out);
    default: return IGAFD_ERR_ARG;
  }
}

}  // namespace


long long igafd_stencil_row_stride(long long N) { return (N + kTile - 1) / kTile * kTile; }

// Zero halo (in elements) around padded vectors, so every x window of every
// tile and offset group lies inside the allocation: p (n_1 n_2 + n_1 + 1)
// + a tile + slack, rounded to 256 bytes.
long long igafd_stencil_halo(int p, const int *n) {
  long long h = (long long)p * ((long long)n[0] * n[1] + n[0] + 1) + kTile + 16;
  return (h + 31) / 32 * 32;
}

// Internal: y = A x (b == null) or y = b - A x. With pcg != 0 the fused dot
// feeds the PCG scalars; with skip_done != 0 the kernel does nothing once the
// PCG convergence flag is set.
static StencilArgs make_args(igafd_patch *P, const double *x, double *y, const double *b, int pcg,
                             int skip_done, int every, unsigned long long *tstat, const double *z) {
  StencilArgs a{};
  a.S = P->stencil;
  a.x = x;
  a.y = y;
  a.b = b;
  a.z = (b && pcg) ? z : nullptr;
  a.n1 = P->n[0];
  a.n2 = P->n[1];
  a.n3 = P->n[2];
  a.N = P->N;
  a.Np = P->stencil_half ? P->sh_ld : P->Np;
  a.oc = P->stencil_half ? P->n_off / 2 : 0;
  a.shH = P->stencil_half ? P->sh_H : 0;
  a.ntiles = (P->N + kTile - 1) / kTile;
  a.partial = pcg ? P->partial : nullptr;
  a.counter = P->counter;
  a.scal = pcg ? P->scal : nullptr;
  a.pcg = pcg;
  a.done = skip_done ? P->scal + S_DONE : nullptr;
  a.err = P->err_flag;
  a.every = every;
  a.tstat = a.partial ? tstat : nullptr;
  return a;
}

static long long grid_cap(igafd_patch *P) {
  const long long ntiles = (P->N + kTile - 1) / kTile;
  return ntiles < IGAFD_RED_BLOCKS ? ntiles : IGAFD_RED_BLOCKS;
}

igafd_status igafd_stencil_launch(igafd_patch *P, const double *x, double *y, const double *b,
                                  int pcg, int skip_done, cudaStream_t s, int every,
                                  unsigned long long *tstat, const double *z) {
  // the kernel reads x windows that reach p planes beyond the box: use a
  // zero-padded copy unless x already is one (PCG search direction / iterate)
  if (x != P->pv && x != P->xpad && x != P->xs) {
    IGAFD_CUDA(cudaMemcpyAsync(P->xpad, x, P->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    x = P->xpad;
  }
  const StencilArgs a = make_args(P, x, y, b, pcg, skip_done, every, tstat, z);
  // persistent grid: the resident CTAs of every SM, never more than the
  // tiles or the partial-sum slots
  const long long cap = grid_cap(P);
  // ring depth; -1 selects the half-stored stencil's kernels (default depth)
  const int st = P->stencil_half ? -1 : P->stencil_stages > 0 ? P->stencil_stages : kStagesDefault;
  const int rows = P->stencil_rows == 2 ? 2 : 1;
  if (P->dim == 3) {
    if (b) return launch_p<3, 1>(P->p, st, rows, a, cap, P->num_sms, s);
    return launch_p<3, 0>(P->p, st, rows, a, cap, P->num_sms, s);
  }
  if (b) return launch_p<2, 1>(P->p, st, 1, a, cap, P->num_sms, s);
  return launch_p<2, 0>(P->p, st, 1, a, cap, P->num_sms, s);
}

// ---- for the batched solve -------------------------------------------------
size_t igafd_stencil_args_bytes() { return sizeof(StencilArgs); }

// The arguments of the PCG's stencil launches on the patch (bytes of a
// StencilArgs): sel 0 q = A p (search direction), else r = b - A x of the
// iterate, with (r, z_old) when flexible; and the single launch's grid,
// whose CTAs a batched launch runs as work items.
igafd_status igafd_stencil_batch_args(igafd_patch *P, int sel, int flexible, int every, void *out,
                                      long long *vgrid) {
  const StencilArgs a = sel == 0 ? make_args(P, P->pv, P->q, nullptr, 1, 0, 0, nullptr, nullptr)
                                 : make_args(P, P->xs, P->r, P->bint, 1, 0, sel == 1 ? every : 0,
                                             nullptr, flexible ? P->z : nullptr);
  memcpy(out, &a, sizeof(a));
  const long long cap = grid_cap(P);
  // ring depth; -1 selects the half-stored stencil's kernels (default depth)
  const int st = P->stencil_half ? -1 : P->stencil_stages > 0 ? P->stencil_stages : kStagesDefault;
  const int rows = P->dim == 3 && P->stencil_rows == 2 ? 2 : 1;
  if (P->dim == 3) {
    if (sel) return launch_p<3, 1>(P->p, st, rows, a, cap, P->num_sms, nullptr, vgrid);
    return launch_p<3, 0>(P->p, st, rows, a, cap, P->num_sms, nullptr, vgrid);
  }
  if (sel) return launch_p<2, 1>(P->p, st, 1, a, cap, P->num_sms, nullptr, vgrid);
  return launch_p<2, 0>(P->p, st, 1, a, cap, P->num_sms, nullptr, vgrid);
}
