// Batched stencil launches: one launch of the product for many problems
// (the batched PCG solve), each work item a CTA of a problem's own grid.
#include "stencil_dev.cuh"

namespace {

// Many problems in one launch: with a queue every (persistent) CTA takes work
// items from it, in order; without one CTA b runs item b. Each item (problem
// i, virtual CTA v) runs CTA v of problem i's own single-problem grid -- the
// same tiles, the same fused dot and the same last-CTA sum -- so each
// problem's result is bitwise that of its own launch. Only the problems still
// unfinished at the start of the pass are listed (the pass's compaction kernel
// writes the list): act_idx[k] is the k-th listed problem's row of args,
// act_start[k] .. act_start[k + 1] its items, *act_count the list's length.
// sel: 0 = q = A p of the PCG iteration (problems not yet done), 1 = the
// periodic true residual (running problems whose iteration count is a
// multiple of args.every), 2 = the convergence confirmation (problems the
// recurrence says converged, status ok, not yet finished). The ring's
// barriers persist across items (one running stage count); the list is
// cached in shared memory when short.
constexpr int kListCache = 64;
template <int DIM, int P, int MODE, int kStages, int R, bool HALF>
__global__ void __launch_bounds__(kTile / R + 32) stencil_batch_kernel(const StencilArgs *args,
                                                                      const int *act_idx,
                                                                      const long long *act_start,
                                                                      const int *act_count, int sel,
                                                                      unsigned long long *queue) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *ring = reinterpret_cast<double *>(smem_raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStages * Geom<P, HALF>::STAGE);
  uint64_t *empty = full + kStages;
  __shared__ volatile int s_abort;
  __shared__ long long s_item;
  __shared__ int s_k, s_run;
  __shared__ StencilArgs s_args;
  __shared__ long long s_start[kListCache + 1];
  __shared__ int s_idx[kListCache];
  const int n = *act_count;
  const bool cached = n <= kListCache;
  if (cached) {
    for (int k = threadIdx.x; k <= n; k += blockDim.x) s_start[k] = act_start[k];
    for (int k = threadIdx.x; k < n; k += blockDim.x) s_idx[k] = act_idx[k];
  }
  if (threadIdx.x == 0) {
    ring_init<kStages, kTile / R>(full, empty);
    s_abort = 0;
  }
  __syncthreads();
  const long long *st = cached ? s_start : act_start;
  const int *ix = cached ? s_idx : act_idx;
  const long long total = n > 0 ? st[n] : 0;
  long long gstage = 0;
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) {
      // persistent: items from the queue; otherwise CTA b runs item b only
      const long long it = queue ? (total > 0 ? (long long)atomicAdd(queue, 1ull) : total)
                                 : (first ? (long long)blockIdx.x : total);
      s_item = it;
      if (it < total) {
        int lo = 0, hi = n - 1;                 // last listed problem with start <= it
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (st[mid] <= it) lo = mid; else hi = mid - 1;
        }
        s_k = lo;
        const StencilArgs &ag = args[ix[lo]];
        const double *sc = ag.scal;
        const bool done = sc[S_DONE] != 0.0;
        bool run;
        if (sel == 0) run = !done;
        else if (sel == 1) run = !done && ag.every > 0 && ((long long)sc[S_ITER]) % ag.every == 0;
        else run = done && sc[S_STATUS] == 0.0 && sc[S_FIN] == 0.0;
        s_run = run ? 1 : 0;
      }
    }
    __syncthreads();
    const long long it = s_item;
    if (it >= total) break;
    if (s_run) {
      // the problem's arguments, copied by one warp
      if (threadIdx.x < 32) {
        const int words = (int)(sizeof(StencilArgs) / 4);
        const unsigned *src = reinterpret_cast<const unsigned *>(&args[ix[s_k]]);
        unsigned *dst = reinterpret_cast<unsigned *>(&s_args);
        for (int w = threadIdx.x; w < words; w += 32) dst[w] = src[w];
      }
      __syncthreads();
      const int k = s_k;
      stencil_cta<DIM, P, MODE, kStages, R, HALF>(s_args, it - st[k], st[k + 1] - st[k], ring, full,
                                            empty, gstage, &s_abort);
    }
    __syncthreads();
    if (s_abort) break;
    first = false;
  }
}

// ---- batched launches (one launch for many problems) ----------------------
template <int DIM, int P, int MODE, int kStages, int R, bool HALF = false>
igafd_status batch_launch_one(const StencilArgs *args, const int *act_idx, const long long *act_start,
                              const int *act_count, int sel, unsigned long long *queue,
                              long long items, int num_sms, cudaStream_t s) {
  const size_t smem =
      (size_t)kStages * Geom<P, HALF>::STAGE * sizeof(double) + 2 * kStages * sizeof(uint64_t);
  constexpr int kBlock = kTile / R + 32;
  auto kern = stencil_batch_kernel<DIM, P, MODE, kStages, R, HALF>;
  static std::atomic<unsigned long long> attr_set{0};
  static std::atomic<int> per_sm_tab[64];
  int per_sm = 1;
  IGAFD_TRY(per_sm_of(kern, kBlock, smem, attr_set, per_sm_tab, &per_sm));
  if (items > 0) {            // a CTA per work item (no queue)
    if (items > 0x7fffffffLL) return IGAFD_ERR_ARG;
    kern<<<(unsigned)items, kBlock, smem, s>>>(args, act_idx, act_start, act_count, sel, nullptr);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
    return IGAFD_OK;
  }
  const unsigned grid = (unsigned)(num_sms * per_sm);
  IGAFD_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
  kern<<<grid, kBlock, smem, s>>>(args, act_idx, act_start, act_count, sel, queue);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

// the stage counts of the single launches (3D; 2D patches use the default
// and one row per thread)
template <int DIM, int P, int MODE>
igafd_status batch_launch_sr(int stages, int rows, const StencilArgs *args, const int *ai,
                             const long long *as, const int *ac, int sel,
                             unsigned long long *queue, long long items, int sms, cudaStream_t s) {
  if (stages < 0) {                               // half-stored stencils: default depth
    if constexpr (DIM == 3)
      if (rows == 2)
        return batch_launch_one<DIM, P, MODE, kStagesDefault, 2, true>(args, ai, as, ac, sel, queue,
                                                                       items, sms, s);
    return batch_launch_one<DIM, P, MODE, kStagesDefault, 1, true>(args, ai, as, ac, sel, queue,
                                                                   items, sms, s);
  }
  if constexpr (DIM == 3) {
    if (rows == 2) {
      if (stages == 3) return batch_launch_one<DIM, P, MODE, 3, 2>(args, ai, as, ac, sel, queue, items, sms, s);
      if (stages == 6) return batch_launch_one<DIM, P, MODE, 6, 2>(args, ai, as, ac, sel, queue, items, sms, s);
      return batch_launch_one<DIM, P, MODE, kStagesDefault, 2>(args, ai, as, ac, sel, queue, items, sms, s);
    }
    if (stages == 3) return batch_launch_one<DIM, P, MODE, 3, 1>(args, ai, as, ac, sel, queue, items, sms, s);
    if (stages == 6) return batch_launch_one<DIM, P, MODE, 6, 1>(args, ai, as, ac, sel, queue, items, sms, s);
  }
  return batch_launch_one<DIM, P, MODE, kStagesDefault, 1>(args, ai, as, ac, sel, queue, items, sms, s);
}

template <int DIM, int MODE>
igafd_status batch_launch_p(int p, int stages, int rows, const StencilArgs *args, const int *ai,
                            const long long *as, const int *ac, int sel, unsigned long long *queue,
                            long long items, int sms, cudaStream_t s) {
  switch (p) {
    case 1: return batch_launch_sr<DIM, 1, MODE>(stages, rows, args, ai, as, ac, sel, queue, items, sms, s);
    case 2: return batch_launch_sr<DIM, 2, MODE>(stages, rows, args, ai, as, ac, sel, queue, items, sms, s);
    case 3: return batch_launch_sr<DIM, 3, MODE>(stages, rows, args, ai, as, ac, sel, queue, items, sms, s);
    case 4: return batch_launch_sr<DIM, 4, MODE>(stages, rows, args, ai, as, ac, sel, queue, items, sms, s);
    case 5: return batch_launch_sr<DIM, 5, MODE>(stages, rows, args, ai, as, ac, sel, queue, items, sms, s);
    case 6: return batch_launch_sr<DIM, 6, MODE>(stages, rows, args, ai, as, ac, sel, queue, items, sms, s);
    case 7: return batch_launch_sr<DIM, 7, MODE>(stages, rows, args, ai, as, ac, sel, queue, items, sms, s);
    default: return IGAFD_ERR_ARG;
  }
}

}  // namespace

// One launch over the listed (unfinished) problems of one class (dim, p,
// rows per thread): args_dev [members] StencilArgs, act_* the pass's list
// (see stencil_batch_kernel); persistent over the queue when items == 0,
// else one CTA per item (items bounds the listed items).
igafd_status igafd_stencil_batch_launch(int dim, int p, int stages, int rows, int sel,
                                        const void *args_dev, const int *act_idx,
                                        const long long *act_start, const int *act_count,
                                        unsigned long long *queue, long long items, int num_sms,
                                        cudaStream_t s) {
  const StencilArgs *args = (const StencilArgs *)args_dev;
  const int *ai = act_idx;
  const long long *as = act_start;
  const int *ac = act_count;
  if (dim == 3) {
    if (sel)
      return batch_launch_p<3, 1>(p, stages, rows, args, ai, as, ac, sel, queue, items, num_sms, s);
    return batch_launch_p<3, 0>(p, stages, rows, args, ai, as, ac, sel, queue, items, num_sms, s);
  }
  const int st2 = stages < 0 ? -1 : 0;            // 2D: the default depth (or the half kernels)
  if (sel) return batch_launch_p<2, 1>(p, st2, 1, args, ai, as, ac, sel, queue, items, num_sms, s);
  return batch_launch_p<2, 0>(p, st2, 1, args, ai, as, ac, sel, queue, items, num_sms, s);
}

// The stage count the batched launch uses for this patch: that of its single
// launch (3D), the default otherwise; -1 for a half-stored stencil.
int igafd_stencil_batch_stages(const igafd_patch *P) {
  if (P->stencil_half) return -1;                // the half-stored stencil's kernels
  const int st = P->stencil_stages > 0 ? P->stencil_stages : kStagesDefault;
  return P->dim == 3 && (st == 3 || st == 6) ? st : kStagesDefault;
}
