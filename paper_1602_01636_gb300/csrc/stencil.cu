// y = A x with A stored as a (2p+1)^d-point FP64 stencil, offset-major:
// S[o][row] with row stride Np (N rounded up to the tile), o = sum_k
// (delta_k + p)(2p+1)^(k-1) (Section 2.1: an interior row of A couples to
// (2p+1)^d columns). Also r = b - A x (true residual).
//
// On GB300 the 343 FP64 FMAs of a p = 3 row take longer on the FP64 pipe
// (2 FMA/clk/SM) than its 2.7 KB of coefficients take to stream from HBM, so
// the kernel is built to keep the FP64 pipe fed from shared memory: a
// persistent grid of CTAs walks 256-row tiles; for every (delta_2, delta_3)
// group a producer warp brings the 2p+1 coefficient runs of the tile
// (contiguous 2 KB each) and the contiguous window of x they multiply into a
// shared-memory ring with bulk asynchronous copies (cp.async.bulk, completion
// on mbarriers), several groups ahead of the eight compute warps. x is read
// from a copy with a zero halo of p planes on both ends, and couplings that
// leave the index box are stored as 0, so every row runs the same
// branch-free (2p+1)^d FMAs and no read leaves the allocation. Every
// mbarrier wait is bounded: on timeout the kernel records an error, waits
// (bounded) for its own copies and returns. Optional fused dot with a
// deterministic last-block reduction.
#include "common.cuh"

#include <atomic>
#include <cstring>

namespace {

constexpr int kTile = 256;                        // rows per tile
// ring depths (offset groups in flight per CTA) the kernel is built for; the
// autotuner picks one per (dimension, degree, sizes), default kStagesDefault
constexpr int kStagesDefault = 4;
constexpr long long kSpin = 1ll << 26;   // mbarrier poll limit (~seconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (long long i = 0; i < kSpin; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Last block of a grid-stride reduction: returns true in every thread of the
// block that finished last (all partials visible).
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

struct StencilArgs {
  const double *S;    // [n_off][Np]
  const double *x;    // interior pointer of a zero-padded vector (halo H)
  double *y;
  const double *b;    // MODE 1
  const double *z;    // MODE 1, optional: also (y, z) -> scal[S_RZOLD] (flexible beta)
  int n1, n2, n3;
  long long N, Np;
  long long ntiles;
  double *partial;    // null: no dot
  unsigned *counter;
  double *scal;       // PCG scalars (pcg != 0)
  int pcg;
  const double *done; // skip when *done != 0
  int *err;           // set on an mbarrier timeout
  int every;          // > 0: run only when scal[S_ITER] is a multiple of every
  unsigned long long *tstat;  // optional device timing (see igafd_patch::tstat)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

template <int P>
struct Geom {
  static constexpr int W = 2 * P + 1;
  static constexpr int XW = (kTile + 2 * P + 2 + 1) & ~1;   // x window (even count)
  static constexpr int STAGE = W * kTile + XW;               // doubles per ring stage
};

// Warp-specialised pipeline: the compute warps take R consecutive rows per
// thread (R = 1: warps 0..7, one row each; R = 2: warps 0..3, two rows each,
// reading both rows' coefficients and the shared x values with 16-byte
// shared-memory loads, which halves the load instructions per FMA); the next
// warp (one elected lane) streams, for every (delta_2, delta_3) group, the
// 2p+1 coefficient runs of the tile and the x window they multiply into a
// ring of kStages shared-memory stages (full/empty mbarriers). The FP64 FMAs
// read both operands from shared memory.
//
// MODE 0: y = A x, dot (x, y) -> alpha = rho / (x, y) when pcg.
// MODE 1: y = b - A x, dot (y, y) -> true (r, r) when pcg; with z given also
// (y, z) -> (r, z_old) of the flexible beta, so that a recomputed residual
// replaces the recurrence one in every scalar that uses it.
// One CTA's share of the product, as CTA vb of a grid of vgrid CTAs: tiles
// vb, vb + vgrid, ..., the fused dot, and (in the CTA that finishes last) the
// dot's fixed-order sum over the vgrid partial sums. The ring's barriers are
// initialised by the caller; gstage counts the ring stages this CTA has
// passed through so far, so a persistent CTA can keep its ring across calls.
template <int DIM, int P, int MODE, int kStages, int R>
__device__ __forceinline__ void stencil_cta(const StencilArgs &a, long long vb, long long vgrid,
                                            double *ring, uint64_t *full, uint64_t *empty,
                                            long long &gstage, volatile int *s_abort) {
  using Gm = Geom<P>;
  constexpr int W = Gm::W;
  constexpr int G = DIM == 3 ? W * W : W;        // (delta_2, delta_3) groups per tile
  constexpr uint32_t kStageBytes = Gm::STAGE * sizeof(double);
  constexpr int kCompute = kTile / R;            // compute threads
  static_assert(R == 1 || R == 2, "one or two rows per thread");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long my_tiles = a.ntiles > vb ? (a.ntiles - 1 - vb) / vgrid + 1 : 0;
  const long long total = my_tiles * G;
  const long long n12 = (long long)a.n1 * a.n2;
  const long long g0 = gstage;                   // global index of this call's first stage

  double dot = 0.0, dot2 = 0.0;
  if (warp == kCompute / 32) {
    // ---------------- producer warp ----------------
    if (lane == 0) {
      long long issued = 0;
      bool ok = true;
      for (long long s = 0; s < total && ok; ++s) {
        const long long gs = g0 + s;
        const int slot = (int)(gs % kStages);
        if (gs >= kStages) {
          const uint32_t par = (uint32_t)(((gs / kStages) - 1) & 1);
          long long it = 0;
          while (!mbar_try_wait(&empty[slot], par)) {
            if (*s_abort || ++it > kSpin) { ok = false; break; }
          }
          if (!ok) break;
        }
        const long long tile = vb + (s / G) * vgrid;
        const int g = (int)(s % G);
        const int d2 = g % W - P, d3 = DIM == 3 ? g / W - P : 0;
        const int ob = (DIM == 3 ? (d3 + P) * W * W : 0) + (d2 + P) * W;
        const long long row0 = tile * kTile;
        long long x0 = row0 + (long long)d3 * n12 + (long long)d2 * a.n1 - P;
        x0 -= (x0 & 1);                                   // 16-byte aligned start
        double *st = ring + (size_t)slot * Gm::STAGE;
        uint64_t *bar = &full[slot];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_tx(bar, kStageBytes);
        for (int d1 = 0; d1 < W; ++d1)
          bulk_g2s(st + d1 * kTile, a.S + (size_t)(ob + d1) * a.Np + row0, kTile * sizeof(double), bar);
        bulk_g2s(st + W * kTile, a.x + x0, Gm::XW * sizeof(double), bar);
        ++issued;
      }
      if (!ok) {
        *s_abort = 1;
        atomicExch(a.err, (int)IGAFD_ERR_TIMEOUT);
      }
      // never leave with copies in flight: wait (bounded) for the last stages issued
      for (long long q = issued - kStages > 0 ? issued - kStages : 0; q < issued; ++q)
        mbar_wait(&full[(g0 + q) % kStages], (uint32_t)(((g0 + q) / kStages) & 1));
    }
  } else {
    // ---------------- compute warps ----------------
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    long long row = 0;                       // first of this thread's R rows
    bool live[R];
    int i2r[R], i3r[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { live[r] = false; i2r[r] = 0; i3r[r] = 0; }
    for (long long s = 0; s < total; ++s) {
      const int g = (int)(s % G);
      if (g == 0) {
        const long long tile = vb + (s / G) * vgrid;
        row = tile * kTile + (long long)R * tid;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          live[r] = row + r < a.N;
          i2r[r] = (int)(((row + r) / a.n1) % a.n2);
          i3r[r] = DIM == 3 ? (int)((row + r) / n12) : 0;
          acc[r] = 0.0;
        }
      }
      const long long gs = g0 + s;
      const int slot = (int)(gs % kStages);
      const uint32_t par = (uint32_t)((gs / kStages) & 1);
      long long it = 0;
      bool ok = true;
      while (!mbar_try_wait(&full[slot], par)) {
        if (*s_abort || ++it > kSpin) { ok = false; break; }
      }
      if (!ok) {
        *s_abort = 1;
        atomicExch(a.err, (int)IGAFD_ERR_TIMEOUT);
        break;
      }
      const int d2 = g % W - P, d3 = DIM == 3 ? g / W - P : 0;
      const long long row0 = row - (long long)R * tid;
      const long long xs0 = row0 + (long long)d3 * n12 + (long long)d2 * a.n1 - P;
      const int sh = (int)(xs0 & 1);                      // window starts at xs0 - sh
      const double *st = ring + (size_t)slot * Gm::STAGE;
      // rows whose (i_2 + delta_2, i_3 + delta_3) leaves the box have only
      // zero coefficients in this group; skip when the whole warp is out
      bool in23 = false;
#pragma unroll
      for (int r = 0; r < R; ++r)
        in23 = in23 || (live[r] && (i2r[r] + d2 >= 0) && (i2r[r] + d2 < a.n2) &&
                        (DIM == 2 || ((i3r[r] + d3 >= 0) && (i3r[r] + d3 < a.n3))));
      if (__any_sync(0xffffffffu, in23)) {
        if constexpr (R == 1) {
          const double *cf = st + tid;
          const double *xw = st + W * kTile + tid + sh;   // xw[j] = x[row + off - P + j]
#pragma unroll
          for (int j = 0; j < W; ++j) acc[0] = fma(cf[j * kTile], xw[j], acc[0]);
        } else {
          // rows row, row + 1: coefficients cf[j] = (S[o_j][row], S[o_j][row + 1]);
          // x[row + off - P + j] = xv[j + sh], x[row + 1 + off - P + j] = xv[j + 1 + sh]
          const double2 *cf = reinterpret_cast<const double2 *>(st + 2 * tid);
          const double2 *xb = reinterpret_cast<const double2 *>(st + W * kTile + 2 * tid);
          constexpr int NP = (W + 1) / 2;                  // pairs covering W + 1 values
          double xv[2 * NP + 2];
          if (sh == 0) {
#pragma unroll
            for (int m = 0; m < NP; ++m) { const double2 v = xb[m]; xv[2 * m] = v.x; xv[2 * m + 1] = v.y; }
#pragma unroll
            for (int j = 0; j < W; ++j) {
              const double2 c = cf[j * (kTile / 2)];
              acc[0] = fma(c.x, xv[j], acc[0]);
              acc[1] = fma(c.y, xv[j + 1], acc[1]);
            }
          } else {
#pragma unroll
            for (int m = 0; m < NP + 1; ++m) { const double2 v = xb[m]; xv[2 * m] = v.x; xv[2 * m + 1] = v.y; }
#pragma unroll
            for (int j = 0; j < W; ++j) {
              const double2 c = cf[j * (kTile / 2)];
              acc[0] = fma(c.x, xv[j + 1], acc[0]);
              acc[1] = fma(c.y, xv[j + 2], acc[1]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot])) : "memory");
      if (g == G - 1) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (!live[r]) continue;
          const double ax = acc[r];
          if (MODE == 0) {
            a.y[row + r] = ax;
            dot = fma(a.x[row + r], ax, dot);
          } else {
            const double rr = a.b[row + r] - ax;
            a.y[row + r] = rr;
            dot = fma(rr, rr, dot);
            if (a.z) dot2 = fma(rr, a.z[row + r], dot2);
          }
        }
      }
    }
  }
  gstage = g0 + total;
  __syncthreads();
  if (*s_abort) {
    if (tid == 0 && a.pcg) {
      a.scal[S_STATUS] = (double)IGAFD_ERR_TIMEOUT;
      a.scal[S_DONE] = 1.0;
    }
    return;
  }
  if (!a.partial) return;
  __shared__ double sh32[32];
  const double bs = block_sum(dot, sh32);
  const double bs2 = (MODE == 1 && a.z) ? block_sum(dot2, sh32) : 0.0;
  if (tid == 0) {
    a.partial[vb] = bs;
    if (MODE == 1 && a.z) a.partial[vgrid + vb] = bs2;
  }
  if (!last_block(a.counter, (unsigned)vgrid)) return;
  const double tot = sum_partials(a.partial, (int)vgrid, sh32);
  const double tot2 = (MODE == 1 && a.z) ? sum_partials(a.partial + vgrid, (int)vgrid, sh32) : 0.0;
  if (tid == 0) {
    *a.counter = 0u;
    if (a.tstat) {   // this block finished last: launch duration = now - first start
      a.tstat[1] += global_ns() - a.tstat[0];
      a.tstat[2] += 1ull;
      a.tstat[0] = ~0ull;
    }
    if (a.pcg) {
      double *scal = a.scal;
      if (MODE == 0) {
        scal[S_PQ] = tot;
        const double alpha = scal[S_RHO] / tot;
        if (!(tot > 0.0) || !isfinite(alpha)) {
          scal[S_STATUS] = (double)IGAFD_ERR_BREAKDOWN;
          scal[S_DONE] = 1.0;
        }
        scal[S_ALPHA] = alpha;
      } else {
        scal[S_TRUE_RR] = tot;
        scal[S_RR] = tot;
        if (a.z) scal[S_RZOLD] = tot2;
      }
    }
  }
}

// Initialise the ring's full/empty barriers of a CTA (thread 0; the caller syncs).
template <int kStages, int kCompute>
__device__ __forceinline__ void ring_init(uint64_t *full, uint64_t *empty) {
  for (int s = 0; s < kStages; ++s) {
    mbar_init(&full[s], 1);
    mbar_init(&empty[s], kCompute / 32);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Warp-specialised pipeline: the compute warps take R consecutive rows per
// thread (R = 1: warps 0..7, one row each; R = 2: warps 0..3, two rows each,
// reading both rows' coefficients and the shared x values with 16-byte
// shared-memory loads, which halves the load instructions per FMA); the next
// warp (one elected lane) streams, for every (delta_2, delta_3) group, the
// 2p+1 coefficient runs of the tile and the x window they multiply into a
// ring of kStages shared-memory stages (full/empty mbarriers). The FP64 FMAs
// read both operands from shared memory.
//
// MODE 0: y = A x, dot (x, y) -> alpha = rho / (x, y) when pcg.
// MODE 1: y = b - A x, dot (y, y) -> true (r, r) when pcg; with z given also
// (y, z) -> (r, z_old) of the flexible beta, so that a recomputed residual
// replaces the recurrence one in every scalar that uses it.
template <int DIM, int P, int MODE, int kStages, int R>
__global__ void __launch_bounds__(kTile / R + 32) stencil_tma_kernel(StencilArgs a) {
  pdl_wait();
  pdl_trigger();
  if (a.done && *a.done != 0.0) return;
  if (a.every > 0 && ((long long)a.scal[S_ITER]) % a.every != 0) return;
  if (a.tstat && threadIdx.x == 0) atomicMin(&a.tstat[0], global_ns());
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *ring = reinterpret_cast<double *>(smem_raw);              // [kStages][STAGE]
  uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStages * Geom<P>::STAGE);
  uint64_t *empty = full + kStages;
  __shared__ volatile int s_abort;
  if (threadIdx.x == 0) {
    ring_init<kStages, kTile / R>(full, empty);
    s_abort = 0;
  }
  __syncthreads();
  long long gstage = 0;
  stencil_cta<DIM, P, MODE, kStages, R>(a, blockIdx.x, gridDim.x, ring, full, empty, gstage, &s_abort);
}

// Many problems in one persistent launch: every CTA takes work items from
// an atomic queue, in order, each item (problem i, virtual CTA v) running CTA
// v of problem i's own single-problem grid -- the same tiles, the same fused
// dot and the same last-CTA sum -- so each problem's result is bitwise that
// of its own launch. Only the problems still unfinished at the start of the
// pass are listed (the pass's compaction kernel writes the list): act_idx[k]
// is the k-th listed problem's row of args, act_start[k] .. act_start[k + 1]
// its items, *act_count the list's length. sel: 0 = q = A p of the PCG
// iteration (problems not yet done), 1 = the periodic true residual (running
// problems whose iteration count is a multiple of args.every), 2 = the
// convergence confirmation (problems the recurrence says converged, status
// ok, not yet finished). The ring's barriers persist across items (one
// running stage count); the list is cached in shared memory when short.
constexpr int kListCache = 64;
template <int DIM, int P, int MODE, int kStages, int R>
__global__ void __launch_bounds__(kTile / R + 32) stencil_batch_kernel(const StencilArgs *args,
                                                                      const int *act_idx,
                                                                      const long long *act_start,
                                                                      const int *act_count, int sel,
                                                                      unsigned long long *queue) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *ring = reinterpret_cast<double *>(smem_raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStages * Geom<P>::STAGE);
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
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = total > 0 ? (long long)atomicAdd(queue, 1ull) : total;
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
      stencil_cta<DIM, P, MODE, kStages, R>(s_args, it - st[k], st[k + 1] - st[k], ring, full,
                                            empty, gstage, &s_abort);
    }
    __syncthreads();
    if (s_abort) break;
  }
}

// Resident CTAs per SM of a kernel with `smem` bytes of dynamic shared
// memory: the attribute and the occupancy are per device, set and measured
// once per device.
template <typename Kern>
igafd_status per_sm_of(Kern kern, int block, size_t smem, std::atomic<unsigned long long> &set,
                       std::atomic<int> *per_sm, int *out) {
  int dev = 0;
  IGAFD_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(set.load() & bit)) {
    IGAFD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nb = 0;
    IGAFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, smem));
    per_sm[dev & 63].store(nb > 0 ? nb : 1);
    set.fetch_or(bit);
  }
  *out = per_sm[dev & 63].load();
  return IGAFD_OK;
}

// One launch of the single-problem kernel, or with grid_out only its grid
// (the resident CTAs of every SM, at most grid_cap).
template <int DIM, int P, int MODE, int kStages, int R>
igafd_status launch_one(const StencilArgs &a, long long grid_cap, int num_sms, cudaStream_t s,
                        long long *grid_out) {
  const size_t smem = (size_t)kStages * Geom<P>::STAGE * sizeof(double) + 2 * kStages * sizeof(uint64_t);
  constexpr int kBlock = kTile / R + 32;
  auto kern = stencil_tma_kernel<DIM, P, MODE, kStages, R>;
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

template <int DIM, int P, int MODE>
igafd_status launch_stages(int stages, int rows, const StencilArgs &a, long long cap, int sms,
                           cudaStream_t s, long long *grid_out) {
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

// ---- batched launches (one persistent launch for many problems) ----------
template <int DIM, int P, int MODE, int R>
igafd_status batch_launch_one(const StencilArgs *args, const int *act_idx, const long long *act_start,
                              const int *act_count, int sel, unsigned long long *queue, int num_sms,
                              cudaStream_t s) {
  constexpr int kStages = kStagesDefault;
  const size_t smem = (size_t)kStages * Geom<P>::STAGE * sizeof(double) + 2 * kStages * sizeof(uint64_t);
  constexpr int kBlock = kTile / R + 32;
  auto kern = stencil_batch_kernel<DIM, P, MODE, kStages, R>;
  static std::atomic<unsigned long long> attr_set{0};
  static std::atomic<int> per_sm_tab[64];
  int per_sm = 1;
  IGAFD_TRY(per_sm_of(kern, kBlock, smem, attr_set, per_sm_tab, &per_sm));
  const unsigned grid = (unsigned)(num_sms * per_sm);
  IGAFD_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
  kern<<<grid, kBlock, smem, s>>>(args, act_idx, act_start, act_count, sel, queue);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

template <int DIM, int MODE>
igafd_status batch_launch_p(int p, int rows, const StencilArgs *args, const int *ai,
                            const long long *as, const int *ac, int sel, unsigned long long *queue,
                            int sms, cudaStream_t s) {
#define IGAFD_BATCH_P(PP)                                                              \
  case PP:                                                                              \
    if (DIM == 3 && rows == 2)                                                          \
      return batch_launch_one<DIM, PP, MODE, 2>(args, ai, as, ac, sel, queue, sms, s); \
    return batch_launch_one<DIM, PP, MODE, 1>(args, ai, as, ac, sel, queue, sms, s);
  switch (p) {
    IGAFD_BATCH_P(1)
    IGAFD_BATCH_P(2)
    IGAFD_BATCH_P(3)
    IGAFD_BATCH_P(4)
    IGAFD_BATCH_P(5)
    IGAFD_BATCH_P(6)
    IGAFD_BATCH_P(7)
    default: return IGAFD_ERR_ARG;
  }
#undef IGAFD_BATCH_P
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
  a.Np = P->Np;
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
  const int st = P->stencil_stages > 0 ? P->stencil_stages : kStagesDefault;
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
  const int st = P->stencil_stages > 0 ? P->stencil_stages : kStagesDefault;
  const int rows = P->dim == 3 && P->stencil_rows == 2 ? 2 : 1;
  if (P->dim == 3) {
    if (sel) return launch_p<3, 1>(P->p, st, rows, a, cap, P->num_sms, nullptr, vgrid);
    return launch_p<3, 0>(P->p, st, rows, a, cap, P->num_sms, nullptr, vgrid);
  }
  if (sel) return launch_p<2, 1>(P->p, st, 1, a, cap, P->num_sms, nullptr, vgrid);
  return launch_p<2, 0>(P->p, st, 1, a, cap, P->num_sms, nullptr, vgrid);
}

// One persistent launch over the listed (unfinished) problems of one class
// (dim, p, rows per thread): args_dev [members] StencilArgs, act_* the
// pass's list (see stencil_batch_kernel).
igafd_status igafd_stencil_batch_launch(int dim, int p, int rows, int sel, const void *args_dev,
                                        const int *act_idx, const long long *act_start,
                                        const int *act_count, unsigned long long *queue,
                                        int num_sms, cudaStream_t s) {
  const StencilArgs *args = (const StencilArgs *)args_dev;
  if (dim == 3) {
    if (sel) return batch_launch_p<3, 1>(p, rows, args, act_idx, act_start, act_count, sel, queue, num_sms, s);
    return batch_launch_p<3, 0>(p, rows, args, act_idx, act_start, act_count, sel, queue, num_sms, s);
  }
  if (sel) return batch_launch_p<2, 1>(p, 1, args, act_idx, act_start, act_count, sel, queue, num_sms, s);
  return batch_launch_p<2, 0>(p, 1, args, act_idx, act_start, act_count, sel, queue, num_sms, s);
}
