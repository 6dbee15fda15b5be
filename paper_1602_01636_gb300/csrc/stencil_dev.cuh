// Device code shared by the single-problem and batched stencil kernels:
// the stencil layout, the arguments, the per-CTA pipeline and the ring set-up.
#pragma once
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
  // half-stored stencil (the HALF kernels): S is [(n_off + 1) / 2][Np] with
  // Np the row stride, offsets from oc (the centre) up, row i at shH + i
  int oc;
  long long shH;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

template <int P, bool HALF = false>
struct Geom {
  static constexpr int W = 2 * P + 1;
  // coefficient run stride in a ring stage: a tile, or (half-stored stencil)
  // a tile and two rows, so that a mirrored run can start one row early
  static constexpr int RS = HALF ? kTile + 2 : kTile;
  static constexpr int XW = (kTile + 2 * P + 2 + 1) & ~1;   // x window (even count)
  static constexpr int STAGE = W * RS + XW;                  // doubles per ring stage
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
//
// HALF: the stencil is stored by its symmetry (offsets from the centre up).
// The run of a stored offset o is S[o - oc][shH + row0 ...]; the run of an
// offset o below the centre (delta < 0) is the mirrored offset's run shifted
// by off(delta) rows, S[mirror(o) - oc][shH + row0 + off ...], fetched from
// the even row at or before its start so that every bulk copy is 16-byte
// aligned; every run is RS = kTile + 2 rows long and the compute warps read a
// mirrored run one row later when its start was odd.
template <int DIM, int P, int MODE, int kStages, int R, bool HALF = false>
__device__ __forceinline__ void stencil_cta(const StencilArgs &a, long long vb, long long vgrid,
                                            double *ring, uint64_t *full, uint64_t *empty,
                                            long long &gstage, volatile int *s_abort) {
  using Gm = Geom<P, HALF>;
  constexpr int W = Gm::W;
  constexpr int RS = Gm::RS;
  constexpr int NOFF = DIM == 3 ? W * W * W : W * W;
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
        if constexpr (!HALF) {
          for (int d1 = 0; d1 < W; ++d1)
            bulk_g2s(st + d1 * kTile, a.S + (size_t)(ob + d1) * a.Np + row0, kTile * sizeof(double),
                     bar);
        } else {
          for (int d1 = 0; d1 < W; ++d1) {
            const int o = ob + d1;
            long long start = a.shH + row0;
            int arr = o - a.oc;
            if (o < a.oc) {                                 // delta < 0: the mirrored run
              arr = NOFF - 1 - o - a.oc;
              start += (d1 - P) + (long long)d2 * a.n1 + (long long)d3 * n12;
            }
            start -= (start & 1);
            bulk_g2s(st + d1 * RS, a.S + (size_t)arr * a.Np + start, RS * sizeof(double), bar);
          }
        }
        bulk_g2s(st + W * RS, a.x + x0, Gm::XW * sizeof(double), bar);
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
      // HALF: run j of this group starts one row late when it is mirrored and
      // its start row was odd
      int hs[W];
#pragma unroll
      for (int j = 0; j < W; ++j) hs[j] = 0;
      if constexpr (HALF) {
        const int ob = (DIM == 3 ? (d3 + P) * W * W : 0) + (d2 + P) * W;
        const long long pb = a.shH + row0 + (long long)d2 * a.n1 + (long long)d3 * n12 - P;
#pragma unroll
        for (int j = 0; j < W; ++j) hs[j] = ob + j < a.oc ? (int)((pb + j) & 1) : 0;
      }
      if (__any_sync(0xffffffffu, in23)) {
        if constexpr (R == 1) {
          const double *cf = st + tid;
          const double *xw = st + W * RS + tid + sh;      // xw[j] = x[row + off - P + j]
#pragma unroll
          for (int j = 0; j < W; ++j) acc[0] = fma(cf[j * RS + hs[j]], xw[j], acc[0]);
        } else if constexpr (HALF) {
          // rows row, row + 1: coefficients st[j RS + 2 tid + hs[j]] and the next;
          // x[row + off - P + j] = xv[j + sh], x[row + 1 + off - P + j] = xv[j + 1 + sh]
          const double *cf = st + 2 * tid;
          const double2 *xb = reinterpret_cast<const double2 *>(st + W * RS + 2 * tid);
          constexpr int NP = (W + 1) / 2;
          double xv[2 * NP + 2];
#pragma unroll
          for (int m = 0; m < NP + 1; ++m) { const double2 v = xb[m]; xv[2 * m] = v.x; xv[2 * m + 1] = v.y; }
          // two 8-byte loads per run (no branch on the shift, so all of the
          // group's loads issue together)
          double c0[W], c1[W];
#pragma unroll
          for (int j = 0; j < W; ++j) {
            c0[j] = cf[j * RS + hs[j]];
            c1[j] = cf[j * RS + hs[j] + 1];
          }
#pragma unroll
          for (int j = 0; j < W; ++j) {
            acc[0] = fma(c0[j], xv[j + sh], acc[0]);
            acc[1] = fma(c1[j], xv[j + 1 + sh], acc[1]);
          }
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

}  // namespace
