// Fast-diagonalization apply on the 5th-generation tensor cores (tcgen05),
// operands in TF32, BF16 or FP16, FP32 accumulation in tensor memory.
//
// Algorithm 3 (Algorithm 1 in 2D) is run as 2d mode products, each a GEMM
//   out[j][m] = sum_i in[m][i] * B[j][i]
// over the tensor viewed as rows m (the other directions) by the contracted
// direction i, which is always the fastest one: every product writes its
// result transposed (new index slowest), so the next direction to contract
// becomes the contiguous one. After the d forward products the layout is the
// original one again (the divide by D_1 (+) D_2 (+) D_3 is fused there), and
// likewise after the d backward products. Forward products use
// B = U_k^T (out_j = sum_i U_k[i][j] in_i), backward ones B = U_k.
//
// Per CTA: a 128-row tile of `in`; K is walked in 64-element chunks through a
// two-stage shared-memory ring in the canonical K-major 128-byte-swizzled
// layout; one thread issues tcgen05.mma (M = 128, N = n_k padded to 16) into
// a TMEM accumulator; eight warps read it back (tcgen05.ld) and store the
// transposed, rescaled result. Intermediates are FP32 in global memory;
// operands are rounded to the chosen type when they are staged. FP16
// operands use a power-of-two scale per tile (and per U_k) so that nothing
// overflows; the scales are removed exactly in the epilogue.
#include "common.cuh"

#include <atomic>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <vector>

namespace {

constexpr int kM = 128;          // rows per tile (MMA M)
constexpr int kKC = 64;          // K elements per stage
constexpr int kThreads = 256;
constexpr long long kSpin = 1ll << 26;

enum OpType { OP_TF32 = 0, OP_BF16 = 1, OP_FP16 = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// SM100 shared-memory matrix descriptor, K-major, 128-byte swizzle:
// start >> 4 in [0,14), LBO >> 4 in [16,30) (unused for this layout),
// SBO >> 4 in [32,46) (1024 B between 8-row groups), version 1 in [46,48),
// layout 2 (SWIZZLE_128B) in [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Byte offset of (row, kbyte) in a K-major tile of `rows` rows stored as
// 128-byte K atoms [katom][row][128 B], 16-byte chunks XOR-swizzled by row%8.
__device__ __forceinline__ uint32_t sw128_off(int row, int kbyte, int rows) {
  const int katom = kbyte >> 7, kb = kbyte & 127, chunk = kb >> 4;
  return katom * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 +
         (((chunk ^ (row & 7)) << 4) | (kb & 15));
}

// FP64 <-> FP32 by integer operations on the IEEE-754 bit fields (on GB300
// the conversion instructions issue on the FP64 pipe, two per clock per SM,
// which would make them the bottleneck of the staging and of the FP64 store).
// f64_to_f32 truncates the mantissa (below the operand rounding that follows)
// and flushes magnitudes under 2^-126 to zero; f32_to_f64 is exact for
// normal numbers and flushes subnormals to zero. Infinities and NaNs are kept.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u, ed = (hi >> 20) & 0x7ffu;
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const int e = (int)ed - 896;
  unsigned r;
  if (ed == 0x7ffu) r = sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
  else if (e >= 255) r = sign | 0x7f800000u;
  else if (e <= 0) r = sign;
  else r = sign | ((unsigned)e << 23) | mant;
  return __uint_as_float(r);
}
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi = sign, lo = 0u;
  if (e == 0xffu) { hi = sign | 0x7ff00000u | (m >> 3); lo = m << 29; }
  else if (e != 0u) { hi = sign | ((e + 896u) << 20) | (m >> 3); lo = m << 29; }
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
// TF32 (10-bit mantissa) rounding to nearest, ties away from zero, on the bits
__device__ __forceinline__ uint32_t tf32_bits(float v) {
  return (__float_as_uint(v) + 0x1000u) & 0xffffe000u;
}

template <int OP> struct Op;
template <> struct Op<OP_TF32> {
  static constexpr int kBytes = 4;
  static constexpr uint32_t kFmt = 2;
  // round to nearest TF32 (the MMA would otherwise drop the low mantissa bits)
  __device__ static void put(unsigned char *p, float v) { *(uint32_t *)p = tf32_bits(v); }
};
template <> struct Op<OP_BF16> {
  static constexpr int kBytes = 2;
  static constexpr uint32_t kFmt = 1;
  __device__ static void put(unsigned char *p, float v) { *(__nv_bfloat16 *)p = __float2bfloat16_rn(v); }
};
template <> struct Op<OP_FP16> {
  static constexpr int kBytes = 2;
  static constexpr uint32_t kFmt = 0;
  __device__ static void put(unsigned char *p, float v) { *(__half *)p = __float2half_rn(v); }
};

struct PassArgs {
  const void *in;        // [M][K] (double for the first pass, float otherwise)
  int in_f64;
  int in_aligned;        // `in` is 16-byte aligned (vector loads allowed)
  void *out;             // [N][M] (double for the last pass, float otherwise)
  int out_f64;
  const unsigned char *Bimg;  // B = U_k^T (forward) or U_k, pre-staged: per K chunk the
                              // exact shared-memory image of the B stage
  const float *b_scale;  // device: power of two folded into the FP16 image of B (null: 1)
  const float *inv_lam;  // divide epilogue (null: none), indexed like out
  long long M;
  int K, N, Np;          // Np: N padded to a multiple of 16 (MMA N)
  int tmem_cols;
  const double *done;    // skip when *done != 0
  int *err;
  // tile shape (autotuned): rows of the input per CTA (128, or 64 with the
  // 128-row MMA on a half-filled A tile), output columns per CTA (a multiple
  // of 16; grid.y covers Np), and K stages in the shared-memory ring (2 or 3)
  int m_tile, n_tile, stages;
};

template <int OP>
__global__ void __launch_bounds__(kThreads) tc_pass_kernel(PassArgs a) {
  pdl_wait();
  pdl_trigger();
  if (a.done && *a.done != 0.0) return;
  using T = Op<OP>;
  constexpr int kRowBytes = kKC * T::kBytes;                 // bytes of one stage row
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = a.stages;                                    // 2 or 3
  const int n0 = (int)blockIdx.y * a.n_tile;                 // first output column of this CTA
  const int nN = a.Np - n0 < a.n_tile ? a.Np - n0 : a.n_tile; // its columns (multiple of 16)
  const int stageA = kM * kRowBytes;                         // multiple of 1024
  const int stageB = nN * kRowBytes;
  const int stageStride = stageA + a.n_tile * kRowBytes;     // multiple of 1024
  unsigned char *sA[3], *sB[3];
  for (int st = 0; st < 3; ++st) {
    sA[st] = base + st * stageStride;
    sB[st] = sA[st] + stageA;
  }
  __shared__ uint64_t bar[3];     // MMA completion per stage
  __shared__ uint64_t bbar[3];    // B-image bulk copy per stage
  __shared__ uint32_t tmem_base;
  __shared__ float s_red[kThreads / 32];
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.x * a.m_tile;
  const int mrows = (int)((a.M - m0) < a.m_tile ? (a.M - m0) : a.m_tile);
  const int K = a.K;
  const int nchunks = (K + kKC - 1) / kKC;

  // per-tile power-of-two scale for FP16 operands
  float a_scale = 1.0f;
  if (OP == OP_FP16) {
    float mx = 0.0f;
    for (int i = tid; i < mrows * K; i += kThreads) {
      const long long idx = (m0 + i / K) * K + i % K;
      const float v = a.in_f64 ? f64_to_f32(((const double *)a.in)[idx]) : ((const float *)a.in)[idx];
      mx = fmaxf(mx, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      float m = 0.0f;
      for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, s_red[w]);
      s_red[0] = m;
    }
    __syncthreads();
    const float m = s_red[0];
    // largest power of two with m * scale <= 2^14
    a_scale = m > 0.0f ? exp2f(14.0f - ceilf(log2f(m))) : 1.0f;
  }

  if (tid == 0) {
    for (int st = 0; st < 3; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[st])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bbar[st])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (T::kFmt << 7) | (T::kFmt << 10) |
                         ((uint32_t)(nN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

  auto wait_on = [&](uint64_t *b, uint32_t parity) -> bool {
    for (long long it = 0; it < kSpin; ++it) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_u32(b)), "r"(parity)
          : "memory");
      if (ok) return true;
    }
    return false;
  };
  auto wait_bar = [&](int st, uint32_t parity) -> bool { return wait_on(&bar[st], parity); };

  for (int c = 0; c < nchunks; ++c) {
    const int st = c % S;
    if (c >= S) {   // the MMAs that read this stage S chunks ago must be done
      if (!wait_bar(st, (uint32_t)(((c - S) / S) & 1))) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
    }
    const int k0 = c * kKC;
    // stage B: rows n0 .. n0 + nN of the pre-staged image of this K chunk, one
    // bulk copy per 128-byte K atom (the image is [atom][Np rows][128 B]; the
    // rows of a tile starting at a multiple of 8 keep their swizzle phase)
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)stageB;
      constexpr int kAtoms = kRowBytes / 128;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bbar[st])),
                   "r"(bytes)
                   : "memory");
      for (int at = 0; at < kAtoms; ++at)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sB[st] + at * nN * 128)),
            "l"(a.Bimg + (size_t)c * a.Np * kRowBytes + (size_t)at * a.Np * 128 + (size_t)n0 * 128),
            "r"((uint32_t)(nN * 128)), "r"(smem_u32(&bbar[st]))
            : "memory");
    }
    // stage A: warp w takes rows 16w..16w+15, lane l columns k0+2l, k0+2l+1;
    // all sixteen loads are issued before the swizzled, rounded stores
    {
      float2 v[16];
      const bool vec = a.in_aligned && (K % 2 == 0) && (k0 + kKC <= K);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int rr = warp * 16 + i;
        const int k = k0 + 2 * lane;
        v[i] = make_float2(0.f, 0.f);
        if (rr < mrows) {
          const long long idx = (m0 + rr) * K + k;
          if (vec) {
            if (a.in_f64) {
              const double2 d = *reinterpret_cast<const double2 *>((const double *)a.in + idx);
              v[i] = make_float2(f64_to_f32(d.x), f64_to_f32(d.y));
            } else {
              v[i] = *reinterpret_cast<const float2 *>((const float *)a.in + idx);
            }
          } else {
            if (k < K) v[i].x = a.in_f64 ? f64_to_f32(((const double *)a.in)[idx]) : ((const float *)a.in)[idx];
            if (k + 1 < K)
              v[i].y = a.in_f64 ? f64_to_f32(((const double *)a.in)[idx + 1]) : ((const float *)a.in)[idx + 1];
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int rr = warp * 16 + i;
        T::put(sA[st] + sw128_off(rr, (2 * lane) * T::kBytes, kM), v[i].x * a_scale);
        T::put(sA[st] + sw128_off(rr, (2 * lane + 1) * T::kBytes, kM), v[i].y * a_scale);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!wait_on(&bbar[st], (uint32_t)((c / S) & 1))) s_fail = 1;
    }
    if (tid == 0 && !s_fail) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int ksteps = kRowBytes / 32;          // 32 bytes of K per MMA
      for (int ks = 0; ks < ksteps; ++ks) {
        const int kbyte = ks * 32;
        const uint32_t ao = (kbyte >> 7) * kM * 128 + (kbyte & 127);
        const uint32_t bo = (kbyte >> 7) * nN * 128 + (kbyte & 127);
        const uint64_t ad = sw128_desc(smem_u32(sA[st]) + ao);
        const uint64_t bd = sw128_desc(smem_u32(sB[st]) + bo);
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        if (OP == OP_TF32)
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bar[st]))
          : "memory");
    }
  }
  // wait for the last MMAs (the commits track all earlier ones too)
  bool ok = !s_fail;
  if (ok && nchunks > 0) {
    const int last = nchunks - 1;
    ok = wait_bar(last % S, (uint32_t)((last / S) & 1));
    if (!ok) s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_fail) {
    // epilogue: warp w reads TMEM lanes 32*(w%4).. and columns of half w/4
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;                  // row within the tile
    const long long m = m0 + r;
    const float unscale = 1.0f / (a_scale * (a.b_scale ? *a.b_scale : 1.0f));
    const int ncol32 = (nN + 31) / 32;
    for (int cb = half; cb < ncol32; cb += 2) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < mrows) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + cb * 32 + j;
          if (cb * 32 + j < nN && n < a.N) {
            const long long o = (long long)n * a.M + m;
            float val = __uint_as_float(v[j]) * unscale;
            if (a.inv_lam) val *= a.inv_lam[o];
            if (a.out_f64) ((double *)a.out)[o] = f32_to_f64(val);
            else ((float *)a.out)[o] = val;
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(a.err, (int)IGAFD_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
}

// U32_k = (float) U_k and D32_k = (float) D_k for every direction (grid.y =
// direction) and the bit pattern of max |U32_k| (non-negative floats order
// like their bits) into umax[k] (zeroed before the launch)
struct U32Args {
  const double *U[3], *D[3];
  float *U32[3], *D32[3];
  int n[3];
  unsigned *umax;
};
__global__ void u32_kernel(U32Args a) {
  const int k = blockIdx.y;
  const int n = k == 0 ? a.n[0] : k == 1 ? a.n[1] : a.n[2];
  const double *U = k == 0 ? a.U[0] : k == 1 ? a.U[1] : a.U[2];
  float *V = k == 0 ? a.U32[0] : k == 1 ? a.U32[1] : a.U32[2];
  const int first = blockIdx.x * blockDim.x + threadIdx.x;
  if (first < n) {
    const double *D = k == 0 ? a.D[0] : k == 1 ? a.D[1] : a.D[2];
    float *D32 = k == 0 ? a.D32[0] : k == 1 ? a.D32[1] : a.D32[2];
    D32[first] = (float)D[first];
  }
  unsigned mx = 0u;
  for (int i = first; i < n * n; i += gridDim.x * blockDim.x) {
    const float v = f64_to_f32(U[i]);
    V[i] = v;
    const unsigned b = __float_as_uint(v) & 0x7fffffffu;
    mx = b > mx ? b : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned w = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = w > mx ? w : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(&a.umax[k], mx);
}

// FP16 staging scale of U_k from max |U_k|: the largest power of two with
// max |U_k| * scale <= 2^14
__device__ __forceinline__ float fp16_scale(unsigned maxbits) {
  const float m = __uint_as_float(maxbits);
  return m > 0.0f ? exp2f(14.0f - ceilf(log2f(m))) : 1.0f;
}


// Shared-memory images of B for every K chunk, one job per (direction,
// forward/backward, operand type): B = U_k^T (forward) or U_k (backward),
// U_k row-major FP32; rows padded to Np and K to whole chunks with zeros,
// rounded to the operand type, FP16 scaled by a power of two, in the
// swizzled stage layout.
struct ImgJob {
  const float *U;
  int n, Np, op, transpose;
  const unsigned *umax;     // FP16: bit pattern of max |U| (the scale follows); null: scale 1
  float *scale;             // FP16: where the scale is recorded for the epilogue
  unsigned char *img;
};
struct ImgBatch {
  ImgJob j[18];
};

__global__ void b_image_kernel(ImgBatch b) {
  const ImgJob J = b.j[blockIdx.y];
  const int n = J.n, Np = J.Np;
  const int nchunks = (n + kKC - 1) / kKC;
  const long long total = (long long)nchunks * Np * kKC;
  const float scale = J.umax ? fp16_scale(*J.umax) : 1.0f;
  if (J.scale && blockIdx.x == 0 && threadIdx.x == 0) *J.scale = scale;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(i % kKC);
    const int r = (int)((i / kKC) % Np);
    const int c = (int)(i / ((long long)kKC * Np));
    const int k = c * kKC + kk;
    float v = 0.0f;
    if (r < n && k < n) v = (J.transpose ? J.U[(size_t)k * n + r] : J.U[(size_t)r * n + k]) * scale;
    if (J.op == OP_TF32)
      Op<OP_TF32>::put(J.img + (size_t)c * Np * kKC * 4 + sw128_off(r, kk * 4, Np), v);
    else if (J.op == OP_BF16)
      Op<OP_BF16>::put(J.img + (size_t)c * Np * kKC * 2 + sw128_off(r, kk * 2, Np), v);
    else
      Op<OP_FP16>::put(J.img + (size_t)c * Np * kKC * 2 + sw128_off(r, kk * 2, Np), v);
  }
}

// ---------------------------------------------------------------------------
// Fused FD for n_k <= 128 with TF32 or BF16 operands: three kernels, each CTA
// running two dependent MMAs with the intermediate passed from TMEM through
// shared memory (never through global memory):
//   SLAB_FWD  (one CTA per slab i3):  Y = X_s U1 (lanes i2, cols j1), then
//             Z^T = Y^T U2 (lanes j1, cols j2): writes T[i3][j2][j1]
//             (2D: the whole tensor is one slab and the divide is fused here)
//   PENCIL    (one CTA per 128 columns c = (j2, j1)): D = T^T U3 (lanes c,
//             cols j3), divide by D1 (+) D2 (+) D3, then Z = D U3^T (lanes c,
//             cols i3): writes T2[i3][c]
//   SLAB_BWD  (one CTA per slab): Y = T2_s U1^T (lanes j2, cols i1), then
//             Z^T = Y^T U2^T (lanes i1, cols i2): writes z[i3][i2][i1] (FP64)
// The accumulator lanes of the second MMA are always the contiguous index of
// the output, so every global store is coalesced.
enum FusedKind { SLAB_FWD = 0, PENCIL = 1, SLAB_BWD = 2 };

struct FusedArgs {
  const void *in;            // SLAB_FWD: r (double); others: float
  int in_f64, in_aligned;
  void *out;                 // SLAB_BWD: z (double); others: float
  int out_f64;
  const unsigned char *B1, *B2;   // images of the first / second B operand
  int Np1, Np2;              // their rows (N of each MMA, multiple of 16)
  int K1, K2;                // contraction lengths (valid)
  int Kp1, Kp2;              // the same padded to whole 64-element chunks (the images' K)
  int Kpad;                  // max(Kp1, Kp2): sizes the shared-memory regions
  int rowsA;                 // valid rows of the first A operand (lanes)
  int n1, n2, n3;
  long long n12;
  const float *inv_lam;      // divide of SLAB_FWD in 2D (null: none)
  const float *d1, *d2, *d3; // PENCIL: FP32 D_k, divided by d1 + d2 + d3 on the fly
  const double *done;
  int *err;
  int ctile;                 // PENCIL: columns per CTA, 128 or 64 (a half-filled MMA tile; autotuned)
};

// Pack E = 16 / kBytes operand values into one 16-byte chunk of the
// swizzled layout (the values are consecutive K elements of one row).
template <int OP> __device__ __forceinline__ uint4 pack_chunk(const float *v);
template <> __device__ __forceinline__ uint4 pack_chunk<OP_TF32>(const float *v) {
  uint32_t t[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) t[e] = tf32_bits(v[e]);
  return make_uint4(t[0], t[1], t[2], t[3]);
}
template <> __device__ __forceinline__ uint4 pack_chunk<OP_BF16>(const float *v) {
  uint32_t t[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    t[e] = *reinterpret_cast<uint32_t *>(&h);
  }
  return make_uint4(t[0], t[1], t[2], t[3]);
}

// Stage A[r][k] = in[(row0 + r) * K + k] (r < rowsA, k < K, zero elsewhere)
// as a K-major swizzled operand of kM rows and Kp columns. Each thread owns
// one 16-byte chunk (E consecutive k of a row) per step, issues the loads of
// U chunks before storing any, and stores each chunk with one 16-byte write:
// consecutive threads take consecutive chunks of a row, so global loads are
// coalesced and the eight threads of a store phase hit eight distinct banks.
template <int OP>
__device__ void stage_rows(unsigned char *R, const void *in, int in_f64, long long row0,
                           int rowsA, int K, int Kp, int aligned, int tid) {
  constexpr int E = 16 / Op<OP>::kBytes;
  constexpr int U = 32 / E;
  const int cpr = Kp / E;
  const int total = kM * cpr;
  const bool vec = aligned && (in_f64 ? (K % 2 == 0) : (K % 4 == 0));
  for (int b0 = 0; b0 < total; b0 += kThreads * U) {
    float v[U][E];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int id = b0 + u * kThreads + tid;
      const int r = id / cpr, k0 = (id - r * cpr) * E;
      const bool rowok = id < total && r < rowsA;
      const long long g = (row0 + r) * K + k0;
      if (in_f64) {
        const double *src = (const double *)in + g;
        if (vec) {
#pragma unroll
          for (int e = 0; e < E; e += 2) {
            double2 d = make_double2(0.0, 0.0);
            if (rowok && k0 + e < K) d = __ldg(reinterpret_cast<const double2 *>(src + e));
            v[u][e] = f64_to_f32(d.x);
            v[u][e + 1] = f64_to_f32(d.y);
          }
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) v[u][e] = (rowok && k0 + e < K) ? f64_to_f32(__ldg(src + e)) : 0.0f;
        }
      } else {
        const float *src = (const float *)in + g;
        if (vec) {
#pragma unroll
          for (int e = 0; e < E; e += 4) {
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rowok && k0 + e < K) f = __ldg(reinterpret_cast<const float4 *>(src + e));
            v[u][e] = f.x; v[u][e + 1] = f.y; v[u][e + 2] = f.z; v[u][e + 3] = f.w;
          }
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) v[u][e] = (rowok && k0 + e < K) ? __ldg(src + e) : 0.0f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int id = b0 + u * kThreads + tid;
      if (id < total) {
        const int r = id / cpr, k0 = (id - r * cpr) * E;
        *reinterpret_cast<uint4 *>(R + sw128_off(r, k0 * Op<OP>::kBytes, kM)) = pack_chunk<OP>(v[u]);
      }
    }
  }
}

// Stage A[c][k] = in[k * n12 + c0 + c] (c0 + c < n12, k < K, zero elsewhere):
// the transpose of a block of 128 columns. A thread loads E consecutive k
// at one c (each load instruction of a warp reads 32 consecutive c) and
// writes them as one chunk of row c; a store phase covers eight consecutive
// rows, whose swizzle puts the chunk in eight distinct banks.
template <int OP>
__device__ void stage_cols(unsigned char *R, const float *in, long long n12, long long c0, int K,
                           int Kp, int aligned, int tid, int ctile) {
  (void)aligned;
  constexpr int E = 16 / Op<OP>::kBytes;
  constexpr int U = 32 / E;
  const int total = kM * (Kp / E);
  for (int b0 = 0; b0 < total; b0 += kThreads * U) {
    float v[U][E];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int id = b0 + u * kThreads + tid;
      const int c = id % kM, k0 = (id / kM) * E;
      const bool ok = id < total && c0 + c < n12 && c < ctile;
      const float *src = in + (long long)k0 * n12 + c0 + c;
#pragma unroll
      for (int e = 0; e < E; ++e) v[u][e] = (ok && k0 + e < K) ? __ldg(src + (long long)e * n12) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int id = b0 + u * kThreads + tid;
      if (id < total) {
        const int c = id % kM, k0 = (id / kM) * E;
        *reinterpret_cast<uint4 *>(R + sw128_off(c, k0 * Op<OP>::kBytes, kM)) = pack_chunk<OP>(v[u]);
      }
    }
  }
}

// CTA resources of the fused kernels: the two mbarriers (B image copies, MMA
// completions; each completes twice per block, so every block waits on
// parities 0 then 1) and 128 TMEM columns, set up once per CTA.
__device__ __forceinline__ void fused_init(uint64_t *bar_mma, uint64_t *bar_b, uint32_t *tmem_slot,
                                           int *s_fail) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_mma)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_b)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_fail = 0;
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Release of the TMEM columns (after the last block's epilogue, which ends
// with a CTA barrier).
__device__ __forceinline__ void fused_fini(uint32_t tmem) {
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// One block (CTA tile) of a fused kernel on the CTA's resources; false when a
// wait ran out (the error is recorded and the CTA must stop: its barriers'
// phases are then unknown).
template <int OP, int KIND>
__device__ __forceinline__ bool tc_fused_item(const FusedArgs &a, const int blk, const uint32_t tmem,
                                              uint64_t *bar_mma_p, uint64_t *bar_b_p,
                                              int *s_fail_p) {
  using T = Op<OP>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int rowBytes = a.Kpad * T::kBytes;              // bytes of K per row
  unsigned char *R1 = base;                              // A operands: 128 rows
  unsigned char *R2 = base + (size_t)kM * rowBytes;      // B operands: up to 128 rows
  uint64_t &bar_mma = *bar_mma_p, &bar_b = *bar_b_p;
  int &s_fail = *s_fail_p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  auto wait_on = [&](uint64_t *b, uint32_t parity) -> bool {
    for (long long it = 0; it < kSpin; ++it) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_u32(b)), "r"(parity)
          : "memory");
      if (ok) return true;
    }
    return false;
  };
  auto load_b = [&](const unsigned char *img, int Np, int Kp) {
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)(Np * Kp * T::kBytes);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_b)),
                   "r"(bytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(R2)),
          "l"(img), "r"(bytes), "r"(smem_u32(&bar_b))
          : "memory");
    }
  };
  auto mma = [&](int Np, int Kp, uint32_t tmem) {
    const uint32_t idesc = (1u << 4) | (T::kFmt << 7) | (T::kFmt << 10) |
                           ((uint32_t)(Np >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int ksteps = Kp * T::kBytes / 32;     // 32 bytes of K per MMA
    for (int ks = 0; ks < ksteps; ++ks) {
      const int kbyte = ks * 32;
      const uint64_t ad = sw128_desc(smem_u32(R1) + (kbyte >> 7) * kM * 128 + (kbyte & 127));
      const uint64_t bd = sw128_desc(smem_u32(R2) + (kbyte >> 7) * Np * 128 + (kbyte & 127));
      const uint32_t acc = ks > 0 ? 1u : 0u;
      if (OP == OP_TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&bar_mma))
        : "memory");
  };
  // read 32 TMEM columns [c0, c0+32) of this warp's lane quarter
  auto tmem_ld32 = [&](uint32_t tmem, int q, int c0, uint32_t *v) {
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  };

  load_b(a.B1, a.Np1, a.Kp1);

  // ---- first A operand: rows = lanes of the first accumulator ----
  const int ctile = KIND == PENCIL && a.ctile == 64 ? 64 : kM;
  if (KIND == PENCIL)
    stage_cols<OP>(R1, (const float *)a.in, a.n12, (long long)blk * ctile, a.K1, a.Kp1, a.in_aligned,
                   tid, ctile);
  else
    stage_rows<OP>(R1, a.in, a.in_f64, (long long)blk * a.n2, a.rowsA, a.K1, a.Kp1, a.in_aligned, tid);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    if (!wait_on(&bar_b, 0)) s_fail = 1;
    else mma(a.Np1, a.Kp1, tmem);
  }
  __syncthreads();
  if (!s_fail && !wait_on(&bar_mma, 0)) s_fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int q = warp & 3, half = warp >> 2;
  const int lane_row = q * 32 + lane;              // accumulator lane of this thread
  if (!s_fail) {
    // second B image into R2 (the first MMA is done with it)
    load_b(a.B2, a.Np2, a.Kp2);
    // zero R1, then write the second A operand from the first accumulator
    const int row2 = a.Kp2 * T::kBytes;
    for (int i = tid; i < kM * row2 / 16; i += kThreads)
      reinterpret_cast<uint4 *>(R1)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int ncol32 = (a.Np1 + 31) / 32;
    // PENCIL: d1[j1] + d2[j2] of this thread's column c = j2 n1 + j1
    const long long cc = (long long)blk * ctile + lane_row;
    const bool c_ok = KIND == PENCIL && cc < a.n12 && lane_row < ctile;
    const float d12 = c_ok ? a.d1[cc % a.n1] + a.d2[cc / a.n1] : 0.0f;
    for (int cb = half; cb < ncol32; cb += 2) {
      uint32_t v[32];
      tmem_ld32(tmem, q, cb * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = cb * 32 + j;
        float x = __uint_as_float(v[j]);
        if (KIND == PENCIL) {
          // divide by D1 (+) D2 (+) D3 at (j3 = col, c = c0 + lane_row); row = lane, k = col
          if (col < a.K2 && c_ok) x = __fdividef(x, d12 + a.d3[col]);
          else x = 0.0f;
          v[j] = __float_as_uint(x);
        } else {
          // row = col (the new lanes), k = lane
          if (col < a.Np1 && lane_row * T::kBytes < row2)
            T::put(R1 + sw128_off(col, lane_row * T::kBytes, kM), lane_row < a.K2 ? x : 0.0f);
        }
      }
      if (KIND == PENCIL) {
        // row = lane, k = the 32 columns: whole 16-byte chunks
        constexpr int E = 16 / T::kBytes;
#pragma unroll
        for (int e0 = 0; e0 < 32; e0 += E) {
          const int k0 = cb * 32 + e0;
          if (k0 * T::kBytes < row2) {
            float f[E];
#pragma unroll
            for (int e = 0; e < E; ++e) f[e] = __uint_as_float(v[e0 + e]);
            *reinterpret_cast<uint4 *>(R1 + sw128_off(lane_row, k0 * T::kBytes, kM)) = pack_chunk<OP>(f);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!wait_on(&bar_b, 1)) s_fail = 1;
      else mma(a.Np2, a.Kp2, tmem);
    }
    __syncthreads();
    if (!s_fail && !wait_on(&bar_mma, 1)) s_fail = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!s_fail) {
    // ---- epilogue: lanes = contiguous output index, columns = strided one ----
    long long obase, ostride;
    int nlanes, ncols;
    if (KIND == PENCIL) {
      obase = (long long)blk * ctile; ostride = a.n12;
      nlanes = (int)((a.n12 - obase) < ctile ? (a.n12 - obase) : ctile); ncols = a.n3;
    } else {
      obase = (long long)blk * a.n12; ostride = a.n1;
      nlanes = a.n1; ncols = a.n2;
    }
    const int ncol32 = (a.Np2 + 31) / 32;
    for (int cb = half; cb < ncol32; cb += 2) {
      uint32_t v[32];
      tmem_ld32(tmem, q, cb * 32, v);
      if (lane_row < nlanes) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = cb * 32 + j;
          if (col < ncols) {
            const long long o = obase + (long long)col * ostride + lane_row;
            float x = __uint_as_float(v[j]);
            if (KIND == SLAB_FWD && a.inv_lam) x *= a.inv_lam[o];
            if (a.out_f64) ((double *)a.out)[o] = f32_to_f64(x);
            else ((float *)a.out)[o] = x;
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(a.err, (int)IGAFD_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  return s_fail == 0;
}

template <int OP, int KIND>
__global__ void __launch_bounds__(kThreads) tc_fused_kernel(FusedArgs a) {
  pdl_wait();
  pdl_trigger();
  if (a.done && *a.done != 0.0) return;
  __shared__ uint64_t bar_mma, bar_b;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  fused_init(&bar_mma, &bar_b, &tmem_slot, &s_fail);
  const uint32_t tmem = tmem_slot;
  tc_fused_item<OP, KIND>(a, blockIdx.x, tmem, &bar_mma, &bar_b, &s_fail);
  fused_fini(tmem);
}

// The same kernel for many problems in one persistent launch: the work items
// are (listed problem k, CTA b of its own launch), act_start[k] <= item <
// act_start[k + 1], over the problems listed in act (indices into args; the
// pass's compaction lists the unfinished ones, largest CTAs first, and zeroes
// *queue). CTAs take items from the queue counter, with the barriers and TMEM
// columns set up once; with a null queue CTA b runs item b only (a grid of
// one CTA per item). Problems whose PCG is done are skipped as in their own
// launch.
constexpr int kFusedListCache = 128;
template <int OP, int KIND>
__global__ void __launch_bounds__(kThreads) tc_fused_batch_kernel(const FusedArgs *args,
                                                                  const int *act,
                                                                  const int *act_start,
                                                                  const int *act_count,
                                                                  unsigned *queue) {
  __shared__ FusedArgs s_a;
  __shared__ int s_st[kFusedListCache + 1];
  __shared__ int s_it, s_lo, s_run;
  __shared__ uint64_t bar_mma, bar_b;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int n = *act_count;
  const int total = n > 0 ? act_start[n] : 0;
  if ((int)blockIdx.x >= total) return;              // uniform over the CTA
  const bool cached = n <= kFusedListCache;
  if (cached)
    for (int k = threadIdx.x; k <= n; k += blockDim.x) s_st[k] = act_start[k];
  fused_init(&bar_mma, &bar_b, &tmem_slot, &s_fail);  // ends with a CTA barrier
  const int *st = cached ? s_st : act_start;
  const uint32_t tmem = tmem_slot;
  int cur = -1;
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) {
      // persistent: items from the queue; otherwise CTA b runs item b only
      const int it = queue ? (int)atomicAdd(queue, 1u) : (first ? (int)blockIdx.x : total);
      int lo = cur < 0 ? 0 : cur, hi = n - 1;       // a CTA's items ascend: search from its current one
      if (it < total)
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (st[mid] <= it) lo = mid; else hi = mid - 1;
        }
      s_it = it;
      s_lo = lo;
    }
    __syncthreads();
    const int it = s_it, lo = s_lo;
    if (it >= total) break;                          // uniform
    if (lo != cur) {
      if (threadIdx.x < 32) {
        const unsigned *src = reinterpret_cast<const unsigned *>(&args[act[lo]]);
        unsigned *dst = reinterpret_cast<unsigned *>(&s_a);
        for (int w = threadIdx.x; w < (int)(sizeof(FusedArgs) / 4); w += 32) dst[w] = src[w];
      }
      __syncthreads();
      if (threadIdx.x == 0) s_run = !(s_a.done && *s_a.done != 0.0);
      cur = lo;
    }
    __syncthreads();
    first = false;
    if (!s_run) continue;                            // uniform
    if (!tc_fused_item<OP, KIND>(s_a, it - st[lo], tmem, &bar_mma, &bar_b, &s_fail)) break;
  }
  fused_fini(tmem);
}

// ---------------------------------------------------------------------------
// Fused FD for n_1 = n_2 = n_3 = 128 (3D): the three kernels of the fused path
// with every size a compile-time constant, 512 threads, both B images fetched
// at the start, and staging, transposition and epilogue addressed through
// per-thread constant swizzle offsets (the generic kernels above spend most
// of their instructions on run-time index arithmetic). Products are those of
// tc_fused_kernel; the slab-forward kernel writes its result as [j2][i3][j1],
// so that the pencil kernel's 128 x 128 input block (j2 = its CTA) is one
// contiguous 64 KB run: a single bulk copy into shared memory and a transpose
// there replace 128 strided row reads from L2.
constexpr int kN = 128;            // dofs per direction on this path
constexpr int kT128 = 512;         // threads per CTA
constexpr int kAtomCol = kN * 128; // bytes of one 128-byte K atom over all 128 rows

// byte offset of (row, kbyte) in a 128-row K-major tile with 128-byte swizzle
__device__ __forceinline__ uint32_t swz128(uint32_t row, uint32_t kbyte) {
  return (kbyte >> 7) * kAtomCol + (row >> 3) * 1024 + (row & 7) * 128 +
         ((((kbyte >> 4) & 7) ^ (row & 7)) << 4) + (kbyte & 15);
}

// FP64 -> operand bits by integer operations on the IEEE-754 fields, rounded
// to nearest (ties away from zero) at the operand's precision; magnitudes
// under 2^-126 flush to zero, above the FP32 range to infinity (NaN kept).
template <int OP> __device__ __forceinline__ uint32_t op_bits_f64(double d);
template <> __device__ __forceinline__ uint32_t op_bits_f64<OP_TF32>(double d) {
  const uint32_t hi = (uint32_t)((unsigned long long)__double_as_longlong(d) >> 32);
  const uint32_t sign = hi & 0x80000000u;
  if (((hi >> 20) & 0x7ffu) == 0x7ffu) return sign | 0x7fc00000u | ((hi & 0xfffffu) ? 0u : 0u);
  const uint32_t mag = (hi & 0x7fffffffu) + 0x200u;          // round at the TF32 mantissa
  const int e = (int)(mag >> 20) - 896;
  if (e <= 0) return sign;
  if (e >= 255) return sign | 0x7f800000u;
  return sign | ((uint32_t)e << 23) | (((mag >> 10) & 0x3ffu) << 13);
}
template <> __device__ __forceinline__ uint32_t op_bits_f64<OP_BF16>(double d) {
  const uint32_t hi = (uint32_t)((unsigned long long)__double_as_longlong(d) >> 32);
  const uint32_t sign = hi & 0x80000000u;
  if (((hi >> 20) & 0x7ffu) == 0x7ffu) return (sign | 0x7fc00000u) >> 16;
  const uint32_t mag = (hi & 0x7fffffffu) + 0x1000u;         // round at the BF16 mantissa
  const int e = (int)(mag >> 20) - 896;
  if (e <= 0) return sign >> 16;
  if (e >= 255) return (sign | 0x7f800000u) >> 16;
  return (sign >> 16) | ((uint32_t)e << 7) | ((mag >> 13) & 0x7fu);
}
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&h);
}

// A[r][k] = src[r * kN + k] (FP64), r, k < 128. Warp w takes half h = w & 1
// of rows g + 8t (g = w >> 1, t < 16): each lane two consecutive elements
// per row, so the row's swizzle term is one constant per thread.
template <int OP>
__device__ __forceinline__ void stage128_rows_f64(unsigned char *R, const double *src, int warp,
                                                  int lane) {
  constexpr int kB = Op<OP>::kBytes;
  const int h = warp & 1, g = warp >> 1;
  const int k = 64 * h + 2 * lane;
  const uint32_t off0 = swz128((uint32_t)g, (uint32_t)(k * kB));
  double2 d[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) d[t] = __ldg(reinterpret_cast<const double2 *>(src + (g + 8 * t) * kN + k));
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    if (OP == OP_TF32)
      *reinterpret_cast<uint2 *>(R + off0 + t * 1024) =
          make_uint2(op_bits_f64<OP_TF32>(d[t].x), op_bits_f64<OP_TF32>(d[t].y));
    else
      *reinterpret_cast<uint32_t *>(R + off0 + t * 1024) =
          op_bits_f64<OP_BF16>(d[t].x) | (op_bits_f64<OP_BF16>(d[t].y) << 16);
  }
}

// A[r][k] = src[r * kN + k] (FP32). Warp w takes rows g + 8 (2t + u) (g = w & 7,
// u = w >> 3, t < 8); each lane four consecutive elements per row.
template <int OP>
__device__ __forceinline__ void stage128_rows_f32(unsigned char *R, const float *src, int warp,
                                                  int lane) {
  constexpr int kB = Op<OP>::kBytes;
  const int g = warp & 7, u = warp >> 3;
  const int k = 4 * lane;
  const uint32_t off0 = swz128((uint32_t)(g + 8 * u), (uint32_t)(k * kB));
  float4 f[8];
#pragma unroll
  for (int t = 0; t < 8; ++t)
    f[t] = __ldg(reinterpret_cast<const float4 *>(src + (g + 8 * (2 * t + u)) * kN + k));
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (OP == OP_TF32)
      *reinterpret_cast<uint4 *>(R + off0 + t * 2048) =
          make_uint4(tf32_bits(f[t].x), tf32_bits(f[t].y), tf32_bits(f[t].z), tf32_bits(f[t].w));
    else
      *reinterpret_cast<uint2 *>(R + off0 + t * 2048) =
          make_uint2(bf16x2_bits(f[t].x, f[t].y), bf16x2_bits(f[t].z, f[t].w));
  }
}

// A[c][k] = raw[k * kN + c] (FP32, the contiguous 128 x 128 block [k][c]
// already in shared memory): the transpose of the block into the K-major
// operand. A warp reads 32 consecutive c of E consecutive k (conflict-free
// 128-byte rows) and writes one 16-byte operand chunk per lane.
template <int OP>
__device__ __forceinline__ void stage128_cols_smem(unsigned char *R, const float *raw, int warp,
                                                   int lane) {
  constexpr int kB = Op<OP>::kBytes;
  constexpr int E = 16 / kB;                  // k per chunk: 4 (TF32) or 8 (BF16)
  constexpr int kTasks = (kN / 32) * (kN / E);
#pragma unroll 2
  for (int t = warp; t < kTasks; t += kT128 / 32) {
    const int c = (t % (kN / 32)) * 32 + lane, k0 = (t / (kN / 32)) * E;
    float v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = raw[(k0 + e) * kN + c];
    *reinterpret_cast<uint4 *>(R + swz128((uint32_t)c, (uint32_t)(k0 * kB))) = pack_chunk<OP>(v);
  }
}

template <int OP, int KIND>
__global__ void __launch_bounds__(kT128, 1) fd128_kernel(FusedArgs a) {
  using T = Op<OP>;
  constexpr int kB = T::kBytes;
  constexpr int kTile = kN * kN * kB;          // bytes of one 128 x 128 operand
  constexpr long long n12 = (long long)kN * kN;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *R1 = base, *R2 = base + kTile, *R3 = base + 2 * kTile;   // A, B1, B2
  __shared__ uint64_t bar_b1, bar_b2, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, blk = blockIdx.x;

  auto wait_on = [&](uint64_t *b, uint32_t parity) -> bool {
    for (long long it = 0; it < kSpin; ++it) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_u32(b)), "r"(parity)
          : "memory");
      if (ok) return true;
    }
    return false;
  };
  auto mma = [&](unsigned char *Bt, uint32_t tmem) {
    const uint32_t idesc = (1u << 4) | (T::kFmt << 7) | (T::kFmt << 10) |
                           ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int ks = 0; ks < kN * kB / 32; ++ks) {
      const uint32_t o = (uint32_t)((ks * 32) >> 7) * kAtomCol + ((ks * 32) & 127);
      const uint64_t ad = sw128_desc(smem_u32(R1) + o);
      const uint64_t bd = sw128_desc(smem_u32(Bt) + o);
      const uint32_t acc = ks > 0 ? 1u : 0u;
      if (OP == OP_TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&bar_mma))
        : "memory");
  };
  auto bulk = [&](unsigned char *dst, const unsigned char *src, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"((uint32_t)kTile)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"((uint32_t)kTile), "r"(smem_u32(bar))
        : "memory");
  };
  auto tmem_ld32 = [&](uint32_t taddr, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  };

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_b1)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_b2)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bulk(R2, a.B1, &bar_b1);
    // the pencil kernel stages its input block through R3 first and fetches
    // the second B image into it after the transpose
    if (KIND != PENCIL) bulk(R3, a.B2, &bar_b2);
  }
  // everything above (barriers, TMEM, the constant B images) overlaps the
  // previous kernel's tail; its outputs are read only from here on
  pdl_wait();
  pdl_trigger();
  const bool skip = a.done && *a.done != 0.0;
  if (skip) {
    // skipped (converged): let the image copies land, free TMEM
    if (tid == 0) {
      wait_on(&bar_b1, 0);
      if (KIND != PENCIL) wait_on(&bar_b2, 0);
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
    return;
  }
  // ---- first A operand ----
  if (KIND == PENCIL) {
    // input block j2 = blk of the slab pass's [j2][i3][j1] output: contiguous
    // 64 KB of FP32 [i3][j1], one bulk copy into R3, transposed into R1
    constexpr uint32_t kRaw = (uint32_t)(n12 * sizeof(float));
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_b2)),
                   "r"(kRaw)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(R3)),
          "l"((const float *)a.in + (long long)blk * n12), "r"(kRaw), "r"(smem_u32(&bar_b2))
          : "memory");
    }
    if (!wait_on(&bar_b2, 0)) s_fail = 1;    // every thread waits for the block
    __syncthreads();
    if (!s_fail) stage128_cols_smem<OP>(R1, reinterpret_cast<const float *>(R3), warp, lane);
    __syncthreads();
    // R3 is free again: the second B image (phase 1 of bar_b2)
    if (tid == 0 && !s_fail) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk(R3, a.B2, &bar_b2);
    }
  } else if (KIND == SLAB_FWD) {
    stage128_rows_f64<OP>(R1, (const double *)a.in + blk * n12, warp, lane);
  } else {
    stage128_rows_f32<OP>(R1, (const float *)a.in + blk * n12, warp, lane);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    if (!wait_on(&bar_b1, 0)) s_fail = 1;
    else mma(R2, tmem);
  }
  __syncthreads();
  if (!s_fail && !wait_on(&bar_mma, 0)) s_fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int q = warp & 3, cg = warp >> 2;              // TMEM lane quarter, 32-column group
  const int lrow = q * 32 + lane;                       // accumulator lane of this thread
  const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cg * 32);
  if (!s_fail) {
    uint32_t v[32];
    tmem_ld32(taddr, v);
    if (KIND == PENCIL) {
      // divide by D1 (+) D2 (+) D3 at column c = blk kN + lrow (= j2 kN + j1), j3 = cg 32 + j;
      // the row's 32 values are whole operand chunks of the second A (k = j3)
      const float d12 = a.d1[lrow] + a.d2[blk];
      constexpr int E = 16 / kB;
#pragma unroll
      for (int e0 = 0; e0 < 32; e0 += E) {
        float f[E];
#pragma unroll
        for (int e = 0; e < E; ++e) f[e] = __fdividef(__uint_as_float(v[e0 + e]), d12 + a.d3[cg * 32 + e0 + e]);
        *reinterpret_cast<uint4 *>(R1 + swz128((uint32_t)lrow, (uint32_t)((cg * 32 + e0) * kB))) =
            pack_chunk<OP>(f);
      }
    } else {
      // transpose: element (row = cg 32 + j, k = lrow)
#pragma unroll
      for (int j = 0; j < 32; ++j)
        T::put(R1 + swz128((uint32_t)(cg * 32 + j), (uint32_t)(lrow * kB)), __uint_as_float(v[j]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0 && !s_fail) {
    if (!wait_on(&bar_b2, KIND == PENCIL ? 1 : 0)) s_fail = 1;
    else mma(R3, tmem);
  }
  __syncthreads();
  if (!s_fail && !wait_on(&bar_mma, 1)) s_fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_fail) {
    uint32_t v[32];
    tmem_ld32(taddr, v);
    // lanes: the output's contiguous index; columns: its strided one
    if (KIND == PENCIL) {
      float *o = (float *)a.out + (long long)blk * kN + lrow + (long long)cg * 32 * n12;
#pragma unroll
      for (int j = 0; j < 32; ++j) o[j * n12] = __uint_as_float(v[j]);
    } else if (KIND == SLAB_FWD) {
      // [j2][i3][j1]: the pencil kernel's block j2 is then contiguous
      float *o = (float *)a.out + (long long)blk * kN + lrow + (long long)cg * 32 * n12;
#pragma unroll
      for (int j = 0; j < 32; ++j) o[j * n12] = __uint_as_float(v[j]);
    } else {
      double *o = (double *)a.out + blk * n12 + lrow + cg * 32 * kN;
#pragma unroll
      for (int j = 0; j < 32; ++j) o[j * kN] = f32_to_f64(__uint_as_float(v[j]));
    }
  } else if (tid == 0) {
    atomicExch(a.err, (int)IGAFD_ERR_TIMEOUT);
    // a wait ran out: give the copies and MMAs this CTA issued a bounded
    // chance to finish before shared memory and TMEM are released
    wait_on(&bar_b1, 0);
    wait_on(&bar_b2, 0);
    if (KIND == PENCIL) wait_on(&bar_b2, 1);
    wait_on(&bar_mma, 0);
    wait_on(&bar_mma, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}
}  // namespace

struct FDMixed {
  float *scale16;                // device [3]: power of two folded into the FP16 images of U_k
  unsigned *umax;                // device [3]: bit pattern of max |U32_k|
  float *d32[3];                 // FP32 copies of D_k (the fused FD's divide)
  unsigned char *img[3][2][3];   // [direction][0: U_k^T, 1: U_k][op] B images
};

// FP32 copies U32_k of the eigenvector matrices and the tensor-core images
// of U_k^T and U_k. Allocates on the first call; later calls (a re-setup of
// P) refill the same buffers. Enqueues a memset and two kernels and does not
// synchronise.
igafd_status igafd_fd_tc_init(igafd_patch *P, cudaStream_t s) {
  FDMixed *F = P->mixed;
  if (!F) {
    F = (FDMixed *)calloc(1, sizeof(FDMixed));
    if (!F) return IGAFD_ERR_OOM;
    P->mixed = F;
  }
  if ((!F->scale16 && cudaMalloc(&F->scale16, 3 * sizeof(float)) != cudaSuccess) ||
      (!F->umax && cudaMalloc(&F->umax, 3 * sizeof(unsigned)) != cudaSuccess)) {
    cudaGetLastError();
    return IGAFD_ERR_OOM;
  }
  const int dim = P->dim;
  int nmax = 0;
  for (int k = 0; k < dim; ++k) nmax = P->n[k] > nmax ? P->n[k] : nmax;
  IGAFD_CUDA(cudaMemsetAsync(F->umax, 0, 3 * sizeof(unsigned), s));
  {
    U32Args ua{};
    for (int k = 0; k < dim; ++k) {
      if (!F->d32[k] && cudaMalloc(&F->d32[k], (size_t)P->n[k] * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return IGAFD_ERR_OOM;
      }
      ua.U[k] = P->U[k]; ua.D[k] = P->D[k]; ua.U32[k] = P->U32[k]; ua.D32[k] = F->d32[k];
      ua.n[k] = P->n[k];
    }
    ua.umax = F->umax;
    long long blocks = ((long long)nmax * nmax + 1023) / 1024;
    if (blocks > 64) blocks = 64;
    if (blocks * 256 < nmax) blocks = (nmax + 255) / 256;   // the D copy takes one thread per entry
    u32_kernel<<<dim3((unsigned)blocks, dim), 256, 0, s>>>(ua);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
  }
  ImgBatch batch{};
  int jobs = 0;
  long long most = 0;
  for (int k = 0; k < dim; ++k) {
    const int n = P->n[k];
    if (n > 256) continue;   // tensor-core FD limited to n_k <= 256
    const int Np = (n + 15) / 16 * 16;
    const int nchunks = (n + kKC - 1) / kKC;
    for (int dir = 0; dir < 2; ++dir) {
      for (int op = 0; op < 3; ++op) {
        const int bytes = op == OP_TF32 ? 4 : 2;
        const size_t sz = (size_t)nchunks * Np * kKC * bytes;
        if (!F->img[k][dir][op] && cudaMalloc(&F->img[k][dir][op], sz) != cudaSuccess) {
          cudaGetLastError();
          return IGAFD_ERR_OOM;
        }
        ImgJob &J = batch.j[jobs++];
        J.U = P->U32[k]; J.n = n; J.Np = Np; J.op = op; J.transpose = dir == 0;
        J.umax = op == OP_FP16 ? F->umax + k : nullptr;
        J.scale = op == OP_FP16 ? F->scale16 + k : nullptr;
        J.img = F->img[k][dir][op];
        const long long total = (long long)nchunks * Np * kKC;
        most = total > most ? total : most;
      }
    }
  }
  if (jobs > 0) {
    const unsigned blocks = (unsigned)((most + 255) / 256);
    b_image_kernel<<<dim3(blocks, jobs), 256, 0, s>>>(batch);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
  }
  return IGAFD_OK;
}

void igafd_fd_tc_free(igafd_patch *P) {
  if (!P || !P->mixed) return;
  cudaFree(P->mixed->scale16);
  cudaFree(P->mixed->umax);
  for (int k = 0; k < 3; ++k) cudaFree(P->mixed->d32[k]);
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 2; ++d)
      for (int o = 0; o < 3; ++o) cudaFree(P->mixed->img[k][d][o]);
  free(P->mixed);
  P->mixed = nullptr;
}

static size_t pass_smem(int op, int n_tile, int stages) {
  const int bytes = op == OP_TF32 ? 4 : 2;
  const size_t row = (size_t)kKC * bytes;
  return 1024 + (size_t)stages * (kM * row + (size_t)n_tile * row);
}

template <int OP>
static igafd_status launch_pass(const PassArgs &a, cudaStream_t s) {
  const size_t smem = pass_smem(OP, a.n_tile, a.stages);
  IGAFD_CUDA(cudaFuncSetAttribute(tc_pass_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  const dim3 grid((unsigned)((a.M + a.m_tile - 1) / a.m_tile),
                  (unsigned)((a.Np + a.n_tile - 1) / a.n_tile));
  IGAFD_CUDA(igafd_launch(tc_pass_kernel<OP>, grid, dim3(kThreads), smem, s, a));
  IGAFD_LAUNCHED(1);
  return IGAFD_OK;
}

// Tensor-core FD. dt selects the operand type: IGAFD_BF16, IGAFD_FP16, or
// IGAFD_TF32 (declared in igafd.h).
constexpr int kFusedMaxSmem = 1024 + (kM + 128) * 128 * 4;

template <int OP, int KIND>
static igafd_status launch_fused(const FusedArgs &a, int grid, cudaStream_t s, int dev) {
  const int bytes = OP == OP_TF32 ? 4 : 2;
  const size_t smem = 1024 + (size_t)(kM + 128) * a.Kpad * bytes;
  // the largest size this kernel is launched with, set once per device
  static std::atomic<unsigned long long> attr_set{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_set.load() & bit)) {
    IGAFD_CUDA(cudaFuncSetAttribute(tc_fused_kernel<OP, KIND>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedMaxSmem));
    attr_set.fetch_or(bit);
  }
  IGAFD_CUDA(igafd_launch(tc_fused_kernel<OP, KIND>, dim3(grid), dim3(kThreads), smem, s, a));
  IGAFD_LAUNCHED(1);
  return IGAFD_OK;
}

// Arguments and CTA counts of the fused FD's kernels (slab forward, pencil in
// 3D, slab backward; grid 0 = not launched) for z = P^{-1} r.
static void fused_args(igafd_patch *P, int op, const double *r, double *z, double *done,
                       FusedArgs out[3], int grid[3]) {
  FDMixed *F = P->mixed;
  const int dim = P->dim;
  const int n1 = P->n[0], n2 = P->n[1], n3 = dim == 3 ? P->n[2] : 1;
  int kmax = n1 > n2 ? n1 : n2;
  if (dim == 3 && n3 > kmax) kmax = n3;
  FusedArgs a{};
  a.n1 = n1; a.n2 = n2; a.n3 = n3;
  a.n12 = (long long)n1 * n2;
  a.Kpad = (kmax + kKC - 1) / kKC * kKC;
  auto kp = [](int n) { return (n + kKC - 1) / kKC * kKC; };
  a.done = done;
  a.err = P->err_flag;
  auto np = [](int n) { return (n + 15) / 16 * 16; };
  // images are padded to whole 64-element K chunks; use the largest K
  float *t1 = (float *)P->fd_a, *t2 = (float *)P->fd_b;
  // slab forward (modes 1 and 2; the divide too in 2D)
  a.in = r; a.in_f64 = 1; a.in_aligned = ((uintptr_t)r % 16) == 0;
  a.out = t1; a.out_f64 = 0;
  a.B1 = F->img[0][0][op]; a.Np1 = np(n1); a.K1 = n1; a.Kp1 = kp(n1);
  a.B2 = F->img[1][0][op]; a.Np2 = np(n2); a.K2 = n2; a.Kp2 = kp(n2);
  a.rowsA = n2;
  a.inv_lam = dim == 2 ? P->inv_lam32 : nullptr;
  out[0] = a;
  grid[0] = n3;
  const float *mid = t1;
  grid[1] = 0;
  if (dim == 3) {
    FusedArgs c = a;
    c.in = t1; c.in_f64 = 0; c.in_aligned = 1;
    c.out = t2; c.out_f64 = 0;
    c.B1 = F->img[2][0][op]; c.Np1 = np(n3); c.K1 = n3; c.Kp1 = kp(n3);
    c.B2 = F->img[2][1][op]; c.Np2 = np(n3); c.K2 = n3; c.Kp2 = kp(n3);
    c.rowsA = kM;
    c.inv_lam = nullptr;
    c.d1 = F->d32[0]; c.d2 = F->d32[1]; c.d3 = F->d32[2];
    c.ctile = P->fd_tile[op][3] == 64 ? 64 : kM;
    out[1] = c;
    grid[1] = (int)((a.n12 + c.ctile - 1) / c.ctile);
    mid = t2;
  }
  FusedArgs b = a;
  b.in = mid; b.in_f64 = 0; b.in_aligned = 1;
  b.out = z; b.out_f64 = 1;
  b.B1 = F->img[0][1][op]; b.Np1 = np(n1); b.K1 = n1; b.Kp1 = kp(n1);
  b.B2 = F->img[1][1][op]; b.Np2 = np(n2); b.K2 = n2; b.Kp2 = kp(n2);
  b.rowsA = n2;
  b.inv_lam = nullptr;
  out[2] = b;
  grid[2] = n3;
}

template <int OP>
static igafd_status fused_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                                double *done) {
  FusedArgs a[3];
  int grid[3];
  fused_args(P, OP, r, z, done, a, grid);
  IGAFD_TRY((launch_fused<OP, SLAB_FWD>(a[0], grid[0], s, P->dev)));
  if (grid[1] > 0) IGAFD_TRY((launch_fused<OP, PENCIL>(a[1], grid[1], s, P->dev)));
  IGAFD_TRY((launch_fused<OP, SLAB_BWD>(a[2], grid[2], s, P->dev)));
  return IGAFD_OK;
}

template <int OP, int KIND>
static igafd_status launch_fd128(const FusedArgs &a, cudaStream_t s, int dev) {
  // R1, R2 (operands) and R3 (second B image; the pencil's FP32 input block first)
  const size_t tile = (size_t)kN * kN * (OP == OP_TF32 ? 4 : 2);
  const size_t smem = 1024 + 2 * tile + (KIND == PENCIL ? (size_t)kN * kN * 4 : tile);
  static std::atomic<unsigned long long> attr_set{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_set.load() & bit)) {
    IGAFD_CUDA(cudaFuncSetAttribute(fd128_kernel<OP, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    attr_set.fetch_or(bit);
  }
  IGAFD_CUDA(igafd_launch(fd128_kernel<OP, KIND>, dim3(kN), dim3(kT128), smem, s, a));
  IGAFD_LAUNCHED(1);
  return IGAFD_OK;
}

// Fused FD with every n_k = 128 in 3D: slab forward (modes 1, 2), pencil
// (mode 3 forward, divide, mode 3 backward), slab backward (modes 2, 1).
template <int OP>
static igafd_status fd128_apply(igafd_patch *P, const double *r, double *z, cudaStream_t s,
                                double *done) {
  FDMixed *F = P->mixed;
  float *t1 = (float *)P->fd_a, *t2 = (float *)P->fd_b;
  FusedArgs a{};
  a.done = done;
  a.err = P->err_flag;
  a.in = r; a.out = t1;
  a.B1 = F->img[0][0][OP]; a.B2 = F->img[1][0][OP];
  IGAFD_TRY((launch_fd128<OP, SLAB_FWD>(a, s, P->dev)));
  a.in = t1; a.out = t2;
  a.B1 = F->img[2][0][OP]; a.B2 = F->img[2][1][OP];
  a.d1 = F->d32[0]; a.d2 = F->d32[1]; a.d3 = F->d32[2];
  IGAFD_TRY((launch_fd128<OP, PENCIL>(a, s, P->dev)));
  a.in = t2; a.out = z;
  a.B1 = F->img[0][1][OP]; a.B2 = F->img[1][1][OP];
  IGAFD_TRY((launch_fd128<OP, SLAB_BWD>(a, s, P->dev)));
  return IGAFD_OK;
}

igafd_status igafd_fd_tc_apply(igafd_patch *P, igafd_dtype dt, const double *r, double *z,
                               cudaStream_t s, double *done) {
  FDMixed *F = P->mixed;
  if (!F) return IGAFD_ERR_ARG;
  const int op = dt == IGAFD_TF32 ? OP_TF32 : dt == IGAFD_BF16 ? OP_BF16 : OP_FP16;
  const int dim = P->dim;
  bool fusable = op != OP_FP16 && P->fd_fused && P->fd_fused_op[op];
  for (int k = 0; k < dim; ++k) fusable = fusable && P->n[k] <= 128;
  if (fusable) {
    // every n_k = 128 in 3D, 16-byte aligned vectors: the compile-time-sized kernels
    const bool n128 = dim == 3 && P->n[0] == kN && P->n[1] == kN && P->n[2] == kN &&
                      (uintptr_t)r % 16 == 0 && (uintptr_t)z % 16 == 0;
    if (n128) {
      if (op == OP_TF32) return fd128_apply<OP_TF32>(P, r, z, s, done);
      return fd128_apply<OP_BF16>(P, r, z, s, done);
    }
    if (op == OP_TF32) return fused_apply<OP_TF32>(P, r, z, s, done);
    return fused_apply<OP_BF16>(P, r, z, s, done);
  }
  for (int k = 0; k < dim; ++k)
    if (P->n[k] > 256) return IGAFD_ERR_ARG;   // one MMA covers N <= 256
  // current layout: dims[0] slowest .. dims[dim-1] fastest (direction indices)
  int dims[3];
  for (int i = 0; i < dim; ++i) dims[i] = dim - 1 - i;
  float *bufs[2] = {(float *)P->fd_a, (float *)P->fd_b};
  const void *in = r;
  int in_f64 = 1, cur = 0;
  for (int pass = 0; pass < 2 * dim; ++pass) {
    const bool forward = pass < dim;
    const int k = dims[dim - 1];                 // contracted direction (fastest)
    const int n = P->n[k];
    PassArgs a{};
    a.in = in;
    a.in_f64 = in_f64;
    a.in_aligned = ((uintptr_t)in % 16) == 0;
    const bool last = pass == 2 * dim - 1;
    a.out = last ? (void *)z : (void *)bufs[cur];
    a.out_f64 = last ? 1 : 0;
    a.Bimg = F->img[k][forward ? 0 : 1][op];
    a.b_scale = op == OP_FP16 ? F->scale16 + k : nullptr;
    a.inv_lam = pass == dim - 1 ? P->inv_lam32 : nullptr;
    a.M = P->N / n;
    a.K = n;
    a.N = n;
    a.Np = (n + 15) / 16 * 16;
    // tile shape of this operand type (autotuned; 128 rows, all columns and
    // two stages by default); a 256-row ring tile would not fit in TMEM
    const int *tile = P->fd_tile[op];
    a.m_tile = tile[0] == 64 ? 64 : kM;
    a.n_tile = a.Np;
    if (tile[1] == 2 && a.Np >= 32) a.n_tile = (a.Np / 2 + 15) / 16 * 16;
    a.stages = tile[2] == 3 ? 3 : 2;
    int cols = 32;
    while (cols < a.n_tile) cols <<= 1;
    a.tmem_cols = cols;
    a.done = done;
    a.err = P->err_flag;
    if (op == OP_TF32) IGAFD_TRY(launch_pass<OP_TF32>(a, s));
    else if (op == OP_BF16) IGAFD_TRY(launch_pass<OP_BF16>(a, s));
    else IGAFD_TRY(launch_pass<OP_FP16>(a, s));
    // rotate: the new index becomes the slowest
    for (int i = dim - 1; i > 0; --i) dims[i] = dims[i - 1];
    dims[0] = k;
    if (!last) {
      in = bufs[cur];
      in_f64 = 0;
      cur ^= 1;
    }
  }
  return IGAFD_OK;
}

// ---- batched solve -----------------------------------------------------------
bool igafd_fd_tc_fused_generic(const igafd_patch *P, igafd_dtype dt) {
  if (!P->mixed || (dt != IGAFD_TF32 && dt != IGAFD_BF16)) return false;
  const int op = dt == IGAFD_TF32 ? OP_TF32 : OP_BF16;
  bool fusable = P->fd_fused && P->fd_fused_op[op];
  for (int k = 0; k < P->dim; ++k) fusable = fusable && P->n[k] <= 128;
  const bool n128 = P->dim == 3 && P->n[0] == kN && P->n[1] == kN && P->n[2] == kN;
  return fusable && !n128;
}

size_t igafd_fd_fused_args_bytes() { return sizeof(FusedArgs); }

// The fused FD's arguments on the PCG's buffers (z = P^{-1} r, skipped once
// the PCG is done), CTA counts per kind and the dynamic shared memory.
igafd_status igafd_fd_fused_batch_args(igafd_patch *P, igafd_dtype dt, void *args3, int *blocks3,
                                       size_t *smem) {
  if (!igafd_fd_tc_fused_generic(P, dt)) return IGAFD_ERR_ARG;
  const int op = dt == IGAFD_TF32 ? OP_TF32 : OP_BF16;
  FusedArgs a[3];
  fused_args(P, op, P->r, P->z, P->scal + S_DONE, a, blocks3);
  memcpy(args3, a, sizeof(a));
  *smem = 1024 + (size_t)(kM + 128) * a[0].Kpad * (op == OP_TF32 ? 4 : 2);
  return IGAFD_OK;
}

template <int OP, int KIND>
static igafd_status batch_fused(const FusedArgs *args, const int *act, const int *act_start,
                                const int *act_count, unsigned *queue, int total, size_t smem,
                                int num_sms, cudaStream_t s) {
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  IGAFD_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_set.load() & bit)) {
    IGAFD_CUDA(cudaFuncSetAttribute(tc_fused_batch_kernel<OP, KIND>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedMaxSmem));
    attr_set.fetch_or(bit);
  }
  // persistent: the CTAs that fit on an SM at once, at most 4 (128 of the 512
  // TMEM columns each), on every SM
  int occ = 0;
  IGAFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tc_fused_batch_kernel<OP, KIND>,
                                                           kThreads, smem));
  occ = occ < 1 ? 1 : occ > 4 ? 4 : occ;
  const long long cap = queue ? (long long)num_sms * occ : (long long)total;
  const int grid = (int)(total < cap ? total : cap);
  tc_fused_batch_kernel<OP, KIND><<<grid, kThreads, smem, s>>>(args, act, act_start, act_count,
                                                                queue);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

igafd_status igafd_fd_fused_batch_launch(igafd_dtype dt, int kind, const void *args_dev,
                                         const int *act, const int *act_start,
                                         const int *act_count, unsigned *queue, int total_blocks,
                                         size_t smem, int num_sms, cudaStream_t s) {
  if (total_blocks <= 0) return IGAFD_OK;
  if (smem > (size_t)kFusedMaxSmem || num_sms < 1) return IGAFD_ERR_ARG;
  const FusedArgs *a = (const FusedArgs *)args_dev;
#define IGAFD_BF(O, K) \
  batch_fused<O, K>(a, act, act_start, act_count, queue, total_blocks, smem, num_sms, s)
  if (dt == IGAFD_TF32) {
    if (kind == 0) return IGAFD_BF(OP_TF32, SLAB_FWD);
    if (kind == 1) return IGAFD_BF(OP_TF32, PENCIL);
    return IGAFD_BF(OP_TF32, SLAB_BWD);
  }
  if (kind == 0) return IGAFD_BF(OP_BF16, SLAB_FWD);
  if (kind == 1) return IGAFD_BF(OP_BF16, PENCIL);
  return IGAFD_BF(OP_BF16, SLAB_BWD);
#undef IGAFD_BF
}

// ---- tensor-core throughput probe ---------------------------------------------
namespace {

// One CTA per launch slot issues back-to-back M = 128, N = 128 tcgen05 MMAs
// of the operand type from a constant shared-memory tile (one 128-byte K
// atom per operand row: four MMAs of 32 bytes of K per round) into one TMEM
// accumulator, then waits (bounded) for their completion. Operands hold 1.0,
// so the accumulator grows by K per MMA and stays finite.
template <int OP>
__global__ void __launch_bounds__(128) tc_probe_kernel(int rounds, int *err) {
  using T = Op<OP>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *A = base, *B = base + kM * 128;
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const uint32_t one = OP == OP_TF32 ? 0x3F800000u : 0x3F803F80u;   // 1.0 (x2 in 16-bit)
  for (int i = threadIdx.x; i < 2 * kM * 128 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t *>(A)[i] = one;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = (1u << 4) | (T::kFmt << 7) | (T::kFmt << 10) |
                           ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t ad = sw128_desc(smem_u32(A) + ks * 32);
        const uint64_t bd = sw128_desc(smem_u32(B) + ks * 32);
        const uint32_t acc = (r > 0 || ks > 0) ? 1u : 0u;
        if (OP == OP_TF32)
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&bar))
        : "memory");
    bool ok = false;
    for (long long it = 0; it < kSpin && !ok; ++it) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(&bar))
          : "memory");
      ok = done != 0;
    }
    if (!ok) atomicExch(err, (int)IGAFD_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

template <int OP>
igafd_status tc_probe(int num_sms, int rounds, int *err, double *flops, float *ms) {
  const size_t smem = 1024 + 2 * (size_t)kM * 128;
  IGAFD_CUDA(cudaFuncSetAttribute(tc_probe_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  const int grid = 2 * num_sms;                   // two CTAs per SM (256 of the 512 TMEM columns)
  cudaEvent_t e0, e1;
  IGAFD_CUDA(cudaEventCreate(&e0));
  IGAFD_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {             // the first launch warms up
    cudaEventRecord(e0);
    tc_probe_kernel<OP><<<grid, 128, smem>>>(rounds, err);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return IGAFD_ERR_CUDA;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0 && t < best) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  IGAFD_CUDA(cudaGetLastError());
  const double k_inst = OP == OP_TF32 ? 8.0 : 16.0;  // K of one 32-byte MMA step
  *flops = 2.0 * kM * 128 * k_inst * 4.0 * rounds * grid;
  *ms = best;
  return IGAFD_OK;
}

}  // namespace

// Dense tensor-core FLOP/s of this device for TF32 (op 0) or BF16 (op 1)
// operands with FP32 accumulation in TMEM (M = N = 128 tcgen05 MMAs).
igafd_status igafd_tc_probe(int op, int num_sms, int rounds, int *err_dev, double *flop_per_s) {
  double flops = 0.0;
  float ms = 0.f;
  if (op == 0) IGAFD_TRY(tc_probe<OP_TF32>(num_sms, rounds, err_dev, &flops, &ms));
  else IGAFD_TRY(tc_probe<OP_BF16>(num_sms, rounds, err_dev, &flops, &ms));
  *flop_per_s = ms > 0.f ? flops / (ms * 1e-3) : 0.0;
  return IGAFD_OK;
}
