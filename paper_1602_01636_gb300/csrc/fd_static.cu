// FP64 fast-diagonalization apply that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while another library
// owns all device memory through its own pool, latency-critical loops where an
// allocation's implicit device synchronisation is not acceptable, or plugins
// that are handed device buffers but no allocation rights. For them this file
// provides igafd_apply_prec_static: the caller passes the eigenpairs, r and z;
// the two intermediate tensors of the mode products live in a file-scope
// static device array of fixed size (igafd.h: IGAFD_STATIC_FD_MAX_DOFS), which
// every GPU that loads the library holds until the process exits.
//
// The host-side name of that array is only a stand-in, never a device
// address: the address is obtained with cudaGetSymbolAddress (with the
// device current) on every call whose stream is not capturing, and cached
// per device for calls made during a stream capture (which must not query
// it). So the first call on a device should come before any stream capture,
// and after a context reset (cudaDeviceReset) the next call outside a capture
// picks up the reloaded module's address. No element of the
// scratch needs to start at zero: every product writes each element of its
// output before the next product reads it. All calls share the one array, so
// calls whose kernels overlap on the GPU (different streams, or concurrent
// host threads) race; serialise them.
#include "common.cuh"

#include <mutex>

static __device__ __align__(256) double g_fd_static_scratch[2 * (size_t)IGAFD_STATIC_FD_MAX_DOFS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};

igafd_status scratch_address(cudaStream_t s, double **out) {
  int dev = -1;
  IGAFD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return IGAFD_ERR_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  IGAFD_CUDA(cudaStreamIsCapturing(s, &cap));
  std::lock_guard<std::mutex> lock(g_mutex);
  if (cap != cudaStreamCaptureStatusNone && !g_scratch_addr[dev]) {
    fprintf(stderr, "igafd_apply_prec_static: the first call on a device must not be captured\n");
    return IGAFD_ERR_ARG;
  }
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fd_static_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "igafd: cudaGetSymbolAddress of the static FD scratch failed: %s\n",
              cudaGetErrorString(e));
      return IGAFD_ERR_CUDA;
    }
    g_scratch_addr[dev] = (double *)p;
  }
  *out = g_scratch_addr[dev];
  return IGAFD_OK;
}

struct StaticGemm {
  const double *A, *B;
  double *C;
  int M, N, K, batch;
  int b_off;          // first batch index of this launch (grid.z covers at most 65535)
  long long sam, sak, sbk, sbn, scm, scn, batA, batB, batC;
  // divide epilogue: C[i] /= D1[i1] + D2[i2] + D3[i3] for the linear index i
  const double *D1, *D2, *D3;
  int n1, n2;
};

// 64x64 FP64 tile, 16-deep K slices, 256 threads with 4x4 outputs each; the
// same mode product as the patch FD, with the eigenvalue sum formed in the
// epilogue instead of read from a precomputed array.
__global__ void __launch_bounds__(256) static_mode_gemm(StaticGemm g) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long long b = (long long)blockIdx.z + g.b_off;
  const double *A = g.A + b * g.batA;
  const double *B = g.B + b * g.batB;
  double *C = g.C + b * g.batC;
  double acc[4][4] = {};
  const bool a_kfast = g.sak == 1, b_nfast = g.sbn == 1;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      int t = tid + 256 * l;
      int mm, kk, nn, kb;
      if (a_kfast) { mm = t / BK; kk = t % BK; } else { kk = t / BM; mm = t % BM; }
      if (b_nfast) { kb = t / BN; nn = t % BN; } else { nn = t / BK; kb = t % BK; }
      int m = m0 + mm, k = k0 + kk, n = n0 + nn, kq = k0 + kb;
      As[kk][mm] = (m < g.M && k < g.K) ? A[m * g.sam + k * g.sak] : 0.0;
      Bs[kb][nn] = (n < g.N && kq < g.K) ? B[kq * g.sbk + n * g.sbn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      long long ci = m * g.scm + n * g.scn;
      double v = acc[i][j];
      if (g.D1) {
        long long li = b * g.batC + ci;
        long long i1 = li % g.n1, i2 = (li / g.n1) % g.n2, i3 = li / ((long long)g.n1 * g.n2);
        double lam = g.D1[i1] + g.D2[i2] + (g.D3 ? g.D3[i3] : 0.0);
        v = v / lam;
      }
      C[ci] = v;
    }
  }
}

StaticGemm mode_desc(const int *n, int dim, int k, const double *U, bool forward, const double *X,
                     double *Y) {
  long long F = 1, S = 1;
  for (int l = 0; l < k; ++l) F *= n[l];
  for (int l = k + 1; l < dim; ++l) S *= n[l];
  const long long nk = n[k];
  StaticGemm g{};
  if (k == 0) {
    g.A = X; g.B = U; g.C = Y;
    g.M = (int)S; g.N = (int)nk; g.K = (int)nk; g.batch = 1;
    g.sam = nk; g.sak = 1;
    if (forward) { g.sbk = nk; g.sbn = 1; } else { g.sbk = 1; g.sbn = nk; }
    g.scm = nk; g.scn = 1;
  } else {
    g.A = U; g.B = X; g.C = Y;
    g.M = (int)nk; g.N = (int)F; g.K = (int)nk; g.batch = (int)S;
    if (forward) { g.sam = 1; g.sak = nk; } else { g.sam = nk; g.sak = 1; }
    g.sbk = F; g.sbn = 1;
    g.scm = F; g.scn = 1;
    g.batB = nk * F; g.batC = nk * F;
  }
  return g;
}

// One mode product; the batch index runs over launches of at most 65535
// (the grid's z extent), so every shape within the dof limit launches.
igafd_status launch_mode(StaticGemm g, cudaStream_t s) {
  const int total = g.batch;
  for (int b0 = 0; b0 < total; b0 += 65535) {
    g.b_off = b0;
    const int nb = total - b0 < 65535 ? total - b0 : 65535;
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, nb);
    static_mode_gemm<<<grid, 256, 0, s>>>(g);
    IGAFD_LAUNCHED(1);
    IGAFD_CUDA(cudaGetLastError());
  }
  return IGAFD_OK;
}

}  // namespace

extern "C" igafd_status igafd_apply_prec_static(int dim, const int *n, const double *const *U,
                                                const double *const *D, const double *r,
                                                double *z, void *stream) {
  if ((dim != 2 && dim != 3) || !n || !U || !D || !r || !z || r == z) return IGAFD_ERR_ARG;
  long long N = 1;
  for (int k = 0; k < dim; ++k) {
    if (n[k] < 1 || !U[k] || !D[k]) return IGAFD_ERR_ARG;
    N *= n[k];
  }
  if (N > IGAFD_STATIC_FD_MAX_DOFS) {
    fprintf(stderr,
            "igafd_apply_prec_static: %lld dofs exceed the static scratch limit of %d dofs "
            "(IGAFD_STATIC_FD_MAX_DOFS); use igafd_apply_prec on a patch instead\n",
            N, IGAFD_STATIC_FD_MAX_DOFS);
    return IGAFD_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *scratch = nullptr;
  IGAFD_TRY(scratch_address(s, &scratch));
  double *bufs[2] = {scratch, scratch + IGAFD_STATIC_FD_MAX_DOFS};
  const double *in = r;
  int cur = 0;
  for (int k = 0; k < dim; ++k) {            // forward U_k^T, divide in the last
    StaticGemm g = mode_desc(n, dim, k, U[k], true, in, bufs[cur]);
    if (k == dim - 1) {
      g.D1 = D[0]; g.D2 = D[1]; g.D3 = dim == 3 ? D[2] : nullptr;
      g.n1 = n[0]; g.n2 = n[1];
    }
    IGAFD_TRY(launch_mode(g, s));
    in = bufs[cur];
    cur ^= 1;
  }
  for (int k = dim - 1; k >= 0; --k) {       // backward U_k, the last writes z
    double *out = k == 0 ? z : bufs[cur];
    StaticGemm g = mode_desc(n, dim, k, U[k], false, in, out);
    IGAFD_TRY(launch_mode(g, s));
    in = out;
    cur ^= 1;
  }
  return IGAFD_OK;
}
