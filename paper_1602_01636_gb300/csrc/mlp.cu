// Small MLP 6 -> 64 -> 64 -> 2 (tanh) that maps per-span features of Q to
// the log span scalings (log wK, log wM) of the 1D pencils. FP16 weights are
// used in the forward pass with FP32 arithmetic; training keeps FP32 master
// weights and Adam moments, accumulates the MSE gradient per block in shared
// memory and refreshes the FP16 copy after each step.
//
// Parameter layout (floats): W1[64][6], b1[64], W2[64][64], b2[64], W3[2][64],
// b3[2]. Inputs are normalised by (x - in_mean) / in_std and outputs mapped
// back by out_mean + out_std * net(x); the normalisation is set by the caller
// and is not trained.
#include "common.cuh"

#include <cuda_fp16.h>

#include <cstdlib>
#include <cstring>

#define H1 64
#define H2 64
#define NIN 6
#define NOUT 2
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + H1 * NIN)
#define OFF_W2 (OFF_B1 + H1)
#define OFF_B2 (OFF_W2 + H2 * H1)
#define OFF_W3 (OFF_B2 + H2)
#define OFF_B3 (OFF_W3 + NOUT * H2)
#define NPARAM (OFF_B3 + NOUT)

static_assert(NPARAM == IGAFD_MLP_PARAMS, "MLP parameter count");

struct igafd_mlp {
  int dev;
  float *w32;      // master weights
  __half *w16;     // forward weights
  float *m, *v;    // Adam moments
  float *grad;
  float *loss;     // device scalar
  float norm[16];  // in_mean[6], in_std[6], out_mean[2], out_std[2]
  int step;
};

namespace {

struct Norm {
  float in_mean[NIN], in_std[NIN], out_mean[NOUT], out_std[NOUT];
};

__device__ void load_weights(const __half *w16, float *sw) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sw[i] = __half2float(w16[i]);
  __syncthreads();
}

// normalised network output o (before out_mean + out_std *) and hidden states
__device__ void net_forward(const float *sw, const float *xn, float *h1, float *h2, float *o) {
  for (int j = 0; j < H1; ++j) {
    float acc = sw[OFF_B1 + j];
#pragma unroll
    for (int i = 0; i < NIN; ++i) acc = fmaf(sw[OFF_W1 + j * NIN + i], xn[i], acc);
    h1[j] = tanhf(acc);
  }
  for (int j = 0; j < H2; ++j) {
    float acc = sw[OFF_B2 + j];
    for (int i = 0; i < H1; ++i) acc = fmaf(sw[OFF_W2 + j * H1 + i], h1[i], acc);
    h2[j] = tanhf(acc);
  }
  for (int j = 0; j < NOUT; ++j) {
    float acc = sw[OFF_B3 + j];
    for (int i = 0; i < H2; ++i) acc = fmaf(sw[OFF_W3 + j * H2 + i], h2[i], acc);
    o[j] = acc;
  }
}

__global__ void mlp_forward_kernel(const __half *w16, Norm nm, const float *X, int rows, float *Y) {
  __shared__ float sw[NPARAM];
  load_weights(w16, sw);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    float xn[NIN], h1[H1], h2[H2], o[NOUT];
    for (int i = 0; i < NIN; ++i) xn[i] = (X[r * NIN + i] - nm.in_mean[i]) / nm.in_std[i];
    net_forward(sw, xn, h1, h2, o);
    for (int j = 0; j < NOUT; ++j) Y[r * NOUT + j] = nm.out_mean[j] + nm.out_std[j] * o[j];
  }
}

// Gradient of L = mean over rows and outputs of (o - t_n)^2, t_n the
// normalised target, with respect to every parameter (added into grad) and
// the loss (added into *loss).
__global__ void mlp_grad_kernel(const __half *w16, Norm nm, const float *X, const float *T, int rows,
                                float *grad, float *loss) {
  __shared__ float sw[NPARAM];
  __shared__ float sg[NPARAM];
  __shared__ float sl;
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sg[i] = 0.0f;
  if (threadIdx.x == 0) sl = 0.0f;
  load_weights(w16, sw);
  const float scale = 2.0f / ((float)rows * NOUT);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    float xn[NIN], h1[H1], h2[H2], o[NOUT], dz2[H2];
    for (int i = 0; i < NIN; ++i) xn[i] = (X[r * NIN + i] - nm.in_mean[i]) / nm.in_std[i];
    net_forward(sw, xn, h1, h2, o);
    float dout[NOUT], l = 0.0f;
    for (int j = 0; j < NOUT; ++j) {
      const float tn = (T[r * NOUT + j] - nm.out_mean[j]) / nm.out_std[j];
      const float d = o[j] - tn;
      l += d * d;
      dout[j] = scale * d;
      atomicAdd(&sg[OFF_B3 + j], dout[j]);
      for (int i = 0; i < H2; ++i) atomicAdd(&sg[OFF_W3 + j * H2 + i], dout[j] * h2[i]);
    }
    atomicAdd(&sl, l / ((float)rows * NOUT));
    for (int i = 0; i < H2; ++i) {
      float s = 0.0f;
      for (int j = 0; j < NOUT; ++j) s = fmaf(sw[OFF_W3 + j * H2 + i], dout[j], s);
      dz2[i] = s * (1.0f - h2[i] * h2[i]);
      atomicAdd(&sg[OFF_B2 + i], dz2[i]);
    }
    for (int j = 0; j < H2; ++j)
      for (int i = 0; i < H1; ++i) atomicAdd(&sg[OFF_W2 + j * H1 + i], dz2[j] * h1[i]);
    for (int i = 0; i < H1; ++i) {
      float s = 0.0f;
      for (int j = 0; j < H2; ++j) s = fmaf(sw[OFF_W2 + j * H1 + i], dz2[j], s);
      const float dz1 = s * (1.0f - h1[i] * h1[i]);
      atomicAdd(&sg[OFF_B1 + i], dz1);
      for (int k = 0; k < NIN; ++k) atomicAdd(&sg[OFF_W1 + i * NIN + k], dz1 * xn[k]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) atomicAdd(&grad[i], sg[i]);
  if (threadIdx.x == 0) atomicAdd(loss, sl);
}

__global__ void adam_kernel(float *w32, __half *w16, float *m, float *v, float *grad, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float w = w32[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w32[i] = w;
  w16[i] = __float2half_rn(w);
  grad[i] = 0.0f;
}

__global__ void refresh_half_kernel(const float *w32, __half *w16) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NPARAM) w16[i] = __float2half_rn(w32[i]);
}

Norm make_norm(const igafd_mlp *M) {
  Norm n;
  memcpy(&n, M->norm, sizeof(n));
  return n;
}

int grid_for(int rows) {
  int g = (rows + 127) / 128;
  return g < 1 ? 1 : (g > 1184 ? 1184 : g);
}

}  // namespace

extern "C" igafd_status igafd_mlp_create(const float *params, igafd_mlp **out) {
  if (!out) return IGAFD_ERR_ARG;
  *out = nullptr;
  igafd_mlp *M = (igafd_mlp *)calloc(1, sizeof(igafd_mlp));
  if (!M) return IGAFD_ERR_OOM;
  cudaGetDevice(&M->dev);
  for (int i = 0; i < NIN; ++i) M->norm[NIN + i] = 1.0f;
  M->norm[2 * NIN + NOUT] = M->norm[2 * NIN + NOUT + 1] = 1.0f;
  bool ok = cudaMalloc(&M->w32, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->w16, NPARAM * sizeof(__half)) == cudaSuccess &&
            cudaMalloc(&M->m, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->v, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->grad, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->loss, sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    igafd_mlp_destroy(M);
    return IGAFD_ERR_OOM;
  }
  cudaMemset(M->m, 0, NPARAM * sizeof(float));
  cudaMemset(M->v, 0, NPARAM * sizeof(float));
  cudaMemset(M->grad, 0, NPARAM * sizeof(float));
  if (params) cudaMemcpy(M->w32, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  else cudaMemset(M->w32, 0, NPARAM * sizeof(float));
  refresh_half_kernel<<<(NPARAM + 255) / 256, 256>>>(M->w32, M->w16);
  IGAFD_LAUNCHED(1);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    igafd_mlp_destroy(M);
    return IGAFD_ERR_CUDA;
  }
  *out = M;
  return IGAFD_OK;
}

extern "C" void igafd_mlp_destroy(igafd_mlp *M) {
  if (!M) return;
  cudaFree(M->w32); cudaFree(M->w16); cudaFree(M->m); cudaFree(M->v);
  cudaFree(M->grad); cudaFree(M->loss);
  free(M);
}

extern "C" igafd_status igafd_mlp_set_normalization(igafd_mlp *M, const float *in_mean,
                                                    const float *in_std, const float *out_mean,
                                                    const float *out_std) {
  if (!M || !in_mean || !in_std || !out_mean || !out_std) return IGAFD_ERR_ARG;
  for (int i = 0; i < NIN; ++i)
    if (!(in_std[i] > 0.0f)) return IGAFD_ERR_ARG;
  for (int j = 0; j < NOUT; ++j)
    if (!(out_std[j] > 0.0f)) return IGAFD_ERR_ARG;
  memcpy(M->norm, in_mean, NIN * sizeof(float));
  memcpy(M->norm + NIN, in_std, NIN * sizeof(float));
  memcpy(M->norm + 2 * NIN, out_mean, NOUT * sizeof(float));
  memcpy(M->norm + 2 * NIN + NOUT, out_std, NOUT * sizeof(float));
  return IGAFD_OK;
}

extern "C" igafd_status igafd_mlp_get_params(const igafd_mlp *M, float *host) {
  if (!M || !host) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaMemcpy(host, M->w32, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
  return IGAFD_OK;
}

extern "C" igafd_status igafd_mlp_set_params(igafd_mlp *M, const float *host) {
  if (!M || !host) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaMemcpy(M->w32, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
  refresh_half_kernel<<<(NPARAM + 255) / 256, 256>>>(M->w32, M->w16);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaDeviceSynchronize());
  return IGAFD_OK;
}

extern "C" igafd_status igafd_mlp_forward(igafd_mlp *M, const float *X, int rows, float *Y,
                                          void *stream) {
  if (!M || !X || !Y || rows < 0) return IGAFD_ERR_ARG;
  if (rows == 0) return IGAFD_OK;
  mlp_forward_kernel<<<grid_for(rows), 128, 0, (cudaStream_t)stream>>>(M->w16, make_norm(M), X, rows, Y);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  return IGAFD_OK;
}

extern "C" igafd_status igafd_mlp_gradient(igafd_mlp *M, const float *X, const float *T, int rows,
                                           float *grad_host, float *loss_host, void *stream) {
  if (!M || !X || !T || rows < 1) return IGAFD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  IGAFD_CUDA(cudaMemsetAsync(M->grad, 0, NPARAM * sizeof(float), s));
  IGAFD_CUDA(cudaMemsetAsync(M->loss, 0, sizeof(float), s));
  mlp_grad_kernel<<<grid_for(rows), 128, 0, s>>>(M->w16, make_norm(M), X, T, rows, M->grad, M->loss);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  if (grad_host)
    IGAFD_CUDA(cudaMemcpyAsync(grad_host, M->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (loss_host) IGAFD_CUDA(cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  IGAFD_CUDA(cudaStreamSynchronize(s));
  IGAFD_CUDA(cudaMemsetAsync(M->grad, 0, NPARAM * sizeof(float), s));
  return IGAFD_OK;
}

extern "C" igafd_status igafd_mlp_train_step(igafd_mlp *M, const float *X, const float *T, int rows,
                                             float lr, float *loss_host, void *stream) {
  if (!M || !X || !T || rows < 1 || !(lr > 0.0f)) return IGAFD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  IGAFD_CUDA(cudaMemsetAsync(M->loss, 0, sizeof(float), s));
  mlp_grad_kernel<<<grid_for(rows), 128, 0, s>>>(M->w16, make_norm(M), X, T, rows, M->grad, M->loss);
  IGAFD_LAUNCHED(1);
  M->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)M->step), c2 = 1.0f - powf(b2, (float)M->step);
  adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(M->w32, M->w16, M->m, M->v, M->grad, lr, b1, b2,
                                                   1e-8f, c1, c2);
  IGAFD_LAUNCHED(1);
  IGAFD_CUDA(cudaGetLastError());
  if (loss_host) {
    IGAFD_CUDA(cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    IGAFD_CUDA(cudaStreamSynchronize(s));
  }
  return IGAFD_OK;
}
