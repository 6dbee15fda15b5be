// C ABI: patch setup (validation, allocation, table/pencil/eigen/stencil
// construction), teardown and queries.
#include "common.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>

namespace {

// Open knot vector on [0, 1]: nondecreasing, first and last value repeated
// exactly deg+1 times, interior multiplicity <= deg (Eq. (knot-vector)).
bool valid_open_knots(const double *kn, int nk, int deg) {
  if (!kn || nk < 2 * (deg + 1)) return false;
  for (int i = 0; i + 1 < nk; ++i)
    if (!(kn[i] <= kn[i + 1]) || !std::isfinite(kn[i])) return false;
  if (kn[0] != 0.0 || kn[nk - 1] != 1.0) return false;
  for (int i = 0; i <= deg; ++i)
    if (kn[i] != 0.0 || kn[nk - 1 - i] != 1.0) return false;
  if (kn[deg + 1] == 0.0 || kn[nk - deg - 2] == 1.0) return false;
  int mult = 1;
  for (int i = deg + 2; i < nk - deg - 1; ++i) {
    mult = (kn[i] == kn[i - 1]) ? mult + 1 : 1;
    if (mult > deg) return false;
  }
  return true;
}

template <typename T>
igafd_status alloc(T **p, size_t count) {
  cudaError_t e = cudaMalloc((void **)p, (count > 0 ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return IGAFD_ERR_OOM;
  }
  return IGAFD_OK;
}

void free_patch(igafd_patch *P) {
  if (!P) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(P->dev);
  for (int k = 0; k < 3; ++k) {
    Dir1D &D = P->dir[k];
    cudaFree(D.knots); cudaFree(D.gknots); cudaFree(D.span); cudaFree(D.z); cudaFree(D.w);
    cudaFree(D.bv); cudaFree(D.bd); cudaFree(D.gspan); cudaFree(D.gv); cudaFree(D.gd);
    cudaFree(D.kknots); cudaFree(D.kspan); cudaFree(D.kv);
    cudaFree(P->U[k]); cudaFree(P->D[k]); cudaFree(P->U32[k]);
    cudaFree(P->wK[k]); cudaFree(P->wM[k]);
  }
  cudaFree(P->ctrl); cudaFree(P->kctrl); cudaFree(P->inv_lam); cudaFree(P->inv_lam32); cudaFree(P->stencil);
  cudaFree(P->fd_a); cudaFree(P->fd_b);
  cudaFree(P->r); cudaFree(P->z); cudaFree(P->pv_base); cudaFree(P->xpad_base);
  cudaFree(P->xs_base); cudaFree(P->bint); cudaFree(P->tstat);
  if (P->loop_exec) cudaGraphExecDestroy(P->loop_exec);
  if (P->loop_graph) cudaGraphDestroy(P->loop_graph);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  cudaFree(P->q); cudaFree(P->xt);
  cudaFree(P->partial); cudaFree(P->counter); cudaFree(P->scal); cudaFree(P->err_flag);
  cudaFree(P->eig_work); cudaFree(P->eig_jobs); cudaFree(P->coef);
  cudaFree(P->lfeat); cudaFree(P->lybar);
  igafd_fd_tc_free(P);
  igafd_adi_free(P);
  for (int i = 0; i < IGAFD_NEV; ++i)
    if (P->ev[i]) cudaEventDestroy(P->ev[i]);
  if (P->host_scal) cudaFreeHost(P->host_scal);
  if (cur >= 0) cudaSetDevice(cur);
  free(P);
}

igafd_status build(igafd_patch *P, const igafd_patch_desc *d, cudaStream_t s) {
  IGAFD_TRY(igafd_setup_tables(P, d, s));
  long long N = 1;
  for (int k = 0; k < 3; ++k) {
    if (k >= P->dim) { P->n[k] = 1; P->nel[k] = 1; }
    if (P->n[k] < 1) return IGAFD_ERR_ARG;
    N *= P->n[k];
  }
  P->N = N;
  P->n_off = 1;
  for (int k = 0; k < P->dim; ++k) P->n_off *= 2 * P->p + 1;
  for (int k = 0; k < P->dim; ++k) {
    size_t nn = (size_t)P->n[k] * P->n[k];
    IGAFD_TRY(alloc(&P->U[k], nn));
    IGAFD_TRY(alloc(&P->D[k], (size_t)P->n[k]));
    IGAFD_TRY(alloc(&P->U32[k], nn));
  }
  IGAFD_TRY(alloc(&P->inv_lam, (size_t)N));
  IGAFD_TRY(alloc(&P->inv_lam32, (size_t)N));
  P->Np = igafd_stencil_row_stride(N);
  const bool with_stencil = !(d->flags & IGAFD_SETUP_NO_STENCIL);
  P->stencil_half = (d->flags & IGAFD_SETUP_HALF_STENCIL) ? 1 : 0;
  if (P->stencil_half) {
    // halo: the largest |off(delta)| plus two rows (the odd-start fetch of a
    // mirrored run reads one row before it and one after), even
    long long mo = 1, str = 1;
    for (int k = 0; k < P->dim; ++k) { mo += (long long)P->p * str; str *= P->n[k]; }
    P->sh_H = (mo + 2 + 1) / 2 * 2;
    P->sh_ld = P->Np + 2 * P->sh_H;
  }
  if (with_stencil)
    IGAFD_TRY(alloc(&P->stencil, P->stencil_half ? (size_t)((P->n_off + 1) / 2) * P->sh_ld
                                                 : (size_t)P->n_off * P->Np));
  IGAFD_TRY(alloc(&P->fd_a, (size_t)N));
  IGAFD_TRY(alloc(&P->fd_b, (size_t)N));
  IGAFD_TRY(alloc(&P->r, (size_t)N));
  IGAFD_TRY(alloc(&P->z, (size_t)N));
  P->halo = igafd_stencil_halo(P->p, P->n);
  IGAFD_TRY(alloc(&P->pv_base, (size_t)(N + 2 * P->halo)));
  IGAFD_TRY(alloc(&P->xpad_base, (size_t)(N + 2 * P->halo)));
  IGAFD_CUDA(cudaMemsetAsync(P->pv_base, 0, (N + 2 * P->halo) * sizeof(double), s));
  IGAFD_CUDA(cudaMemsetAsync(P->xpad_base, 0, (N + 2 * P->halo) * sizeof(double), s));
  IGAFD_TRY(alloc(&P->xs_base, (size_t)(N + 2 * P->halo)));
  IGAFD_CUDA(cudaMemsetAsync(P->xs_base, 0, (N + 2 * P->halo) * sizeof(double), s));
  IGAFD_TRY(alloc(&P->bint, (size_t)N));
  IGAFD_TRY(alloc(&P->tstat, (size_t)4));
  P->pv = P->pv_base + P->halo;
  P->xpad = P->xpad_base + P->halo;
  P->xs = P->xs_base + P->halo;
  IGAFD_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  IGAFD_TRY(alloc(&P->q, (size_t)N));
  IGAFD_TRY(alloc(&P->xt, (size_t)N));
  IGAFD_TRY(alloc(&P->partial, (size_t)IGAFD_PARTIAL_SLOTS * IGAFD_RED_BLOCKS));
  IGAFD_TRY(alloc(&P->counter, (size_t)8));
  IGAFD_TRY(alloc(&P->scal, (size_t)S_COUNT + 1));
  IGAFD_TRY(alloc(&P->coef, 2 * (size_t)IGAFD_COEF_CAP));
  IGAFD_TRY(alloc(&P->err_flag, (size_t)1));
  if (cudaHostAlloc((void **)&P->host_scal, (S_COUNT + 1) * sizeof(double), cudaHostAllocDefault) !=
      cudaSuccess) {
    cudaGetLastError();
    P->host_scal = nullptr;
    return IGAFD_ERR_OOM;
  }
  for (int i = 0; i < IGAFD_NEV; ++i) IGAFD_CUDA(cudaEventCreate(&P->ev[i]));
  IGAFD_CUDA(cudaMemsetAsync(P->counter, 0, 8 * sizeof(unsigned), s));
  IGAFD_CUDA(cudaMemsetAsync(P->scal, 0, (S_COUNT + 1) * sizeof(double), s));
  if (with_stencil) IGAFD_TRY(igafd_setup_stencil(P, s));
  // a full-space patch (a piece of a multi-patch operator) has no P: its
  // pencils include the boundary functions, so its K_k are singular
  if (P->dshift) IGAFD_TRY(igafd_build_prec(P, s));
  igafd_tune_lookup(P);
  IGAFD_CUDA(cudaStreamSynchronize(s));
  return IGAFD_OK;
}

}  // namespace

// P's setup (Section 4.1) on the patch's own buffers: pencils (span-scaled
// when scalings are set), generalized eigendecompositions, 1/(D1 (+) D2 (+)
// D3), FP32 and tensor-core copies of U_k. Synchronises the stream.
igafd_status igafd_build_prec(igafd_patch *P, cudaStream_t s) {
  IGAFD_TRY(igafd_setup_pencils_eig(P, s, P->scaled ? P->wK : nullptr, P->scaled ? P->wM : nullptr));
  IGAFD_TRY(igafd_fd_tc_init(P, s));   // also the FP32 copies U32_k
  IGAFD_CUDA(cudaStreamSynchronize(s));
  return IGAFD_OK;
}

extern "C" igafd_status igafd_setup_prec(igafd_patch *P, void *stream) {
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // a full-space patch has no preconditioner
  if (!P) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  return igafd_build_prec(P, (cudaStream_t)stream);
}

extern "C" igafd_status igafd_set_eig_route(igafd_patch *P, int route) {
  if (!P || (route != 0 && route != 1)) return IGAFD_ERR_ARG;
  P->eig_route = route;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_setup_patch(const igafd_patch_desc *d, void *stream,
                                          igafd_patch **out) {
  if (!out) return IGAFD_ERR_ARG;
  *out = nullptr;
  if (!d || (d->dim != 2 && d->dim != 3) || d->p < 1 || d->p > IGAFD_MAXP || d->geo_p < 1 ||
      d->geo_p > IGAFD_MAXP || !d->n_knots || !d->knots || !d->geo_n_knots || !d->geo_knots ||
      !d->ctrl || !(d->kappa > 0.0) || !std::isfinite(d->kappa))
    return IGAFD_ERR_ARG;
  if (d->kappa_ctrl) {
    if (d->kappa_p < 0 || d->kappa_p > IGAFD_MAXP || !d->kappa_n_knots || !d->kappa_knots)
      return IGAFD_ERR_ARG;
    size_t kc = 1;
    for (int k = 0; k < d->dim; ++k) {
      if (!valid_open_knots(d->kappa_knots[k], d->kappa_n_knots[k], d->kappa_p)) return IGAFD_ERR_ARG;
      kc *= (size_t)(d->kappa_n_knots[k] - d->kappa_p - 1);
    }
    for (size_t i = 0; i < kc; ++i)   // positive control values: kappa > 0 everywhere
      if (!(d->kappa_ctrl[i] > 0.0) || !std::isfinite(d->kappa_ctrl[i])) return IGAFD_ERR_ARG;
  }
  for (int k = 0; k < d->dim; ++k) {
    if (!valid_open_knots(d->knots[k], d->n_knots[k], d->p)) return IGAFD_ERR_ARG;
    if (!valid_open_knots(d->geo_knots[k], d->geo_n_knots[k], d->geo_p)) return IGAFD_ERR_ARG;
    if (d->n_knots[k] - d->p - 1 < 3) return IGAFD_ERR_ARG;   // at least one interior dof
    if (d->n_knots[k] - d->p - 3 > 1024) return IGAFD_ERR_ARG; // eigen-solver limit
  }
  if ((d->flags & IGAFD_SETUP_HALF_STENCIL) &&
      (d->flags & (IGAFD_SETUP_NO_STENCIL | IGAFD_SETUP_FULL_SPACE)))
    return IGAFD_ERR_ARG;
  if (d->flags & ~(IGAFD_SETUP_NO_STENCIL | IGAFD_SETUP_FULL_SPACE | IGAFD_SETUP_HALF_STENCIL))
    return IGAFD_ERR_ARG;
  igafd_patch *P = (igafd_patch *)calloc(1, sizeof(igafd_patch));
  if (!P) return IGAFD_ERR_OOM;
  P->dim = d->dim;
  P->p = d->p;
  P->dshift = (d->flags & IGAFD_SETUP_FULL_SPACE) ? 0 : 1;
  P->geo_p = d->geo_p;
  P->kappa_p = d->kappa_ctrl ? d->kappa_p : 0;
  P->kappa = d->kappa;
  P->fd_fused = 1;
  for (int o = 0; o < 3; ++o) P->fd_fused_op[o] = 1;
  P->stencil_rows = 1;
  if (cudaGetDevice(&P->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->dev) != cudaSuccess) {
    free(P);
    return IGAFD_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  igafd_status st = build(P, d, s);
  if (st == IGAFD_OK) {
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    P->setup_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != IGAFD_OK) {
    cudaStreamSynchronize(s);
    free_patch(P);
    return st;
  }
  *out = P;
  return IGAFD_OK;
}

extern "C" void igafd_destroy_patch(igafd_patch *P) {
  if (!P) return;
  cudaSetDevice(P->dev);
  cudaDeviceSynchronize();
  free_patch(P);
}

extern "C" igafd_status igafd_patch_query(const igafd_patch *P, igafd_patch_info *info) {
  if (!P || !info) return IGAFD_ERR_ARG;
  memset(info, 0, sizeof(*info));
  info->dim = P->dim;
  info->p = P->p;
  for (int k = 0; k < 3; ++k) {
    info->n[k] = P->n[k];
    info->nel[k] = P->nel[k];
  }
  info->N = P->N;
  info->n_offsets = P->n_off;
  info->min_detJ = P->min_detJ;
  info->q_bound = P->q_bound;
  info->setup_ms = P->setup_ms;
  info->eig_ms = P->eig_ms;
  info->stencil_bytes =
      P->stencil ? (long long)(P->stencil_half ? (P->n_off + 1) / 2 : P->n_off) * P->N *
                       (long long)sizeof(double)
                 : 0;
  info->stencil_half = P->stencil_half;
  info->stencil_stages = P->stencil_stages > 0 ? P->stencil_stages : 4;
  info->stencil_rows = P->stencil_rows == 2 ? 2 : 1;
  for (int k = 0; k < 3; ++k) {
    info->eig_refined[k] = k < P->dim && P->eig_used[k] == 0 ? 1 : 0;
    info->eig_check[k][0] = k < P->dim ? P->eig_check[k][0] : 0.0;
    info->eig_check[k][1] = k < P->dim ? P->eig_check[k][1] : 0.0;
    // the form the next apply takes (FP16 and any n_k > 128 run per mode product)
    bool shape_ok = true;
    for (int d = 0; d < P->dim; ++d) shape_ok = shape_ok && P->n[d] <= 128;
    info->fd_fused[k] = P->fd_fused && P->fd_fused_op[k] && k != 2 && shape_ok ? 1 : 0;
    info->fd_tile[k][0] = P->fd_tile[k][0] == 64 ? 64 : 128;
    info->fd_tile[k][1] = P->fd_tile[k][1] == 2 ? 2 : 1;
    info->fd_tile[k][2] = P->fd_tile[k][2] == 3 ? 3 : 2;
    info->fd_tile[k][3] = P->fd_tile[k][3] == 64 ? 64 : 128;
  }
  return IGAFD_OK;
}

extern "C" igafd_status igafd_get_eigen(const igafd_patch *P, int k, double *U_host,
                                        double *D_host) {
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // a full-space patch has no preconditioner
  if (!P || k < 0 || k >= P->dim) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  IGAFD_CUDA(cudaDeviceSynchronize());
  size_t n = P->n[k];
  if (U_host) IGAFD_CUDA(cudaMemcpy(U_host, P->U[k], n * n * sizeof(double), cudaMemcpyDeviceToHost));
  if (D_host) IGAFD_CUDA(cudaMemcpy(D_host, P->D[k], n * sizeof(double), cudaMemcpyDeviceToHost));
  return IGAFD_OK;
}

extern "C" igafd_status igafd_copy_stencil(const igafd_patch *P, double *dst, void *stream) {
  if (!P || !dst || !P->stencil) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  if (P->stencil_half) return igafd_stencil_expand(P, dst, (cudaStream_t)stream);
  IGAFD_CUDA(cudaMemcpy2DAsync(dst, P->N * sizeof(double), P->stencil, P->Np * sizeof(double),
                               P->N * sizeof(double), P->n_off, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return IGAFD_OK;
}

extern "C" const char *igafd_status_str(igafd_status s) {
  switch (s) {
    case IGAFD_OK: return "ok";
    case IGAFD_ERR_ARG: return "invalid argument";
    case IGAFD_ERR_CUDA: return "CUDA runtime error";
    case IGAFD_ERR_NOT_SPD: return "1D mass matrix not positive definite";
    case IGAFD_ERR_EIG: return "eigen-solve did not converge";
    case IGAFD_ERR_FOLDED: return "geometry map folds (det J <= 0)";
    case IGAFD_ERR_BREAKDOWN: return "PCG breakdown";
    case IGAFD_ERR_NOT_CONVERGED: return "PCG did not converge";
    case IGAFD_ERR_TIMEOUT: return "device wait timed out";
    case IGAFD_ERR_OOM: return "out of device memory";
    default: return "unknown status";
  }
}
