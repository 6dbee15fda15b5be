// Autotuner for the hot kernels of a patch.
//
// The stencil pipeline is built for several ring depths (offset groups in
// flight per CTA: 3, 4, 6) and, in 3D, for one or two rows per compute
// thread. The best choice depends on the degree (bytes per stage grow with
// 2p+1, trading shared memory per CTA against resident CTAs per SM) and on
// the sizes, so it is measured: each candidate applies A a few times to the
// patch's own search-direction buffer, timed with CUDA events, and the
// fastest is kept in the patch. The tensor-core FD is built in two forms for
// TF32 and BF16 operands: fused (two mode products per CTA, 128-row tiles of
// whole slabs or column blocks, the intermediate kept on chip; three kernels)
// and one kernel per mode product (128-row tiles, K in 64-wide chunks
// through a two-stage ring; 2d kernels). Which is faster depends on the
// sizes (ragged n_k pad the fused tiles), so both are timed on the patch's
// own residual buffer and the faster is kept per operand type. Results are cached per
// process, keyed by (dim, p, n_1, n_2, n_3, SM count), and, when the
// environment variable IGAFD_TUNE_CACHE names a file, in that file (one JSON
// object per line), so later processes reuse them without measuring.
#include "common.cuh"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

namespace {

constexpr int kNumCand = 6;

struct TuneEntry {
  int stages, rows;
  float ms[kNumCand];   // candidate c: depth kCandidates[c % 3], rows 1 + c / 3
  int fd_fused[2];      // TF32, BF16: 1 fused, 0 per mode product
  float fd_ms[4];       // TF32 fused, TF32 per mode, BF16 fused, BF16 per mode: the best
                        // time of each form over its tile shapes (-1: not timed)
  int fd_tile[3][4];    // TF32, BF16, FP16: the chosen tile shape (igafd_patch::fd_tile)
  float fp16_ms;        // FP16 (per mode product only): the best time
};

void default_tiles(TuneEntry &e) {
  for (int o = 0; o < 3; ++o) {
    e.fd_tile[o][0] = 128; e.fd_tile[o][1] = 1; e.fd_tile[o][2] = 2; e.fd_tile[o][3] = 128;
  }
  e.fp16_ms = -1.0f;
}

std::mutex g_tune_mutex;
std::map<std::string, TuneEntry> g_tune;
bool g_tune_loaded = false;
const int kCandidates[3] = {3, 4, 6};

std::string tune_key(const igafd_patch *P) {
  char buf[128];
  snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%d:sm%d%s", P->dim, P->p, P->n[0], P->n[1], P->n[2],
           P->num_sms, P->stencil_half ? ":half" : "");
  return buf;
}

// lines: {"key": "3:3:128:128:128:sm152", "stencil_stages": 4, "stencil_rows": 2,
//         "ms": [six times, -1 where not measured], "fd_fused": [1, 1],
//         "fd_ms": [four times]}
void load_file_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = getenv("IGAFD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    char key[128];
    TuneEntry e{};
    e.fd_fused[0] = e.fd_fused[1] = 1;
    for (int i = 0; i < 4; ++i) e.fd_ms[i] = -1.0f;
    default_tiles(e);
    int t[12];
    const int got = sscanf(line,
               " {\"key\": \"%127[^\"]\", \"stencil_stages\": %d, \"stencil_rows\": %d, "
               "\"ms\": [%f, %f, %f, %f, %f, %f], \"fd_fused\": [%d, %d], "
               "\"fd_ms\": [%f, %f, %f, %f], \"fd_tile\": [[%d, %d, %d, %d], [%d, %d, %d, %d], "
               "[%d, %d, %d, %d]], \"fp16_ms\": %f",
               key, &e.stages, &e.rows, &e.ms[0], &e.ms[1], &e.ms[2], &e.ms[3], &e.ms[4],
               &e.ms[5], &e.fd_fused[0], &e.fd_fused[1], &e.fd_ms[0], &e.fd_ms[1], &e.fd_ms[2],
               &e.fd_ms[3], &t[0], &t[1], &t[2], &t[3], &t[4], &t[5], &t[6], &t[7], &t[8], &t[9],
               &t[10], &t[11], &e.fp16_ms);
    // 28: every field; 15: written before tile shapes were tuned; 9: before the FD was
    if (got == 28 || got == 15 || got == 9) {
      if (got == 9) e.fd_fused[0] = e.fd_fused[1] = 1;
      if (got == 28)
        for (int i = 0; i < 12; ++i) e.fd_tile[i / 4][i % 4] = t[i];
      g_tune[key] = e;
    }
  }
  fclose(f);
}

void append_file_locked(const std::string &key, const TuneEntry &e) {
  const char *path = getenv("IGAFD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  const int(*t)[4] = e.fd_tile;
  fprintf(f,
          "{\"key\": \"%s\", \"stencil_stages\": %d, \"stencil_rows\": %d, "
          "\"ms\": [%.5f, %.5f, %.5f, %.5f, %.5f, %.5f], \"fd_fused\": [%d, %d], "
          "\"fd_ms\": [%.5f, %.5f, %.5f, %.5f], \"fd_tile\": [[%d, %d, %d, %d], [%d, %d, %d, %d], "
          "[%d, %d, %d, %d]], \"fp16_ms\": %.5f}\n",
          key.c_str(), e.stages, e.rows, e.ms[0], e.ms[1], e.ms[2], e.ms[3], e.ms[4], e.ms[5],
          e.fd_fused[0], e.fd_fused[1], e.fd_ms[0], e.fd_ms[1], e.fd_ms[2], e.fd_ms[3], t[0][0],
          t[0][1], t[0][2], t[0][3], t[1][0], t[1][1], t[1][2], t[1][3], t[2][0], t[2][1], t[2][2],
          t[2][3], e.fp16_ms);
  fclose(f);
}

}  // namespace

// Apply a cached choice (if any) at set-up time; measures nothing.
void igafd_tune_lookup(igafd_patch *P) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  load_file_locked();
  auto it = g_tune.find(tune_key(P));
  if (it != g_tune.end()) {
    P->stencil_stages = it->second.stages;
    P->stencil_rows = it->second.rows;
    P->fd_fused_op[0] = it->second.fd_fused[0];
    P->fd_fused_op[1] = it->second.fd_fused[1];
    memcpy(P->fd_tile, it->second.fd_tile, sizeof(P->fd_tile));
  }
}

// Time `reps` tensor-core FD applies (after one untimed) of operand type dt
// on the patch's residual buffer; ms per apply into *ms.
static igafd_status time_fd(igafd_patch *P, igafd_dtype dt, cudaStream_t s, cudaEvent_t e0,
                            cudaEvent_t e1, float *ms) {
  constexpr int reps = 5;
  IGAFD_TRY(igafd_fd_tc_apply(P, dt, P->r, P->z, s, nullptr));
  IGAFD_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) IGAFD_TRY(igafd_fd_tc_apply(P, dt, P->r, P->z, s, nullptr));
  IGAFD_CUDA(cudaEventRecord(e1, s));
  IGAFD_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  IGAFD_CUDA(cudaEventElapsedTime(&t, e0, e1));
  *ms = t / reps;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_autotune(igafd_patch *P, int flags, void *stream) {
  if (P && !P->dshift) return IGAFD_ERR_ARG;   // full-space patches are not tuned
  if (!P || !P->stencil) return IGAFD_ERR_ARG;
  IGAFD_CUDA(cudaSetDevice(P->dev));
  const std::string key = tune_key(P);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_file_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end() && !(flags & 1)) {
      P->stencil_stages = it->second.stages;
      P->stencil_rows = it->second.rows;
      P->fd_fused_op[0] = it->second.fd_fused[0];
      P->fd_fused_op[1] = it->second.fd_fused[1];
      memcpy(P->fd_tile, it->second.fd_tile, sizeof(P->fd_tile));
      return IGAFD_OK;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  IGAFD_CUDA(cudaEventCreate(&e0));
  IGAFD_CUDA(cudaEventCreate(&e1));
  TuneEntry best{};
  best.stages = 4;
  best.rows = 1;
  float best_ms = 1e30f;
  const int saved = P->stencil_stages, saved_rows = P->stencil_rows;
  const int ncand = P->dim == 3 ? kNumCand : 3;
  igafd_status st = IGAFD_OK;
  for (int c = 0; c < kNumCand; ++c) best.ms[c] = -1.0f;
  for (int c = 0; c < ncand && st == IGAFD_OK; ++c) {
    // a half-stored stencil runs at the default depth: only its rows are tuned
    if (P->stencil_half && kCandidates[c % 3] != 4) continue;
    P->stencil_stages = kCandidates[c % 3];
    P->stencil_rows = 1 + c / 3;
    st = igafd_stencil_launch(P, P->pv, P->q, nullptr, 0, 0, s);     // warm-up
    if (st != IGAFD_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 5 && st == IGAFD_OK; ++r) st = igafd_stencil_launch(P, P->pv, P->q, nullptr, 0, 0, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = IGAFD_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best.ms[c] = ms / 5;
    if (best.ms[c] < best_ms) {
      best_ms = best.ms[c];
      best.stages = kCandidates[c % 3];
      best.rows = 1 + c / 3;
    }
  }
  // Tensor-core FD per operand type: its form (fused, which needs every
  // n_k <= 128, or one kernel per mode product) and that form's tile shape,
  // every candidate timed on the patch. Fused: the pencil kernel's columns
  // per CTA (128, or 64 on a half-filled MMA tile; the compile-time-sized
  // n_k = 128 kernels have none). Per mode product: rows per CTA {128, 64},
  // one or two column tiles, and a third K stage where some n_k > 128 and it
  // fits in shared memory.
  const bool have_tc = P->mixed != nullptr;
  bool shape_ok = have_tc;
  int nmax = 0, npmin = 1 << 30;
  for (int k = 0; k < P->dim; ++k) {
    shape_ok = shape_ok && P->n[k] <= 128;
    nmax = P->n[k] > nmax ? P->n[k] : nmax;
    const int np = (P->n[k] + 15) / 16 * 16;
    npmin = np < npmin ? np : npmin;
  }
  const bool n128 = P->dim == 3 && P->n[0] == 128 && P->n[1] == 128 && P->n[2] == 128;
  const int saved_fused = P->fd_fused, saved_op[2] = {P->fd_fused_op[0], P->fd_fused_op[1]};
  int saved_tile[3][4];
  memcpy(saved_tile, P->fd_tile, sizeof(saved_tile));
  for (int i = 0; i < 4; ++i) best.fd_ms[i] = -1.0f;
  default_tiles(best);
  best.fd_fused[0] = best.fd_fused[1] = shape_ok ? 1 : 0;
  const igafd_dtype dts[3] = {IGAFD_TF32, IGAFD_BF16, IGAFD_FP16};
  P->fd_fused = 1;
  bool fits256 = true;
  for (int k = 0; k < P->dim; ++k) fits256 = fits256 && P->n[k] <= 256;
  for (int o = 0; o < 3 && st == IGAFD_OK && have_tc && fits256; ++o) {
    const int bytes = o == 0 ? 4 : 2;
    float best_o = 1e30f;
    auto trial = [&](int fused, int m, int nd, int stg, int pm) {
      if (o < 2) P->fd_fused_op[o] = fused;
      P->fd_tile[o][0] = m; P->fd_tile[o][1] = nd; P->fd_tile[o][2] = stg; P->fd_tile[o][3] = pm;
      float ms = 0.f;
      st = time_fd(P, dts[o], s, e0, e1, &ms);
      if (st != IGAFD_OK) return;
      float *slot = o < 2 ? &best.fd_ms[2 * o + (fused ? 0 : 1)] : &best.fp16_ms;
      if (*slot < 0.f || ms < *slot) *slot = ms;
      if (ms < best_o) {
        best_o = ms;
        if (o < 2) best.fd_fused[o] = fused;
        best.fd_tile[o][0] = m; best.fd_tile[o][1] = nd; best.fd_tile[o][2] = stg;
        best.fd_tile[o][3] = pm;
      }
    };
    if (o < 2 && shape_ok) {
      trial(1, 128, 1, 2, 128);
      if (P->dim == 3 && !n128 && st == IGAFD_OK) trial(1, 128, 1, 2, 64);
    }
    for (int m = 128; m >= 64 && st == IGAFD_OK; m -= 64)
      for (int nd = 1; nd <= 2 && st == IGAFD_OK; ++nd) {
        if (nd == 2 && npmin < 32) continue;
        for (int stg = 2; stg <= 3 && st == IGAFD_OK; ++stg) {
          if (stg == 3) {            // only with more than two K chunks, and if it fits
            const int npm = (nmax + 15) / 16 * 16;
            const int nt = nd == 2 ? (npm / 2 + 15) / 16 * 16 : npm;
            const size_t smem = 1024 + (size_t)3 * (128 + nt) * 64 * bytes;
            if (nmax <= 128 || smem > 227 * 1024) continue;
          }
          trial(0, m, nd, stg, 128);
        }
      }
  }
  memcpy(P->fd_tile, saved_tile, sizeof(saved_tile));
  P->fd_fused = saved_fused;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != IGAFD_OK) {
    P->stencil_stages = saved;
    P->stencil_rows = saved_rows;
    P->fd_fused_op[0] = saved_op[0];
    P->fd_fused_op[1] = saved_op[1];
    return st;
  }
  P->stencil_stages = best.stages;
  P->stencil_rows = best.rows;
  P->fd_fused_op[0] = best.fd_fused[0];
  P->fd_fused_op[1] = best.fd_fused[1];
  memcpy(P->fd_tile, best.fd_tile, sizeof(P->fd_tile));
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[key] = best;
  append_file_locked(key, best);
  return IGAFD_OK;
}

extern "C" igafd_status igafd_set_stencil_stages(igafd_patch *P, int stages) {
  if (!P || (stages != 3 && stages != 4 && stages != 6)) return IGAFD_ERR_ARG;
  P->stencil_stages = stages;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_set_stencil_rows(igafd_patch *P, int rows) {
  if (!P || (rows != 1 && rows != 2) || (rows == 2 && P->dim != 3)) return IGAFD_ERR_ARG;
  P->stencil_rows = rows;
  return IGAFD_OK;
}

extern "C" igafd_status igafd_set_fd_fused(igafd_patch *P, int fused) {
  if (!P || (fused != 0 && fused != 1)) return IGAFD_ERR_ARG;
  P->fd_fused = fused;
  for (int o = 0; o < 3; ++o) P->fd_fused_op[o] = 1;   // an explicit choice overrides the autotuner
  return IGAFD_OK;
}

extern "C" igafd_status igafd_set_fd_tile(igafd_patch *P, igafd_dtype dtype, const int *tile) {
  if (!P || !tile) return IGAFD_ERR_ARG;
  const int o = dtype == IGAFD_TF32 ? 0 : dtype == IGAFD_BF16 ? 1 : dtype == IGAFD_FP16 ? 2 : -1;
  if (o < 0 || (tile[0] != 64 && tile[0] != 128) || (tile[1] != 1 && tile[1] != 2) ||
      (tile[2] != 2 && tile[2] != 3) || (tile[3] != 64 && tile[3] != 128))
    return IGAFD_ERR_ARG;
  const int bytes = o == 0 ? 4 : 2;
  int nmax = 0;
  for (int k = 0; k < P->dim; ++k) nmax = P->n[k] > nmax ? P->n[k] : nmax;
  const int npm = (nmax + 15) / 16 * 16;
  const int nt = tile[1] == 2 ? (npm / 2 + 15) / 16 * 16 : npm;
  if (1024 + (size_t)tile[2] * (128 + nt) * 64 * bytes > 227 * 1024) return IGAFD_ERR_ARG;
  for (int i = 0; i < 4; ++i) P->fd_tile[o][i] = tile[i];
  return IGAFD_OK;
}
