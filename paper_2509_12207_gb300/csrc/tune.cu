// Conv tile autotuner: for one layer shape, times every tile that supports it by replaying a
// captured CUDA graph of a few launches (tensor maps encoded once, at capture, so only device
// time is measured) and remembers the fastest.  pp_conv3x3 and the release units use the
// remembered tile whenever they are asked for the library's choice (tile = -1).  The table can
// be written to and read back from a text file, so a deployment tunes once.
#include "pp_internal.h"

#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

namespace pp {
namespace {

using Key = std::tuple<int, int, int, int, int, int, int>;  // dtype, batch, H, W, cin, cout, stride
struct Entry {
  int tile;
  float us;
};
std::mutex g_mu;
std::map<Key, Entry> g_table;

}  // namespace

int tuned_tile(int dtype, const ConvShape& c) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(Key(dtype, c.batch, c.H, c.W, c.cin, c.cout, c.stride));
  return it == g_table.end() ? -1 : it->second.tile;
}

void tune_record(int dtype, int batch, int H, int W, int cin, int cout, int stride, int tile) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[Key(dtype, batch, H, W, cin, cout, stride)] = Entry{tile, 0.f};
}

}  // namespace pp

using namespace pp;

extern "C" {

int pp_conv_autotune(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout,
                     int32_t stride, int32_t dtype, const void* in, const void* w,
                     const float* scale_shift, void* out, int32_t reps, int32_t* best_tile,
                     float* best_us) {
  return pp_conv_autotune_ws(batch, H, W, cin, cout, stride, dtype, in, w, scale_shift, out,
                             nullptr, 0, reps, best_tile, best_us);
}

int pp_conv_autotune_ws(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout,
                        int32_t stride, int32_t dtype, const void* in, const void* w,
                        const float* scale_shift, void* out, void* workspace,
                        size_t workspace_bytes, int32_t reps, int32_t* best_tile, float* best_us) {
  if (reps <= 0 || reps > 1000 || !best_tile) return fail(PP_EINVAL, "conv_autotune: bad argument");
  const int n = pp_conv_tile_count(dtype);
  if (n <= 0) return fail(PP_EINVAL, "conv_autotune: bad dtype");
  cudaStream_t s;
  int st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "autotune stream");
  if (st) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = -1;
  float best_t = 1e30f;
  for (int t = 0; t < n; ++t) {
    // a first plain launch validates the tile for this shape (and sets kernel attributes)
    if (pp_conv3x3_ws(batch, H, W, cin, cout, stride, dtype, in, w, scale_shift, out, t, workspace,
                      workspace_bytes, s) != PP_OK) {
      cudaGetLastError();
      continue;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = fail(PP_EDEVICE, "conv_autotune: tile %d failed on the device", t);
      break;
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = cuda_status(cudaGetLastError(), "conv_autotune: capture");
      break;
    }
    int lst = PP_OK;
    for (int r = 0; r < reps && lst == PP_OK; ++r)
      lst = pp_conv3x3_ws(batch, H, W, cin, cout, stride, dtype, in, w, scale_shift, out, t, workspace,
                          workspace_bytes, s);
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (lst != PP_OK || ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      continue;
    }
    float ms = 0;
    const bool ok = cudaGraphLaunch(ge, s) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess &&
                    cudaGraphLaunch(ge, s) == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
                    cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    if (!ok) {
      st = cuda_status(cudaGetLastError(), "conv_autotune: timing");
      break;
    }
    const float us = ms * 1000.f / (float)reps;
    if (us < best_t) {
      best_t = us;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st) return st;
  if (best < 0) return fail(PP_EINVAL, "conv_autotune: no tile supports this shape");
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[Key(dtype, batch, H, W, cin, cout, stride)] = Entry{best, best_t};
  }
  *best_tile = best;
  if (best_us) *best_us = best_t;
  return PP_OK;
}

int pp_conv_tune_save(const char* path) {
  if (!path) return fail(PP_EINVAL, "conv_tune_save: NULL path");
  FILE* f = fopen(path, "w");
  if (!f) return fail(PP_EINVAL, "conv_tune_save: cannot open %s", path);
  std::lock_guard<std::mutex> lk(g_mu);
  fprintf(f, "# pp conv tiles: dtype batch H W cin cout stride tile us\n");
  for (const auto& kv : g_table) {
    const Key& k = kv.first;
    fprintf(f, "%d %d %d %d %d %d %d %d %.3f\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
            std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), kv.second.tile,
            kv.second.us);
  }
  fclose(f);
  return PP_OK;
}

int pp_conv_tune_load(const char* path) {
  if (!path) return fail(PP_EINVAL, "conv_tune_load: NULL path");
  FILE* f = fopen(path, "r");
  if (!f) return fail(PP_EINVAL, "conv_tune_load: cannot open %s", path);
  char line[256];
  int n = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int v[8];
    float us = 0;
    if (sscanf(line, "%d %d %d %d %d %d %d %d %f", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
               &v[7], &us) != 9)
      continue;
    if (v[7] < 0 || v[7] >= pp_conv_tile_count(v[0])) continue;
    g_table[Key(v[0], v[1], v[2], v[3], v[4], v[5], v[6])] = Entry{v[7], us};
    ++n;
  }
  fclose(f);
  return n;
}

void pp_conv_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
}

}  // extern "C"
