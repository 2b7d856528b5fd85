// A release unit's device state: buffers for up to B frames, the whole-frame launch sequence
// (voxelise -> PointNet -> scatter -> backbone) and one CUDA graph per batch size.
#pragma once

#include <vector>

#include "pp_internal.h"

namespace pp {

struct LayerSpec {
  int cin, cout, stride, H, W, Ho, Wo;
};

struct Model {
  Geom g;
  std::vector<LayerSpec> layers;
  std::vector<int> block_end;  // index of the last layer of each block
  int precision;               // PP_F32 / PP_BF16
  int conv_dtype;              // PP_F32 (CUDA cores), PP_F32_TC (3xTF32) or PP_BF16
  // device weights
  float* pfn_w = nullptr;        // [64][9]
  float* pfn_ss = nullptr;       // [2][64]
  std::vector<void*> conv_w;     // packed per precision
  std::vector<float*> conv_ss;   // [2][cout]
  size_t bytes = 0;
  int upload(const pp_config* cfg, int precision, cudaStream_t s);
  void release();
};

class Pipeline {
 public:
  // tune: autotune every conv layer for unit sizes 1..max_batch before capturing the graphs
  int init(const Model* m, int max_batch, int cap_points, bool graphs, bool tune, cudaStream_t s);
  void release();
  // Stages `n` frames (device or host pointers, cudaMemcpyDefault) into slots 0..n-1 and
  // enqueues the whole front end for them on `s` (graph or plain launches).
  int run(int n, const float* const* frames, const int* counts, bool use_graph, cudaStream_t s);
  // Enqueues the kernels for slots 0..n-1 (points and counts already in place).
  int enqueue(int n, cudaStream_t s);
  size_t bytes() const { return bytes_; }
  int max_batch() const { return B_; }
  int cap() const { return cap_; }
  // Output of layer `layer` (padded NHWC) for slot `i`.
  const void* layer_out(int layer, int i) const;
  const Model* model() const { return m_; }
  int* num_pillars_dev() const { return num_; }
  float4* points_dev() const { return points_; }
  int* counts_dev() const { return n_dev_; }
  int* counts_host() const { return n_host_; }
  // pinned copy of num_pillars, written at the end of every run (valid once it completes)
  const int* num_pillars_host() const { return num_host_; }

 private:
  const Model* m_ = nullptr;
  int B_ = 0, cap_ = 0;
  size_t bytes_ = 0;
  float4* points_ = nullptr;
  int* n_dev_ = nullptr;
  int* n_host_ = nullptr;    // pinned [B]
  int* num_host_ = nullptr;  // pinned [B]
  int *cell_ = nullptr, *poc_ = nullptr, *coord_ = nullptr, *npts_ = nullptr, *num_ = nullptr;
  unsigned* cnt_ = nullptr;
  float4* pts_ = nullptr;
  void* vox_ws_ = nullptr;
  VoxWork vw_{};
  float* feat_ = nullptr;
  void* canvas_ = nullptr;
  std::vector<void*> act_;
  std::vector<cudaGraphExec_t> graphs_;
  std::vector<void*> allocs_;
  int alloc(void** p, size_t n);
};

}  // namespace pp
