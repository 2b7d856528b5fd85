// A release unit's device state: buffers for up to B frames, the whole-frame launch sequence
// (voxelise -> PointNet -> scatter -> backbone) and one CUDA graph per batch size.
#pragma once

#include <vector>

#include "pp_internal.h"

namespace pp {

struct LayerSpec {
  int cin, cout, stride, H, W, Ho, Wo;
};

constexpr int kMaxUnit = 8;  // frames per release unit

// Per-launch table a unit's kernels read from device memory, so that one captured graph serves
// any frames: counts, where each frame's points are, where its block outputs go.
struct UnitTable {
  int32_t counts[kMaxUnit];
  int32_t pad[kMaxUnit];
  const float4* src[kMaxUnit];   // frame's points (a borrowed buffer, or a staging row)
  char* dst[kMaxUnit];           // frame's result slot (NULL: leave outputs in the unit)
  float4* mirror[kMaxUnit];      // where the first voxelise pass copies points read over the
                                 // host link (a borrowed page-locked frame), else NULL
  const float4* gsrc[kMaxUnit];  // where the point gather reads: the frame in device memory
  char* hdst[kMaxUnit];          // page-locked host copy of the frame's final output (device
                                 // view of the mapping; written over the host link), else NULL
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
  // neck + head (head_outputs > 0): per block a transposed conv of kernel = stride =
  // up_stride[b] into channels [b * up_c, (b + 1) * up_c) of the neck map, then the 1x1 head
  int head_outputs = 0;
  int head_c = 0;                // head_outputs rounded up to 64 (the GEMM's N)
  int up_c = 0, neck_c = 0;      // channels per upsampled block, of the neck map
  std::vector<int> up_stride;
  std::vector<void*> up_w;       // packed for pp_upsample
  std::vector<float*> up_ss;     // [2][up_c]
  void* head_w = nullptr;        // packed for pp_head
  float* head_ss = nullptr;      // [2][head_c]: 1 and the bias
  size_t bytes = 0;
  int upload(const pp_config* cfg, int precision, cudaStream_t s);
  bool keep_blocks = false;      // result slots hold every block's output (else the last one's)
  // Blocks whose outputs a result slot holds, in order (none with a head: the head map).
  std::vector<int> kept_blocks() const;
  // Result slot layout: each kept block's padded NHWC output at a 256-byte aligned offset
  // (block_off[k] for kept_blocks()[k]; with a head: the head map alone, one offset).
  size_t result_layout(std::vector<size_t>* block_off) const;
  int out_h() const { return layers[block_end[0]].Ho; }  // neck / head map size (block 0's)
  int out_w() const { return layers[block_end[0]].Wo; }
  // Bytes of a frame's final output (last block, or the head map), padded NHWC.
  size_t final_bytes() const;
  void release();
};

class Pipeline {
 public:
  // tune: autotune every conv layer for unit sizes 1..max_batch before capturing the graphs
  // stream_k: own a stream-K workspace and let the autotuner consider stream-K tiles
  int init(const Model* m, int max_batch, int cap_points, bool graphs, bool tune, bool stream_k,
           cudaStream_t s);
  void release();
  // Enqueues the whole front end for `n` frames on `s` (graph or plain launches).  Frame i is
  // read in place when direct[i] (a 16-byte aligned device or page-locked host buffer), else
  // staged into slot i (host or device pointer, cudaMemcpyDefault).  A direct frame with
  // host_mapped[i] is read over the host link once, by the first voxelise pass, which copies it
  // into slot i for the point gather.  When dst[i] is set, the blocks' outputs are copied to it
  // (result_layout) inside the same graph.  direct / host_mapped / dst may be NULL.
  // hdst[i] (may be NULL): a page-locked host buffer (its device view) that also receives the
  // frame's final output (last block, or the head map), written by the same copy kernel over
  // the host link.
  int run(int n, const float* const* frames, const int* counts, const bool* direct,
          char* const* dst, bool use_graph, cudaStream_t s, const bool* host_mapped = nullptr,
          char* const* hdst = nullptr);
  // Enqueues the kernels for slots 0..n-1 (points and counts already in place).
  int enqueue(int n, cudaStream_t s);
  size_t bytes() const { return bytes_; }
  int max_batch() const { return B_; }
  int cap() const { return cap_; }
  // Output of layer `layer` (padded NHWC) for slot `i`.
  const void* layer_out(int layer, int i) const;
  // Neck map / head map (padded NHWC, value plane) for slot `i`; NULL without a head.
  const void* neck_out(int i) const;
  const void* head_out(int i) const;
  const Model* model() const { return m_; }
  int* num_pillars_dev() const { return num_; }
  // pinned copy of num_pillars, written at the end of every run (valid once it completes)
  const int* num_pillars_host() const { return num_host_; }
  // The device error words as the run's last kernel saw them (valid once the run completes):
  // the tensor-core conv's sticky word (a bounded wait ran out: that conv skipped its stores)
  // in the low 31 bits, bit 31 for the voxeliser's (a point count outside [0, capacity]).
  // Nonzero means the run's outputs are not to be trusted.
  unsigned device_error_host() const { return (unsigned)num_host_[B_]; }

 private:
  const Model* m_ = nullptr;
  int B_ = 0, cap_ = 0;
  size_t bytes_ = 0;
  float4* points_ = nullptr;
  UnitTable* tab_dev_ = nullptr;
  UnitTable* tab_host_ = nullptr;  // pinned; rewritten only once the previous run completed
  UnitTable* tab_map_ = nullptr;   // its device view (read by the first kernel of a run)
  int* num_host_ = nullptr;        // pinned [B + 1], written by the unit's last kernel: the
                                   // pillar counts, then the device error words
  const unsigned* tc_err_ = nullptr;  // device address of the tensor-core conv's error word
  int* num_host_dev_ = nullptr;    // its device view
  cudaEvent_t tab_ev_ = nullptr;   // after the last run (whose first kernel read the table)
  std::vector<size_t> res_off_;
  size_t hout_off_ = 0, hout_bytes_ = 0;  // the final output inside a result slot
  int sms_ = 1;
  int *cell_ = nullptr, *poc_ = nullptr, *coord_ = nullptr, *npts_ = nullptr, *num_ = nullptr;
  unsigned* cnt_ = nullptr;
  void* vox_ws_ = nullptr;
  VoxWork vw_{};
  void* canvas_ = nullptr;   // persists across runs: updated in place (pp_scatter_update)
  int* drawn_ = nullptr;     // [B][P] cells drawn into each slot's canvas by its last frame
  int* drawn_num_ = nullptr; // [B]
  void* conv_ws_ = nullptr;  // stream-K workspace shared by the unit's (stream-ordered) convs
  size_t conv_ws_bytes_ = 0;
  std::vector<void*> act_;
  void* neck_ = nullptr;     // [planes][B][H0+2][W0+2][neck_c]
  void* head_ = nullptr;     // [planes][B][H0+2][W0+2][head_c]
  std::vector<cudaGraphExec_t> graphs_;
  std::vector<void*> allocs_;
  int alloc(void** p, size_t n);
};

}  // namespace pp
