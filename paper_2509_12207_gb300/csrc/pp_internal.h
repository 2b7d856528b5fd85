// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

#include "pp.h"

namespace pp {

// Records `msg` as this thread's last error and returns `code` (for `return fail(...)`).
int fail(int code, const char* fmt, ...);
// Maps a CUDA error to PP_EDEVICE with a message naming `what`; PP_OK for cudaSuccess.
int cuda_status(cudaError_t e, const char* what);
void clear_error();
const char* last_error();

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// SM count of the current device, looked up once per device (152 if the query fails).
int device_sms();
// Sets the dynamic shared-memory limit of kernel `func` to `bytes` on the current device, once
// per device: `done` is the caller's per-kernel set of devices already configured (bit d for
// device d; devices from 64 on are configured on every call).  Thread-safe.
int smem_attr_once(const void* func, int bytes, std::atomic<uint64_t>* done, const char* what);

// The tensor-core conv's sticky device error word (conv_tc.cu): read (and optionally clear) it,
// set bits in it, or get its device address on the current device (for kernels that copy it).
int tc_error_read(unsigned* code, bool clear);
int tc_error_set(unsigned bits);
int tc_error_address(const unsigned** out);

// Programmatic dependent launch.  Kernels that follow another kernel of the library in a stream
// (or graph) are launched with programmatic stream serialisation: they may start while their
// predecessor drains, run their prologue (shared-memory carve-up, barrier init, TMEM
// allocation, tensor-map prefetch), and block in pdl_wait() -- which returns once the
// predecessor grid has completed and its memory is visible -- before they touch any global data
// a predecessor writes or reads.  Every kernel launched this way calls pdl_wait() first
// thing after its prologue.  The persistent tensor-core kernels call pdl_trigger() from their
// MMA thread when it starts the CTA's last tile (one-tile CTAs right after their TMEM
// allocation): never before the CTA's own TMEM allocation, so that a dependent CTA sharing the
// SM cannot take the columns a predecessor CTA still has to allocate; and late, so that the
// next layer's CTAs, which hold an SM while they wait, take only SMs that are about to free up.
// The short kernels do not trigger (a CTA's exit is its trigger): dependents launched at their
// start held SM slots while blocked and measured slower.  PP_PDL=0 in the environment turns
// it off (plain stream order).
bool pdl_enabled();
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}
#endif

// Kernel-side copy of the geometry with derived sizes.
struct Geom {
  float xmin, xmax, ymin, ymax, zmin, zmax, vx, vy;
  int nx, ny, G, P;
  uint64_t nx_magic;  // ceil(2^64 / nx) for nx >= 2 (cell / nx by one multiply-high), else 0
};

int check_geometry(const pp_geometry* g, Geom* out);

// ---- voxelisation (vox.cu)
struct VoxWork {
  int* err;          // [1] sticky error word
  int* slot;         // [B][cap] arrival slot of a point inside its cell
  int* csr;          // [B][cap] point indices grouped by kept pillar
  int* pillar_start; // [B][P]
  int* pillar_cnt;   // [B][P]
  int2* tile_sums;   // [B][ntiles] (occupied cells, points) per tile of cells
  int ntiles;
};
constexpr int kVoxTile = 2048;        // cells per scan tile (256 threads x 8)
size_t vox_workspace_bytes(const Geom& g, int batch, int cap);
VoxWork vox_carve(void* ws, const Geom& g, int batch, int cap);
// srcs: optional device table of per-frame point pointers (frame b reads srcs[b][0..n));
// NULL = frame b is row b of `points` ([batch][cap]).
// How a release unit feeds the voxeliser (the stage entry points pass none).  Its per-launch
// table lives in page-locked host memory: the first kernel reads its own entries there (device
// view of the mapping) and copies the whole table to device memory for the kernels after it,
// so that no copy precedes the unit's graph.  The unit's cell counts start at zero and the scan
// leaves them zero again (no clearing pass).
struct VoxUnitIO {
  const int* first_counts = nullptr;           // host-mapped table entries the first kernel reads
  const float4* const* first_srcs = nullptr;
  float4* const* first_mirrors = nullptr;
  const uint4* table_src = nullptr;            // host-mapped table ...
  uint4* table_dst = nullptr;                  // ... copied here (table_words 16-byte words)
  int table_words = 0;
  // the counts start zero (no memset); the scan then leaves each kept cell's pillar start + 1
  // there for the bucket pass (a dropped cell's count back at zero), and the PointNet pass
  // (select_pfn_launch's cnt_zero) zeroes the kept cells' entries again for the next launch
  bool cnt_clean = false;
  // a release unit's persistent canvas (canvas != NULL): the bucket pass also zeroes the cells
  // drawn for each slot's previous frame (drawn / drawn_num) that hold no kept pillar now, in
  // `canvas_chunks` 16-byte chunks per pixel (both planes of the split FP32 form, lo != NULL)
  uint4* canvas = nullptr;
  uint4* canvas_lo = nullptr;
  int canvas_chunks = 0;
  const int* drawn = nullptr;
  const int* drawn_num = nullptr;
};
// pts == NULL: stop after the bucket step (the caller runs select_pfn_launch, which gathers
// each pillar's points itself).  mirrors: device table of per-frame destinations (NULL
// entries skip) into which the first pass copies the points it reads.
int vox_launch(const Geom& g, int batch, int cap, const float4* points, const int* n_points,
               int* cell, unsigned* cnt, int* pillar_of_cell, int* coord, int* npts,
               int* num_pillars, float4* pts, const VoxWork& w, cudaStream_t s,
               const float4* const* srcs = nullptr, float4* const* mirrors = nullptr,
               const VoxUnitIO* io = nullptr);

// ---- PointNet and scatter (pfn.cu)
int pfn_launch(const Geom& g, int batch, const float4* pts, const int* npts, const int* coord,
               const int* num_pillars, const float* pfn_w, const float* scale_shift,
               float* feat, cudaStream_t s);
// Point selection + PointNet in one launch, from the voxelisation workspace (csr, pillar
// start / count) of the same batch: feat as pfn_launch computes it, without the pts buffer.
// cnt_zero (a release unit whose count array the scan turned into the bucket's lookup): each
// kept pillar's cell entry is set back to zero.
// With `canvas` (a release unit): each pillar's 64 features also go straight to its cell of the
// persistent canvas (FP32 value + TF32 remainder plane `lo`, or BF16 round to nearest even, in
// `chunks` 16-byte chunks per pixel), its cell to drawn[b][p] and the pillar count to
// drawn_num[b]; feat may then be NULL.
int select_pfn_launch(const Geom& g, int batch, int cap, const float4* points, const float4* const* srcs,
                      const VoxWork& w, const int* coord, const int* num_pillars, const float* pfn_w,
                      const float* ss, float* feat, cudaStream_t s, int chunks = 0, int* drawn = nullptr,
                      int* drawn_num = nullptr, uint4* canvas = nullptr, uint4* lo = nullptr,
                      unsigned* cnt_zero = nullptr);
// lo[i] = TF32 remainder of x[i] (x, lo 16-byte aligned when n >= 4).
int tf32_split_launch(const float* x, float* lo, size_t n, cudaStream_t s);
// PP_F32_TC: `plane` = elements between the canvas's value and remainder planes (0 = this
// batch's plane size).
int scatter_launch(const Geom& g, int batch, const float* feat, const int* pillar_of_cell,
                   void* canvas, int dtype, cudaStream_t s, size_t plane = 0);
// Incremental scatter (pp_scatter_update): zero the stale cells of the previous frame, write the
// new pillars, record them in drawn / drawn_num.  plane: floats per plane of a split FP32 canvas
// (0 = batch-sized).
int scatter_update_launch(const Geom& g, int batch, const float* feat, const int* coord, const int* num_pillars,
                          const int* pillar_of_cell, int* drawn, int* drawn_num, void* canvas, int dtype,
                          cudaStream_t s, size_t plane = 0);

// ---- conv (conv_simt.cu, conv_tc.cu)
struct ConvShape {
  int batch, H, W, cin, cout, stride, Ho, Wo;
  // split FP32 (PP_F32_TC): elements between the value and remainder planes of the input and
  // the output; 0 = this batch's plane size (planes packed for exactly `batch` frames)
  size_t in_plane = 0, out_plane = 0;
  // the weights and the folded BN scale/shift were written before the previous kernel in the
  // stream started (a release unit's, packed at creation): a kernel may load them before its
  // dependent-launch wait
  bool static_w = false;
  // a release unit's last layer: frame b's output goes to frame_dst[b] + frame_off (its result
  // slot, a padded [Ho+2][Wo+2][cout] map whose border stays zero) when that entry is non-NULL,
  // else to the output buffer as usual; frame_dst is a device array of batch pointers (the
  // unit table's), read when the epilogue runs.  skip_lo: split FP32 output without its
  // remainder plane (no later layer reads it).  Tensor-core convs only.
  char* const* frame_dst = nullptr;
  size_t frame_off = 0;
  bool skip_lo = false;
};
// The persistent tensor-core kernel as a general implicit GEMM (see conv_tc.cu PArgs): taps 9 =
// 3x3 conv, 1 = pointwise; up > 1 = transposed conv with kernel = stride = up (GEMM N =
// up * up * co_blk); output written at channel offset out_coff of an out_c-channel map; relu 0 =
// bias-only epilogue (scale_shift = [1.., bias..]).  Zero fields take the 3x3-conv defaults.
struct GemmOpts {
  int taps = 9, up = 1, co_blk = 0, out_c = 0, out_coff = 0, relu = 1;
};
// dtype PP_BF16 (mode 0) or PP_F32_TC (mode 1, split FP32 operands); tile: persistent tile
// index or -1 (shape heuristic).
int gemm_tc_launch(int dtype, const ConvShape& c, const GemmOpts& g, const void* in, const void* w,
                   const float* ss, void* out, int tile, cudaStream_t s);
int conv_f32_launch(const ConvShape& c, const float* in, const float* w_kn, const float* ss,
                    float* out, int tile, cudaStream_t s);
int conv_f32_tile_count();
int conv_bf16_launch(const ConvShape& c, const __nv_bfloat16* in, const __nv_bfloat16* w_nk,
                     const float* ss, __nv_bfloat16* out, int tile, cudaStream_t s);
int conv_bf16_tile_count();
// ws: stream-K workspace (conv_sk_workspace_bytes, zeroed once; NULL = no stream-K tiles).
int conv_f32tc_launch(const ConvShape& c, const float* in, const float* w_split, const float* ss,
                      float* out, int tile, cudaStream_t s, void* ws = nullptr, size_t ws_bytes = 0);
size_t conv_sk_workspace_bytes(const ConvShape& c);
int conv_f32tc_tile_count();
int conv_tc_tile_info(int dtype, int tile, int* bh, int* bw, int* bn, int* persistent);
// Tile the autotuner found fastest for this dtype and shape, or -1 (tune.cu).
int tuned_tile(int dtype, const ConvShape& c);
// Records `tile` as the library's choice for this (dtype, layer shape) without timing it.
void tune_record(int dtype, int batch, int H, int W, int cin, int cout, int stride, int tile);
int conv_pack_launch(const float* w_oihw, int cin, int cout, int dtype, void* dst, cudaStream_t s);

// ---- synthetic GPU load (synth.cu): kernels of set utilisation and duration
struct SynthBuf {
  void* ab = nullptr;  // [2][SMs][slice] float4 inputs
  void* c = nullptr;   // [units][SMs][slice] float4 outputs, one region per synthetic unit
  int sms = 0, units = 0;
};
int synth_alloc(SynthBuf* b, int units);
void synth_free(SynthBuf* b);
int synth_ctas(const SynthBuf& b, double util);  // round(util x SMs), 1..SMs
// n_kernels launches of `iters` passes each with `ctas` CTAs on s, into unit `unit`'s region.
int synth_launch(const SynthBuf& b, int unit, int ctas, int iters, int n_kernels, cudaStream_t s);
// Passes per launch that make one launch of `ctas` CTAs last about kernel_us (synchronous).
int synth_calibrate(const SynthBuf& b, int ctas, double kernel_us, cudaStream_t s, int* iters);

}  // namespace pp
