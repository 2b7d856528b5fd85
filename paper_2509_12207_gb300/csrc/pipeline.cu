// Release unit: device buffers for up to B frames, the whole pillar front end as one launch
// sequence (voxelise -> point selection + PointNet -> incremental scatter -> conv3x3 layers), and
// one CUDA graph per batch size 1..B so that a unit launch costs one cudaGraphLaunch.  Per-frame
// point counts live in device memory, so a graph replays any mix of uneven frames: grids are
// sized for the unit's capacity and blocks past a frame's count exit at once.
#include "pipeline.h"

#include <algorithm>
#include <cstring>
#include <new>

namespace pp {

namespace {

// Where the block outputs of slot 0 are, how far apart the slots lie, and where each block goes
// inside a result slot.
struct ResultCopy {
  const int* num;   // [B] pillars per frame ...
  int* num_host;    // ... copied to the unit's pinned host array (device view of the mapping)
  int err_at;       // num_host[err_at] receives the device error words (B, the capacity)
  int direct;       // block written into the result slots by the last conv itself (-1: none):
                    // not copied; its host copy (hblock) is read from the slot
  const unsigned* tc_err;  // the tensor-core conv's sticky error word
  const int* vox_err;      // the voxeliser's sticky error word
  int nblocks;
  int hblock;  // the block (the unit's final output) also copied to a frame's host buffer
  const char* src[PP_MAX_BLOCKS];
  size_t bytes[PP_MAX_BLOCKS];  // one slot's block output = the distance between slots
  size_t off[PP_MAX_BLOCKS];
};

// Copies every frame's block outputs into its result slot (tab->dst[frame]) and, when the frame
// has one, its final output (block rc.hblock) into its page-locked host buffer (tab->hdst[frame],
// at offset 0, over the host link); gridDim.y = frame.  Pure 16-byte streaming copy (all sizes
// are multiples of 128 bytes, all bases 16-byte aligned).
__global__ void __launch_bounds__(256) result_copy(ResultCopy rc, const UnitTable* __restrict__ tab) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const int f = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    rc.num_host[f] = rc.num[f];  // over the host link
    // every conv of this run has completed: its error word says whether one skipped its stores
    if (f == 0) rc.num_host[rc.err_at] = (int)((*rc.tc_err & 0x7fffffffu) | (*rc.vox_err ? 0x80000000u : 0u));
  }
  char* dst = tab->dst[f];
  char* hdst = tab->hdst[f];
  if (!dst) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int b = 0; b < rc.nblocks; ++b) {
    const bool direct = b == rc.direct;
    uint4* h = hdst && b == rc.hblock ? reinterpret_cast<uint4*>(hdst) : nullptr;
    if (direct && !h) continue;  // already in the slot, nothing to send to the host
    const uint4* s = direct ? reinterpret_cast<const uint4*>(dst + rc.off[b])
                            : reinterpret_cast<const uint4*>(rc.src[b] + (size_t)f * rc.bytes[b]);
    // a direct block only goes to the host (its slot is the source)
    uint4* d = direct ? nullptr : reinterpret_cast<uint4*>(dst + rc.off[b]);
    const size_t n = rc.bytes[b] / 16;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
      const uint4 v0 = __ldcs(s + i), v1 = __ldcs(s + i + stride);
      const uint4 v2 = __ldcs(s + i + 2 * stride), v3 = __ldcs(s + i + 3 * stride);
      if (d) {
        d[i] = v0;
        d[i + stride] = v1;
        d[i + 2 * stride] = v2;
        d[i + 3 * stride] = v3;
      }
      if (h) {
        h[i] = v0;
        h[i + stride] = v1;
        h[i + 2 * stride] = v2;
        h[i + 3 * stride] = v3;
      }
    }
    for (; i < n; i += stride) {
      const uint4 v = __ldcs(s + i);
      if (d) d[i] = v;
      if (h) h[i] = v;
    }
  }
}

int layers_of(const pp_config* cfg, std::vector<LayerSpec>* out, std::vector<int>* block_end,
              int H0, int W0) {
  if (cfg->n_blocks <= 0 || cfg->n_blocks > PP_MAX_BLOCKS)
    return fail(PP_EINVAL, "config: n_blocks must be 1..%d", PP_MAX_BLOCKS);
  int cin = 64, H = H0, W = W0;
  for (int b = 0; b < cfg->n_blocks; ++b) {
    if (cfg->convs[b] <= 0 || cfg->convs[b] > 16 || cfg->chans[b] <= 0 || cfg->chans[b] % 64 ||
        cfg->chans[b] > 1024 || (cfg->strides[b] != 1 && cfg->strides[b] != 2))
      return fail(PP_EINVAL, "config: block %d: convs 1..16, chans multiple of 64, stride 1/2", b);
    for (int i = 0; i < cfg->convs[b]; ++i) {
      LayerSpec l;
      l.cin = cin;
      l.cout = cfg->chans[b];
      l.stride = i == 0 ? cfg->strides[b] : 1;
      if (l.stride == 2 && ((H & 1) || (W & 1)))
        return fail(PP_EINVAL, "config: stride 2 on an odd map (%d x %d)", H, W);
      l.H = H;
      l.W = W;
      l.Ho = (H - 1) / l.stride + 1;
      l.Wo = (W - 1) / l.stride + 1;
      out->push_back(l);
      cin = l.cout;
      H = l.Ho;
      W = l.Wo;
    }
    block_end->push_back((int)out->size() - 1);
  }
  return PP_OK;
}
}  // namespace

int Model::upload(const pp_config* cfg, int prec, cudaStream_t s) {
  int st = check_geometry(&cfg->geom, &g);
  if (st) return st;
  precision = prec;
  keep_blocks = cfg->keep_blocks != 0;
  conv_dtype = prec == PP_BF16 ? PP_BF16 : (cfg->fp32_cuda_cores ? PP_F32 : PP_F32_TC);
  layers.clear();
  block_end.clear();
  st = layers_of(cfg, &layers, &block_end, g.ny, g.nx);
  if (st) return st;
  if (!cfg->pfn_w || !cfg->pfn_bn || !cfg->conv_w || !cfg->conv_bn)
    return fail(PP_EINVAL, "config: NULL weights");
  auto dev_alloc = [&](void** p, size_t n) -> int {
    if (cudaMalloc(p, n) != cudaSuccess) {
      cudaGetLastError();
      return fail(PP_ENOMEM, "cudaMalloc(%zu) for weights failed", n);
    }
    bytes += n;
    return PP_OK;
  };
  float ss[2 * 1024];
  if ((st = dev_alloc((void**)&pfn_w, 64 * 9 * sizeof(float)))) return st;
  if ((st = dev_alloc((void**)&pfn_ss, 2 * 64 * sizeof(float)))) return st;
  if ((st = pp_bn_fold(cfg->pfn_bn, 64, 1e-3f, ss))) return st;
  if ((st = cuda_status(cudaMemcpy(pfn_w, cfg->pfn_w, 64 * 9 * sizeof(float), cudaMemcpyHostToDevice), "upload pfn_w"))) return st;
  if ((st = cuda_status(cudaMemcpy(pfn_ss, ss, 2 * 64 * sizeof(float), cudaMemcpyHostToDevice), "upload pfn_ss"))) return st;
  for (size_t l = 0; l < layers.size(); ++l) {
    const LayerSpec& L = layers[l];
    if (!cfg->conv_w[l] || !cfg->conv_bn[l]) return fail(PP_EINVAL, "config: NULL layer %zu weights", l);
    const size_t wbytes = (size_t)L.cout * L.cin * 9 * sizeof(float);
    float* tmp = nullptr;
    if ((st = cuda_status(cudaMalloc(&tmp, wbytes), "weights staging"))) return st;
    void* packed = nullptr;
    float* ssd = nullptr;
    st = dev_alloc(&packed, pp_conv_packed_bytes(L.cin, L.cout, conv_dtype));
    if (!st) st = dev_alloc((void**)&ssd, 2 * L.cout * sizeof(float));
    if (!st) st = cuda_status(cudaMemcpy(tmp, cfg->conv_w[l], wbytes, cudaMemcpyHostToDevice), "upload conv_w");
    if (!st) st = conv_pack_launch(tmp, L.cin, L.cout, conv_dtype, packed, s);
    if (!st) st = cuda_status(cudaStreamSynchronize(s), "pack weights");
    if (!st) st = pp_bn_fold(cfg->conv_bn[l], L.cout, 1e-3f, ss);
    if (!st) st = cuda_status(cudaMemcpy(ssd, ss, 2 * L.cout * sizeof(float), cudaMemcpyHostToDevice), "upload conv_ss");
    cudaFree(tmp);
    conv_w.push_back(packed);
    conv_ss.push_back(ssd);
    if (st) return st;
  }
  head_outputs = cfg->head_outputs;
  if (head_outputs == 0) return PP_OK;
  // neck + head
  const int nb = (int)block_end.size();
  if (head_outputs < 0 || head_outputs > 1024 || cfg->up_channels <= 0 || cfg->up_channels % 64 ||
      cfg->up_channels > 1024)
    return fail(PP_EINVAL, "config: head_outputs 0..1024, up_channels a multiple of 64 up to 1024");
  if (conv_dtype == PP_F32) return fail(PP_EINVAL, "config: the neck and head need tensor-core convs");
  if (!cfg->up_w || !cfg->up_bn || !cfg->head_w || !cfg->head_b) return fail(PP_EINVAL, "config: NULL head weights");
  up_c = cfg->up_channels;
  neck_c = nb * up_c;
  head_c = (head_outputs + 63) / 64 * 64;
  for (int b = 0; b < nb; ++b) {
    const LayerSpec& L = layers[block_end[b]];
    const int up = out_h() / L.Ho;
    if (up < 1 || up > 8 || up * L.Ho != out_h() || up * L.Wo != out_w())
      return fail(PP_EINVAL, "config: block %d (%d x %d) does not upsample to block 0 (%d x %d)", b, L.Ho, L.Wo,
                  out_h(), out_w());
    if (!cfg->up_w[b] || !cfg->up_bn[b]) return fail(PP_EINVAL, "config: NULL upsampling weights %d", b);
    void* packed = nullptr;
    float* ssd = nullptr;
    st = dev_alloc(&packed, pp_upsample_packed_bytes(L.cout, up_c, up, conv_dtype));
    if (!st) st = dev_alloc((void**)&ssd, 2 * up_c * sizeof(float));
    if (!st) st = pp_upsample_pack_weights(cfg->up_w[b], L.cout, up_c, up, conv_dtype, packed);
    if (!st) st = pp_bn_fold(cfg->up_bn[b], up_c, 1e-3f, ss);
    if (!st) st = cuda_status(cudaMemcpy(ssd, ss, 2 * up_c * sizeof(float), cudaMemcpyHostToDevice), "upload up_ss");
    up_stride.push_back(up);
    up_w.push_back(packed);
    up_ss.push_back(ssd);
    if (st) return st;
  }
  if ((st = dev_alloc(&head_w, pp_head_packed_bytes(neck_c, head_outputs, conv_dtype)))) return st;
  if ((st = dev_alloc((void**)&head_ss, 2 * head_c * sizeof(float)))) return st;
  return pp_head_pack_weights(cfg->head_w, cfg->head_b, neck_c, head_outputs, conv_dtype, head_w, head_ss);
}

size_t Model::result_layout(std::vector<size_t>* block_off) const {
  const size_t elt = precision == PP_F32 ? 4 : 2;
  size_t off = 0;
  block_off->clear();
  if (head_outputs > 0) {
    block_off->push_back(0);
    return align_up((size_t)(out_h() + 2) * (out_w() + 2) * head_c * elt, 256);
  }
  for (int b : kept_blocks()) {
    const LayerSpec& L = layers[block_end[b]];
    block_off->push_back(off);
    off += align_up((size_t)(L.Ho + 2) * (L.Wo + 2) * L.cout * elt, 256);
  }
  return off;
}

std::vector<int> Model::kept_blocks() const {
  std::vector<int> v;
  if (head_outputs > 0) return v;
  for (int b = keep_blocks ? 0 : (int)block_end.size() - 1; b < (int)block_end.size(); ++b) v.push_back(b);
  return v;
}

size_t Model::final_bytes() const {
  const size_t elt = precision == PP_F32 ? 4 : 2;
  if (head_outputs > 0) return (size_t)(out_h() + 2) * (out_w() + 2) * head_c * elt;
  const LayerSpec& L = layers[block_end.back()];
  return (size_t)(L.Ho + 2) * (L.Wo + 2) * L.cout * elt;
}

void Model::release() {
  cudaFree(pfn_w);
  cudaFree(pfn_ss);
  for (void* p : conv_w) cudaFree(p);
  for (float* p : conv_ss) cudaFree(p);
  for (void* p : up_w) cudaFree(p);
  for (float* p : up_ss) cudaFree(p);
  cudaFree(head_w);
  cudaFree(head_ss);
  pfn_w = pfn_ss = nullptr;
  head_w = nullptr;
  head_ss = nullptr;
  conv_w.clear();
  conv_ss.clear();
  up_w.clear();
  up_ss.clear();
  up_stride.clear();
}

int Pipeline::alloc(void** p, size_t n) {
  n = align_up(n < 256 ? 256 : n, 256);
  if (cudaMalloc(p, n) != cudaSuccess) {
    cudaGetLastError();
    return fail(PP_ENOMEM, "cudaMalloc(%zu) failed", n);
  }
  allocs_.push_back(*p);
  bytes_ += n;
  return PP_OK;
}

int Pipeline::init(const Model* m, int max_batch, int cap_points, bool graphs, bool tune, bool stream_k,
                   cudaStream_t s) {
  m_ = m;
  B_ = max_batch;
  cap_ = cap_points;
  const Geom& g = m->g;
  const size_t elt = m->precision == PP_F32 ? 4 : 2;
  int st = PP_OK;
#define PP_ALLOC(ptr, n) \
  if ((st = alloc(reinterpret_cast<void**>(&ptr), (n)))) return st
  if (B_ < 1 || B_ > kMaxUnit) return fail(PP_EINVAL, "pipeline: max_batch 1..%d", kMaxUnit);
  PP_ALLOC(points_, (size_t)B_ * cap_ * sizeof(float4));
  PP_ALLOC(tab_dev_, sizeof(UnitTable));
  PP_ALLOC(cell_, (size_t)B_ * cap_ * sizeof(int));
  PP_ALLOC(cnt_, (size_t)B_ * g.G * sizeof(unsigned));
  PP_ALLOC(poc_, (size_t)B_ * g.G * sizeof(int));
  PP_ALLOC(coord_, (size_t)B_ * g.P * sizeof(int));
  PP_ALLOC(npts_, (size_t)B_ * g.P * sizeof(int));
  PP_ALLOC(num_, (size_t)B_ * sizeof(int));
  PP_ALLOC(vox_ws_, vox_workspace_bytes(g, B_, cap_));
  // split FP32 (3xTF32 convs): every conv operand carries its TF32 remainder plane
  const size_t planes = m->conv_dtype == PP_F32_TC ? 2 : 1;
  PP_ALLOC(canvas_, planes * B_ * (g.ny + 2) * (g.nx + 2) * 64 * elt);
  PP_ALLOC(drawn_, (size_t)B_ * g.P * sizeof(int));
  PP_ALLOC(drawn_num_, (size_t)B_ * sizeof(int));
  // the canvas is updated in place frame after frame: it starts zero with nothing drawn
  if ((st = cuda_status(cudaMemsetAsync(canvas_, 0, planes * B_ * (g.ny + 2) * (g.nx + 2) * 64 * elt, s),
                        "clear canvas")))
    return st;
  if ((st = cuda_status(cudaMemsetAsync(drawn_num_, 0, (size_t)B_ * sizeof(int), s), "clear drawn"))) return st;
  for (const LayerSpec& L : m->layers) {
    void* a = nullptr;
    const size_t n = planes * B_ * (L.Ho + 2) * (L.Wo + 2) * L.cout * elt;
    PP_ALLOC(a, n);
    act_.push_back(a);
    // borders stay zero forever: convs write interiors only
    if ((st = cuda_status(cudaMemsetAsync(a, 0, n, s), "clear activations"))) return st;
  }
  if (m->head_outputs > 0) {
    const size_t px = planes * B_ * (m->out_h() + 2) * (m->out_w() + 2) * elt;
    PP_ALLOC(neck_, px * m->neck_c);
    PP_ALLOC(head_, px * m->head_c);
    if ((st = cuda_status(cudaMemsetAsync(neck_, 0, px * m->neck_c, s), "clear neck"))) return st;
    if ((st = cuda_status(cudaMemsetAsync(head_, 0, px * m->head_c, s), "clear head"))) return st;
  }
  if (m->conv_dtype == PP_F32_TC && stream_k) {
    // one stream-K workspace, sized for the widest layer at the unit's capacity (a smaller
    // batch needs fewer arrival counters), zeroed once; every completed conv leaves it zero
    for (const LayerSpec& L : m->layers) {
      ConvShape c{B_, L.H, L.W, L.cin, L.cout, L.stride, L.Ho, L.Wo};
      conv_ws_bytes_ = std::max(conv_ws_bytes_, conv_sk_workspace_bytes(c));
    }
    PP_ALLOC(conv_ws_, conv_ws_bytes_);
    if ((st = cuda_status(cudaMemsetAsync(conv_ws_, 0, conv_ws_bytes_, s), "clear conv workspace"))) return st;
  }
#undef PP_ALLOC
  if ((st = cuda_status(cudaMemsetAsync(vox_ws_, 0, 256, s), "clear vox error word"))) return st;
  if ((st = cuda_status(cudaMemsetAsync(tab_dev_, 0, sizeof(UnitTable), s), "clear unit table"))) return st;
  if ((st = cuda_status(cudaMallocHost(&tab_host_, sizeof(UnitTable)), "pinned unit table"))) return st;
  memset(tab_host_, 0, sizeof(UnitTable));
  if ((st = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void**>(&tab_map_), tab_host_, 0),
                        "unit table mapping")))
    return st;
  // cell counts start zero; every launch's scan leaves them zero again
  if ((st = cuda_status(cudaMemsetAsync(cnt_, 0, (size_t)B_ * g.G * sizeof(unsigned), s), "clear counts"))) return st;
  if ((st = cuda_status(cudaEventCreateWithFlags(&tab_ev_, cudaEventDisableTiming), "table event"))) return st;
  m->result_layout(&res_off_);
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if ((st = cuda_status(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev), "SM count"))) return st;
  }
  if ((st = cuda_status(cudaMallocHost(&num_host_, (size_t)(B_ + 1) * sizeof(int)), "pinned pillar counts"))) return st;
  memset(num_host_, 0, (size_t)(B_ + 1) * sizeof(int));
  if ((st = tc_error_address(&tc_err_))) return st;
  if ((st = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void**>(&num_host_dev_), num_host_, 0),
                        "pinned pillar counts mapping")))
    return st;
  vw_ = vox_carve(vox_ws_, g, B_, cap_);
  if (tune) {
    // time every conv tile of every layer at the largest unit size on this unit's own buffers
    // and use the fastest for every unit size: the tiles differ in their accumulation order,
    // and one tile per layer keeps a frame's result bit-identical whatever the number of
    // frames its unit carries.  The launches below (and the captured graphs) then use it.
    if ((st = cuda_status(cudaStreamSynchronize(s), "pre-tune sync"))) return st;
    const void* x = canvas_;
    for (size_t l = 0; l < m->layers.size() && st == PP_OK; ++l) {
      const LayerSpec& L = m->layers[l];
      int best = -1;
      st = pp_conv_autotune_ws(B_, L.H, L.W, L.cin, L.cout, L.stride, m->conv_dtype, x, m->conv_w[l],
                               m->conv_ss[l], act_[l], conv_ws_, conv_ws_bytes_, 5, &best, nullptr);
      for (int b = 1; b < B_ && st == PP_OK; ++b)
        tune_record(m->conv_dtype, b, L.H, L.W, L.cin, L.cout, L.stride, best);
      x = act_[l];
    }
    if (st) return st;
  }
  // one eager pass sets kernel attributes and validates every launch before capture
  if ((st = enqueue(B_, s))) return st;
  if ((st = cuda_status(cudaStreamSynchronize(s), "pipeline warm-up"))) return st;
  graphs_.assign(B_ + 1, nullptr);
  if (graphs) {
    cudaStream_t cs;
    if ((st = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream"))) return st;
    for (int b = 1; b <= B_ && st == PP_OK; ++b) {
      cudaGraph_t graph = nullptr;
      st = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
      if (st) break;
      const int est = enqueue(b, cs);
      const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      if (est) { st = est; if (graph) cudaGraphDestroy(graph); break; }
      if ((st = cuda_status(ee, "end capture"))) break;
      st = cuda_status(cudaGraphInstantiate(&graphs_[b], graph, 0), "instantiate graph");
      cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cs);
    if (st) return st;
  }
  return PP_OK;
}

void Pipeline::release() {
  for (cudaGraphExec_t g : graphs_)
    if (g) cudaGraphExecDestroy(g);
  graphs_.clear();
  for (void* p : allocs_) cudaFree(p);
  allocs_.clear();
  act_.clear();
  if (tab_host_) cudaFreeHost(tab_host_);
  if (num_host_) cudaFreeHost(num_host_);
  if (tab_ev_) cudaEventDestroy(tab_ev_);
  tab_host_ = nullptr;
  num_host_ = nullptr;
  tab_ev_ = nullptr;
  bytes_ = 0;
}

int Pipeline::enqueue(int n, cudaStream_t s) {
  const Model& m = *m_;
  const Geom& g = m.g;
  // voxelise up to the bucketing; point selection runs fused into PointNet
  // the unit table is read from its page-locked host copy by the first kernel, which copies it
  // to tab_dev_ for the rest; the counts stay zero between launches
  VoxUnitIO io;
  io.first_counts = tab_map_->counts;
  io.first_srcs = tab_map_->src;
  io.first_mirrors = tab_map_->mirror;
  io.table_src = reinterpret_cast<const uint4*>(tab_map_);
  io.table_dst = reinterpret_cast<uint4*>(tab_dev_);
  io.table_words = (int)(sizeof(UnitTable) / sizeof(uint4));
  io.cnt_clean = true;
  // the canvas keeps each slot's previous frame: the bucket pass zeroes its stale cells, the
  // point selection + PointNet pass writes every kept pillar's features straight into its cell
  // (the incremental scatter of pp_scatter_update, without a feature buffer or launches of its
  // own)
  const bool split = m.conv_dtype == PP_F32_TC;
  const int chunks = m.precision == PP_BF16 ? 8 : 16;
  uint4* cv = static_cast<uint4*>(canvas_);
  uint4* cv_lo = split ? cv + (size_t)B_ * (g.ny + 2) * (g.nx + 2) * 16 : nullptr;
  io.canvas = cv;
  io.canvas_lo = cv_lo;
  io.canvas_chunks = chunks;
  io.drawn = drawn_;
  io.drawn_num = drawn_num_;
  int st = vox_launch(g, n, cap_, points_, tab_dev_->counts, cell_, cnt_, poc_, coord_, npts_, num_,
                      nullptr, vw_, s, tab_dev_->src, tab_dev_->mirror, &io);
  if (!st)
    st = select_pfn_launch(g, n, cap_, points_, tab_dev_->gsrc, vw_, coord_, num_, m.pfn_w, m.pfn_ss, nullptr, s,
                           chunks, drawn_, drawn_num_, cv, cv_lo, cnt_);
  const void* x = canvas_;
  // without a head the last layer's output is the frames' result: its tensor-core epilogue
  // writes it straight into each frame's result slot (the unit table's dst; frames without a
  // slot fall back to the unit's buffer), and a split FP32 last layer skips the remainder plane
  // no later layer would read
  const bool direct = m.head_outputs == 0 && m.conv_dtype != PP_F32;
  for (size_t l = 0; l < m.layers.size() && !st; ++l) {
    const LayerSpec& L = m.layers[l];
    ConvShape c{n, L.H, L.W, L.cin, L.cout, L.stride, L.Ho, L.Wo};
    c.static_w = true;  // packed once at creation
    if (direct && l + 1 == m.layers.size()) {
      c.frame_dst = tab_dev_->dst;
      c.frame_off = res_off_.back();
      c.skip_lo = split;
    }
    if (split) {  // planes are laid out for the unit's capacity, not for this batch
      c.in_plane = (size_t)B_ * (L.H + 2) * (L.W + 2) * L.cin;
      c.out_plane = (size_t)B_ * (L.Ho + 2) * (L.Wo + 2) * L.cout;
    }
    if (m.conv_dtype == PP_F32)
      st = conv_f32_launch(c, (const float*)x, (const float*)m.conv_w[l], m.conv_ss[l],
                           (float*)act_[l], -1, s);
    else if (m.conv_dtype == PP_F32_TC)
      st = conv_f32tc_launch(c, (const float*)x, (const float*)m.conv_w[l], m.conv_ss[l],
                             (float*)act_[l], -1, s, conv_ws_, conv_ws_bytes_);
    else
      st = conv_bf16_launch(c, (const __nv_bfloat16*)x, (const __nv_bfloat16*)m.conv_w[l],
                            m.conv_ss[l], (__nv_bfloat16*)act_[l], -1, s);
    x = act_[l];
  }
  if (st) return st;
  ResultCopy rc{};
  rc.num = num_;
  rc.num_host = num_host_dev_;
  rc.err_at = B_;
  rc.direct = -1;
  rc.tc_err = tc_err_;
  rc.vox_err = vw_.err;
  if (m.head_outputs > 0) {
    // neck: every block's output upsampled into its channel range of the neck map; then the head
    const int H0 = m.out_h(), W0 = m.out_w();
    const size_t px = (size_t)B_ * (H0 + 2) * (W0 + 2);
    for (size_t b = 0; b < m.block_end.size() && !st; ++b) {
      const LayerSpec& L = m.layers[m.block_end[b]];
      const int up = m.up_stride[b];
      ConvShape c{n, L.Ho, L.Wo, L.cout, up * up * m.up_c, 1, L.Ho, L.Wo};
      c.in_plane = (size_t)B_ * (L.Ho + 2) * (L.Wo + 2) * L.cout;
      c.out_plane = px * m.neck_c;
      GemmOpts o;
      o.taps = 1;
      o.up = up;
      o.co_blk = m.up_c;
      o.out_c = m.neck_c;
      o.out_coff = (int)b * m.up_c;
      st = gemm_tc_launch(m.conv_dtype, c, o, act_[m.block_end[b]], m.up_w[b], m.up_ss[b], neck_, -1, s);
    }
    if (!st) {
      ConvShape c{n, H0, W0, m.neck_c, m.head_c, 1, H0, W0};
      c.in_plane = px * m.neck_c;
      c.out_plane = px * m.head_c;
      GemmOpts o;
      o.taps = 1;
      o.relu = 0;
      st = gemm_tc_launch(m.conv_dtype, c, o, neck_, m.head_w, m.head_ss, head_, -1, s);
    }
    if (st) return st;
    rc.nblocks = 1;
    rc.hblock = 0;
    rc.src[0] = static_cast<const char*>(head_);
    rc.bytes[0] = (size_t)(H0 + 2) * (W0 + 2) * m.head_c * (m.precision == PP_F32 ? 4 : 2);
    rc.off[0] = res_off_[0];
    hout_off_ = rc.off[0];
    hout_bytes_ = rc.bytes[0];
  } else {
    const std::vector<int> kept = m.kept_blocks();
    rc.nblocks = (int)kept.size();
    rc.hblock = rc.nblocks - 1;  // the last block: the unit's final output
    for (int k = 0; k < rc.nblocks; ++k) {
      const int l = m.block_end[kept[k]];
      const LayerSpec& L = m.layers[l];
      rc.src[k] = static_cast<const char*>(act_[l]);
      rc.bytes[k] = (size_t)(L.Ho + 2) * (L.Wo + 2) * L.cout * (m.precision == PP_F32 ? 4 : 2);
      rc.off[k] = res_off_[k];
    }
    hout_off_ = rc.off[rc.hblock];
    hout_bytes_ = rc.bytes[rc.hblock];
    if (direct) rc.direct = rc.hblock;  // the last block, written by the last conv
  }
  return cuda_status(launch_pdl(result_copy, dim3(std::max(1, 8 * sms_ / n), n), dim3(256), 0, s, rc,
                                (const UnitTable*)tab_dev_),
                     "result copy");
}

int Pipeline::run(int n, const float* const* frames, const int* counts, const bool* direct,
                  char* const* dst, bool use_graph, cudaStream_t s, const bool* host_mapped,
                  char* const* hdst) {
  if (n <= 0 || n > B_) return fail(PP_EINVAL, "pipeline run: batch %d outside 1..%d", n, B_);
  for (int i = 0; i < n; ++i) {
    if (counts[i] < 0 || counts[i] > cap_)
      return fail(PP_EINVAL, "pipeline run: frame %d has %d points (cap %d)", i, counts[i], cap_);
    if (counts[i] > 0 && !frames[i]) return fail(PP_EINVAL, "pipeline run: NULL frame %d", i);
    if (direct && direct[i] && (reinterpret_cast<uintptr_t>(frames[i]) & 15u))
      return fail(PP_EINVAL, "pipeline run: frame %d is not 16-byte aligned", i);
  }
  // the previous run on this unit reads the pinned table from its first kernel: wait for that
  // run to finish before rewriting it (a release unit is reused only once it completed)
  int st = cuda_status(cudaEventSynchronize(tab_ev_), "unit table reuse");
  if (st) return st;
  UnitTable& t = *tab_host_;
  memset(&t, 0, sizeof(t));
  // Host frames and host outputs of a unit that batches several frames move by copy engine
  // (into the unit's point slots before its kernels, out of its result slots after them), so
  // that the transfers overlap the kernels of other units in flight; a one-frame unit reads its
  // points and writes its output over the host link from its own kernels (no copy on its
  // critical path).
  const bool ce = n > 1;
  for (int i = 0; i < n; ++i) {
    t.counts[i] = counts[i];
    t.dst[i] = dst ? dst[i] : nullptr;
    t.hdst[i] = hdst && t.dst[i] && !ce ? hdst[i] : nullptr;
    if (direct && direct[i] && !(host_mapped && host_mapped[i] && ce)) {
      t.src[i] = reinterpret_cast<const float4*>(frames[i]);
      t.gsrc[i] = t.src[i];
      if (host_mapped && host_mapped[i]) {
        // read once over the host link (coalesced); the scattered gather reads the copy
        t.mirror[i] = points_ + (size_t)i * cap_;
        t.gsrc[i] = t.mirror[i];
      }
      continue;
    }
    t.src[i] = points_ + (size_t)i * cap_;
    t.gsrc[i] = t.src[i];
    if (counts[i] > 0 &&
        (st = cuda_status(cudaMemcpyAsync(points_ + (size_t)i * cap_, frames[i],
                                          (size_t)counts[i] * sizeof(float4), cudaMemcpyDefault, s),
                          "stage points")))
      return st;
  }
  if (use_graph && graphs_.size() > (size_t)n && graphs_[n])
    st = cuda_status(cudaGraphLaunch(graphs_[n], s), "graph launch");
  else
    st = enqueue(n, s);
  if (!st && ce && hdst && dst)
    for (int i = 0; i < n && !st; ++i)
      if (hdst[i] && dst[i])
        st = cuda_status(cudaMemcpyAsync(hdst[i], dst[i] + hout_off_, hout_bytes_, cudaMemcpyDeviceToHost, s),
                         "host output copy");
  if (!st) st = cuda_status(cudaEventRecord(tab_ev_, s), "unit table event");
  return st;  // the result copy kernel has written num_host_ (pillar counts) over the host link
}

const void* Pipeline::neck_out(int i) const {
  if (!neck_) return nullptr;
  return static_cast<const char*>(neck_) +
         (size_t)i * (m_->out_h() + 2) * (m_->out_w() + 2) * m_->neck_c * (m_->precision == PP_F32 ? 4 : 2);
}

const void* Pipeline::head_out(int i) const {
  if (!head_) return nullptr;
  return static_cast<const char*>(head_) +
         (size_t)i * (m_->out_h() + 2) * (m_->out_w() + 2) * m_->head_c * (m_->precision == PP_F32 ? 4 : 2);
}

const void* Pipeline::layer_out(int layer, int i) const {
  const LayerSpec& L = m_->layers[layer];
  const size_t elt = m_->precision == PP_F32 ? 4 : 2;
  return static_cast<const char*>(act_[layer]) + (size_t)i * (L.Ho + 2) * (L.Wo + 2) * L.cout * elt;
}

}  // namespace pp

// ------------------------------------------------------------------ C ABI

struct pp_pipeline {
  pp::Model model;
  pp::Pipeline pipe;
};

using namespace pp;

extern "C" {

int pp_pipeline_create(const pp_config* cfg, int32_t precision, pp_pipeline** out) {
  if (!cfg || !out) return fail(PP_EINVAL, "pipeline_create: NULL argument");
  if (precision != PP_F32 && precision != PP_BF16) return fail(PP_EINVAL, "pipeline_create: bad precision");
  if (cfg->max_batch < 1 || cfg->max_batch > 8 || cfg->cap_points < 1 || cfg->cap_points > (1 << 24))
    return fail(PP_EINVAL, "pipeline_create: max_batch 1..8, cap_points 1..2^24");
  pp_pipeline* p = new (std::nothrow) pp_pipeline();
  if (!p) return fail(PP_ENOMEM, "pipeline_create: host allocation");
  cudaStream_t s;
  int st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
  if (!st) st = p->model.upload(cfg, precision, s);
  if (!st)
    st = p->pipe.init(&p->model, cfg->max_batch, cfg->cap_points, cfg->use_graphs != 0, cfg->autotune != 0,
                      cfg->stream_k != 0, s);
  if (!st) st = cuda_status(cudaStreamSynchronize(s), "pipeline init");
  cudaStreamDestroy(s);
  if (st) {
    p->pipe.release();
    p->model.release();
    delete p;
    return st;
  }
  *out = p;
  return PP_OK;
}

int pp_pipeline_run(pp_pipeline* p, int32_t n, const float* const* frames, const int32_t* counts,
                    int32_t use_graph, void* stream) {
  if (!p || !frames || !counts) return fail(PP_EINVAL, "pipeline_run: NULL argument");
  return p->pipe.run(n, frames, counts, nullptr, nullptr, use_graph != 0, static_cast<cudaStream_t>(stream));
}

int pp_pipeline_output(pp_pipeline* p, int32_t i, int32_t block, const void** dev, int32_t* c,
                       int32_t* h, int32_t* w) {
  if (!p || !dev || i < 0 || i >= p->pipe.max_batch()) return fail(PP_EINVAL, "pipeline_output: bad argument");
  if (block == -1) {
    *dev = p->pipe.num_pillars_dev() + i;
    return PP_OK;
  }
  if (block == -2 || block == -3) {
    if (p->model.head_outputs <= 0) return fail(PP_EINVAL, "pipeline_output: no neck or head configured");
    *dev = block == -2 ? p->pipe.head_out(i) : p->pipe.neck_out(i);
    if (c) *c = block == -2 ? p->model.head_c : p->model.neck_c;
    if (h) *h = p->model.out_h();
    if (w) *w = p->model.out_w();
    return PP_OK;
  }
  if (block < 0 || block >= (int)p->model.block_end.size()) return fail(PP_EINVAL, "pipeline_output: bad block");
  const int l = p->model.block_end[block];
  const LayerSpec& L = p->model.layers[l];
  *dev = p->pipe.layer_out(l, i);
  if (c) *c = L.cout;
  if (h) *h = L.Ho;
  if (w) *w = L.Wo;
  return PP_OK;
}

size_t pp_pipeline_bytes(pp_pipeline* p) { return p ? p->pipe.bytes() + p->model.bytes : 0; }

int pp_pipeline_destroy(pp_pipeline* p) {
  if (!p) return PP_OK;
  cudaDeviceSynchronize();
  p->pipe.release();
  p->model.release();
  delete p;
  return PP_OK;
}

}  // extern "C"
