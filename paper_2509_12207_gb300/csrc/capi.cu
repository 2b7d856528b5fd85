// C-ABI stage entry points: argument validation, then the launches in the kernel files.
#include "pp_internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace pp {

namespace {
thread_local char g_err[512] = {0};
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PP_OK;
  return fail(PP_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_err[0] = 0; }

bool pdl_enabled() {
  static const bool on = [] {
    const char* v = getenv("PP_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}

const char* last_error() { return g_err; }

int check_geometry(const pp_geometry* g, Geom* out) {
  if (!g) return fail(PP_EINVAL, "geometry is NULL");
  if (g->nx <= 0 || g->ny <= 0 || g->max_pillars <= 0 || g->max_pts != 32)
    return fail(PP_EINVAL, "geometry: nx, ny, max_pillars must be > 0 and max_pts == 32");
  if ((int64_t)g->nx * g->ny > (int64_t)1 << 28 || g->max_pillars > (1 << 24))
    return fail(PP_EINVAL, "geometry too large");
  if (!(g->vx > 0.f) || !(g->vy > 0.f) || !(g->xmax > g->xmin) || !(g->ymax > g->ymin) ||
      !(g->zmax > g->zmin))
    return fail(PP_EINVAL, "geometry: empty range or non-positive voxel size");
  out->xmin = g->xmin; out->xmax = g->xmax;
  out->ymin = g->ymin; out->ymax = g->ymax;
  out->zmin = g->zmin; out->zmax = g->zmax;
  out->vx = g->vx; out->vy = g->vy;
  out->nx = g->nx; out->ny = g->ny;
  out->G = g->nx * g->ny;
  out->P = g->max_pillars;
  out->nx_magic = g->nx > 1 ? UINT64_MAX / (uint64_t)g->nx + 1u : 0u;
  return PP_OK;
}

int device_sms() {
  constexpr int kDev = 64;
  static std::atomic<int> cache[kDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  int n = dev < kDev ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = 152;
  }
  if (dev < kDev) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

int smem_attr_once(const void* func, int bytes, std::atomic<uint64_t>* done, const char* what) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, what);
  const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
  if (bit && (done->load(std::memory_order_acquire) & bit)) return PP_OK;
  // setting it twice (two threads racing here) is harmless
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return cuda_status(e, what);
  if (bit) done->fetch_or(bit, std::memory_order_acq_rel);
  return PP_OK;
}

}  // namespace pp

using namespace pp;

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

namespace pp {
namespace {

// float -> bf16 bits, round to nearest even (NaN kept quiet)
uint16_t bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return (uint16_t)((u >> 16) | 0x40u);
  const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(r >> 16);
}

// Packs a K-major GEMM weight matrix given element by element (value(n, k), n < N, k < K, rows
// n >= n_valid zero) for `dtype` and copies it to the device: BF16 [N][K] bf16; F32_TC [2][N][K]
// float (TF32 part, remainder).
template <class F>
int pack_gemm(int N, int n_valid, int K, int dtype, F value, void* dst) {
  const size_t nk = (size_t)N * K;
  std::vector<uint16_t> b16;
  std::vector<float> f32;
  if (dtype == PP_BF16) b16.assign(nk, 0); else f32.assign(2 * nk, 0.f);
  for (int n = 0; n < n_valid; ++n)
    for (int k = 0; k < K; ++k) {
      const float v = value(n, k);
      if (dtype == PP_BF16) {
        b16[(size_t)n * K + k] = bf16_bits(v);
      } else {
        uint32_t u;
        memcpy(&u, &v, 4);
        u &= 0xFFFFE000u;
        float hi;
        memcpy(&hi, &u, 4);
        f32[(size_t)n * K + k] = hi;
        f32[nk + (size_t)n * K + k] = v - hi;
      }
    }
  const cudaError_t e = dtype == PP_BF16 ? cudaMemcpy(dst, b16.data(), nk * 2, cudaMemcpyHostToDevice)
                                         : cudaMemcpy(dst, f32.data(), 2 * nk * 4, cudaMemcpyHostToDevice);
  return cuda_status(e, "upload packed GEMM weights");
}

int head_pad(int cout) { return (cout + 63) / 64 * 64; }

}  // namespace
}  // namespace pp

extern "C" {

const char* pp_version(void) { return "pp 0.1 sm_103a"; }

const char* pp_last_error(void) { return pp::last_error(); }

size_t pp_voxelize_workspace_bytes(const pp_geometry* g, int32_t batch, int32_t cap_points) {
  Geom gg;
  if (check_geometry(g, &gg) != PP_OK || batch <= 0 || cap_points < 0) return 0;
  return vox_workspace_bytes(gg, batch, cap_points);
}

int pp_voxelize(const pp_geometry* g, int32_t batch, int32_t cap_points, const float* points,
                const int32_t* n_points, int32_t* cell, uint32_t* cnt, int32_t* pillar_of_cell,
                int32_t* coord, int32_t* npts, int32_t* num_pillars, float* pts,
                void* workspace, size_t workspace_bytes, void* stream) {
  Geom gg;
  int st = check_geometry(g, &gg);
  if (st) return st;
  if (batch <= 0 || batch > 4096 || cap_points < 0 || cap_points > (1 << 27))
    return fail(PP_EINVAL, "voxelize: batch or cap_points out of range");
  if (!n_points || !cnt || !pillar_of_cell || !coord || !npts || !num_pillars || !pts ||
      !workspace || (cap_points > 0 && (!points || !cell)))
    return fail(PP_EINVAL, "voxelize: NULL buffer");
  if (!aligned16(points) || !aligned16(pts) || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return fail(PP_EINVAL, "voxelize: points/pts need 16-byte, workspace 256-byte alignment");
  if (workspace_bytes < vox_workspace_bytes(gg, batch, cap_points))
    return fail(PP_EINVAL, "voxelize: workspace too small");
  VoxWork w = vox_carve(workspace, gg, batch, cap_points);
  return vox_launch(gg, batch, cap_points, reinterpret_cast<const float4*>(points), n_points,
                    cell, cnt, pillar_of_cell, coord, npts, num_pillars,
                    reinterpret_cast<float4*>(pts), w, static_cast<cudaStream_t>(stream));
}

int pp_voxelize_pointnet(const pp_geometry* g, int32_t batch, int32_t cap_points, const float* points,
                         const int32_t* n_points, int32_t* cell, uint32_t* cnt, int32_t* pillar_of_cell,
                         int32_t* coord, int32_t* npts, int32_t* num_pillars, const float* pfn_w,
                         const float* scale_shift, float* feat, void* workspace, size_t workspace_bytes,
                         void* stream) {
  Geom gg;
  int st = check_geometry(g, &gg);
  if (st) return st;
  if (batch <= 0 || batch > 4096 || cap_points < 0 || cap_points > (1 << 27))
    return fail(PP_EINVAL, "voxelize_pointnet: batch or cap_points out of range");
  if (!n_points || !cnt || !pillar_of_cell || !coord || !npts || !num_pillars || !pfn_w || !scale_shift ||
      !feat || !workspace || (cap_points > 0 && (!points || !cell)))
    return fail(PP_EINVAL, "voxelize_pointnet: NULL buffer");
  if (!aligned16(points) || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return fail(PP_EINVAL, "voxelize_pointnet: points need 16-byte, workspace 256-byte alignment");
  if (workspace_bytes < vox_workspace_bytes(gg, batch, cap_points))
    return fail(PP_EINVAL, "voxelize_pointnet: workspace too small");
  VoxWork w = vox_carve(workspace, gg, batch, cap_points);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float4* p4 = reinterpret_cast<const float4*>(points);
  st = vox_launch(gg, batch, cap_points, p4, n_points, cell, cnt, pillar_of_cell, coord, npts, num_pillars,
                  nullptr, w, s);
  if (st) return st;
  return select_pfn_launch(gg, batch, cap_points, p4, nullptr, w, coord, num_pillars, pfn_w, scale_shift, feat, s);
}

int pp_voxelize_check(const void* workspace, void* stream) {
  if (!workspace) return fail(PP_EINVAL, "voxelize_check: NULL workspace");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = cuda_status(cudaStreamSynchronize(s), "voxelize_check sync");
  if (st) return st;
  int err = 0;
  st = cuda_status(cudaMemcpy(&err, workspace, sizeof(int), cudaMemcpyDeviceToHost),
                   "voxelize_check read");
  if (st) return st;
  if (err) {
    cudaMemset(const_cast<void*>(workspace), 0, sizeof(int));
    return fail(PP_EINVAL, "voxelize: a n_points value was outside [0, cap_points]");
  }
  return PP_OK;
}

int pp_pointnet(const pp_geometry* g, int32_t batch, const float* pts, const int32_t* npts,
                const int32_t* coord, const int32_t* num_pillars, const float* pfn_w,
                const float* scale_shift, float* feat, void* stream) {
  Geom gg;
  int st = check_geometry(g, &gg);
  if (st) return st;
  if (batch <= 0 || batch > 4096) return fail(PP_EINVAL, "pointnet: batch out of range");
  if (!pts || !npts || !coord || !num_pillars || !pfn_w || !scale_shift || !feat)
    return fail(PP_EINVAL, "pointnet: NULL buffer");
  if (!aligned16(pts)) return fail(PP_EINVAL, "pointnet: pts must be 16-byte aligned");
  return pfn_launch(gg, batch, reinterpret_cast<const float4*>(pts), npts, coord, num_pillars,
                    pfn_w, scale_shift, feat, static_cast<cudaStream_t>(stream));
}

int pp_scatter(const pp_geometry* g, int32_t batch, const float* feat,
               const int32_t* pillar_of_cell, void* canvas, int32_t dtype, void* stream) {
  Geom gg;
  int st = check_geometry(g, &gg);
  if (st) return st;
  if (batch <= 0 || batch > 4096) return fail(PP_EINVAL, "scatter: batch out of range");
  if (dtype != PP_F32 && dtype != PP_BF16 && dtype != PP_F32_TC) return fail(PP_EINVAL, "scatter: bad dtype");
  if (!feat || !pillar_of_cell || !canvas) return fail(PP_EINVAL, "scatter: NULL buffer");
  if (!aligned16(feat) || !aligned16(canvas))
    return fail(PP_EINVAL, "scatter: feat and canvas must be 16-byte aligned");
  return scatter_launch(gg, batch, feat, pillar_of_cell, canvas, dtype,
                        static_cast<cudaStream_t>(stream));
}

int pp_scatter_update(const pp_geometry* g, int32_t batch, const float* feat, const int32_t* coord,
                      const int32_t* num_pillars, const int32_t* pillar_of_cell, int32_t* drawn,
                      int32_t* drawn_num, void* canvas, int32_t dtype, void* stream) {
  Geom gg;
  int st = check_geometry(g, &gg);
  if (st) return st;
  if (batch <= 0 || batch > 4096) return fail(PP_EINVAL, "scatter_update: batch out of range");
  if (dtype != PP_F32 && dtype != PP_BF16 && dtype != PP_F32_TC) return fail(PP_EINVAL, "scatter_update: bad dtype");
  if (!feat || !coord || !num_pillars || !pillar_of_cell || !drawn || !drawn_num || !canvas)
    return fail(PP_EINVAL, "scatter_update: NULL buffer");
  if (!aligned16(feat) || !aligned16(canvas))
    return fail(PP_EINVAL, "scatter_update: feat and canvas must be 16-byte aligned");
  return scatter_update_launch(gg, batch, feat, coord, num_pillars, pillar_of_cell, drawn, drawn_num, canvas, dtype,
                               static_cast<cudaStream_t>(stream));
}

int pp_tf32_split(const float* x, float* lo, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !lo))) return fail(PP_EINVAL, "tf32_split: bad argument");
  if (n == 0) return PP_OK;
  if (!aligned16(x) || !aligned16(lo)) return fail(PP_EINVAL, "tf32_split: x and lo must be 16-byte aligned");
  const char *a = reinterpret_cast<const char*>(x), *b = reinterpret_cast<const char*>(lo);
  if (a < b + n * 4 && b < a + n * 4) return fail(PP_EINVAL, "tf32_split: x and lo overlap");
  return tf32_split_launch(x, lo, (size_t)n, static_cast<cudaStream_t>(stream));
}

static int conv_shape(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t stride,
                      ConvShape* c) {
  if (batch <= 0 || H <= 0 || W <= 0 || cin <= 0 || cout <= 0 || cin % 64 || cout % 64 ||
      cin > 1024 || cout > 1024 || (stride != 1 && stride != 2))
    return fail(PP_EINVAL, "conv3x3: unsupported shape (cin, cout multiples of 64, stride 1/2)");
  if ((int64_t)batch * (H + 2) * (W + 2) > ((int64_t)1 << 31) / 2)
    return fail(PP_EINVAL, "conv3x3: activation too large");
  if (stride == 2 && ((H & 1) || (W & 1)))
    return fail(PP_EINVAL, "conv3x3: stride 2 needs even H and W");
  c->batch = batch; c->H = H; c->W = W; c->cin = cin; c->cout = cout; c->stride = stride;
  c->Ho = (H - 1) / stride + 1;
  c->Wo = (W - 1) / stride + 1;
  return PP_OK;
}

size_t pp_conv_workspace_bytes(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout,
                               int32_t stride, int32_t dtype) {
  ConvShape c;
  if (dtype != PP_F32_TC || conv_shape(batch, H, W, cin, cout, stride, &c) != PP_OK) return 0;
  return conv_sk_workspace_bytes(c);
}

int pp_conv3x3(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t stride,
               int32_t dtype, const void* in, const void* w, const float* scale_shift,
               void* out, int32_t tile, void* stream) {
  return pp_conv3x3_ws(batch, H, W, cin, cout, stride, dtype, in, w, scale_shift, out, tile,
                       nullptr, 0, stream);
}

int pp_conv3x3_ws(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t stride,
                  int32_t dtype, const void* in, const void* w, const float* scale_shift,
                  void* out, int32_t tile, void* workspace, size_t workspace_bytes, void* stream) {
  ConvShape c;
  int st = conv_shape(batch, H, W, cin, cout, stride, &c);
  if (st) return st;
  if (!in || !w || !scale_shift || !out) return fail(PP_EINVAL, "conv3x3: NULL buffer");
  if (!aligned16(in) || !aligned16(w) || !aligned16(out))
    return fail(PP_EINVAL, "conv3x3: buffers must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == PP_F32)
    return conv_f32_launch(c, static_cast<const float*>(in), static_cast<const float*>(w),
                           scale_shift, static_cast<float*>(out), tile, s);
  if (dtype == PP_BF16)
    return conv_bf16_launch(c, static_cast<const __nv_bfloat16*>(in),
                            static_cast<const __nv_bfloat16*>(w), scale_shift,
                            static_cast<__nv_bfloat16*>(out), tile, s);
  if (dtype == PP_F32_TC)
    return conv_f32tc_launch(c, static_cast<const float*>(in), static_cast<const float*>(w),
                             scale_shift, static_cast<float*>(out), tile, s, workspace, workspace_bytes);
  return fail(PP_EINVAL, "conv3x3: bad dtype");
}

int pp_conv_tile_count(int32_t dtype) {
  return dtype == PP_F32 ? conv_f32_tile_count()
       : dtype == PP_BF16 ? conv_bf16_tile_count()
       : dtype == PP_F32_TC ? conv_f32tc_tile_count() : 0;
}

int pp_conv_tile_info(int32_t dtype, int32_t tile, int32_t* bh, int32_t* bw, int32_t* bn,
                      int32_t* persistent) {
  if (!bh || !bw || !bn || !persistent) return fail(PP_EINVAL, "conv_tile_info: NULL argument");
  if (dtype == PP_F32) {
    static const int tiles[4][2] = {{128, 64}, {64, 64}, {128, 128}, {64, 128}};
    if (tile < 0 || tile >= 4) return fail(PP_EINVAL, "conv_tile_info: bad tile");
    *bh = 1; *bw = tiles[tile][0]; *bn = tiles[tile][1]; *persistent = 0;
    return PP_OK;
  }
  if (conv_tc_tile_info(dtype, tile, bh, bw, bn, persistent) != PP_OK)
    return fail(PP_EINVAL, "conv_tile_info: bad dtype or tile");
  return PP_OK;
}

size_t pp_conv_packed_bytes(int32_t cin, int32_t cout, int32_t dtype) {
  if (cin <= 0 || cout <= 0 || cin % 64 || cout % 64) return 0;
  if (dtype == PP_F32_TC) return (size_t)2 * 9 * cin * cout * 4;
  return (size_t)9 * cin * cout * (dtype == PP_F32 ? 4 : 2);
}

int pp_conv_pack_weights(const float* w_oihw, int32_t cin, int32_t cout, int32_t dtype,
                         void* w_packed, void* stream) {
  if (!w_oihw || !w_packed || cin <= 0 || cout <= 0 ||
      (dtype != PP_F32 && dtype != PP_BF16 && dtype != PP_F32_TC))
    return fail(PP_EINVAL, "pack_weights: bad argument");
  // the shapes pp_conv3x3 takes: a buffer packed for any other cin would be read past its end
  if (cin % 64 || cout % 64) return fail(PP_EINVAL, "pack_weights: cin and cout must be multiples of 64");
  return conv_pack_launch(w_oihw, cin, cout, dtype, w_packed, static_cast<cudaStream_t>(stream));
}

// ---- neck (transposed-conv upsampling) and detection head on the tensor-core GEMM

size_t pp_upsample_packed_bytes(int32_t cin, int32_t cout, int32_t up, int32_t dtype) {
  if (cin <= 0 || cin % 64 || cout <= 0 || cout % 64 || up < 1 || up > 8 ||
      (dtype != PP_BF16 && dtype != PP_F32_TC))
    return 0;
  return (size_t)up * up * cout * cin * (dtype == PP_BF16 ? 2 : 8);
}

int pp_upsample_pack_weights(const float* w, int32_t cin, int32_t cout, int32_t up, int32_t dtype,
                             void* w_packed) {
  if (!w || !w_packed || cin <= 0 || cout <= 0 || up < 1 || up > 8 || (dtype != PP_BF16 && dtype != PP_F32_TC))
    return fail(PP_EINVAL, "upsample_pack_weights: bad argument");
  // GEMM column n = (dy * up + dx) * cout + co  <-  w[ci][co][dy][dx]
  return pack_gemm(up * up * cout, up * up * cout, cin, dtype,
                   [&](int n, int k) {
                     const int q = n / cout, co = n % cout;
                     return w[(((size_t)k * cout + co) * up + q / up) * up + q % up];
                   },
                   w_packed);
}

size_t pp_head_packed_bytes(int32_t cin, int32_t cout, int32_t dtype) {
  if (cin <= 0 || cin % 64 || cout <= 0 || cout > 1024 || (dtype != PP_BF16 && dtype != PP_F32_TC)) return 0;
  return (size_t)head_pad(cout) * cin * (dtype == PP_BF16 ? 2 : 8);
}

int pp_head_pack_weights(const float* w, const float* bias, int32_t cin, int32_t cout, int32_t dtype,
                         void* w_packed, float* scale_shift) {
  if (!w || !bias || !w_packed || !scale_shift || cin <= 0 || cout <= 0 || (dtype != PP_BF16 && dtype != PP_F32_TC))
    return fail(PP_EINVAL, "head_pack_weights: bad argument");
  const int np = head_pad(cout);
  int st = pack_gemm(np, cout, cin, dtype, [&](int n, int k) { return w[(size_t)n * cin + k]; }, w_packed);
  if (st) return st;
  std::vector<float> ss(2 * (size_t)np, 0.f);
  for (int n = 0; n < np; ++n) ss[n] = 1.f;
  for (int n = 0; n < cout; ++n) ss[np + n] = bias[n];
  return cuda_status(cudaMemcpy(scale_shift, ss.data(), ss.size() * 4, cudaMemcpyHostToDevice), "upload head bias");
}

int pp_upsample(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t up, int32_t dtype,
                const void* in, const void* w_packed, const float* scale_shift, void* out, int32_t out_c,
                int32_t out_coff, int32_t tile, void* stream) {
  if (batch <= 0 || H <= 0 || W <= 0 || cin <= 0 || cin % 64 || cout <= 0 || cout % 64 || up < 1 || up > 8 ||
      out_c % 64 || out_coff % 64 || out_coff < 0 || out_coff + cout > out_c || cout > 1024)
    return fail(PP_EINVAL, "upsample: unsupported shape (cin, cout, out_c, out_coff multiples of 64)");
  if (!in || !w_packed || !scale_shift || !out) return fail(PP_EINVAL, "upsample: NULL buffer");
  ConvShape c;
  c.batch = batch; c.H = H; c.W = W; c.cin = cin; c.cout = up * up * cout; c.stride = 1; c.Ho = H; c.Wo = W;
  GemmOpts g;
  g.taps = 1; g.up = up; g.co_blk = cout; g.out_c = out_c; g.out_coff = out_coff; g.relu = 1;
  return gemm_tc_launch(dtype, c, g, in, w_packed, scale_shift, out, tile, static_cast<cudaStream_t>(stream));
}

int pp_head(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dtype, const void* in,
            const void* w_packed, const float* scale_shift, void* out, int32_t tile, void* stream) {
  if (batch <= 0 || H <= 0 || W <= 0 || cin <= 0 || cin % 64 || cout <= 0 || cout > 1024)
    return fail(PP_EINVAL, "head: unsupported shape (cin multiple of 64)");
  if (!in || !w_packed || !scale_shift || !out) return fail(PP_EINVAL, "head: NULL buffer");
  ConvShape c;
  c.batch = batch; c.H = H; c.W = W; c.cin = cin; c.cout = head_pad(cout); c.stride = 1; c.Ho = H; c.Wo = W;
  GemmOpts g;
  g.taps = 1; g.relu = 0;
  return gemm_tc_launch(dtype, c, g, in, w_packed, scale_shift, out, tile, static_cast<cudaStream_t>(stream));
}

int pp_bn_fold(const float* bn, int32_t c, float eps, float* out) {
  if (!bn || !out || c <= 0) return fail(PP_EINVAL, "bn_fold: bad argument");
  for (int i = 0; i < c; ++i) {
    const double gamma = bn[i], beta = bn[c + i], mean = bn[2 * c + i], var = bn[3 * c + i];
    if (!(var + eps > 0.0)) return fail(PP_EINVAL, "bn_fold: var + eps must be > 0");
    const double sc = gamma / std::sqrt(var + (double)eps);
    out[i] = (float)sc;
    out[c + i] = (float)(beta - mean * sc);
  }
  return PP_OK;
}

int pp_device_error_set(uint32_t bits) { return tc_error_set(bits); }

int pp_device_error(uint32_t* code, int32_t clear) {
  if (!code) return fail(PP_EINVAL, "device_error: NULL");
  unsigned v = 0;
  int st = tc_error_read(&v, clear != 0);
  *code = v;
  return st;
}

}  // extern "C"
