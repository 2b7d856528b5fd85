// C-ABI stage entry points: argument validation, then the launches in the kernel files.
#include "pp_internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

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
  return PP_OK;
}

int tc_error_read(unsigned* code, bool clear);

}  // namespace pp

using namespace pp;

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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
  if (cin <= 0 || cout <= 0) return 0;
  if (dtype == PP_F32_TC) return (size_t)2 * 9 * cin * cout * 4;
  return (size_t)9 * cin * cout * (dtype == PP_F32 ? 4 : 2);
}

int pp_conv_pack_weights(const float* w_oihw, int32_t cin, int32_t cout, int32_t dtype,
                         void* w_packed, void* stream) {
  if (!w_oihw || !w_packed || cin <= 0 || cout <= 0 ||
      (dtype != PP_F32 && dtype != PP_BF16 && dtype != PP_F32_TC))
    return fail(PP_EINVAL, "pack_weights: bad argument");
  return conv_pack_launch(w_oihw, cin, cout, dtype, w_packed, static_cast<cudaStream_t>(stream));
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

int pp_device_error(uint32_t* code, int32_t clear) {
  if (!code) return fail(PP_EINVAL, "device_error: NULL");
  unsigned v = 0;
  int st = tc_error_read(&v, clear != 0);
  *code = v;
  return st;
}

}  // extern "C"
