// PointNet (PFN) over pillars and the BEV scatter, batched over frames (PointPillars front end
// of the paper's 3D-perception chains, Section 6 / Table 4).
//
// pfn_fused: one warp per pillar.  The pillar's means come from a warp butterfly over lane j =
// point j; lane c owns channels c and c+32 and runs Linear(9->64) + folded BN + ReLU over the
// valid points (each point broadcast by shuffles), keeping a running max in registers.  The
// linear layer is evaluated regrouped (dev::PfnLane): the five offset features are affine in
// the point with per-pillar constants, so a point costs four FMAs per channel.  The regrouped
// weights are staged in shared memory once per block and held in registers by each lane.
// pfn_select_fused (a release unit's path): the same, with the voxeliser's point selection
// done by the warp itself (sort of the pillar's point indices, point loaded into lane j).
//
// bev_scatter: a single gather pass over the whole padded canvas -- every 16-byte chunk of every
// pixel is written exactly once (feature row of the pillar at that cell, zeros elsewhere and on
// the border), so no separate clear is needed and all stores are coalesced 16-byte vectors.
#include "pillar_dev.cuh"

namespace pp {
namespace {

constexpr int kWarps = 8;
// Resident blocks per SM of the fused selection + PointNet kernel: its registers (launch
// bounds) and its grid are both sized for this many, so the grid is one wave.
constexpr int kSelectBlocksPerSM = 3;

// x minus x with its 13 low mantissa bits cleared (exact in FP32): what a TF32 read drops.
__device__ __forceinline__ float tf32_rem(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// One pillar's features (lane c holds channels 2c and 2c + 1) into its canvas pixel: FP32 (chunks
// 16) as one 256-byte row per plane, the TF32 remainder plane beside it when lo != NULL; BF16
// (chunks 8) rounded to nearest even, one 128-byte row.
// The values and roundings are those of canvas_write on the same features.
__device__ __forceinline__ void canvas_put(size_t pix, int chunks, float m0, float m1, int lane,
                                           uint4* __restrict__ canvas, uint4* __restrict__ lo) {
  if (chunks == 16) {
    reinterpret_cast<float2*>(canvas)[pix * 32 + lane] = make_float2(m0, m1);
    if (lo) reinterpret_cast<float2*>(lo)[pix * 32 + lane] = make_float2(tf32_rem(m0), tf32_rem(m1));
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(m0, m1);
    reinterpret_cast<unsigned*>(canvas)[pix * 32 + lane] = *reinterpret_cast<unsigned*>(&h);
  }
}

// Stages the regrouped PointNet weights (dev::pfn_combine, one row per channel) and the table
// of 1 / n for n = 1..32 in shared memory; each lane then keeps its two channels' weights in
// registers (dev::pfn_lane).
__device__ __forceinline__ void pfn_stage_weights(const float* pfn_w, const float* ss,
                                                  float (*comb)[dev::kPfnComb], float* inv_s) {
  if (threadIdx.x < 64) dev::pfn_combine(pfn_w, ss, threadIdx.x, comb[threadIdx.x]);
  if (threadIdx.x < 33) inv_s[threadIdx.x] = threadIdx.x ? 1.f / (float)threadIdx.x : 0.f;
  __syncthreads();
}

__global__ void __launch_bounds__(256) pfn_fused(Geom g, const float4* __restrict__ pts,
                                                 const int* __restrict__ npts,
                                                 const int* __restrict__ coord,
                                                 const int* __restrict__ num_pillars,
                                                 const float* __restrict__ pfn_w,
                                                 const float* __restrict__ ss,
                                                 float* __restrict__ feat) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  __shared__ float comb[64][dev::kPfnComb];
  __shared__ float inv_s[33];
  pfn_stage_weights(pfn_w, ss, comb, inv_s);
  const dev::PfnLane L = dev::pfn_lane(comb, threadIdx.x & 31);
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int np = num_pillars[b];
  // each warp walks pillars p, p + gridDim.x * kWarps, ... (warp-uniform; no block barrier
  // follows), so the weights staged above serve several pillars
  for (int p = blockIdx.x * kWarps + wid; p < np; p += gridDim.x * kWarps) {
    const size_t q = (size_t)b * g.P + p;
    float m0, m1;
    const int n = npts[q];
    dev::pfn_pillar(g, pts[q * 32 + lane], n, coord[q], lane, L, inv_s[n], m0, m1);
    reinterpret_cast<float2*>(feat)[q * 32 + lane] = make_float2(m0, m1);
  }
}

// Point selection fused with PointNet (the release unit's path): each warp sorts its pillar's
// point indices (the 32 lowest, as vox_select does), loads lane j's point straight into a
// register and runs the pillar's PointNet, so the gathered points never go through memory.
__global__ void __launch_bounds__(256, kSelectBlocksPerSM) pfn_select_fused(Geom g, int cap, const float4* __restrict__ points,
                                                        const float4* const* __restrict__ srcs,
                                                        const int* __restrict__ csr,
                                                        const int* __restrict__ pillar_start,
                                                        const int* __restrict__ pillar_cnt,
                                                        const int* __restrict__ coord,
                                                        const int* __restrict__ num_pillars,
                                                        const float* __restrict__ pfn_w,
                                                        const float* __restrict__ ss,
                                                        float* __restrict__ feat, int chunks,
                                                        int* __restrict__ drawn, int* __restrict__ drawn_num,
                                                        uint4* __restrict__ canvas, uint4* __restrict__ lo,
                                                        unsigned* __restrict__ cnt_zero) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  __shared__ float comb[64][dev::kPfnComb];
  __shared__ float inv_s[33];
  pfn_stage_weights(pfn_w, ss, comb, inv_s);
  const dev::PfnLane L = dev::pfn_lane(comb, threadIdx.x & 31);
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int np = num_pillars[b];
  // the bucket pass has read the previous frame's drawn list: this frame's replaces it
  if (canvas && blockIdx.x == 0 && threadIdx.x == 0) drawn_num[b] = np;
  const float4* src = dev::frame_src(points, srcs, b, cap);
  const int* csr_b = csr + (size_t)b * cap;
  const int stride = gridDim.x * kWarps;
  // Software pipeline over the warp's pillars p, p + stride, ...: in the iteration of pillar p
  // the warp loads the metadata of pillar p + 3 and the first 32 point indices of pillar p + 2,
  // sorts the indices of pillar p + 1 and starts its point gather, then runs pillar p's
  // PointNet on the points gathered one iteration earlier, so every load has a whole
  // iteration's work to arrive in.
  auto meta = [&](int pp, int& cnt, int& st, int& cl) {
    cnt = 0; st = 0; cl = 0;
    if (pp < np) {
      const size_t q = (size_t)b * g.P + pp;
      cnt = pillar_cnt[q];
      st = pillar_start[q];
      cl = coord[q];
    }
  };
  auto firsts = [&](int pp, int cnt, int st) { return pp < np && lane < cnt ? csr_b[st + lane] : INT_MAX; };
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  int p = blockIdx.x * kWarps + wid;
  int c0, s0, l0, c1, s1, l1, c2, s2, l2;  // metadata of pillars p, p + stride, p + 2 stride
  meta(p, c0, s0, l0);
  meta(p + stride, c1, s1, l1);
  meta(p + 2 * stride, c2, s2, l2);
  int f1 = firsts(p + stride, c1, s1);
  float4 v0 = zero;
  if (p < np) {
    const int best = dev::lowest_32_from(firsts(p, c0, s0), csr_b + s0, c0, lane);
    if (lane < c0) v0 = src[best];
  }
  for (; p < np; p += stride) {
    const size_t q = (size_t)b * g.P + p;
    int c3, s3, l3;
    meta(p + 3 * stride, c3, s3, l3);
    const int f2 = firsts(p + 2 * stride, c2, s2);
    float4 v1 = zero;
    if (p + stride < np) {  // warp-uniform
      const int best = dev::lowest_32_from(f1, csr_b + s1, c1, lane);
      if (lane < c1) v1 = src[best];
    }
    float m0, m1;
    const int n0 = c0 < 32 ? c0 : 32;
    dev::pfn_pillar(g, v0, n0, l0, lane, L, inv_s[n0], m0, m1);
    if (feat) {
      reinterpret_cast<float2*>(feat)[q * 32 + lane] = make_float2(m0, m1);
    }
    if (canvas) {
      canvas_put(dev::canvas_pixel(g, b, l0), chunks, m0, m1, lane, canvas, lo);
      if (lane == 0) drawn[q] = l0;
    }
    // a release unit's count array: the kept cell's entry (its bucket lookup) back to zero
    if (cnt_zero && lane == 0) cnt_zero[(size_t)b * g.G + l0] = 0u;
    c0 = c1; s0 = s1; l0 = l1;
    c1 = c2; s1 = s2; l1 = l2;
    c2 = c3; s2 = s3; l2 = l3;
    f1 = f2;
    v0 = v1;
  }
}

__device__ __forceinline__ float4 tf32_rem4(float4 v) {
  return make_float4(tf32_rem(v.x), tf32_rem(v.y), tf32_rem(v.z), tf32_rem(v.w));
}

// FP32 canvas: 16 chunks of 4 channels per pixel; with `lo`, also the TF32 remainder plane.
__global__ void bev_scatter_f32(Geom g, int batch, const float4* __restrict__ feat,
                                const int* __restrict__ pillar_of_cell,
                                float4* __restrict__ canvas, float4* __restrict__ lo) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const int Wp = g.nx + 2, Hp = g.ny + 2;
  const size_t total = (size_t)batch * Hp * Wp * 16;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int chunk = (int)(t & 15);
    const size_t pix = t >> 4;
    const int x = (int)(pix % Wp);
    const size_t r = pix / Wp;
    const int y = (int)(r % Hp);
    const int b = (int)(r / Hp);
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x >= 1 && x <= g.nx && y >= 1 && y <= g.ny) {
      const int p = pillar_of_cell[(size_t)b * g.G + (size_t)(y - 1) * g.nx + (x - 1)];
      if (p >= 0) val = feat[((size_t)b * g.P + p) * 16 + chunk];
    }
    canvas[t] = val;
    if (lo) lo[t] = tf32_rem4(val);
  }
}

__global__ void tf32_split_kernel(const float4* __restrict__ x, float4* __restrict__ lo, size_t n4) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    lo[i] = tf32_rem4(x[i]);
}

__global__ void tf32_split_tail(const float* __restrict__ x, float* __restrict__ lo, size_t from, size_t n) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const size_t i = from + threadIdx.x;
  if (i < n) lo[i] = tf32_rem(x[i]);
}

// BF16 canvas: 8 chunks of 8 channels (16 bytes) per pixel, round to nearest even.
__global__ void bev_scatter_bf16(Geom g, int batch, const float4* __restrict__ feat,
                                 const int* __restrict__ pillar_of_cell,
                                 uint4* __restrict__ canvas) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const int Wp = g.nx + 2, Hp = g.ny + 2;
  const size_t total = (size_t)batch * Hp * Wp * 8;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int chunk = (int)(t & 7);
    const size_t pix = t >> 3;
    const int x = (int)(pix % Wp);
    const size_t r = pix / Wp;
    const int y = (int)(r % Hp);
    const int b = (int)(r / Hp);
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (x >= 1 && x <= g.nx && y >= 1 && y <= g.ny) {
      const int p = pillar_of_cell[(size_t)b * g.G + (size_t)(y - 1) * g.nx + (x - 1)];
      if (p >= 0) {
        const float4* src = feat + ((size_t)b * g.P + p) * 16 + chunk * 2;
        const float4 a = src[0], c = src[1];
        __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(a.z, a.w);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(c.x, c.y);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(c.z, c.w);
        val.x = *reinterpret_cast<unsigned*>(&h0);
        val.y = *reinterpret_cast<unsigned*>(&h1);
        val.z = *reinterpret_cast<unsigned*>(&h2);
        val.w = *reinterpret_cast<unsigned*>(&h3);
      }
    }
    canvas[t] = val;
  }
}

// Incremental scatter into a canvas that persists across frames (see pp_scatter_update).
// Stale cells: cells drawn for the slot's previous frame that hold no kept pillar now; each
// thread zeroes one 16-byte chunk of one (both planes of the split FP32 form).  Cells that hold
// a pillar now are left to canvas_write, so the two kernels never touch the same cell.
using dev::canvas_pixel;

__global__ void canvas_clear_stale(Geom g, int batch, int chunks, const int* __restrict__ pillar_of_cell,
                                   const int* __restrict__ drawn, const int* __restrict__ drawn_num,
                                   uint4* __restrict__ canvas, uint4* __restrict__ lo) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const size_t total = (size_t)batch * g.P * chunks;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int chunk = (int)(t % chunks);
    const size_t q = t / chunks;
    const int b = (int)(q / g.P), j = (int)(q % g.P);
    if (j >= drawn_num[b]) continue;
    const int c = drawn[q];
    if (pillar_of_cell[(size_t)b * g.G + c] >= 0) continue;
    const size_t off = canvas_pixel(g, b, c) * chunks + chunk;
    canvas[off] = make_uint4(0u, 0u, 0u, 0u);
    if (lo) lo[off] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Writes every kept pillar's features at its cell (FP32 value + TF32 remainder plane, or BF16
// round to nearest even) and records the cells drawn for this frame.
__global__ void canvas_write(Geom g, int batch, int chunks, const float4* __restrict__ feat,
                             const int* __restrict__ coord, const int* __restrict__ num_pillars,
                             int* __restrict__ drawn, int* __restrict__ drawn_num, uint4* __restrict__ canvas,
                             uint4* __restrict__ lo) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const size_t total = (size_t)batch * g.P * chunks;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int chunk = (int)(t % chunks);
    const size_t q = t / chunks;
    const int b = (int)(q / g.P), p = (int)(q % g.P);
    const int n = num_pillars[b];
    if (p == 0 && chunk == 0) drawn_num[b] = n;
    if (p >= n) continue;
    const int c = coord[q];
    if (chunk == 0) drawn[q] = c;
    const size_t off = canvas_pixel(g, b, c) * chunks + chunk;
    if (chunks == 16) {  // FP32: 4 channels per chunk
      const float4 v = feat[q * 16 + chunk];
      canvas[off] = *reinterpret_cast<const uint4*>(&v);
      if (lo) {
        const float4 r = tf32_rem4(v);
        lo[off] = *reinterpret_cast<const uint4*>(&r);
      }
    } else {             // BF16: 8 channels per chunk
      const float4 a = feat[q * 16 + chunk * 2], d = feat[q * 16 + chunk * 2 + 1];
      __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(a.z, a.w);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(d.x, d.y);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(d.z, d.w);
      uint4 val;
      val.x = *reinterpret_cast<unsigned*>(&h0);
      val.y = *reinterpret_cast<unsigned*>(&h1);
      val.z = *reinterpret_cast<unsigned*>(&h2);
      val.w = *reinterpret_cast<unsigned*>(&h3);
      canvas[off] = val;
    }
  }
}

int sm_count() {
  return device_sms();
}

}  // namespace

int pfn_launch(const Geom& g, int batch, const float4* pts, const int* npts, const int* coord,
               const int* num_pillars, const float* pfn_w, const float* ss, float* feat,
               cudaStream_t s) {
  // about 4 blocks per SM over the batch; warps loop over their pillars
  int bx = (g.P + kWarps - 1) / kWarps;
  const int bx_max = (4 * sm_count() + batch - 1) / batch;
  if (bx > bx_max) bx = bx_max;
  return cuda_status(launch_pdl(pfn_fused, dim3(bx > 0 ? bx : 1, batch), dim3(kWarps * 32), 0, s, g, pts, npts,
                                coord, num_pillars, pfn_w, ss, feat),
                     "pointnet launch");
}

int select_pfn_launch(const Geom& g, int batch, int cap, const float4* points, const float4* const* srcs,
                      const VoxWork& w, const int* coord, const int* num_pillars, const float* pfn_w,
                      const float* ss, float* feat, cudaStream_t s, int chunks, int* drawn, int* drawn_num,
                      uint4* canvas, uint4* lo, unsigned* cnt_zero) {
  int bx = (g.P + kWarps - 1) / kWarps;
  const int bx_max = (kSelectBlocksPerSM * sm_count() + batch - 1) / batch;
  if (bx > bx_max) bx = bx_max;
  return cuda_status(launch_pdl(pfn_select_fused, dim3(bx > 0 ? bx : 1, batch), dim3(kWarps * 32), 0, s, g, cap,
                                points, srcs, (const int*)w.csr, (const int*)w.pillar_start,
                                (const int*)w.pillar_cnt, coord, num_pillars, pfn_w, ss, feat, chunks, drawn,
                                drawn_num, canvas, lo, cnt_zero),
                     "select + pointnet launch");
}

int scatter_launch(const Geom& g, int batch, const float* feat, const int* pillar_of_cell,
                   void* canvas, int dtype, cudaStream_t s, size_t plane) {
  const size_t pixels = (size_t)batch * (g.ny + 2) * (g.nx + 2);
  const size_t chunks = pixels * (dtype == PP_BF16 ? 8 : 16);
  size_t blocks = (chunks + 255) / 256;
  const size_t cap = (size_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  cudaError_t e;
  if (dtype == PP_F32 || dtype == PP_F32_TC)
    e = launch_pdl(bev_scatter_f32, dim3((unsigned)blocks), dim3(256), 0, s, g, batch, (const float4*)feat,
                   pillar_of_cell, (float4*)canvas,
                   dtype == PP_F32_TC ? (float4*)canvas + (plane ? plane / 4 : chunks) : (float4*)nullptr);
  else
    e = launch_pdl(bev_scatter_bf16, dim3((unsigned)blocks), dim3(256), 0, s, g, batch, (const float4*)feat,
                   pillar_of_cell, (uint4*)canvas);
  return cuda_status(e, "scatter launch");
}

int scatter_update_launch(const Geom& g, int batch, const float* feat, const int* coord, const int* num_pillars,
                          const int* pillar_of_cell, int* drawn, int* drawn_num, void* canvas, int dtype,
                          cudaStream_t s, size_t plane) {
  const int chunks = dtype == PP_BF16 ? 8 : 16;
  const size_t pixels = (size_t)batch * (g.ny + 2) * (g.nx + 2);
  uint4* cv = static_cast<uint4*>(canvas);
  // the remainder plane follows the value plane (plane: floats per plane, default this batch's)
  uint4* lo = dtype == PP_F32_TC ? cv + (plane ? plane / 4 : pixels * 16) : nullptr;
  const size_t work = (size_t)batch * g.P * chunks;
  size_t blocks = (work + 255) / 256;
  const size_t cap = (size_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  cudaError_t e = launch_pdl(canvas_clear_stale, dim3((unsigned)blocks), dim3(256), 0, s, g, batch, chunks,
                             pillar_of_cell, (const int*)drawn, (const int*)drawn_num, cv, lo);
  if (e == cudaSuccess)
    e = launch_pdl(canvas_write, dim3((unsigned)blocks), dim3(256), 0, s, g, batch, chunks, (const float4*)feat,
                   coord, num_pillars, drawn, drawn_num, cv, lo);
  return cuda_status(e, "scatter update launch");
}

int tf32_split_launch(const float* x, float* lo, size_t n, cudaStream_t s) {
  const size_t n4 = n / 4;
  if (n4) {
    size_t blocks = (n4 + 255) / 256;
    const size_t cap = (size_t)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    const cudaError_t e = launch_pdl(tf32_split_kernel, dim3((unsigned)blocks), dim3(256), 0, s, (const float4*)x,
                                     (float4*)lo, n4);
    if (e != cudaSuccess) return cuda_status(e, "tf32 split launch");
  }
  if (n % 4)
    return cuda_status(launch_pdl(tf32_split_tail, dim3(1), dim3(4), 0, s, x, lo, n4 * 4, n), "tf32 split launch");
  return PP_OK;
}

}  // namespace pp
