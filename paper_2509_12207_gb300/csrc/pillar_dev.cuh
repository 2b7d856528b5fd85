// Device helpers shared by the voxelisation and PointNet kernels: the warp sort that picks a
// pillar's lowest point indices, and the PointNet of one pillar (one warp, lane j = point j).
#pragma once

#include <climits>

#include "pp_internal.h"

namespace pp {
namespace dev {

constexpr unsigned kFullMask = 0xffffffffu;

// Frame b's points: srcs[b] when a per-frame pointer table is given, else row b of the batch.
__device__ __forceinline__ const float4* frame_src(const float4* points, const float4* const* srcs, int b,
                                                   int cap) {
  return srcs ? srcs[b] : points + (size_t)b * cap;
}

// Ascending bitonic sort of one int per lane across a warp.  With `upto` < 32 (warp-uniform)
// the network stops after its merges of width `upto` (rounded up to a power of two): lanes
// 0..upto-1 are then sorted among themselves, which is the whole sort when every lane from
// `upto` on holds INT_MAX (a pillar of at most `upto` points).
__device__ __forceinline__ int warp_sort(int v, int lane, int upto = 32) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
    if (k >= 2 * upto && k > 2) break;  // blocks of k / 2 >= upto lanes are sorted already
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int o = __shfl_xor_sync(kFullMask, v, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
      v = keep_min ? min(v, o) : max(v, o);
    }
  }
  return v;
}

// Sorts a bitonic sequence held one per lane into ascending order.
__device__ __forceinline__ int warp_bitonic_merge(int v, int lane) {
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const int o = __shfl_xor_sync(kFullMask, v, j);
    v = (lane & j) == 0 ? min(v, o) : max(v, o);
  }
  return v;
}

// The 32 smallest of `count` point indices seg[0..count), ascending, one per lane (INT_MAX past
// count): a warp sort of the first 32 (`first`: lane's entry of them, already loaded), then a
// bitonic merge with each further sorted chunk.
__device__ __forceinline__ int lowest_32_from(int first, const int* seg, int count, int lane) {
  int best = warp_sort(first, lane, count);
  for (int k = 32; k < count; k += 32) {
    int v = warp_sort(k + lane < count ? seg[k + lane] : INT_MAX, lane);
    v = __shfl_sync(kFullMask, v, 31 - lane);          // reversed: best ++ v is bitonic
    best = warp_bitonic_merge(min(best, v), lane);     // lower half = 32 smallest of the union
  }
  return best;
}

__device__ __forceinline__ int lowest_32(const int* seg, int count, int lane) {
  return lowest_32_from(lane < count ? seg[lane] : INT_MAX, seg, count, lane);
}

// PointNet of one pillar: lane j holds point v of the pillar (valid for j < n, n >= 1) at grid
// cell `cell`.  Builds the 9 features (x, y, z, r, offsets to the mean of the valid points, x/y
// offsets to the cell centre) into f_w[32][10], then lane c computes channels c and c+32:
// max over the valid points of ReLU(scale * (W . f) + shift).  w_s [9][64] (transposed
// weights), sc_s / sh_s [64] in shared memory.
__device__ __forceinline__ void pfn_pillar(const Geom& g, float4 v, int n, int cell, int lane,
                                           float (*f_w)[10], const float (*w_s)[64], const float* sc_s,
                                           const float* sh_s, float& m0, float& m1) {
  const bool valid = lane < n;
  float sx = valid ? v.x : 0.f, sy = valid ? v.y : 0.f, sz = valid ? v.z : 0.f;
  for (int o = 16; o; o >>= 1) {
    sx += __shfl_xor_sync(kFullMask, sx, o);
    sy += __shfl_xor_sync(kFullMask, sy, o);
    sz += __shfl_xor_sync(kFullMask, sz, o);
  }
  const float inv = 1.f / (float)n;
  const float mx = sx * inv, my = sy * inv, mz = sz * inv;
  const int ix = cell % g.nx, iy = cell / g.nx;
  const float xc = g.xmin + ((float)ix + 0.5f) * g.vx;
  const float yc = g.ymin + ((float)iy + 0.5f) * g.vy;
  float* f = f_w[lane];
  f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
  f[4] = v.x - mx; f[5] = v.y - my; f[6] = v.z - mz;
  f[7] = v.x - xc; f[8] = v.y - yc;
  __syncwarp();
  const float s0 = sc_s[lane], s1 = sc_s[lane + 32];
  const float h0 = sh_s[lane], h1 = sh_s[lane + 32];
  m0 = 0.f;  // ReLU outputs are >= 0 and every pillar has >= 1 point
  m1 = 0.f;
  for (int j = 0; j < n; ++j) {
    const float* fj = f_w[j];
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      a0 = fmaf(fj[k], w_s[k][lane], a0);
      a1 = fmaf(fj[k], w_s[k][lane + 32], a1);
    }
    m0 = fmaxf(m0, fmaxf(fmaf(a0, s0, h0), 0.f));
    m1 = fmaxf(m1, fmaxf(fmaf(a1, s1, h1), 0.f));
  }
  __syncwarp();  // f_w is rewritten by the next pillar
}

// Padded canvas pixel [b][iy + 1][ix + 1] of cell `cell` = iy * nx + ix of frame b.
__device__ __forceinline__ size_t canvas_pixel(const Geom& g, int b, int cell) {
  const int iy = cell / g.nx, ix = cell - iy * g.nx;
  return ((size_t)b * (g.ny + 2) + iy + 1) * (g.nx + 2) + ix + 1;
}

}  // namespace dev
}  // namespace pp
