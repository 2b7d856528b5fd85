// Device helpers shared by the voxelisation and PointNet kernels: the warp sort that picks a
// pillar's lowest point indices, and the PointNet of one pillar (one warp, lane j = point j).
#pragma once

#include <climits>

#include "pp_internal.h"

namespace pp {
namespace dev {

constexpr unsigned kFullMask = 0xffffffffu;

// cell / nx for a cell index 0 <= cell < 2^31: the high word of cell times
// g.nx_magic = ceil(2^64 / nx) (nx >= 2; Lemire, Kaser and Kurz, "Faster remainder by direct
// computation", 2019: exact for every 32-bit dividend), set with the geometry on the host.
__device__ __forceinline__ int nx_div(const Geom& g, int cell) {
  return g.nx > 1 ? (int)__umul64hi(g.nx_magic, (uint64_t)(unsigned)cell) : cell;
}

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

// PointNet weights of lane c's two channels (2c and 2c + 1), BN folded in: with BN scale s,
// shift h and weight rows w[0..8] over the features (x, y, z, r, x - x_mean, y - y_mean,
// z - z_mean, x - x_centre, y - y_centre), a channel's pre-activation is
//   s (w . f) + h = ax x + ay y + az z + ar r + (h - m4 x_mean - m5 y_mean - m6 z_mean
//                                                  - m7 x_centre - m8 y_centre)
// with ax = s (w0 + w4 + w7), ay = s (w1 + w5 + w8), az = s (w2 + w6), ar = s w3 and
// mk = s wk: the same affine map of the point, regrouped so that the per-point work is four
// FMAs per channel and the pillar's means and cell centre enter once per pillar.
struct PfnLane {
  float ax[2], ay[2], az[2], ar[2], m4[2], m5[2], m6[2], m7[2], m8[2], h[2];
};
constexpr int kPfnComb = 10;  // floats per channel in the staged table

// One channel's regrouped weights (row c of W [64][9] and the folded scale / shift ss [2][64])
// into t[0..9] = ax, ay, az, ar, m4, m5, m6, m7, m8, h.
__device__ __forceinline__ void pfn_combine(const float* __restrict__ w, const float* __restrict__ ss, int c,
                                            float* t) {
  const float sc = ss[c];
  const float* r = w + c * 9;
  t[0] = sc * (r[0] + r[4] + r[7]);
  t[1] = sc * (r[1] + r[5] + r[8]);
  t[2] = sc * (r[2] + r[6]);
  t[3] = sc * r[3];
  t[4] = sc * r[4];
  t[5] = sc * r[5];
  t[6] = sc * r[6];
  t[7] = sc * r[7];
  t[8] = sc * r[8];
  t[9] = ss[64 + c];
}

__device__ __forceinline__ PfnLane pfn_lane(const float (*comb)[kPfnComb], int lane) {
  PfnLane L;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float* t = comb[2 * lane + i];
    L.ax[i] = t[0]; L.ay[i] = t[1]; L.az[i] = t[2]; L.ar[i] = t[3];
    L.m4[i] = t[4]; L.m5[i] = t[5]; L.m6[i] = t[6]; L.m7[i] = t[7]; L.m8[i] = t[8];
    L.h[i] = t[9];
  }
  return L;
}

// PointNet of one pillar: lane j holds point v of the pillar (valid for j < n, n >= 1) at grid
// cell `cell`; lane c returns channels 2c and 2c + 1: the max over the valid points of
// ReLU(s (W . f) + h) for the 9 features f of the point (x, y, z, r, offsets to the mean of the
// valid points, x/y offsets to the cell centre), evaluated in the regrouped form of PfnLane.
// inv_n: 1 / n (table in shared memory).
__device__ __forceinline__ void pfn_pillar(const Geom& g, float4 v, int n, int cell, int lane, const PfnLane& L,
                                           float inv_n, float& m0, float& m1) {
  const bool valid = lane < n;
  float sx = valid ? v.x : 0.f, sy = valid ? v.y : 0.f, sz = valid ? v.z : 0.f;
  // butterfly sums over lanes 0..2^k-1 (2^k >= n): the stages of a 32-lane butterfly above
  // them would only add zeros, so this is the full sum, bit for bit, in every lane below 2^k
  for (int o = n > 1 ? 1 << (31 - __clz(n - 1)) : 0; o; o >>= 1) {
    sx += __shfl_xor_sync(kFullMask, sx, o);
    sy += __shfl_xor_sync(kFullMask, sy, o);
    sz += __shfl_xor_sync(kFullMask, sz, o);
  }
  // every lane takes the means from lane 0 (the lanes >= 2^k hold partial sums)
  const float mx = __shfl_sync(kFullMask, sx, 0) * inv_n;
  const float my = __shfl_sync(kFullMask, sy, 0) * inv_n;
  const float mz = __shfl_sync(kFullMask, sz, 0) * inv_n;
  const int iy = nx_div(g, cell), ix = cell - iy * g.nx;
  const float xc = g.xmin + ((float)ix + 0.5f) * g.vx;
  const float yc = g.ymin + ((float)iy + 0.5f) * g.vy;
  float c[2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
    c[i] = L.h[i] - (L.m4[i] * mx + L.m7[i] * xc + L.m5[i] * my + L.m8[i] * yc + L.m6[i] * mz);
  m0 = 0.f;  // ReLU outputs are >= 0 and every pillar has >= 1 point
  m1 = 0.f;
  for (int j = 0; j < n; ++j) {
    const float px = __shfl_sync(kFullMask, v.x, j), py = __shfl_sync(kFullMask, v.y, j);
    const float pz = __shfl_sync(kFullMask, v.z, j), pr = __shfl_sync(kFullMask, v.w, j);
    const float a0 = fmaf(L.ax[0], px, fmaf(L.ay[0], py, fmaf(L.az[0], pz, fmaf(L.ar[0], pr, c[0]))));
    const float a1 = fmaf(L.ax[1], px, fmaf(L.ay[1], py, fmaf(L.az[1], pz, fmaf(L.ar[1], pr, c[1]))));
    m0 = fmaxf(m0, a0);
    m1 = fmaxf(m1, a1);
  }
}

// Padded canvas pixel [b][iy + 1][ix + 1] of cell `cell` = iy * nx + ix of frame b.
__device__ __forceinline__ size_t canvas_pixel(const Geom& g, int b, int cell) {
  const int iy = nx_div(g, cell), ix = cell - iy * g.nx;
  return ((size_t)b * (g.ny + 2) + iy + 1) * (g.nx + 2) + ix + 1;
}

}  // namespace dev
}  // namespace pp
