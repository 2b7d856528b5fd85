// FP32 conv3x3 + folded BN + ReLU on CUDA cores: implicit GEMM over padded NHWC.
//
// GEMM view per frame: M = Ho*Wo output pixels, N = cout, K = 9*cin ordered (ky, kx, ci).
// The one-pixel zero border of the padded input means no halo test in the inner loop; ragged M
// tiles clamp their loads to the last pixel and mask their stores.  A tiles (pixels x 16
// channels) are loaded to registers and stored transposed ([k][m]) so each thread reads its
// rows as float4; B tiles come from weights packed [9*cin][cout] by 16-byte cp.async.  Two
// shared-memory stages overlap the next tile's loads with this tile's FMAs.  This is the exact
// path (FP32 throughout, no TF32).
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int BK = 16;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n"); }

template <int BM, int BN, int TN>
__global__ void __launch_bounds__((BM / 8) * (BN / TN))
conv3x3_f32(ConvShape c, const float* __restrict__ in, const float* __restrict__ w,
            const float* __restrict__ ss, float* __restrict__ out) {
  constexpr int THR = (BM / 8) * (BN / TN);
  constexpr int TX = BN / TN;  // threads along N
  static_assert(THR == 2 * BM, "A-tile loader assumes 2*BM threads");
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];

  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int b = blockIdx.z;
  const int n0 = blockIdx.y * BN;
  const int m0 = blockIdx.x * BM;
  const int Mtot = c.Ho * c.Wo;
  const int Hp = c.H + 2, Wp = c.W + 2;

  // this thread's two A rows (pixel m, channel quads q and q+2)
  const int am = t % BM;
  const int aq = t / BM;  // 0 or 1
  int mm = m0 + am;
  if (mm >= Mtot) mm = Mtot - 1;
  const int oy = mm / c.Wo, ox = mm % c.Wo;
  const float* abase = in + (((size_t)b * Hp + (size_t)oy * c.stride) * Wp + (size_t)ox * c.stride) * c.cin;

  const int kchunks = c.cin / BK;
  const int KT = 9 * kchunks;

  auto a_ptr = [&](int kt) {
    const int tap = kt / kchunks, cc = kt % kchunks;
    const int ky = tap / 3, kx = tap % 3;
    return abase + ((size_t)ky * Wp + kx) * c.cin + cc * BK;
  };
  auto load_b = [&](int kt, int stage) {
    const float* wb = w + (size_t)kt * BK * c.cout + n0;
#pragma unroll
    for (int r = 0; r < (BK * BN / 4 + THR - 1) / THR; ++r) {
      const int idx = t + r * THR;
      if (idx < BK * BN / 4) {
        const int k = idx / (BN / 4), nq = idx % (BN / 4);
        cp_async16(&Bs[stage][k][nq * 4], wb + (size_t)k * c.cout + nq * 4);
      }
    }
    cp_async_commit();
  };
  auto store_a = [&](int stage, const float4& v0, const float4& v1) {
    As[stage][aq * 4 + 0][am] = v0.x;
    As[stage][aq * 4 + 1][am] = v0.y;
    As[stage][aq * 4 + 2][am] = v0.z;
    As[stage][aq * 4 + 3][am] = v0.w;
    As[stage][aq * 4 + 8][am] = v1.x;
    As[stage][aq * 4 + 9][am] = v1.y;
    As[stage][aq * 4 + 10][am] = v1.z;
    As[stage][aq * 4 + 11][am] = v1.w;
  };

  float acc[8][TN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  {
    const float* ap = a_ptr(0);
    const float4 v0 = *reinterpret_cast<const float4*>(ap + aq * 4);
    const float4 v1 = *reinterpret_cast<const float4*>(ap + aq * 4 + 8);
    load_b(0, 0);
    store_a(0, v0, v1);
    cp_async_wait_all();
    __syncthreads();
  }

  for (int kt = 0; kt < KT; ++kt) {
    const int cur = kt & 1, nxt = cur ^ 1;
    float4 v0, v1;
    const bool more = kt + 1 < KT;
    if (more) {
      const float* ap = a_ptr(kt + 1);
      v0 = *reinterpret_cast<const float4*>(ap + aq * 4);
      v1 = *reinterpret_cast<const float4*>(ap + aq * 4 + 8);
      load_b(kt + 1, nxt);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][BM / 2 + ty * 4]);
      float bv[TN];
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
      bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
      if (TN == 8) {
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][BN / 2 + tx * 4]);
        bv[TN - 4] = b1.x; bv[TN - 3] = b1.y; bv[TN - 2] = b1.z; bv[TN - 1] = b1.w;
      }
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      store_a(nxt, v0, v1);
      cp_async_wait_all();
    }
    __syncthreads();
  }

  // epilogue: folded BN + ReLU, float4 stores into the padded output interior
  float sc[TN], sh[TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int n = n0 + (j < 4 ? tx * 4 + j : BN / 2 + tx * 4 + (j - 4));
    sc[j] = ss[n];
    sh[j] = ss[c.cout + n];
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : BM / 2 + ty * 4 + (i - 4));
    if (m >= Mtot) continue;
    const int y = m / c.Wo, x = m % c.Wo;
    float* o = out + (((size_t)b * (c.Ho + 2) + y + 1) * (c.Wo + 2) + x + 1) * c.cout + n0;
    float4 r0;
    r0.x = fmaxf(fmaf(acc[i][0], sc[0], sh[0]), 0.f);
    r0.y = fmaxf(fmaf(acc[i][1], sc[1], sh[1]), 0.f);
    r0.z = fmaxf(fmaf(acc[i][2], sc[2], sh[2]), 0.f);
    r0.w = fmaxf(fmaf(acc[i][3], sc[3], sh[3]), 0.f);
    *reinterpret_cast<float4*>(o + tx * 4) = r0;
    if (TN == 8) {
      float4 r1;
      r1.x = fmaxf(fmaf(acc[i][TN - 4], sc[TN - 4], sh[TN - 4]), 0.f);
      r1.y = fmaxf(fmaf(acc[i][TN - 3], sc[TN - 3], sh[TN - 3]), 0.f);
      r1.z = fmaxf(fmaf(acc[i][TN - 2], sc[TN - 2], sh[TN - 2]), 0.f);
      r1.w = fmaxf(fmaf(acc[i][TN - 1], sc[TN - 1], sh[TN - 1]), 0.f);
      *reinterpret_cast<float4*>(o + BN / 2 + tx * 4) = r1;
    }
  }
}

// OIHW float -> packed layout (see pp_conv_pack_weights).
__global__ void pack_weights(const float* __restrict__ w, int cin, int cout, int dtype,
                             void* __restrict__ dst) {
  const int total = cout * cin * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int kx = i % 3, ky = (i / 3) % 3, ci = (i / 9) % cin, co = i / (9 * cin);
    const int k = (ky * 3 + kx) * cin + ci;
    if (dtype == PP_F32) {
      static_cast<float*>(dst)[(size_t)k * cout + co] = w[i];
    } else if (dtype == PP_F32_TC) {
      // hi: the value with its 13 low mantissa bits cleared (a TF32 value); lo: the rest
      const float hi = __uint_as_float(__float_as_uint(w[i]) & 0xFFFFE000u);
      float* d = static_cast<float*>(dst);
      d[(size_t)co * 9 * cin + k] = hi;
      d[(size_t)cout * 9 * cin + (size_t)co * 9 * cin + k] = w[i] - hi;
    } else {
      static_cast<__nv_bfloat16*>(dst)[(size_t)co * 9 * cin + k] = __float2bfloat16_rn(w[i]);
    }
  }
}

struct TileF32 {
  int bm, bn;
};
constexpr TileF32 kTiles[] = {{128, 64}, {64, 64}, {128, 128}, {64, 128}};

int sms() {
  return device_sms();
}

}  // namespace

int conv_f32_tile_count() { return (int)(sizeof(kTiles) / sizeof(kTiles[0])); }

int conv_f32_launch(const ConvShape& c, const float* in, const float* w, const float* ss,
                    float* out, int tile, cudaStream_t s) {
  const int M = c.Ho * c.Wo;
  if (tile < 0) tile = tuned_tile(PP_F32, c);
  if (tile < 0) {
    // fewest waves of (CTAs per SM ~ 2) first, then larger tiles
    int best = 0;
    double best_cost = 1e30;
    for (int i = 0; i < conv_f32_tile_count(); ++i) {
      if (c.cout % kTiles[i].bn) continue;
      const double ctas = (double)((M + kTiles[i].bm - 1) / kTiles[i].bm) * (c.cout / kTiles[i].bn) * c.batch;
      const double per_wave = (double)sms() * (kTiles[i].bm * kTiles[i].bn >= 8192 ? 2 : 4);
      const double waves = ceil(ctas / per_wave);
      const double cost = waves * kTiles[i].bm * kTiles[i].bn / (kTiles[i].bm * kTiles[i].bn >= 8192 ? 2.0 : 4.0);
      if (cost < best_cost - 1e-9) { best_cost = cost; best = i; }
    }
    tile = best;
  }
  if (tile >= conv_f32_tile_count() || c.cout % kTiles[tile].bn)
    return fail(PP_EINVAL, "conv f32: tile %d unsupported for cout %d", tile, c.cout);
  const int bm = kTiles[tile].bm, bn = kTiles[tile].bn;
  const dim3 grid((M + bm - 1) / bm, c.cout / bn, c.batch);
  cudaError_t e;
  switch (tile) {
    case 0: e = launch_pdl(conv3x3_f32<128, 64, 4>, grid, dim3(256), 0, s, c, in, w, ss, out); break;
    case 1: e = launch_pdl(conv3x3_f32<64, 64, 4>, grid, dim3(128), 0, s, c, in, w, ss, out); break;
    case 2: e = launch_pdl(conv3x3_f32<128, 128, 8>, grid, dim3(256), 0, s, c, in, w, ss, out); break;
    default: e = launch_pdl(conv3x3_f32<64, 128, 8>, grid, dim3(128), 0, s, c, in, w, ss, out); break;
  }
  return cuda_status(e, "conv f32 launch");
}

int conv_pack_launch(const float* w_oihw, int cin, int cout, int dtype, void* dst, cudaStream_t s) {
  const int total = cout * cin * 9;
  pack_weights<<<(total + 255) / 256, 256, 0, s>>>(w_oihw, cin, cout, dtype, dst);
  return cuda_status(cudaGetLastError(), "pack weights launch");
}

}  // namespace pp
