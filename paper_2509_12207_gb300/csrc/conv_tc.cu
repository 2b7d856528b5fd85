// BF16 conv3x3 + folded BN + ReLU on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// Implicit GEMM over padded NHWC bf16:  M = output pixels, N = cout, K = 9*cin in (ky, kx, ci)
// order.  One CTA computes a 128 x BN output tile whose 128 pixels form a bh x bw box of one
// frame (bh*bw = 128), so one tiled TMA copy fetches the whole A operand of a (tap, 64-channel)
// K block: the zero border of the padded layout supplies the halo, and stride 2 is expressed
// by viewing each padded row/column pair as (index/2, index%2) in a 5-D tensor map.  The
// weights ([cout][9*cin] bf16) come in by a 2-D tensor map.  Both land in shared memory in the
// 128-byte-swizzled K-major layout that tcgen05.mma reads directly.
//
// Warp roles (128 threads):  warp 0 lane 0 issues TMA into a STAGES-deep ring (full/empty
// mbarriers); warp 1 lane 0 issues tcgen05.mma (M=128, N=BN, K=16) accumulating in TMEM and
// frees each stage with tcgen05.commit; then all four warps read the accumulator back with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows), apply BN + ReLU in FP32, round
// to bf16 and store.  Every mbarrier wait is bounded (%globaltimer); on timeout the kernel sets
// the library's device error word, skips its stores, frees its TMEM and returns.
#include "pp_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

namespace pp {

__device__ unsigned g_tc_error;  // sticky device error word of the tensor-core conv

namespace {

constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s per wait
constexpr int kBM = 128;
constexpr int kBK = 64;                              // channels per K block (128 bytes)
constexpr uint32_t kABytes = kBM * kBK * 2;          // 16 KiB

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned tc_error_now() {
  return *reinterpret_cast<volatile unsigned*>(&g_tc_error);
}
// Bounded wait; false on timeout (after recording `code` in the device error word) or once
// another CTA has recorded an error, so that one failure does not cost a timeout per CTA.  The
// barrier is polled in a tight loop; the clock and the error word (a global load) are looked at
// only every 256 polls, so a completed phase is seen within one poll.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned code) {
  if (mbar_try(bar, parity)) return true;
  uint64_t t0 = 0;
  for (uint32_t n = 1;; ++n) {
    if (mbar_try(bar, parity)) return true;
    if ((n & 255u) == 0u) {
      if (tc_error_now() != 0u) return false;
      const uint64_t t = now_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kTimeoutNs) {
        atomicOr(&g_tc_error, code);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_3d(void* dst, const CUtensorMap* m, uint64_t* bar, int c0,
                                       int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tma_5d(void* dst, const CUtensorMap* m, uint64_t* bar, int c0,
                                       int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* m, uint64_t* bar, int c0,
                                       int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// Named barrier `id` over `n` threads that also ANDs a predicate across them.
__device__ __forceinline__ bool bar_and(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// Stores 32 rows of 128 bytes, row l held by lane l as v[0..7], through a 4 KiB per-warp shared
// buffer, so that every store instruction writes four whole 128-byte lines (lane l writes bytes
// 16 (l % 8) .. of row 4 i + l / 8) instead of 32 lines by 16 bytes.  dst_row: this lane's
// row destination in global memory, or NULL to skip the row.  The buffer is XOR-swizzled by
// row, so both the row writes and the transposed reads are free of bank conflicts.
__device__ __forceinline__ void warp_rows_store(uint4* wbuf, const uint4 (&v)[8], char* dst_row, int lane) {
#pragma unroll
  for (int j = 0; j < 8; ++j) wbuf[lane * 8 + (j ^ (lane & 7))] = v[j];
  __syncwarp();
  const unsigned long long mine = reinterpret_cast<unsigned long long>(dst_row);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = 4 * i + (lane >> 3), col = lane & 7;
    const unsigned long long d = __shfl_sync(0xffffffffu, mine, row);
    const uint4 x = wbuf[row * 8 + (col ^ (row & 7))];
    if (d) *reinterpret_cast<uint4*>(d + (unsigned long long)col * 16) = x;
  }
  __syncwarp();
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)(16u >> 4) << 16;             // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024u >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D f32, A/B bf16, both K-major, M=128, N=BN.
template <int BN>
__device__ __forceinline__ uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive TMEM columns of this warp's 32 lanes into v[0..31]; no wait (see tmem_wait).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  ConvShape c;
  int bh, bw, tiles_x, tiles_y;
  const float* ss;
  __nv_bfloat16* out;
};

template <int BN, int STAGES, bool S2>
__global__ void __launch_bounds__(128, 1)
conv3x3_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           TcArgs args) {
  constexpr uint32_t kBBytes = BN * kBK * 2;
  constexpr uint32_t kCols = BN < 32 ? 32 : BN;  // power of two >= 32 (BN is 64/128/256)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * kBBytes);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  float* s_ss = reinterpret_cast<float*>(tmem_slot + 4);  // [2][BN]

  const ConvShape& c = args.c;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = blockIdx.x;
  const int tx = bx % args.tiles_x;
  const int ty = (bx / args.tiles_x) % args.tiles_y;
  const int b = bx / (args.tiles_x * args.tiles_y);
  const int n0 = blockIdx.y * BN;
  const int oy0 = ty * args.bh, ox0 = tx * args.bw;

  // a previous failure (sticky until the host clears it) turns every later CTA into a no-op
  __shared__ unsigned s_abort;
  if (threadIdx.x == 0) s_abort = tc_error_now();
  __syncthreads();
  if (s_abort != 0u) return;
  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < STAGES; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], 1);
      }
      mbar_init(accum, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    }
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_trigger();  // after this CTA's TMEM allocation: the next kernel may launch
  pdl_wait();     // the previous kernel's outputs are complete and visible
  for (int i = threadIdx.x; i < BN; i += blockDim.x) {
    s_ss[i] = args.ss[n0 + i];
    s_ss[BN + i] = args.ss[c.cout + n0 + i];
  }
  __syncthreads();

  const int kchunks = c.cin / kBK;
  const int KB = 9 * kchunks;
  const int Hp2 = (c.H + 2) / 2;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, 1u)) break;
      const int tap = kb / kchunks, cc = kb % kchunks;
      const int ky = tap / 3, kx = tap % 3;
      mbar_expect_tx(&full[s], kABytes + kBBytes);
      if (S2)
        tma_5d(sA + s * kABytes, &tmA, &full[s], cc * kBK, kx & 1, ox0 + (kx >> 1), ky & 1,
               b * Hp2 + oy0 + (ky >> 1));
      else
        tma_3d(sA + s * kABytes, &tmA, &full[s], cc * kBK, ox0 + kx, b * (c.H + 2) + oy0 + ky);
      tma_2d(sB + s * kBBytes, &tmB, &full[s], tap * c.cin + cc * kBK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id = idesc<BN>();
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, 2u)) break;
      tc_fence_after();
      const uint8_t* a = sA + s * kABytes;
      const uint8_t* bb = sB + s * kBBytes;
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k)
        mma_bf16(tmem, sdesc(a + k * 32), sdesc(bb + k * 32), id, (kb | k) != 0);
      mma_commit(&empty[s]);
    }
    mma_commit(accum);
  }
  __syncwarp();

  // epilogue: TMEM -> registers -> BN + ReLU -> bf16 -> global
  const bool ok = mbar_wait(accum, 0u, 4u);
  __syncwarp();
  tc_fence_after();
  const int r = warp * 32 + lane;
  const int oy = oy0 + r / args.bw, ox = ox0 + r % args.bw;
  const bool store = ok && oy < c.Ho && ox < c.Wo;
  char* fdst = c.frame_dst ? c.frame_dst[b] : nullptr;  // the frame's result slot, if any
  __nv_bfloat16* o = fdst ? reinterpret_cast<__nv_bfloat16*>(fdst + c.frame_off) +
                                ((size_t)(oy + 1) * (c.Wo + 2) + ox + 1) * c.cout + n0
                          : args.out + (((size_t)b * (c.Ho + 2) + oy + 1) * (c.Wo + 2) + ox + 1) * c.cout + n0;
#pragma unroll 1
  for (int j = 0; j < BN / 16; ++j) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 16), v);
    if (store) {
      uint32_t pk[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = j * 16 + 2 * i;
        const float a0 = fmaxf(fmaf(v[2 * i], s_ss[n], s_ss[BN + n]), 0.f);
        const float a1 = fmaxf(fmaf(v[2 * i + 1], s_ss[n + 1], s_ss[BN + n + 1]), 0.f);
        __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
        pk[i] = *reinterpret_cast<uint32_t*>(&h);
      }
      uint4* dst = reinterpret_cast<uint4*>(o + j * 16);
      dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
}

// ---------------------------------------------------------------------------- FP32 via 3xTF32
//
// The same implicit GEMM for FP32 activations, on the tensor cores with FP32-level accuracy:
// every operand x is split into hi = x with its 13 low mantissa bits cleared (exactly a TF32
// value) and lo = x - hi (exact in FP32, < 2^-10 |x|), and the product is accumulated as
// hi*hi' + hi*lo' + lo*hi' (the dropped lo*lo' term is < 2^-20 of the product).  The tensor
// core reads a TF32 operand from an FP32 word by dropping those 13 bits, so an FP32 tensor
// already is its own hi part.  Weights come pre-split from packing ([2][cout][9*cin]: hi plane,
// lo plane); activations travel as split FP32, two planes [2][B][H+2][W+2][C] (the values, then
// their remainders lo), written by the producer of the tensor (the scatter, or the previous
// conv's epilogue, which has the FP32 value in a register anyway), so the A remainder arrives by
// TMA like the A tile itself.  The tensor core's FP32 accumulation is not round-to-nearest, so
// long accumulation chains drift: the MMAs accumulate only `fold` K blocks into one TMEM buffer,
// and reducer warps add each finished buffer into FP32 registers (round to nearest).

// x - (x with its 13 low mantissa bits cleared): exact in FP32 (the cleared bits times the
// exponent's unit); what a TF32 read of x drops.
__device__ __forceinline__ float tf32_remainder(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}
__device__ __forceinline__ float4 tf32_remainder4(float4 v) {
  return make_float4(tf32_remainder(v.x), tf32_remainder(v.y), tf32_remainder(v.z), tf32_remainder(v.w));
}

template <int BN>
__device__ __forceinline__ uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

// ---------------------------------------------------------------------------- persistent
//
// Persistent form of both tensor-core convs: one CTA per SM walks the output tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... (N tile innermost, so CTAs sharing an A tile run
// side by side and the second read hits L2).  The TMA ring and the MMA thread run over the
// concatenated K blocks of all the CTA's tiles without draining, and
// accumulation goes to TMEM buffers in turn (four where 512 columns hold them, else two):
// while the reducer warps read one buffer (and, at the end of a tile, apply BN + ReLU and
// store), the MMAs fill the next.  For BF16 a buffer
// holds a whole tile's accumulation and a ring stage carries KPS K blocks (p_kps: 2-4, so
// 8-16 MMAs per handshake); for 3xTF32 a buffer holds `fold` K blocks, which the reducers add into FP32
// registers, and each K step is two MMAs: A_hi x [B_hi | B_lo] (N = 2 BN, the two products land
// side by side in TMEM) and A_lo x B_hi (N = BN, into the first half); the reducers sum the
// halves.  Loop counters advance incrementally (no division in the steady state) and shared
// memory descriptors are built once and offset by addition.  192 threads: warp 0 TMA, warp 1
// TMEM allocation + MMA, warps 2-5 reduce and store (TMEM lane quarters 2, 3, 0, 1).
// HALO (3xTF32, BN 64, stride 1): a tile is 128 consecutive pixels of the output laid out over
// the padded width W + 2 (the two padding columns of each row are computed and not stored), so
// that for every tap the 128 input pixels are consecutive too: input pixel = output pixel +
// ky (W + 2) + kx in the flattened padded image.  A ring stage holds 130 consecutive input
// pixels (32 channels, value and remainder) and the weights of the three kx taps, and the MMAs
// of tap kx read the row range from pixel kx on (a K-major 128-byte-swizzled operand may start
// at any 128-byte row of its buffer), so one load serves three taps: 82 KiB per three K blocks
// instead of 144 KiB, at any width.  A stage is one accumulation group (fold 3), in the order
// ky, channel chunk, kx.
// HALO with NBS > 0 (split rings): A and B have rings of their own -- STAGES A slots, each one
// (ky, chunk) input range (34 KiB), and NBS B slots, each one tap's weights (value and
// remainder: 16 KiB at BN 64, 32 KiB at BN 128); the MMAs of a group wait for the A slot once and
// for each tap's B slot in turn, and free each B slot after its tap and the A slot after the
// third.  With BN 128 this is what makes three taps fit at all (130 KiB of TMA per three K
// blocks instead of 192 KiB for the plain BN 128 tile); with either BN a deeper ring than the
// unified stage allows: a stage is held from its TMA issue until its MMAs complete, so the
// ring's depth, not its bytes, sets how much of that round trip is hidden.
// HALO with KXN (kx folded into N; BN 64, unified stages): the three kx taps' weights are
// stacked along N (B = 192 rows: the value taps kx = 0, 1, 2, then the remainder taps), and
// the A operand is the stage's input range from its first pixel on, unshifted.  A K step is
// three MMAs of N = 192 -- A_hi x B_hi, A_hi x B_lo, A_lo x B_hi, all into one 192-column
// accumulator -- so that accumulator row j holds, for each tap kx, the products of input pixel
// p0 + j with that tap's weights; output pixel p0 + i takes tap kx from row i + kx.  A tile is
// 126 output pixels (rows 126 and 127 only feed the rows before them).  Per K step the MMAs
// read 30 KiB of operands for 288 tensor cycles (106 B per clock) where the shifted-A halo
// tile reads 14 KiB per 96 (149 B per clock, above the ~128 B per clock that shared memory
// serves): the N = 64 MMAs of the shifted form run at 0.66 of the tensor rate, N = 192 at the
// full rate.  The reducer warps of a lane quarter split the output channels (0-31 and 32-63),
// each holding its channels' columns of all three taps; at the tile's end a warp adds tap 1
// from the next row and tap 2 from the row after (warp shuffles; the next lane quarter's first
// two rows through shared memory).

struct PArgs {
  ConvShape c;
  int bh, bw, tiles_x, tiles_y, tiles_n, total, fold;
  // GEMM shape and epilogue mapping (3x3 conv: taps 9, up 1, co_blk = out_c = cout, relu 1).
  // taps 1 = pointwise (1x1) GEMM over the centre tap.  up > 1: a transposed conv with kernel =
  // stride = up, GEMM column n = (dy * up + dx) * co_blk + co written to output pixel
  // (up * y + dy, up * x + dx), channel out_coff + co of an out_c-channel [Hout+2][Wout+2] map.
  int taps, up, co_blk, out_c, out_coff, Hout, Wout, relu;
  size_t plane;  // 3xTF32: elements from the output's value plane to its remainder plane
  const float* ss;
  void* out;
  int sk;         // 3xTF32 stream-K partition (else whole tiles per CTA)
  float* ws;      // stream-K: [2 * gridDim.x][128][BN] partial tiles
  unsigned* sem;  // stream-K: [total] arrival counters, zero between launches
};

// Reducer warps of the persistent conv: eight for the BN 64 halo tiles (two per TMEM lane
// quarter, each owning half of the tile's columns, so that the accumulation groups are drained
// and the last tile's epilogue is written by two warps per scheduler), four otherwise (where
// eight 4 KiB transposing buffers would not fit beside the rings).
template <int MODE, int BN, bool HALO>
__host__ __device__ constexpr int p_red_warps() {
  return MODE == 1 && HALO && BN == 64 ? 8 : 4;
}
template <int MODE, int BN, bool HALO>
__host__ __device__ constexpr int p_threads() {
  return 64 + 32 * p_red_warps<MODE, BN, HALO>();
}

template <int MODE, int BN, int STAGES, int KPS, bool S2, bool SK, bool HALO = false, int NBS = 0,
          bool KXN = false>
__global__ void __launch_bounds__(p_threads<MODE, BN, HALO>(), 1)
conv3x3_tcp(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
            const __grid_constant__ CUtensorMap tmB, PArgs args) {
  constexpr int BK = MODE == 1 ? 32 : 64;                  // channels per K block (128 B rows)
  constexpr uint32_t kA = 128 * 128;                       // A tile bytes of one K block
  constexpr uint32_t kB = BN * 128;                        // B tile bytes of one K block, one plane
  constexpr uint32_t kAK = MODE == 1 ? 2 * kA : kA;        // per K block: A (+ lo)
  constexpr uint32_t kBK = MODE == 1 ? 2 * kB : kB;        // per K block: B (+ lo plane)
  constexpr uint32_t kHaloRow = (KXN ? 128 : 130) * 128;   // HALO: one padded input row, one plane
  constexpr uint32_t kHaloA = (kHaloRow + 1023) / 1024 * 1024;
  static_assert(!HALO || (MODE == 1 && (BN == 64 || BN == 128) && !S2 && KPS == 3),
                "halo rows: 3xTF32, BN 64 or 128, stride 1");
  static_assert(NBS == 0 || HALO, "split rings: halo tiles only");
  static_assert(!HALO || BN == 64 || NBS > 0, "a unified halo stage holds three taps of BN 64 only");
  static_assert(!KXN || (HALO && BN == 64 && NBS == 0 && !SK), "kx in N: the unified BN 64 halo tile");
  constexpr bool kSplit = HALO && NBS > 0;                 // A and B in separate rings
  constexpr int NB = kSplit ? NBS : 0;                     // B ring slots (one tap each)
  constexpr uint32_t kStageA = HALO ? 2 * kHaloA : KPS * kAK;
  constexpr uint32_t kStageB = KPS * kBK;
  constexpr uint32_t kBRegion = kSplit ? (uint32_t)NB * kBK : (uint32_t)STAGES * kStageB;
  // unified halo stage: where tap kx's value and remainder weights go (KXN: the three value
  // taps stacked, then the three remainder taps)
  auto b_hi = [](int kx) -> uint32_t { return KXN ? (uint32_t)kx * kB : (uint32_t)kx * kBK; };
  auto b_lo = [](int kx) -> uint32_t { return KXN ? 3u * kB + (uint32_t)kx * kB : (uint32_t)kx * kBK + kB; };
  constexpr int NACC = KXN ? 3 * BN : MODE == 1 ? 2 * BN : BN;  // TMEM columns per accumulator buffer
  // accumulator buffers in TMEM (512 columns): four where they fit, so that the MMAs can run
  // up to three groups ahead of the reducers while they store a finished tile
  constexpr int NBUF = 512 / NACC >= 4 ? 4 : 2;
  constexpr uint32_t kCols = KXN ? 512 : NBUF * NACC;      // (an allocation is a power of two)
  constexpr int kRed0 = 2;                                 // first reducer warp
  constexpr int kRW = p_red_warps<MODE, BN, HALO>();       // reducer warps
  constexpr int kRT = 32 * kRW;                            // reducer threads
  constexpr int BNW = BN * 4 / kRW;                        // columns of the tile per reducer warp
  extern __shared__ uint8_t smem_raw[];
  __shared__ unsigned s_abort;
  __shared__ unsigned s_arrived;  // stream-K: arrivals at the current shared tile before this CTA
  if (threadIdx.x == 0) s_abort = tc_error_now();
  __syncthreads();
  if (s_abort != 0u) return;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + STAGES * kStageA;
  uint8_t* sO = sB + kBRegion;                             // epilogue: 4 KiB transposing buffer per reducer warp
  constexpr uint32_t kStageO = (uint32_t)kRW * 4096u;
  uint64_t* full = reinterpret_cast<uint64_t*>(sO + kStageO);  // (split rings: the A ring's)
  uint64_t* empty = full + STAGES;
  uint64_t* kdone = empty + STAGES;
  uint64_t* kfree = kdone + NBUF;
  uint64_t* fullB = kfree + NBUF;                          // split rings: the B ring's
  uint64_t* emptyB = fullB + NB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(emptyB + NB);
  float* s_scale = reinterpret_cast<float*>(tmem_slot + 4);  // [cout] folded BN scale
  float* s_shift = s_scale + args.co_blk;                    // [co_blk] folded BN shift (or bias)

  const ConvShape& c = args.c;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kchunks = c.cin / BK;
  // work units of one tile: K blocks, or for the halo tiles accumulation groups (one ky and one
  // channel chunk, the three kx taps of one loaded input range), ky outer, chunk inner
  const int KB = HALO ? 3 * kchunks : args.taps * kchunks;
  const int fold = MODE == 1 ? args.fold : KB;
  const int Hp2 = (c.H + 2) / 2;

  const float lo_clamp = args.relu ? 0.f : __uint_as_float(0xff800000u);  // ReLU, or none (-inf: bias-only epilogue)
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < NBUF; ++i) {
      mbar_init(&kdone[i], 1);
      mbar_init(&kfree[i], kRT);
    }
    for (int i = 0; i < NB; ++i) {
      mbar_init(&fullB[i], 1);
      mbar_init(&emptyB[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    if (MODE == 1) asm volatile("prefetch.tensormap [%0];" ::"l"(&tmAlo) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto decode = [&](int t, int& b, int& oy0, int& ox0, int& n0) {
    const int nt = t % args.tiles_n;
    const int r = t / args.tiles_n;
    const int tx = r % args.tiles_x;
    const int ty = (r / args.tiles_x) % args.tiles_y;
    b = r / (args.tiles_x * args.tiles_y);
    oy0 = ty * args.bh;
    ox0 = tx * args.bw;
    n0 = nt * BN;
  };
  // Work pieces of this CTA, i = 0, 1, ...: (tile t, K blocks [k0, k1)).  Plain: whole tiles
  // t = blockIdx.x + i * gridDim.x.  Stream-K: the K blocks of all tiles laid end to end and cut
  // into gridDim.x equal ranges, one per CTA; a tile cut between CTAs is finished by the CTA
  // that completes it last (partial sums through args.ws, arrivals counted in args.sem).
  const long W = (long)args.total * KB;
  auto cta_start = [&](long cta) -> long { return cta * W / gridDim.x; };
  const long r_lo = SK ? cta_start(blockIdx.x) : 0, r_hi = SK ? cta_start(blockIdx.x + 1) : 0;
  auto piece = [&](int i, int& t, int& k0, int& k1) -> bool {
    if (!SK) {
      t = blockIdx.x + i * gridDim.x;
      k0 = 0;
      k1 = KB;
      return t < args.total;
    }
    t = (int)(r_lo / KB) + i;
    const long b0 = (long)t * KB;
    k0 = (int)(r_lo > b0 ? r_lo - b0 : 0);
    k1 = (int)(r_hi < b0 + KB ? r_hi - b0 : KB);
    return b0 < r_hi && k1 > k0;
  };

  // Weights and folded BN written before the previous kernel started (a release unit's,
  // packed at creation) are fetched while that kernel drains: the scale/shift table, and for
  // the halo tiles the weight taps of the first stages (B slots) of this CTA's first piece, so
  // that only the input rows wait for the dependent-launch release.  npre: stages (unified
  // halo stages) or B slots (split rings) already loaded that way.
  int npre = 0;
  if (c.static_w) {
    for (int i = threadIdx.x; i < args.co_blk; i += blockDim.x) {
      s_scale[i] = args.ss[i];
      s_shift[i] = args.ss[args.co_blk + i];
    }
    int t, k0, k1;
    if (HALO && piece(0, t, k0, k1)) {
      int b, oy0, ox0, n0;
      decode(t, b, oy0, ox0, n0);
      npre = kSplit ? (NB < 3 * (k1 - k0) ? NB : 3 * (k1 - k0)) : (STAGES < k1 - k0 ? STAGES : k1 - k0);
      if (warp == 0 && lane == 0) {
        for (int f = 0; f < npre; ++f) {
          const int gi = k0 + (kSplit ? f / 3 : f);
          const int ky = gi / kchunks, cc = gi % kchunks;
          for (int kx = kSplit ? f % 3 : 0; kx < (kSplit ? f % 3 + 1 : 3); ++kx) {
            uint64_t* bar = kSplit ? &fullB[f] : &full[f];
            uint8_t* bb = kSplit ? sB + f * kBK : sB + f * kStageB;
            if (kSplit) mbar_expect_tx(bar, kBK);
            else if (kx == 0) mbar_expect_tx(bar, 2u * kHaloRow + 3u * kBK);
            const int kk = (ky * 3 + kx) * c.cin + cc * BK;
            tma_3d(bb + (kSplit ? 0u : b_hi(kx)), &tmB, bar, kk, n0, 0);
            tma_3d(bb + (kSplit ? kB : b_lo(kx)), &tmB, bar, kk, n0, 1);
          }
        }
      }
    }
  }
  pdl_wait();     // the previous kernel's outputs are complete and visible
  if (!c.static_w) {
    for (int i = threadIdx.x; i < args.co_blk; i += blockDim.x) {
      s_scale[i] = args.ss[i];
      s_shift[i] = args.ss[args.co_blk + i];
    }
  }
  __syncthreads();

  if (warp == 0) {
    if (kSplit && lane == 0) {
      int sa = 0, sb = 0, fb = 0;  // fb: B fills so far
      uint32_t pa = 0, pb = 0;
      bool ok = true;
      int t, k0, k1;
      for (int i = 0; ok && piece(i, t, k0, k1); ++i) {
        int b, oy0, ox0, n0;
        decode(t, b, oy0, ox0, n0);
        for (int gi = k0; gi < k1 && ok; ++gi) {
          const int ky = gi / kchunks, cc = gi % kchunks;
          if (!mbar_wait(&empty[sa], pa ^ 1u, 1u)) { ok = false; break; }
          mbar_expect_tx(&full[sa], 2u * kHaloRow);
          uint8_t* a = sA + sa * kStageA;
          // flattened padded input pixels pix .. pix + 129 (ox0: the tile's first output pixel)
          const int pix = (b * (c.H + 2) + ky) * (c.W + 2) + ox0;
          tma_2d(a, &tmA, &full[sa], cc * BK, pix);
          tma_2d(a + kHaloA, &tmAlo, &full[sa], cc * BK, pix);
          if (++sa == STAGES) { sa = 0; pa ^= 1u; }
          for (int kx = 0; kx < 3; ++kx) {
            if (fb++ >= npre) {  // (the first npre were loaded before the dependent-launch wait)
              if (!mbar_wait(&emptyB[sb], pb ^ 1u, 1u)) { ok = false; break; }
              mbar_expect_tx(&fullB[sb], kBK);
              uint8_t* bb = sB + sb * kBK;
              const int kk = (ky * 3 + kx) * c.cin + cc * BK;
              tma_3d(bb, &tmB, &fullB[sb], kk, n0, 0);
              tma_3d(bb + kB, &tmB, &fullB[sb], kk, n0, 1);
            }
            if (++sb == NB) { sb = 0; pb ^= 1u; }
          }
        }
      }
    } else if (HALO && lane == 0) {
      int s = 0, fs = 0;  // fs: stage fills so far
      uint32_t ph = 0;
      bool ok = true;
      int t, k0, k1;
      for (int i = 0; ok && piece(i, t, k0, k1); ++i) {
        int b, oy0, ox0, n0;
        decode(t, b, oy0, ox0, n0);
        for (int gi = k0; gi < k1 && ok; ++gi) {
          const int ky = gi / kchunks, cc = gi % kchunks;
          // the first npre stages have their weights (and the byte count) in already
          const bool pre = fs++ < npre;
          if (!mbar_wait(&empty[s], ph ^ 1u, 1u)) { ok = false; break; }
          if (!pre) mbar_expect_tx(&full[s], 2u * kHaloRow + 3u * kBK);
          uint8_t* a = sA + s * kStageA;
          // flattened padded input pixels pix .. pix + 129 (ox0: the tile's first output pixel)
          const int pix = (b * (c.H + 2) + ky) * (c.W + 2) + ox0;
          tma_2d(a, &tmA, &full[s], cc * BK, pix);
          tma_2d(a + kHaloA, &tmAlo, &full[s], cc * BK, pix);
          for (int kx = 0; kx < 3 && !pre; ++kx) {
            uint8_t* bb = sB + s * kStageB;
            const int kk = (ky * 3 + kx) * c.cin + cc * BK;
            tma_3d(bb + b_hi(kx), &tmB, &full[s], kk, n0, 0);
            tma_3d(bb + b_lo(kx), &tmB, &full[s], kk, n0, 1);
          }
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
      }
    } else if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      int t, k0, k1;
      for (int i = 0; ok && piece(i, t, k0, k1); ++i) {
        int b, oy0, ox0, n0;
        decode(t, b, oy0, ox0, n0);
        // channel chunk, tap, K offset of the next K block
        // pointwise GEMMs read the centre tap (the unpadded pixel) only
        int cc = k0 % kchunks, kk = k0 * BK;
        int kx = args.taps == 9 ? (k0 / kchunks) % 3 : 1, ky = args.taps == 9 ? k0 / kchunks / 3 : 1;
        for (int kb0 = k0; kb0 < k1; kb0 += KPS) {
          const int nk = k1 - kb0 < KPS ? k1 - kb0 : KPS;
          if (!mbar_wait(&empty[s], ph ^ 1u, 1u)) { ok = false; break; }
          mbar_expect_tx(&full[s], (uint32_t)nk * (kAK + kBK));
          for (int j = 0; j < nk; ++j) {
            uint8_t* a = sA + s * kStageA + j * kAK;
            if (S2) {
              tma_5d(a, &tmA, &full[s], cc * BK, kx & 1, ox0 + (kx >> 1), ky & 1,
                     b * Hp2 + oy0 + (ky >> 1));
              if (MODE == 1)
                tma_5d(a + kA, &tmAlo, &full[s], cc * BK, kx & 1, ox0 + (kx >> 1), ky & 1,
                       b * Hp2 + oy0 + (ky >> 1));
            } else {
              tma_3d(a, &tmA, &full[s], cc * BK, ox0 + kx, b * (c.H + 2) + oy0 + ky);
              if (MODE == 1) tma_3d(a + kA, &tmAlo, &full[s], cc * BK, ox0 + kx, b * (c.H + 2) + oy0 + ky);
            }
            uint8_t* bb = sB + s * kStageB + j * kBK;
            if (MODE == 1) {
              tma_3d(bb, &tmB, &full[s], kk, n0, 0);
              tma_3d(bb + kB, &tmB, &full[s], kk, n0, 1);
            } else {
              tma_2d(bb, &tmB, &full[s], kk, n0);
            }
            kk += BK;
            if (++cc == kchunks) {
              cc = 0;
              if (args.taps == 9 && ++kx == 3) { kx = 0; ++ky; }
            }
          }
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    if (kSplit && lane == 0) {
      const uint32_t id = idesc_tf32<2 * BN>();
      const uint32_t id2 = idesc_tf32<BN>();
      const uint64_t dA0 = sdesc(sA), dB0 = sdesc(sB);
      int sa = 0, sb = 0, gg = 0;
      uint32_t pa = 0, pb = 0;
      bool ok = true;
      int t, k0, k1;
      for (int i = 0; ok && piece(i, t, k0, k1); ++i) {
        for (int g = k0; g < k1; ++g) {  // one A slot = one accumulation group
          const int buf = gg & (NBUF - 1);
          if (gg >= NBUF && !mbar_wait(&kfree[buf], (uint32_t)(gg / NBUF - 1) & 1u, 16u)) { ok = false; break; }
          if (!mbar_wait(&full[sa], pa, 2u)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * NACC);
          const uint64_t da = dA0 + ((uint64_t)(sa * kStageA) >> 4);
          for (int kx = 0; kx < 3; ++kx) {
            if (!mbar_wait(&fullB[sb], pb, 2u)) { ok = false; break; }
            tc_fence_after();
            const uint64_t db = dB0 + ((uint64_t)(sb * kBK) >> 4);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              // tap kx: the row from pixel kx on; K step k: 8 channels = 32 bytes into each row
              const uint64_t a_k = da + (uint64_t)((kx * 128 + k * 32) >> 4);
              const uint64_t b_k = db + (uint64_t)((k * 32) >> 4);
              mma_tf32(d, a_k, b_k, id, (kx == 0 && k == 0) ? 0u : 1u);     // A_hi x [B_hi|B_lo]
              mma_tf32(d, a_k + (kHaloA >> 4), b_k, id2, 1u);               // A_lo x B_hi
            }
            mma_commit(&emptyB[sb]);
            if (++sb == NB) { sb = 0; pb ^= 1u; }
          }
          if (!ok) break;
          mma_commit(&empty[sa]);
          mma_commit(&kdone[buf]);
          ++gg;
          if (++sa == STAGES) { sa = 0; pa ^= 1u; }
        }
      }
    } else if (HALO && lane == 0) {
      const uint32_t id = idesc_tf32<2 * BN>();
      const uint32_t id2 = idesc_tf32<BN>();
      const uint64_t dA0 = sdesc(sA), dB0 = sdesc(sB);
      int s = 0, gg = 0;
      uint32_t ph = 0;
      bool ok = true;
      int t, k0, k1;
      for (int i = 0; ok && piece(i, t, k0, k1); ++i) {
        for (int g = k0; g < k1; ++g) {  // one stage = one accumulation group
          // KXN: args.fold groups per accumulation buffer (12 MMAs each into one column block;
          // two groups give a buffer the 24 accumulations the shifted-A tile gives one group),
          // dividing the reducers' TMEM reads; a tile's last buffer may hold fewer
          const int gl = KXN ? (g - k0) % args.fold : 0;
          const bool fresh = gl == 0;
          const bool close = !KXN || gl == args.fold - 1 || g + 1 == k1;
          const int buf = gg & (NBUF - 1);
          if (fresh && gg >= NBUF && !mbar_wait(&kfree[buf], (uint32_t)(gg / NBUF - 1) & 1u, 16u)) { ok = false; break; }
          if (!mbar_wait(&full[s], ph, 2u)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * NACC);
          const uint64_t da = dA0 + ((uint64_t)(s * kStageA) >> 4);
          const uint64_t db = dB0 + ((uint64_t)(s * kStageB) >> 4);
          if (KXN) {
            const uint32_t id3 = idesc_tf32<3 * BN>();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              // K step k: 8 channels = 32 bytes into each row; the three taps side by side in N
              const uint64_t a_k = da + (uint64_t)((k * 32) >> 4);
              const uint64_t bh = db + (uint64_t)((b_hi(0) + k * 32) >> 4);
              const uint64_t bl = db + (uint64_t)((b_lo(0) + k * 32) >> 4);
              mma_tf32(d, a_k, bh, id3, (fresh && k == 0) ? 0u : 1u);      // A_hi x B_hi
              mma_tf32(d, a_k, bl, id3, 1u);                               // A_hi x B_lo
              mma_tf32(d, a_k + (kHaloA >> 4), bh, id3, 1u);               // A_lo x B_hi
            }
          } else {
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                // tap kx: the row from pixel kx on; K step k: 8 channels = 32 bytes into each row
                const uint64_t a_k = da + (uint64_t)((kx * 128 + k * 32) >> 4);
                const uint64_t b_k = db + (uint64_t)((b_hi(kx) + k * 32) >> 4);
                mma_tf32(d, a_k, b_k, id, (kx == 0 && k == 0) ? 0u : 1u);     // A_hi x [B_hi|B_lo]
                mma_tf32(d, a_k + (kHaloA >> 4), b_k, id2, 1u);               // A_lo x B_hi
              }
            }
          }
          mma_commit(&empty[s]);
          if (close) {
            mma_commit(&kdone[buf]);
            ++gg;
          }
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
      }
    } else if (lane == 0) {
      const uint32_t id = MODE == 1 ? idesc_tf32<2 * BN>() : idesc<BN>();
      const uint32_t id2 = idesc_tf32<BN>();
      const uint64_t dA0 = sdesc(sA), dB0 = sdesc(sB);
      int s = 0, gg = 0, inq = 0;  // inq: K blocks already in the current group
      uint32_t ph = 0;
      bool ok = true;
      int t, k0, k1;
      for (int i = 0; ok && piece(i, t, k0, k1); ++i) {
        for (int kb0 = k0; kb0 < k1; kb0 += KPS) {
          const int nk = k1 - kb0 < KPS ? k1 - kb0 : KPS;
          const int buf = gg & (NBUF - 1);
          if (inq == 0 && gg >= NBUF && !mbar_wait(&kfree[buf], (uint32_t)(gg / NBUF - 1) & 1u, 16u)) { ok = false; break; }
          if (!mbar_wait(&full[s], ph, 2u)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * NACC);
          const uint64_t da = dA0 + ((uint64_t)(s * kStageA) >> 4);
          const uint64_t db = dB0 + ((uint64_t)(s * kStageB) >> 4);
#pragma unroll
          for (int j = 0; j < KPS; ++j) {
            if (j < nk) {
              const bool fresh = inq == 0 && j == 0;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const uint64_t a_k = da + (uint64_t)((j * kAK + k * 32) >> 4);
                const uint64_t b_k = db + (uint64_t)((j * kBK + k * 32) >> 4);
                if (MODE == 1) {
                  mma_tf32(d, a_k, b_k, id, (fresh && k == 0) ? 0u : 1u);           // A_hi x [B_hi|B_lo]
                  mma_tf32(d, a_k + (kA >> 4), b_k, id2, 1u);                      // A_lo x B_hi
                } else {
                  mma_bf16(d, a_k, b_k, id, (fresh && k == 0) ? 0u : 1u);
                }
              }
            }
          }
          mma_commit(&empty[s]);
          inq += nk;
          if (inq >= fold || kb0 + nk == k1) {
            mma_commit(&kdone[buf]);
            ++gg;
            inq = 0;
          }
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp >= kRed0) {
    // The next kernel may launch once this CTA's last accumulation has been read out of TMEM:
    // its CTAs then take SMs as ours exit.  Launched earlier, they would sit on the SMs this
    // grid leaves free, waiting for it to end, where kernels of other streams (units of other
    // chains, at other priorities) could run.
    auto last_piece_trigger = [&](int pi) {
      int t2, a2, b2;
      if (warp == kRed0 && lane == 0 && !piece(pi + 1, t2, a2, b2)) pdl_trigger();
    };
    const int q = warp & 3;  // TMEM lane quarter this warp may read
    const int r = q * 32 + lane;
    const int h0 = ((warp - kRed0) >> 2) * BNW;  // first of this warp's BNW columns of the tile
    const bool lead = threadIdx.x == kRed0 * 32;  // one reducer thread for the CTA's arrivals
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    int gg = 0;
    bool ok = true;
    int t, k0, k1;
    for (int pi = 0; ok && piece(pi, t, k0, k1); ++pi) {
      const int gpt = (k1 - k0 + fold - 1) / fold;  // accumulation groups of this piece
      int b, oy0, ox0, n0;
      decode(t, b, oy0, ox0, n0);
      // HALO: output pixel ox0 + r of the image laid out over the padded width
      const int oy = HALO ? (ox0 + r) / (c.W + 2) : oy0 + r / args.bw;
      const int ox = HALO ? (ox0 + r) % (c.W + 2) : ox0 + r % args.bw;
      // (KXN: rows 126 and 127 of the accumulator only feed taps 1 and 2 of the rows before)
      const bool in_range = oy < c.Ho && ox < c.Wo && (!KXN || r < 126);
      // output pixel of this row for this N tile (a transposed conv spreads the N tiles of one
      // input pixel over its up x up output block); first channel written and its BN index
      const int qb = n0 / args.co_blk, nb = n0 - qb * args.co_blk;
      const int opy = args.up * oy + qb / args.up, opx = args.up * ox + qb % args.up;
      const size_t pix = ((size_t)b * (args.Hout + 2) + opy + 1) * (args.Wout + 2) + opx + 1;
      const size_t obase = pix * args.out_c + args.out_coff + nb;
      // a release unit's last layer writes the frame's result slot directly
      char* fdst = c.frame_dst ? c.frame_dst[b] : nullptr;
      const size_t fbase = ((size_t)(opy + 1) * (args.Wout + 2) + opx + 1) * args.out_c + args.out_coff + nb;
      if (MODE == 1) {
        // KXN: this warp's BNW channels of tap kx at acc[kx * BNW ...] (three taps); else one
        constexpr int NT = KXN ? 3 : 1;
        float acc[NT * BNW];
#pragma unroll
        for (int i = 0; i < NT * BNW; ++i) acc[i] = 0.f;
        for (int g = 0; g < gpt; ++g, ++gg) {
          const int buf = gg & (NBUF - 1);
          ok = mbar_wait(&kdone[buf], (uint32_t)(gg / NBUF) & 1u, 4u);
          ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the epilogue shuffles need all lanes
          if (!ok) break;
          tc_fence_after();
          if (KXN) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              uint32_t v[32];
              tmem_ld32_nowait(trow + (uint32_t)(buf * NACC + t * BN + h0), v);
              tmem_wait();
#pragma unroll
              for (int i = 0; i < 32; ++i) acc[t * BNW + i] += __uint_as_float(v[i]);
            }
          } else {
#pragma unroll
            for (int j = 0; j < BNW / 32; ++j) {
              uint32_t v[32], w[32];
              tmem_ld32_nowait(trow + (uint32_t)(buf * NACC + h0 + j * 32), v);
              tmem_ld32_nowait(trow + (uint32_t)(buf * NACC + BN + h0 + j * 32), w);
              tmem_wait();
#pragma unroll
              for (int i = 0; i < 32; ++i) acc[j * 32 + i] += __uint_as_float(v[i]) + __uint_as_float(w[i]);
            }
          }
          tc_fence_before();
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&kfree[buf])) : "memory");
        }
        last_piece_trigger(pi);
        if (KXN) {
          // output row r = tap 0 of row r + tap 1 of row r + 1 + tap 2 of row r + 2: the rows
          // above come by shuffles; lane 31 (tap 1) and lanes 30, 31 (tap 2) take theirs from
          // the first two rows of the next lane quarter, which the warp holding the same
          // channels there publishes in its transposing buffer (quarter 3 has none: its lanes
          // 30 and 31 are rows 126 and 127, not outputs)
          static_assert(!KXN || BNW == 32, "kx in N: 32 channels per reducer warp");
          float* mine = reinterpret_cast<float*>(sO + (warp - kRed0) * 4096);
          if (lane == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) mine[i] = acc[BNW + i];
          }
          if (lane < 2) {
#pragma unroll
            for (int i = 0; i < 32; ++i) mine[32 + 32 * lane + i] = acc[2 * BNW + i];
          }
          ok = bar_and(1, kRT, ok);
          const int hk = (warp - kRed0) >> 2;
          const float* next = reinterpret_cast<const float*>(sO + (4 * hk + ((q + 1 + 4 - kRed0) & 3)) * 4096);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            float t1 = __shfl_down_sync(0xffffffffu, acc[BNW + i], 1);
            float t2 = __shfl_down_sync(0xffffffffu, acc[2 * BNW + i], 2);
            if (q < 3 && lane == 31) t1 = next[i];
            if (q < 3 && lane >= 30) t2 = next[32 + 32 * (lane - 30) + i];
            acc[i] = (acc[i] + t1) + t2;
          }
          bar_and(1, kRT, true);  // the buffers are the stores' transposing buffers next
        }
        if (SK && (k0 > 0 || k1 < KB)) {
          // Part of a tile shared with neighbouring CTAs: publish this partial sum (slot 2c for
          // the piece a CTA starts with, 2c + 1 for the one it ends with), count the arrival,
          // and let the last of the tile's CTAs add the partials in CTA order and finish it.
          // slot layout [slot][BN/4][128 rows] of float4: a warp's stores and loads of one
          // float4 column are 512 contiguous bytes
          const long tb = (long)t * KB;
          const int slot = 2 * blockIdx.x + (r_lo < tb ? 1 : 0);
          float4* mine = reinterpret_cast<float4*>(args.ws) + ((size_t)slot * (BN / 4) + h0 / 4) * 128 + r;
#pragma unroll
          for (int i = 0; i < BNW / 4; ++i)
            mine[i * 128] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
          __threadfence();
          ok = bar_and(1, kRT, ok);
          if (!ok) break;
          if (lead) s_arrived = atomicAdd(&args.sem[t], 1u);
          bar_and(1, kRT, true);
          auto cta_of = [&](long idx) -> int {
            long cc = idx * gridDim.x / W;
            while (cc > 0 && cta_start(cc) > idx) --cc;
            while (cta_start(cc + 1) <= idx) ++cc;
            return (int)cc;
          };
          const int cf = cta_of(tb), cl = cta_of(tb + KB - 1);
          if (s_arrived != (unsigned)(cl - cf)) continue;  // another CTA finishes this tile
          __threadfence();
          // sum every piece's partial (this CTA's too, as stored) in CTA order, one whole piece
          // per pass so that the BN/4 loads of a pass are all in flight together
          for (int cc = cf; cc <= cl; ++cc) {
            const int sl = 2 * cc + (cta_start(cc) < tb ? 1 : 0);
            const float4* src = reinterpret_cast<const float4*>(args.ws) + ((size_t)sl * (BN / 4) + h0 / 4) * 128 + r;
#pragma unroll
            for (int i = 0; i < BNW / 4; ++i) {
              const float4 p = __ldcg(src + i * 128);
              if (cc == cf) {
                acc[4 * i] = p.x; acc[4 * i + 1] = p.y; acc[4 * i + 2] = p.z; acc[4 * i + 3] = p.w;
              } else {
                acc[4 * i] += p.x; acc[4 * i + 1] += p.y; acc[4 * i + 2] += p.z; acc[4 * i + 3] += p.w;
              }
            }
          }
          if (lead) args.sem[t] = 0u;  // counters are zero again for the next launch
        }
        {
          // value plane and remainder plane (split FP32, the next layer's A operand), 32
          // channels (128 B per pixel) at a time through the warp's transposing buffer
          if (!ok) break;
          uint4* wbuf = reinterpret_cast<uint4*>(sO + (warp - kRed0) * 4096);
          float* orow = (fdst ? reinterpret_cast<float*>(fdst + c.frame_off) + fbase
                              : static_cast<float*>(args.out) + obase) + h0;
#pragma unroll
          for (int k = 0; k < BNW / 32; ++k) {
            uint4 hv[8], lv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int n = nb + h0 + 32 * k + 4 * j;
              const float* a = acc + 32 * k + 4 * j;
              float4 u;
              u.x = fmaxf(fmaf(a[0], s_scale[n + 0], s_shift[n + 0]), lo_clamp);
              u.y = fmaxf(fmaf(a[1], s_scale[n + 1], s_shift[n + 1]), lo_clamp);
              u.z = fmaxf(fmaf(a[2], s_scale[n + 2], s_shift[n + 2]), lo_clamp);
              u.w = fmaxf(fmaf(a[3], s_scale[n + 3], s_shift[n + 3]), lo_clamp);
              const float4 l = tf32_remainder4(u);
              hv[j] = make_uint4(__float_as_uint(u.x), __float_as_uint(u.y), __float_as_uint(u.z), __float_as_uint(u.w));
              lv[j] = make_uint4(__float_as_uint(l.x), __float_as_uint(l.y), __float_as_uint(l.z), __float_as_uint(l.w));
            }
            warp_rows_store(wbuf, hv, in_range ? reinterpret_cast<char*>(orow + 32 * k) : nullptr, lane);
            if (!c.skip_lo)
              warp_rows_store(wbuf, lv, in_range ? reinterpret_cast<char*>(orow + args.plane + 32 * k) : nullptr, lane);
          }
        }
      } else {
        const int buf = gg & (NBUF - 1);
        ok = mbar_wait(&kdone[buf], (uint32_t)(gg / NBUF) & 1u, 4u);
        ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the epilogue shuffles need all lanes
        if (!ok) break;
        last_piece_trigger(pi);
        tc_fence_after();
        __nv_bfloat16* o = fdst ? reinterpret_cast<__nv_bfloat16*>(fdst + c.frame_off) + fbase
                                : static_cast<__nv_bfloat16*>(args.out) + obase;
#pragma unroll 1
        for (int j = 0; j < BN / 64; ++j) {
          uint32_t v[64];
          tmem_ld32_nowait(trow + (uint32_t)(buf * NACC + j * 64), v);
          tmem_ld32_nowait(trow + (uint32_t)(buf * NACC + j * 64 + 32), v + 32);
          tmem_wait();
          {
            uint32_t pk[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int n = nb + j * 64 + 2 * i;
              const float a0 = fmaxf(fmaf(__uint_as_float(v[2 * i]), s_scale[n], s_shift[n]), lo_clamp);
              const float a1 = fmaxf(fmaf(__uint_as_float(v[2 * i + 1]), s_scale[n + 1], s_shift[n + 1]), lo_clamp);
              __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
              pk[i] = *reinterpret_cast<uint32_t*>(&h);
            }
            uint4 hv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) hv[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
            // 64 channels = 128 B per pixel, through the warp's transposing buffer
            warp_rows_store(reinterpret_cast<uint4*>(sO + q * 4096), hv,
                            in_range ? reinterpret_cast<char*>(o + j * 64) : nullptr, lane);
          }
        }
        tc_fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&kfree[buf])) : "memory");
        ++gg;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
}

// ---------------------------------------------------------------------------- row streaming
//
// BF16 conv for 64 input and 64 output channels that moves each input row into shared memory
// once.  A tensor-core A operand in the 128-byte-swizzled K-major layout may start at any
// 128-byte row of a swizzled buffer (the swizzle follows the absolute address), so the nine
// taps of an output row are nine row-shifted views of three resident input rows.  A CTA owns a
// strip of output rows (frame, up to 126 (stride 1) or 127 (stride 2) output columns, a run of
// rows): all 9 weight taps (72 KiB) stay resident, input rows stream through an 8-slot ring of
// 128-pixel rows (stride 2 keeps the even and odd input columns as two planes, so a tap is
// plane kx & 1 shifted by kx >> 1), and each output row is 9 taps x 4 MMAs (M = 128 output
// pixels, N = 64, K = 16) into one of two TMEM buffers while the epilogue warps drain the
// other.  Per output row the ring takes one new input row (two at stride 2) instead of nine
// 16 KiB A tiles and nine weight tiles.

struct RArgs {
  ConvShape c;
  int pv, nseg, rc, nchunks, units;  // valid outputs per segment, segments, rows per chunk
  const float* ss;
  __nv_bfloat16* out;
};

template <bool S2>
__global__ void __launch_bounds__(192, 1)
conv3x3_rows(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             RArgs args) {
  constexpr int NS = 8;                 // ring slots of one 128-pixel x 64-channel row plane
  constexpr uint32_t kRow = 128 * 128;  // 16 KiB
  constexpr uint32_t kTap = 64 * 128;   // one tap of the 64 x 64 weights, 8 KiB
  constexpr int kPlanes = S2 ? 2 : 1;   // ring slots per input row
  extern __shared__ uint8_t smem_raw[];
  __shared__ unsigned s_abort;
  if (threadIdx.x == 0) s_abort = tc_error_now();
  __syncthreads();
  if (s_abort != 0u) return;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* sW = smem;                    // [9][64 rows][128 B]
  uint8_t* sR = sW + 9 * kTap;           // [NS][128 rows][128 B]
  uint64_t* full = reinterpret_cast<uint64_t*>(sR + NS * kRow);
  uint64_t* empty = full + NS;
  uint64_t* wbar = empty + NS;
  uint64_t* kdone = wbar + 1;
  uint64_t* kfree = kdone + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(kfree + 2);
  float* s_scale = reinterpret_cast<float*>(tmem_slot + 4);
  float* s_shift = s_scale + 64;

  const ConvShape& c = args.c;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(wbar, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&kdone[i], 1);
      mbar_init(&kfree[i], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    if (args.c.static_w) {
      // weights that no preceding kernel writes: fetch them while that kernel drains
      mbar_expect_tx(wbar, 9 * kTap);
      for (int t = 0; t < 9; ++t) tma_2d(sW + t * kTap, &tmB, wbar, t * 64, 0);
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(128u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();     // the previous kernel's outputs are complete and visible
  if (threadIdx.x < 64) {
    s_scale[threadIdx.x] = args.ss[threadIdx.x];
    s_shift[threadIdx.x] = args.ss[64 + threadIdx.x];
  }
  __syncthreads();
  const int Hp = c.H + 2, Hp2 = Hp / 2;

  auto decode = [&](int u, int& b, int& ox0, int& r0, int& r1) {
    const int ch = u % args.nchunks;
    const int r = u / args.nchunks;
    const int seg = r % args.nseg;
    b = r / args.nseg;
    ox0 = seg * args.pv;
    r0 = ch * args.rc;
    r1 = r0 + args.rc < c.Ho ? r0 + args.rc : c.Ho;
  };

  if (warp == 0) {
    if (lane == 0) {
      if (!c.static_w) {
        mbar_expect_tx(wbar, 9 * kTap);
        for (int t = 0; t < 9; ++t) tma_2d(sW + t * kTap, &tmB, wbar, t * 64, 0);
      }
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < args.units && ok; u += gridDim.x) {
        int b, ox0, r0, r1;
        decode(u, b, ox0, r0, r1);
        const int in0 = r0 * (S2 ? 2 : 1);
        const int nin = S2 ? 2 * (r1 - r0) + 1 : (r1 - r0) + 2;
        for (int i = 0; i < nin && ok; ++i) {
          const int ir = in0 + i;  // padded input row
          for (int p = 0; p < kPlanes; ++p) {
            if (!mbar_wait(&empty[s], ph ^ 1u, 1u)) { ok = false; break; }
            mbar_expect_tx(&full[s], kRow);
            if (S2)
              tma_5d(sR + s * kRow, &tmA, &full[s], 0, p, ox0, ir & 1, b * Hp2 + (ir >> 1));
            else
              tma_3d(sR + s * kRow, &tmA, &full[s], 0, ox0, b * Hp + ir);
            if (++s == NS) { s = 0; ph ^= 1u; }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc<64>();
      const uint64_t dW = sdesc(sW), dR = sdesc(sR);
      bool ok = mbar_wait(wbar, 0u, 2u);
      int fw = 0, fr = 0;  // ring fills waited / released so far (fill order)
      int gg = 0;
      for (int u = blockIdx.x; u < args.units && ok; u += gridDim.x) {
        if (u + (int)gridDim.x >= args.units) pdl_trigger();  // last unit: the next kernel may launch
        int b, ox0, r0, r1;
        decode(u, b, ox0, r0, r1);
        const int base = fw;  // fill index of this unit's first row plane
        for (int oy = r0; oy < r1 && ok; ++oy) {
          const int li = oy - r0;
          // planes this output row needs: rows li..li+2 (stride 1) or 2li..2li+2 (stride 2)
          const int last = S2 ? (2 * li + 2) * 2 + 1 : li + 2;
          while (ok && fw <= base + last) {
            ok = mbar_wait(&full[fw % NS], (uint32_t)(fw / NS) & 1u, 2u);
            ++fw;
          }
          const int buf = gg & 1;
          if (ok && gg >= 2) ok = mbar_wait(&kfree[buf], (uint32_t)((gg >> 1) - 1) & 1u, 16u);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * 64);
#pragma unroll
          for (int ky = 0; ky < 3; ++ky) {
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
              const int plane = S2 ? base + (2 * li + ky) * 2 + (kx & 1) : base + li + ky;
              const int shift = S2 ? (kx >> 1) : kx;
              const uint64_t a0 = dR + (uint64_t)(((plane % NS) * kRow + shift * 128) >> 4);
              const uint64_t b0 = dW + (uint64_t)(((ky * 3 + kx) * kTap) >> 4);
#pragma unroll
              for (int k = 0; k < 4; ++k)
                mma_bf16(d, a0 + (uint64_t)(k * 2), b0 + (uint64_t)(k * 2), id,
                         (ky | kx | k) != 0 ? 1u : 0u);
            }
            // an input row's planes go back to the ring right after the last tap that reads
            // them (the commit fires once those MMAs are done): stride 1 frees row li after
            // ky = 0, stride 2 frees rows 2li and 2li+1 after ky = 0 and ky = 1
            const int upto = S2 ? (ky < 2 ? base + (2 * li + ky + 1) * 2 : fr)
                                : (ky == 0 ? base + li + 1 : fr);
            while (fr < upto) {
              mma_commit(&empty[fr % NS]);
              ++fr;
            }
          }
          mma_commit(&kdone[buf]);
          ++gg;
          if (oy + 1 == r1) {  // end of the strip: the remaining rows are not needed any more
            while (fr < fw) {
              mma_commit(&empty[fr % NS]);
              ++fr;
            }
          }
        }
      }
    }
  } else {
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    int gg = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < args.units && ok; u += gridDim.x) {
      int b, ox0, r0, r1;
      decode(u, b, ox0, r0, r1);
      const int ox = ox0 + r;
      const bool col_ok = r < args.pv && ox < c.Wo;
      for (int oy = r0; oy < r1; ++oy, ++gg) {
        const int buf = gg & 1;
        ok = mbar_wait(&kdone[buf], (uint32_t)(gg >> 1) & 1u, 4u);
        __syncwarp();
        if (!ok) break;
        tc_fence_after();
        uint32_t v[64];
        tmem_ld32_nowait(trow + (uint32_t)(buf * 64), v);
        tmem_ld32_nowait(trow + (uint32_t)(buf * 64 + 32), v + 32);
        tmem_wait();
        tc_fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&kfree[buf])) : "memory");
        if (col_ok) {
          uint32_t pk[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float a0 = fmaxf(fmaf(__uint_as_float(v[2 * i]), s_scale[2 * i], s_shift[2 * i]), 0.f);
            const float a1 = fmaxf(fmaf(__uint_as_float(v[2 * i + 1]), s_scale[2 * i + 1], s_shift[2 * i + 1]), 0.f);
            __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
            pk[i] = *reinterpret_cast<uint32_t*>(&h);
          }
          char* fdst = c.frame_dst ? c.frame_dst[b] : nullptr;  // the frame's result slot, if any
          uint4* dst = reinterpret_cast<uint4*>(
              fdst ? reinterpret_cast<__nv_bfloat16*>(fdst + c.frame_off) + ((size_t)(oy + 1) * (c.Wo + 2) + ox + 1) * 64
                   : args.out + (((size_t)b * (c.Ho + 2) + oy + 1) * (c.Wo + 2) + ox + 1) * 64);
#pragma unroll
          for (int i = 0; i < 8; ++i) dst[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u));
  }
}

// ---------------------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

struct TileTC {
  int bh, bw, bn, stages;
};
// bh*bw must be 128.  The table is the autotuner's search space.
constexpr TileTC kTilesTC[] = {
    {8, 16, 64, 4},  {4, 32, 64, 4},  {16, 8, 64, 4},  {2, 64, 64, 4}, {1, 128, 64, 4},
    {8, 16, 128, 4}, {4, 32, 128, 4}, {16, 8, 128, 4}, {8, 16, 256, 3}, {4, 32, 256, 3},
    {16, 8, 256, 3}, {8, 16, 64, 6},
};

template <int BN, int STAGES>
constexpr size_t smem_bytes() {
  return 1024 + (size_t)STAGES * (kABytes + BN * kBK * 2) + (2 * STAGES + 1) * 8 + 16 +
         2 * BN * sizeof(float);
}

template <int BN, int STAGES, bool S2>
int launch_tc(const CUtensorMap& a, const CUtensorMap& w, const TcArgs& args, dim3 grid,
              cudaStream_t s) {
  constexpr size_t bytes = smem_bytes<BN, STAGES>();
  static std::atomic<uint64_t> attr_set{0};  // per instantiation: devices configured
  if (int st = smem_attr_once(reinterpret_cast<const void*>(conv3x3_tc<BN, STAGES, S2>), (int)bytes, &attr_set,
                              "conv tc smem attribute"))
    return st;
  return cuda_status(launch_pdl(conv3x3_tc<BN, STAGES, S2>, grid, dim3(128), bytes, s, a, w, args),
                     "conv tc launch");
}



}  // namespace

int conv_tcp_tile_count(int mode);
int conv_tcp_sk_twin(int tile);
int conv_tcp_launch(int mode, const ConvShape& c, const void* in, const void* w, const float* ss,
                    void* out, int ptile, cudaStream_t s, void* ws = nullptr, size_t ws_bytes = 0,
                    const GemmOpts& g = GemmOpts());
int conv_rows_launch(const ConvShape& c, const void* in, const void* w, const float* ss, void* out,
                     cudaStream_t s, int strips_per_cta = 2);
// BF16 tiles: kTilesTC, then the persistent ones, then the row-streaming kernel with about two
// row strips per CTA and with one (longer) strip per CTA
int conv_bf16_tile_count() { return (int)(sizeof(kTilesTC) / sizeof(kTilesTC[0])) + conv_tcp_tile_count(0) + 2; }

int conv_bf16_launch(const ConvShape& c, const __nv_bfloat16* in, const __nv_bfloat16* w,
                     const float* ss, __nv_bfloat16* out, int tile, cudaStream_t s) {
  auto enc = encode_fn();
  if (!enc) return fail(PP_EDEVICE, "cuTensorMapEncodeTiled is unavailable");
  if (tile < 0) tile = tuned_tile(PP_BF16, c);
  const int n_old = (int)(sizeof(kTilesTC) / sizeof(kTilesTC[0]));
  const int n_p = conv_tcp_tile_count(0);
  if ((tile < 0 && c.cin == 64 && c.cout == 64) || tile == n_old + n_p)
    return conv_rows_launch(c, in, w, ss, out, s, 2);
  if (tile == n_old + n_p + 1) return conv_rows_launch(c, in, w, ss, out, s, 1);
  if (tile < 0 || tile >= n_old) return conv_tcp_launch(0, c, in, w, ss, out, tile < 0 ? -1 : tile - n_old, s);
  if (tile < 0 || tile >= conv_bf16_tile_count() || c.cout % kTilesTC[tile].bn)
    return fail(PP_EINVAL, "conv bf16: tile %d unsupported for cout %d", tile, c.cout);
  const TileTC t = kTilesTC[tile];
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(w)) & 15u)
    return fail(PP_EINVAL, "conv bf16: operands must be 16-byte aligned");
  const int Hp = c.H + 2, Wp = c.W + 2;
  CUtensorMap ta, tw;
  CUresult r;
  if (c.stride == 1) {
    cuuint64_t dims[3] = {(cuuint64_t)c.cin, (cuuint64_t)Wp, (cuuint64_t)Hp * c.batch};
    cuuint64_t strides[2] = {(cuuint64_t)c.cin * 2, (cuuint64_t)Wp * c.cin * 2};
    cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)t.bw, (cuuint32_t)t.bh};
    cuuint32_t es[3] = {1, 1, 1};
    r = enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(in), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[5] = {(cuuint64_t)c.cin, 2, (cuuint64_t)Wp / 2, 2, (cuuint64_t)(Hp / 2) * c.batch};
    cuuint64_t strides[4] = {(cuuint64_t)c.cin * 2, (cuuint64_t)c.cin * 4,
                             (cuuint64_t)Wp * c.cin * 2, (cuuint64_t)Wp * c.cin * 4};
    cuuint32_t box[5] = {(cuuint32_t)kBK, 1, (cuuint32_t)t.bw, 1, (cuuint32_t)t.bh};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    r = enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(in), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return fail(PP_EDEVICE, "conv bf16: activation tensor map (%d)", (int)r);
  {
    const int K = 9 * c.cin;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)c.cout};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)t.bn};
    cuuint32_t es[2] = {1, 1};
    r = enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(w), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return fail(PP_EDEVICE, "conv bf16: weight tensor map (%d)", (int)r);
  TcArgs args;
  args.c = c;
  args.bh = t.bh;
  args.bw = t.bw;
  args.tiles_x = (c.Wo + t.bw - 1) / t.bw;
  args.tiles_y = (c.Ho + t.bh - 1) / t.bh;
  args.ss = ss;
  args.out = out;
  const dim3 grid((unsigned)(args.tiles_x * args.tiles_y * c.batch), (unsigned)(c.cout / t.bn));
  const bool s2 = c.stride == 2;
#define PP_TC_CASE(BN, ST)                                                       \
  if (t.bn == BN && t.stages == ST)                                              \
    return s2 ? launch_tc<BN, ST, true>(ta, tw, args, grid, s)                   \
              : launch_tc<BN, ST, false>(ta, tw, args, grid, s);
  PP_TC_CASE(64, 4)
  PP_TC_CASE(64, 6)
  PP_TC_CASE(128, 4)
  PP_TC_CASE(256, 3)
#undef PP_TC_CASE
  return fail(PP_EINVAL, "conv bf16: no kernel for tile %d", tile);
}

int conv_f32tc_tile_count() { return conv_tcp_tile_count(1); }

int conv_f32tc_launch(const ConvShape& c, const float* in, const float* w_split, const float* ss,
                      float* out, int tile, cudaStream_t s, void* ws, size_t ws_bytes) {
  if (c.cin % 32) return fail(PP_EINVAL, "conv f32 tensor: cin must be a multiple of 32");
  if (tile < 0) {
    tile = tuned_tile(PP_F32_TC, c);
    // a stream-K choice needs a workspace; without one, the same tile without stream-K
    if (!ws || ws_bytes < conv_sk_workspace_bytes(c)) tile = conv_tcp_sk_twin(tile);
  }
  return conv_tcp_launch(1, c, in, w_split, ss, out, tile, s, ws, ws_bytes);
}

namespace {

struct TileP {
  int bh, bw, bn;
};
// Persistent tiles (bh*bw = 128).  Stages fill ~192 KiB of shared memory: BF16 stage = 16 KiB A
// + BN x 128 B; 3xTF32 stage = 32 KiB A (+lo) + 2 x BN x 128 B.
constexpr TileP kTilesPB[] = {{8, 16, 64}, {4, 32, 64}, {16, 8, 64}, {2, 64, 64}, {8, 16, 128},
                              {4, 32, 128}, {16, 8, 128}, {8, 16, 256}, {4, 32, 256}};
constexpr TileP kTilesPF[] = {{8, 16, 64}, {4, 32, 64}, {16, 8, 64}, {2, 64, 64}, {8, 16, 128},
                              {4, 32, 128}, {16, 8, 128}};
constexpr int kNPB = (int)(sizeof(kTilesPB) / sizeof(kTilesPB[0]));
constexpr int kNPF = (int)(sizeof(kTilesPF) / sizeof(kTilesPF[0]));
// 3xTF32 tiles from 2 kNPF on: 128 consecutive output pixels (over the padded width) whose three
// kx taps share one loaded 130-pixel input range (stride-1 3x3 convs); their output channels and
// ring shapes are listed with the shared-memory sizes below (kHalo)

// Ring depth and K blocks per stage.  BF16 stage = KPS x (16 KiB A + BN x 128 B); 3xTF32
// stage = KPS x (32 KiB A (+lo) + 2 x BN x 128 B).  All fill ~192 KiB of shared memory.  Two K
// blocks per stage halve the per-stage handshakes (measured on the full-size frame: 3xTF32
// BN 64 layers 12-16 % faster with 2 stages of 2 K blocks than with 3 stages of 1; BF16 layers
// up to 11 % faster with 2 stages of 4 / 3 K blocks than with 4 / 3 stages of 2).
template <int MODE, int BN>
constexpr int p_kps() {
  return MODE == 1 ? (BN == 64 ? 2 : 1) : (BN == 64 ? 4 : BN == 128 ? 3 : 2);
}
template <int MODE, int BN>
constexpr int p_stages() {
  return MODE == 1 ? (BN == 64 ? 2 : 3) : 2;
}
template <int MODE, int BN>
constexpr size_t p_smem() {
  return 1024 + (size_t)p_stages<MODE, BN>() * p_kps<MODE, BN>() *
                    ((MODE == 1 ? 2 : 1) * 16384 + (MODE == 1 ? 2 : 1) * BN * 128) +
         4 * 4096 +                                   // epilogue transposing buffers
         (2 * p_stages<MODE, BN>() + 8) * 8 + 16;  // full/empty per stage, kdone/kfree x 4
}
// halo tiles (3xTF32): NB = 0: ST unified stages of (two 130-row planes rounded to 1 KiB, three
// taps of B value and remainder), BN 64 only; NB > 0: an A ring of ST slots (two 130-row planes)
// and a B ring of NB slots (one tap, value and remainder), with their own full/empty barriers
template <int BN, int ST, int NB>
constexpr size_t p_smem_halo() {
  return NB == 0 ? 1024 + (size_t)ST * (2 * 17408 + 3 * 2 * BN * 128) + p_red_warps<1, BN, true>() * 4096 +
                       (2 * ST + 8) * 8 + 16
                 : 1024 + (size_t)ST * 2 * 17408 + (size_t)NB * 2 * BN * 128 + p_red_warps<1, BN, true>() * 4096 +
                       (2 * ST + 8 + 2 * NB) * 8 + 16;
}
// The halo variants, tiles 2 kNPF + i: (output channels, A stages, B slots (0 = unified
// stages), stream-K, kx folded into N).  The stream-K ones cut the accumulation groups of all
// tiles into one equal range per SM, as the stream-K twins of the plain tiles cut their K
// blocks.  The kx-in-N one (last) computes 126 output pixels per tile.
struct HaloVariant {
  int bn, stages, bslots;
  bool sk, kxn;
};
constexpr HaloVariant kHalo[] = {{64, 2, 0, false, false}, {128, 2, 4, false, false}, {64, 3, 5, false, false},
                                 {128, 3, 3, false, false}, {64, 2, 0, true, false},  {128, 2, 4, true, false},
                                 {64, 2, 0, false, true}};
// output pixels per halo tile
constexpr int halo_bw(const HaloVariant& v) { return v.kxn ? 126 : 128; }
// accumulation groups per TMEM buffer of the kx-in-N tile
constexpr int kKxnFold = 2;
constexpr int kNHalo = (int)(sizeof(kHalo) / sizeof(kHalo[0]));

int num_sms() {
  return device_sms();
}

template <int MODE, int BN, bool S2, bool SK, bool HALO = false, int HST = 2, int NBS = 0, bool KXN = false>
int launch_p(const CUtensorMap& a, const CUtensorMap& alo, const CUtensorMap& w, const PArgs& args,
             cudaStream_t s) {
  constexpr int ST = HALO ? HST : p_stages<MODE, BN>();
  constexpr int KPS = HALO ? 3 : p_kps<MODE, BN>();
  // + folded BN (cout <= 1024)
  constexpr size_t bytes = (HALO ? p_smem_halo<BN, HST, NBS>() : p_smem<MODE, BN>()) + 2 * 1024 * sizeof(float);
  static_assert(bytes <= 227 * 1024, "persistent conv shared memory");
  static std::atomic<uint64_t> attr_set{0};  // per instantiation: devices configured
  if (int st = smem_attr_once(reinterpret_cast<const void*>(conv3x3_tcp<MODE, BN, ST, KPS, S2, SK, HALO, NBS, KXN>),
                              (int)bytes, &attr_set, "persistent conv smem attribute"))
    return st;
  // stream-K: one range per CTA, never an empty one (an empty range would be counted among the
  // CTAs that share a tile but never arrive), so at most one CTA per K block (per accumulation
  // group for the halo tiles)
  const long kblocks = (long)args.total * (HALO ? 3 : 9) * (args.c.cin / (MODE == 1 ? 32 : 64));
  const int grid = SK ? (int)(kblocks < num_sms() ? kblocks : num_sms())
                           : (args.total < num_sms() ? args.total : num_sms());
  return cuda_status(launch_pdl(conv3x3_tcp<MODE, BN, ST, KPS, S2, SK, HALO, NBS, KXN>, dim3(grid),
                                dim3(p_threads<MODE, BN, HALO>()), bytes, s, a,
                                alo, w, args),
                     "persistent conv launch");
}

// Persistent tile choice: fewest "waves" of tile work over the SMs, each tile costing its MMA
// time plus a fixed per-tile overhead.
// co_blk: an N tile may not straddle a block of co_blk GEMM columns (transposed conv)
int pick_tile_p(const ConvShape& c, const TileP* tiles, int n, int co_blk) {
  int best = -1;
  double best_cost = 1e30;
  for (int i = 0; i < n; ++i) {
    const TileP& t = tiles[i];
    if (c.cout % t.bn || co_blk % t.bn) continue;
    const double tx = (c.Wo + t.bw - 1) / t.bw, ty = (c.Ho + t.bh - 1) / t.bh;
    const double total = tx * ty * c.batch * (c.cout / t.bn);
    const double per_sm = ceil(total / num_sms());
    const double cost = per_sm * (t.bn + 48.0);
    if (cost < best_cost - 1e-9) { best_cost = cost; best = i; }
  }
  return best;
}

}  // namespace

// mode 0: BF16 in/out, weights [cout][9cin] bf16; mode 1: split FP32 in/out ([2][B][H+2][W+2][C]:
// values, TF32 remainders) via 3xTF32, weights [2][cout][9cin] fp32 (hi, lo planes).
int conv_tcp_launch(int mode, const ConvShape& c, const void* in, const void* w, const float* ss,
                    void* out, int ptile, cudaStream_t s, void* ws, size_t ws_bytes, const GemmOpts& g) {
  auto enc = encode_fn();
  if (!enc) return fail(PP_EDEVICE, "cuTensorMapEncodeTiled is unavailable");
  const int co_blk = g.co_blk ? g.co_blk : c.cout, out_c = g.out_c ? g.out_c : co_blk;
  if ((g.taps != 9 && g.taps != 1) || g.up < 1 || (g.taps == 1 && c.stride != 1) ||
      g.up * g.up * co_blk != c.cout || co_blk % 64 || out_c % 64 || g.out_coff % 64 ||
      g.out_coff + co_blk > out_c || co_blk > 1024)
    return fail(PP_EINVAL, "persistent conv: bad GEMM options");
  const TileP* tiles = mode == 1 ? kTilesPF : kTilesPB;
  const int n = mode == 1 ? kNPF : kNPB;
  // 3xTF32 tiles kNPF..2 kNPF-1: the same tiles with the stream-K partition; 2 kNPF + i: halo
  // variant kHalo[i]
  const bool halo = mode == 1 && ptile >= 2 * n && ptile < 2 * n + kNHalo;
  const HaloVariant hv = halo ? kHalo[ptile - 2 * n] : kHalo[0];
  const int halo_bn = hv.bn;
  if (halo && (c.stride != 1 || g.taps != 9 || g.up != 1 || c.cout % halo_bn || co_blk % halo_bn))
    return fail(PP_EINVAL, "persistent conv: the halo tile needs a stride-1 3x3 conv with cout a multiple of %d",
                halo_bn);
  const bool sk = mode == 1 && ptile >= n && (!halo || hv.sk);
  if (sk && !halo) ptile -= n;
  if (!halo && ptile < 0) ptile = pick_tile_p(c, tiles, n, co_blk);
  if (!halo && (ptile < 0 || ptile >= n || c.cout % tiles[ptile].bn || co_blk % tiles[ptile].bn))
    return fail(PP_EINVAL, "persistent conv: tile %d unsupported for cout %d", ptile, c.cout);
  const TileP t = halo ? TileP{1, halo_bw(hv), halo_bn} : tiles[ptile];
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(w)) & 15u)
    return fail(PP_EINVAL, "persistent conv: operands must be 16-byte aligned");
  const int BK = mode == 1 ? 32 : 64;
  const size_t el = mode == 1 ? 4 : 2;
  const CUtensorMapDataType dt = mode == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const int Hp = c.H + 2, Wp = c.W + 2;
  CUtensorMap ta, talo, tw;
  CUresult r = CUDA_SUCCESS;
  for (int plane = 0; plane < (mode == 1 ? 2 : 1) && r == CUDA_SUCCESS; ++plane) {
    const size_t in_plane = c.in_plane ? c.in_plane : (size_t)c.batch * Hp * Wp * c.cin;
    void* base = static_cast<char*>(const_cast<void*>(in)) + (size_t)plane * in_plane * el;
    CUtensorMap* m = plane ? &talo : &ta;
    if (halo) {
      // the flattened padded image: bw + 2 consecutive pixels per load for bw outputs
      cuuint64_t dims[2] = {(cuuint64_t)c.cin, (cuuint64_t)Hp * Wp * c.batch};
      cuuint64_t strides[1] = {(cuuint64_t)c.cin * el};
      cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)(t.bw + 2)};
      cuuint32_t es[2] = {1, 1};
      r = enc(m, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else if (c.stride == 1) {
      cuuint64_t dims[3] = {(cuuint64_t)c.cin, (cuuint64_t)Wp, (cuuint64_t)Hp * c.batch};
      cuuint64_t strides[2] = {(cuuint64_t)c.cin * el, (cuuint64_t)Wp * c.cin * el};
      cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)t.bw, (cuuint32_t)t.bh};
      cuuint32_t es[3] = {1, 1, 1};
      r = enc(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      cuuint64_t dims[5] = {(cuuint64_t)c.cin, 2, (cuuint64_t)Wp / 2, 2, (cuuint64_t)(Hp / 2) * c.batch};
      cuuint64_t strides[4] = {(cuuint64_t)c.cin * el, (cuuint64_t)c.cin * 2 * el,
                               (cuuint64_t)Wp * c.cin * el, (cuuint64_t)Wp * c.cin * 2 * el};
      cuuint32_t box[5] = {(cuuint32_t)BK, 1, (cuuint32_t)t.bw, 1, (cuuint32_t)t.bh};
      cuuint32_t es[5] = {1, 1, 1, 1, 1};
      r = enc(m, dt, 5, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
  }
  if (mode != 1) talo = ta;
  if (r != CUDA_SUCCESS) return fail(PP_EDEVICE, "persistent conv: activation tensor map (%d)", (int)r);
  {
    const int K = g.taps * c.cin;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)c.cout, (cuuint64_t)(mode == 1 ? 2 : 1)};
    cuuint64_t strides[2] = {(cuuint64_t)K * el, (cuuint64_t)K * c.cout * el};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)t.bn, 1};
    cuuint32_t es[3] = {1, 1, 1};
    r = enc(&tw, dt, mode == 1 ? 3 : 2, const_cast<void*>(w), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return fail(PP_EDEVICE, "persistent conv: weight tensor map (%d)", (int)r);
  PArgs args;
  args.c = c;
  args.bh = t.bh;
  args.bw = t.bw;
  // halo-row tiles: runs of bw output pixels laid out over the padded width, per image
  args.tiles_x = halo ? (c.Ho * (c.W + 2) + t.bw - 1) / t.bw : (c.Wo + t.bw - 1) / t.bw;
  args.tiles_y = halo ? 1 : (c.Ho + t.bh - 1) / t.bh;
  args.tiles_n = c.cout / t.bn;
  args.total = args.tiles_x * args.tiles_y * c.batch * args.tiles_n;
  // work units per TMEM accumulation buffer (a halo unit is one group; the kx-in-N tile takes
  // two groups per buffer; the plain 3xTF32 tiles four K blocks, 32 accumulations into a
  // column: 1-4 % faster than two on the stride-2 layers of the full-size frame, the frame's
  // error unchanged at 3e-5)
  args.fold = halo ? (hv.kxn ? kKxnFold : 1) : 4;
  args.taps = g.taps;
  args.up = g.up;
  args.co_blk = co_blk;
  args.out_c = out_c;
  args.out_coff = g.out_coff;
  args.Hout = g.up * c.Ho;
  args.Wout = g.up * c.Wo;
  args.relu = g.relu;
  args.plane = c.out_plane ? c.out_plane : (size_t)c.batch * (args.Hout + 2) * (args.Wout + 2) * out_c;
  args.ss = ss;
  args.out = out;
  args.sk = sk ? 1 : 0;
  args.ws = nullptr;
  args.sem = nullptr;
  if (sk) {
    // counters after partial slots sized for the widest N tile, at the same offset for every
    // tile, so that launches with different tiles can share one workspace
    const size_t part = (size_t)2 * num_sms() * 128 * 128 * sizeof(float);
    if (!ws || ws_bytes < part + (size_t)args.total * sizeof(unsigned) || (reinterpret_cast<uintptr_t>(ws) & 255u))
      return fail(PP_EINVAL, "persistent conv: stream-K tile needs a 256-byte aligned workspace of %zu bytes",
                  part + (size_t)args.total * sizeof(unsigned));
    args.ws = static_cast<float*>(ws);
    args.sem = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + part);
  }
  const bool s2 = c.stride == 2;
#define PP_P(M, N, K) return s2 ? launch_p<M, N, true, K>(ta, talo, tw, args, s) : launch_p<M, N, false, K>(ta, talo, tw, args, s)
  if (mode == 1) {
    if (halo) {
      switch (ptile - 2 * n) {
        case 0: return launch_p<1, 64, false, false, true, 2, 0>(ta, talo, tw, args, s);
        case 1: return launch_p<1, 128, false, false, true, 2, 4>(ta, talo, tw, args, s);
        case 2: return launch_p<1, 64, false, false, true, 3, 5>(ta, talo, tw, args, s);
        case 3: return launch_p<1, 128, false, false, true, 3, 3>(ta, talo, tw, args, s);
        case 4: return launch_p<1, 64, false, true, true, 2, 0>(ta, talo, tw, args, s);
        case 5: return launch_p<1, 128, false, true, true, 2, 4>(ta, talo, tw, args, s);
        default: return launch_p<1, 64, false, false, true, 2, 0, true>(ta, talo, tw, args, s);
      }
    }
    if (t.bn == 64) { if (sk) PP_P(1, 64, true); PP_P(1, 64, false); }
    if (t.bn == 128) { if (sk) PP_P(1, 128, true); PP_P(1, 128, false); }
  } else {
    if (t.bn == 64) PP_P(0, 64, false);
    if (t.bn == 128) PP_P(0, 128, false);
    if (t.bn == 256) PP_P(0, 256, false);
  }
#undef PP_P
  return fail(PP_EINVAL, "persistent conv: no kernel for tile %d", ptile);
}

// Row-streaming BF16 conv (64 -> 64 channels).
// strips_per_cta: the output rows are cut into strips of rc >= 4 rows so that there are about
// strips_per_cta strips per SM (2: a CTA runs two shorter strips; 1: one longer strip each, so
// that the ring is filled once per CTA)
int conv_rows_launch(const ConvShape& c, const void* in, const void* w, const float* ss, void* out,
                     cudaStream_t s, int strips_per_cta) {
  if (strips_per_cta < 1 || strips_per_cta > 2) return fail(PP_EINVAL, "row conv: 1 or 2 strips per CTA");
  auto enc = encode_fn();
  if (!enc) return fail(PP_EDEVICE, "cuTensorMapEncodeTiled is unavailable");
  if (c.cin != 64 || c.cout != 64) return fail(PP_EINVAL, "row conv: needs 64 input and 64 output channels");
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(w)) & 15u)
    return fail(PP_EINVAL, "row conv: operands must be 16-byte aligned");
  const int Hp = c.H + 2, Wp = c.W + 2;
  CUtensorMap ta, tw;
  CUresult r;
  if (c.stride == 1) {
    cuuint64_t dims[3] = {64, (cuuint64_t)Wp, (cuuint64_t)Hp * c.batch};
    cuuint64_t strides[2] = {128, (cuuint64_t)Wp * 128};
    cuuint32_t box[3] = {64, 128, 1};
    cuuint32_t es[3] = {1, 1, 1};
    r = enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(in), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[5] = {64, 2, (cuuint64_t)Wp / 2, 2, (cuuint64_t)(Hp / 2) * c.batch};
    cuuint64_t strides[4] = {128, 256, (cuuint64_t)Wp * 128, (cuuint64_t)Wp * 256};
    cuuint32_t box[5] = {64, 1, 128, 1, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    r = enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(in), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return fail(PP_EDEVICE, "row conv: activation tensor map (%d)", (int)r);
  {
    cuuint64_t dims[2] = {9 * 64, 64};
    cuuint64_t strides[1] = {9 * 64 * 2};
    cuuint32_t box[2] = {64, 64};
    cuuint32_t es[2] = {1, 1};
    r = enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(w), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return fail(PP_EDEVICE, "row conv: weight tensor map (%d)", (int)r);
  RArgs a;
  a.c = c;
  a.pv = c.stride == 2 ? 127 : 126;
  a.nseg = (c.Wo + a.pv - 1) / a.pv;
  const int sms = num_sms();
  const long rows = (long)c.batch * a.nseg * c.Ho;
  const long slots = (long)strips_per_cta * sms;
  int rc = (int)((rows + slots - 1) / slots);
  if (rc < 4) rc = 4;
  if (rc > c.Ho) rc = c.Ho;
  a.rc = rc;
  a.nchunks = (c.Ho + rc - 1) / rc;
  a.units = c.batch * a.nseg * a.nchunks;
  a.ss = ss;
  a.out = static_cast<__nv_bfloat16*>(out);
  constexpr size_t bytes = 1024 + 9 * 64 * 128 + 8 * 128 * 128 + (2 * 8 + 5) * 8 + 16 + 2 * 64 * 4;
  const int grid = a.units < sms ? a.units : sms;
  if (c.stride == 2) {
    static std::atomic<uint64_t> attr{0};
    if (int st = smem_attr_once(reinterpret_cast<const void*>(conv3x3_rows<true>), (int)bytes, &attr,
                                "row conv smem attribute"))
      return st;
    const cudaError_t e = launch_pdl(conv3x3_rows<true>, dim3(grid), dim3(192), bytes, s, ta, tw, a);
    if (e != cudaSuccess) return cuda_status(e, "row conv launch");
  } else {
    static std::atomic<uint64_t> attr{0};
    if (int st = smem_attr_once(reinterpret_cast<const void*>(conv3x3_rows<false>), (int)bytes, &attr,
                                "row conv smem attribute"))
      return st;
    const cudaError_t e = launch_pdl(conv3x3_rows<false>, dim3(grid), dim3(192), bytes, s, ta, tw, a);
    if (e != cudaSuccess) return cuda_status(e, "row conv launch");
  }
  return PP_OK;
}

int conv_tcp_tile_count(int mode) { return mode == 1 ? 2 * kNPF + kNHalo : kNPB; }
// the tile to launch instead of stream-K tile `tile` when there is no workspace (the tile itself
// if it is not a stream-K one)
int conv_tcp_sk_twin(int tile) {
  if (tile >= kNPF && tile < 2 * kNPF) return tile - kNPF;
  const int h = tile - 2 * kNPF;
  if (h >= 0 && h < kNHalo && kHalo[h].sk)
    for (int i = 0; i < kNHalo; ++i)
      if (!kHalo[i].sk && kHalo[i].bn == kHalo[h].bn && kHalo[i].stages == kHalo[h].stages &&
          kHalo[i].bslots == kHalo[h].bslots)
        return 2 * kNPF + i;
  return tile;
}

int gemm_tc_launch(int dtype, const ConvShape& c, const GemmOpts& g, const void* in, const void* w,
                   const float* ss, void* out, int tile, cudaStream_t s) {
  if (dtype != PP_BF16 && dtype != PP_F32_TC) return fail(PP_EINVAL, "tensor-core GEMM: dtype must be BF16 or F32_TC");
  const int mode = dtype == PP_F32_TC ? 1 : 0;
  if (c.cin % (mode == 1 ? 32 : 64)) return fail(PP_EINVAL, "tensor-core GEMM: bad cin");
  // tiles are numbered as for the 3x3 conv; only the persistent (non-stream-K) ones apply
  const int first = mode == 1 ? 0 : (int)(sizeof(kTilesTC) / sizeof(kTilesTC[0]));
  if (tile >= 0 && (tile < first || tile >= first + (mode == 1 ? kNPF : kNPB)))
    return fail(PP_EINVAL, "tensor-core GEMM: tile %d is not a persistent tile", tile);
  return conv_tcp_launch(mode, c, in, w, ss, out, tile < 0 ? -1 : tile - first, s, nullptr, 0, g);
}

// Workspace for any stream-K tile of this shape: partial tiles for two pieces per CTA at the
// widest N tile, then one arrival counter per output tile of the narrowest.
size_t conv_sk_workspace_bytes(const ConvShape& c) {
  size_t tiles = 0;
  for (int i = 0; i < kNPF; ++i) {
    const TileP& t = kTilesPF[i];
    if (c.cout % t.bn) continue;
    const size_t n = (size_t)((c.Wo + t.bw - 1) / t.bw) * ((c.Ho + t.bh - 1) / t.bh) * c.batch * (c.cout / t.bn);
    if (n > tiles) tiles = n;
  }
  if (c.stride == 1 && c.cout % 64 == 0) {
    // halo tiles: 128-pixel runs of the output over the padded width, 64 channels at the narrowest
    const size_t n = ((size_t)c.Ho * (c.W + 2) + 127) / 128 * c.batch * (c.cout / 64);
    if (n > tiles) tiles = n;
  }
  return (size_t)2 * num_sms() * 128 * 128 * sizeof(float) + align_up(tiles * sizeof(unsigned), 256);
}

int conv_tc_tile_info(int dtype, int tile, int* bh, int* bw, int* bn, int* persistent) {
  if (dtype == PP_BF16) {
    const int n0 = (int)(sizeof(kTilesTC) / sizeof(kTilesTC[0]));
    if (tile < 0 || tile > n0 + kNPB + 1) return PP_EINVAL;
    if (tile >= n0 + kNPB) { *bh = 1; *bw = 128; *bn = 64; *persistent = 2; return PP_OK; }  // row streaming
    if (tile < n0) { *bh = kTilesTC[tile].bh; *bw = kTilesTC[tile].bw; *bn = kTilesTC[tile].bn; *persistent = 0; }
    else { const TileP& t = kTilesPB[tile - n0]; *bh = t.bh; *bw = t.bw; *bn = t.bn; *persistent = 1; }
    return PP_OK;
  }
  if (dtype == PP_F32_TC) {
    if (tile < 0 || tile >= 2 * kNPF + kNHalo) return PP_EINVAL;
    const HaloVariant* hv = tile >= 2 * kNPF ? &kHalo[tile - 2 * kNPF] : nullptr;
    const TileP t = hv ? TileP{1, halo_bw(*hv), hv->bn} : kTilesPF[tile % kNPF];
    *bh = t.bh; *bw = t.bw; *bn = t.bn;
    *persistent = tile < kNPF ? 1 : tile < 2 * kNPF ? 3 : hv->sk ? 5 : hv->kxn ? 6 : 4;
    return PP_OK;
  }
  return PP_EINVAL;
}

int tc_error_set(unsigned bits) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_status(e, "read device error word");
  v |= bits;
  e = cudaMemcpyToSymbol(g_tc_error, &v, sizeof(unsigned));
  return cuda_status(e, "set device error word");
}

int tc_error_address(const unsigned** out) {
  // the symbol's device address differs per device: looked up with that device current, once
  constexpr int kDev = 64;
  static std::atomic<const unsigned*> addr[kDev];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "current device");
  const unsigned* p = dev < kDev ? addr[dev].load(std::memory_order_acquire) : nullptr;
  if (!p) {
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_tc_error);
    if (e != cudaSuccess) return cuda_status(e, "device error word address");
    p = static_cast<const unsigned*>(q);
    if (dev < kDev) addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return PP_OK;
}

int tc_error_read(unsigned* code, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(code, g_tc_error, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_status(e, "read device error word");
  if (clear && *code) {
    const unsigned zero = 0;
    e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_status(e, "clear device error word");
  }
  return PP_OK;
}

}  // namespace pp
