// Voxelisation of LiDAR points into pillars (point -> cell -> pillar), batched over frames.
//
// The paper's 3D-perception chains run PointPillars (Section 6, Table 4); this is its first
// stage, made deterministic: pillars are the occupied cells in ascending cell order (at most
// P), and each keeps its 32 lowest-index points in ascending index order.
//
// Five launches per batch, gridDim.y = frame:
//   1. vox_cell_count   cell per point; warp-aggregated atomic count per cell, which also hands
//                       each point an arrival slot inside its cell (order arbitrary)
//   2. vox_tile_sums    per tile of 2048 cells: (occupied cells, points)
//   3. vox_scan         exclusive scans over cells -> pillar id (rank of occupied cell, kept if
//                       < P), pillar's first point offset; writes coord / npts / num_pillars
//   4. vox_bucket       point i -> csr[pillar_start + slot]: points grouped by kept pillar
//   5. vox_select       one warp per pillar: the 32 smallest point indices of its group, sorted
//                       by warp bitonic sort/merge, gathered into pts (zero padded)
// A release unit stops after step 4: its PointNet kernel does step 5 itself (pfn.cu,
// pfn_select_fused), so the gathered points stay in registers.
// Nothing depends on the order in which atomics land, so the output is bit-identical across
// runs.  The cell index follows the binary32 contract of pp.h (__fsub_rn / __fdiv_rn, floorf).
#include "pillar_dev.cuh"

namespace pp {
namespace {

using dev::frame_src;
constexpr unsigned kFull = dev::kFullMask;

__device__ __forceinline__ int frame_points(const int* n_points, int b, int cap, int* err) {
  int n = n_points[b];
  if (n < 0 || n > cap) {
    if (err && threadIdx.x == 0 && blockIdx.x == 0) atomicOr(err, 1);
    return 0;
  }
  return n;
}


// Points per thread per pass of the point kernels: their loads (and atomics) are issued
// together so that one memory round trip covers several points.
constexpr int kVoxU = 4;
// 32-bit words of the per-warp bit table of the count kernel's no-repeated-cell test (a power
// of two): 16,384 bits, so that 32 distinct cells share a bit with probability ~3 %.
constexpr int kVoxTabWords = 512;

__global__ void vox_cell_count(Geom g, int cap, const float4* __restrict__ points,
                               const float4* const* __restrict__ srcs,
                               float4* const* __restrict__ mirrors,
                               const int* __restrict__ n_points, int* __restrict__ cell,
                               int* __restrict__ slot, unsigned* __restrict__ cnt, int* err,
                               const uint4* __restrict__ table_src, uint4* __restrict__ table_dst,
                               int table_words) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  // a release unit's per-launch table: copied from host memory for the kernels that follow
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < table_words) table_dst[threadIdx.x] = table_src[threadIdx.x];
  const int b = blockIdx.y;
  // the frame's count and pointers: one thread per block reads them (in a release unit from
  // page-locked host memory, where each read crosses the host link) and shares them
  __shared__ int s_n;
  __shared__ const float4* s_src;
  __shared__ float4* s_mirror;
  if (threadIdx.x == 0) {
    s_n = frame_points(n_points, b, cap, err);
    s_src = frame_src(points, srcs, b, cap);
    s_mirror = mirrors ? mirrors[b] : nullptr;
  }
  __syncthreads();
  const int n = s_n;
  const float4* src = s_src;
  float4* mirror = s_mirror;  // copy of a frame read over the host link
  const int lane = threadIdx.x & 31;
  unsigned* cnt_b = cnt + (size_t)b * g.G;
  const int cell_bits = g.G > 1 ? 32 - __clz(g.G - 1) : 1;  // bits of the largest cell index
  __shared__ __align__(16) unsigned s_tab[8][kVoxTabWords];    // per warp (256 threads)
  unsigned* tab = s_tab[threadIdx.x >> 5];
  for (int i = lane; i < kVoxTabWords / 4; i += 32) reinterpret_cast<uint4*>(tab)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  // grid-stride over the frame's points, kVoxU coalesced blocks of blockDim.x points per pass
  // (block-uniform trip count: whole warps stay together)
  for (int i0 = blockIdx.x * blockDim.x * kVoxU; i0 < n; i0 += gridDim.x * blockDim.x * kVoxU) {
    float4 p[kVoxU];
#pragma unroll
    for (int u = 0; u < kVoxU; ++u) {
      const int i = i0 + u * blockDim.x + threadIdx.x;
      p[u] = i < n ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (mirror) {
#pragma unroll
      for (int u = 0; u < kVoxU; ++u) {
        const int i = i0 + u * blockDim.x + threadIdx.x;
        if (i < n) mirror[i] = p[u];
      }
    }
    int c[kVoxU];
#pragma unroll
    for (int u = 0; u < kVoxU; ++u) {
      const int i = i0 + u * blockDim.x + threadIdx.x;
      c[u] = -1;
      if (i < n) {
        bool ok = p[u].x >= g.xmin && p[u].x < g.xmax && p[u].y >= g.ymin && p[u].y < g.ymax &&
                  p[u].z >= g.zmin && p[u].z < g.zmax;
        if (ok) {
          const float qx = floorf(__fdiv_rn(__fsub_rn(p[u].x, g.xmin), g.vx));
          const float qy = floorf(__fdiv_rn(__fsub_rn(p[u].y, g.ymin), g.vy));
          ok = qx >= 0.f && qx < (float)g.nx && qy >= 0.f && qy < (float)g.ny;
          if (ok) c[u] = (int)qy * g.nx + (int)qx;
        }
        cell[(size_t)b * cap + i] = c[u];
      }
    }
    // warp-aggregated counting: lanes with the same cell elect the lowest as leader, which adds
    // their number to the cell's count; the old count is the group's first arrival slot.  A
    // lane's peers (the lanes holding its cell) come from one ballot per bit of the cell index:
    // the lanes that agree with it on every bit.  That is the set __match_any_sync returns, at
    // a lower cost when the 32 cells are mostly distinct.  First a cheap exact test: every
    // lane sets the bit of a per-warp bit table chosen by the low bits of its cell with an
    // atomic OR that returns the word's old value; a lane that finds its bit already set
    // shares it with another lane (the same cell, or another cell with the same low bits).
    // If no lane does, no two lanes share a cell, every lane is its own group and the ballots
    // are skipped.  The lanes then clear the words they set.
    unsigned peers[kVoxU], base[kVoxU];
#pragma unroll
    for (int u = 0; u < kVoxU; ++u) {
      const unsigned valid = __ballot_sync(kFull, c[u] >= 0);
      const int word = (c[u] >> 5) & (kVoxTabWords - 1);
      const unsigned bitm = 1u << (c[u] & 31);
      const bool clash = c[u] >= 0 && (atomicOr(&tab[word], bitm) & bitm) != 0u;
      const unsigned clashes = __ballot_sync(kFull, clash);
      __syncwarp();  // every lane's atomic on the table before any lane clears a word
      if (c[u] >= 0) tab[word] = 0u;
      __syncwarp();  // the table clear before the next group's atomics
      unsigned pm = valid & (1u << lane);
      if (clashes) {
        pm = valid;
        for (int k = 0; k < cell_bits; ++k) {
          const unsigned bit = (unsigned)(c[u] >> k) & 1u;
          const unsigned on = __ballot_sync(kFull, bit);
          pm &= bit ? on : ~on;
        }
      }
      peers[u] = 0u;
      base[u] = 0u;
      if (c[u] >= 0) {
        peers[u] = pm;
        if (lane == __ffs(pm) - 1) base[u] = atomicAdd(&cnt_b[c[u]], (unsigned)__popc(pm));
      }
    }
    // each lane reads its group leader's old count with one whole-warp indexed shuffle (a
    // shuffle over each group's own mask would split the warp into one pass per group)
#pragma unroll
    for (int u = 0; u < kVoxU; ++u) {
      const int leader = peers[u] ? __ffs(peers[u]) - 1 : lane;
      const unsigned first = __shfl_sync(kFull, base[u], leader);
      const int i = i0 + u * blockDim.x + threadIdx.x;
      if (c[u] >= 0) slot[(size_t)b * cap + i] = (int)first + __popc(peers[u] & ((1u << lane) - 1u));
    }
  }
}

// Sums of (occupied, points) over one tile of kVoxTile cells; 256 threads.
__global__ void vox_tile_sums(Geom g, const unsigned* __restrict__ cnt, int2* __restrict__ sums,
                              int ntiles) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const int b = blockIdx.y;
  const unsigned* c = cnt + (size_t)b * g.G;
  const int base = blockIdx.x * kVoxTile;
  int occ = 0, pts = 0;
  for (int j = threadIdx.x; j < kVoxTile; j += blockDim.x) {
    const int k = base + j;
    const unsigned v = k < g.G ? c[k] : 0u;
    occ += v != 0u;
    pts += (int)v;
  }
  for (int o = 16; o; o >>= 1) {
    occ += __shfl_xor_sync(kFull, occ, o);
    pts += __shfl_xor_sync(kFull, pts, o);
  }
  __shared__ int2 red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_int2(occ, pts);
  __syncthreads();
  if (threadIdx.x == 0) {
    int2 t = make_int2(0, 0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t.x += red[w].x; t.y += red[w].y; }
    sums[(size_t)b * ntiles + blockIdx.x] = t;
  }
}

// Pillar ranks over one tile of kVoxTile cells, 256 threads: warp w owns the 256 consecutive
// cells from base + 256 w as 8 rows of 32 (lane l takes cell 32 i + l of row i), so every load
// and store of a row is one coalesced 128-byte line.  A cell's rank (pillar id, kept if < P) is
// the number of occupied cells before it in the frame and its first point offset the number of
// points before it: the preceding tiles' sums, plus the preceding warps' totals in this tile,
// plus a warp scan along the rows.
__global__ void __launch_bounds__(256) vox_scan(Geom g, const unsigned* __restrict__ cnt,
                                                const int2* __restrict__ sums, int ntiles,
                                                int* __restrict__ pillar_of_cell,
                                                int* __restrict__ coord, int* __restrict__ npts,
                                                int* __restrict__ pillar_start,
                                                int* __restrict__ pillar_cnt,
                                                int* __restrict__ num_pillars,
                                                unsigned* __restrict__ cnt_starts) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const int b = blockIdx.y;
  const unsigned* c = cnt + (size_t)b * g.G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ int2 pre_red[8], warp_tot[8];
  // prefix of the preceding tiles' sums
  int2 pre = make_int2(0, 0);
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += blockDim.x) {
    const int2 s = sums[(size_t)b * ntiles + t];
    pre.x += s.x; pre.y += s.y;
  }
  for (int o = 16; o; o >>= 1) {
    pre.x += __shfl_xor_sync(kFull, pre.x, o);
    pre.y += __shfl_xor_sync(kFull, pre.y, o);
  }
  if (lane == 0) pre_red[wid] = pre;
  const int wbase = blockIdx.x * kVoxTile + wid * 256;
  unsigned v[8];
  int2 tot = make_int2(0, 0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = wbase + 32 * i + lane;
    v[i] = k < g.G ? c[k] : 0u;
    tot.x += v[i] != 0u;
    tot.y += (int)v[i];
  }
  for (int o = 16; o; o >>= 1) {
    tot.x += __shfl_xor_sync(kFull, tot.x, o);
    tot.y += __shfl_xor_sync(kFull, tot.y, o);
  }
  if (lane == 0) warp_tot[wid] = tot;
  __syncthreads();
  int2 before = make_int2(0, 0), tile = make_int2(0, 0);
  pre = make_int2(0, 0);
  for (int w = 0; w < 8; ++w) {
    pre.x += pre_red[w].x; pre.y += pre_red[w].y;
    tile.x += warp_tot[w].x; tile.y += warp_tot[w].y;
    if (w < wid) { before.x += warp_tot[w].x; before.y += warp_tot[w].y; }
  }
  int rank = pre.x + before.x, start = pre.y + before.y;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = wbase + 32 * i + lane;
    const int occ = v[i] != 0u ? 1 : 0, pts = (int)v[i];
    int io = occ, ip = pts;  // inclusive scan along the row
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(kFull, io, o);
      const int d = __shfl_up_sync(kFull, ip, o);
      if (lane >= o) { io += a; ip += d; }
    }
    if (k < g.G) {
      const int r = rank + io - occ;
      int pid = -1;
      if (occ && r < g.P) {
        pid = r;
        const size_t q = (size_t)b * g.P + r;
        coord[q] = k;
        npts[q] = pts < 32 ? pts : 32;
        pillar_start[q] = start + ip - pts;
        pillar_cnt[q] = pts;
      }
      pillar_of_cell[(size_t)b * g.G + k] = pid;
      // a release unit: the count becomes the bucket pass's lookup -- a kept cell's first point
      // offset + 1, zero for a cell the pillar cap dropped (this CTA is the count's last
      // reader; the PointNet pass zeroes the kept cells' entries for the next launch)
      if (cnt_starts && occ) cnt_starts[(size_t)b * g.G + k] = pid >= 0 ? (unsigned)(start + ip - pts) + 1u : 0u;
    }
    rank += __shfl_sync(kFull, io, 31);
    start += __shfl_sync(kFull, ip, 31);
  }
  if (blockIdx.x == (unsigned)(ntiles - 1) && threadIdx.x == 0) {
    const int all = pre.x + tile.x;
    num_pillars[b] = all < g.P ? all : g.P;
  }
}

__global__ void vox_bucket(Geom g, int cap, const int* __restrict__ n_points,
                           const int* __restrict__ cell, const int* __restrict__ slot,
                           const int* __restrict__ pillar_of_cell,
                           const int* __restrict__ pillar_start, int* __restrict__ csr,
                           const unsigned* __restrict__ cnt_starts, int chunks,
                           const int* __restrict__ drawn, const int* __restrict__ drawn_num,
                           uint4* __restrict__ canvas, uint4* __restrict__ lo) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const int b = blockIdx.y;
  if (canvas) {
    // a release unit's canvas: zero the cells drawn for this slot's previous frame that hold no
    // kept pillar now (the scan has completed, so pillar_of_cell is this frame's); the cells
    // that do hold one are rewritten by the PointNet pass that follows, never touched here
    const size_t work = (size_t)drawn_num[b] * chunks;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < work; t += (size_t)gridDim.x * blockDim.x) {
      const int j = (int)(t / chunks), chunk = (int)(t % chunks);
      const int c = drawn[(size_t)b * g.P + j];
      if (pillar_of_cell[(size_t)b * g.G + c] >= 0) continue;
      const size_t off = dev::canvas_pixel(g, b, c) * chunks + chunk;
      canvas[off] = make_uint4(0u, 0u, 0u, 0u);
      if (lo) lo[off] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  const int n = frame_points(n_points, b, cap, nullptr);
  const size_t rb = (size_t)b * cap;
  // kVoxU points per thread per pass, each dependent load issued for all of them at once
  for (int i0 = blockIdx.x * blockDim.x * kVoxU; i0 < n; i0 += gridDim.x * blockDim.x * kVoxU) {
    int c[kVoxU], sl[kVoxU], p[kVoxU];
#pragma unroll
    for (int u = 0; u < kVoxU; ++u) {
      const int i = i0 + u * blockDim.x + threadIdx.x;
      c[u] = i < n ? cell[rb + i] : -1;
      sl[u] = i < n ? slot[rb + i] : 0;
    }
    if (cnt_starts) {
      // a release unit: one lookup per point, the cell's first point offset + 1 left by the
      // scan (0: the cell was dropped by the pillar cap)
      unsigned st[kVoxU];
#pragma unroll
      for (int u = 0; u < kVoxU; ++u) st[u] = c[u] >= 0 ? cnt_starts[(size_t)b * g.G + c[u]] : 0u;
#pragma unroll
      for (int u = 0; u < kVoxU; ++u)
        if (st[u]) csr[rb + (st[u] - 1u) + sl[u]] = i0 + u * blockDim.x + threadIdx.x;
      continue;
    }
#pragma unroll
    for (int u = 0; u < kVoxU; ++u) p[u] = c[u] >= 0 ? pillar_of_cell[(size_t)b * g.G + c[u]] : -1;
#pragma unroll
    for (int u = 0; u < kVoxU; ++u)
      if (p[u] >= 0) csr[rb + pillar_start[(size_t)b * g.P + p[u]] + sl[u]] = i0 + u * blockDim.x + threadIdx.x;
  }
}

__global__ void __launch_bounds__(256) vox_select(Geom g, int cap,
                                                  const float4* __restrict__ points,
                                                  const float4* const* __restrict__ srcs,
                                                  const int* __restrict__ csr,
                                                  const int* __restrict__ pillar_start,
                                                  const int* __restrict__ pillar_cnt,
                                                  const int* __restrict__ num_pillars,
                                                  float4* __restrict__ pts) {
  pdl_wait();  // predecessor's outputs complete and visible (exiting lets the next kernel launch)
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= num_pillars[b]) return;  // warp-uniform
  const size_t q = (size_t)b * g.P + p;
  const int count = pillar_cnt[q];
  const int* seg = csr + (size_t)b * cap + pillar_start[q];
  const int best = dev::lowest_32(seg, count, lane);
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (lane < count) out = frame_src(points, srcs, b, cap)[best];
  pts[q * 32 + lane] = out;
}

}  // namespace

size_t vox_workspace_bytes(const Geom& g, int batch, int cap) {
  const int ntiles = (g.G + kVoxTile - 1) / kVoxTile;
  size_t s = 256;                                            // err
  s += align_up((size_t)batch * cap * sizeof(int), 256) * 2;  // slot, csr
  s += align_up((size_t)batch * g.P * sizeof(int), 256) * 2;  // pillar_start, pillar_cnt
  s += align_up((size_t)batch * ntiles * sizeof(int2), 256);
  return s;
}

VoxWork vox_carve(void* ws, const Geom& g, int batch, int cap) {
  VoxWork w;
  char* p = static_cast<char*>(ws);
  w.ntiles = (g.G + kVoxTile - 1) / kVoxTile;
  w.err = reinterpret_cast<int*>(p);
  p += 256;
  w.slot = reinterpret_cast<int*>(p);
  p += align_up((size_t)batch * cap * sizeof(int), 256);
  w.csr = reinterpret_cast<int*>(p);
  p += align_up((size_t)batch * cap * sizeof(int), 256);
  w.pillar_start = reinterpret_cast<int*>(p);
  p += align_up((size_t)batch * g.P * sizeof(int), 256);
  w.pillar_cnt = reinterpret_cast<int*>(p);
  p += align_up((size_t)batch * g.P * sizeof(int), 256);
  w.tile_sums = reinterpret_cast<int2*>(p);
  return w;
}

int vox_launch(const Geom& g, int batch, int cap, const float4* points, const int* n_points,
               int* cell, unsigned* cnt, int* pillar_of_cell, int* coord, int* npts,
               int* num_pillars, float4* pts, const VoxWork& w, cudaStream_t s,
               const float4* const* srcs, float4* const* mirrors, const VoxUnitIO* io) {
  const VoxUnitIO none;
  if (!io) io = &none;
  cudaError_t e = cudaSuccess;
  if (!io->cnt_clean) e = cudaMemsetAsync(cnt, 0, (size_t)batch * g.G * sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_status(e, "memset cnt");
  // point kernels: grid-stride, about 8 blocks of 256 threads per SM over the whole batch (a
  // grid sized for the capacity costs microseconds of empty blocks when frames are short)
  const int sms = device_sms();
  int px = (cap + 256 * kVoxU - 1) / (256 * kVoxU);
  const int px_max = (8 * sms + batch - 1) / batch;
  if (px > px_max) px = px_max;
  const dim3 pg(px > 0 ? px : 1, batch);
  // dependent launches throughout (the count's predecessor may also be the counts' memset)
  // the first kernel reads the unit table's host copy (its device copy is written by this kernel)
  e = launch_pdl(vox_cell_count, pg, dim3(256), 0, s, g, cap, points, io->first_srcs ? io->first_srcs : srcs,
                 io->first_mirrors ? io->first_mirrors : mirrors,
                 io->first_counts ? io->first_counts : n_points, cell, w.slot, cnt, w.err, io->table_src,
                 io->table_dst, io->table_words);
  if (e == cudaSuccess)
    e = launch_pdl(vox_tile_sums, dim3(w.ntiles, batch), dim3(256), 0, s, g, (const unsigned*)cnt, w.tile_sums,
                   w.ntiles);
  if (e == cudaSuccess)
    e = launch_pdl(vox_scan, dim3(w.ntiles, batch), dim3(256), 0, s, g, (const unsigned*)cnt,
                   (const int2*)w.tile_sums, w.ntiles, pillar_of_cell, coord, npts, w.pillar_start, w.pillar_cnt,
                   num_pillars, io->cnt_clean ? cnt : (unsigned*)nullptr);
  if (e == cudaSuccess)
    e = launch_pdl(vox_bucket, pg, dim3(256), 0, s, g, cap, n_points, (const int*)cell, (const int*)w.slot,
                   (const int*)pillar_of_cell, (const int*)w.pillar_start, w.csr,
                   io->cnt_clean ? cnt : (unsigned*)nullptr, io->canvas_chunks, io->drawn,
                   io->drawn_num, io->canvas, io->canvas_lo);
  if (e == cudaSuccess && pts)
    e = launch_pdl(vox_select, dim3((g.P + 7) / 8, batch), dim3(256), 0, s, g, cap, points, srcs,
                   (const int*)w.csr, (const int*)w.pillar_start, (const int*)w.pillar_cnt,
                   (const int*)num_pillars, pts);
  return cuda_status(e, "voxelize launch");
}

}  // namespace pp
