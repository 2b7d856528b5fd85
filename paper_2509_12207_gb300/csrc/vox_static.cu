// pp_voxelize_static: pp_voxelize for callers that cannot allocate device memory.
//
// Its scratch (arrival slots, grouped point indices, per-pillar offsets, tile sums, error
// word) lives in one file-scope __device__ array of fixed size instead of a caller workspace.
// Every GPU that loads the library holds that array until the process exits.  Host code must
// not use the array's name as a device address (on the host it names a host-side shadow), so
// the device address is looked up with cudaGetSymbolAddress once per device and cached.
#include "pp_internal.h"

#include <mutex>

namespace pp {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)PP_VOX_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_vox_scratch[PP_VOX_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on first use).
int scratch_address(void** out) {
  int dev = 0;
  int st = cuda_status(cudaGetDevice(&dev), "voxelize_static: get device");
  if (st) return st;
  if (dev < 0 || dev >= kMaxDevices) return fail(PP_EINVAL, "voxelize_static: device %d unsupported", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    st = cuda_status(cudaGetSymbolAddress(&p, g_vox_scratch), "voxelize_static: cudaGetSymbolAddress");
    if (st) return st;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return PP_OK;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" int pp_voxelize_static(const pp_geometry* g, int32_t batch, int32_t cap_points,
                                  const float* points, const int32_t* n_points, int32_t* cell,
                                  uint32_t* cnt, int32_t* pillar_of_cell, int32_t* coord,
                                  int32_t* npts, int32_t* num_pillars, float* pts, void* stream) {
  Geom gg;
  int st = check_geometry(g, &gg);
  if (st) return st;
  if (batch <= 0 || batch > 4096 || cap_points < 0 || cap_points > (1 << 27))
    return fail(PP_EINVAL, "voxelize_static: batch or cap_points out of range");
  if (!n_points || !cnt || !pillar_of_cell || !coord || !npts || !num_pillars || !pts ||
      (cap_points > 0 && (!points || !cell)))
    return fail(PP_EINVAL, "voxelize_static: NULL buffer");
  if ((reinterpret_cast<uintptr_t>(points) | reinterpret_cast<uintptr_t>(pts)) & 15u)
    return fail(PP_EINVAL, "voxelize_static: points and pts must be 16-byte aligned");
  const size_t need = vox_workspace_bytes(gg, batch, cap_points);
  if (need > kStaticScratchBytes)
    return fail(PP_EINVAL,
                "voxelize_static: this batch needs %zu bytes of scratch, the static array holds "
                "%zu; use pp_voxelize with a caller workspace or a smaller batch",
                need, kStaticScratchBytes);
  void* scratch = nullptr;
  if ((st = scratch_address(&scratch))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents; the error word must start at zero (every
  // other scratch region is fully written before it is read within a call)
  if ((st = cuda_status(cudaMemsetAsync(scratch, 0, 256, s), "voxelize_static: clear error word")))
    return st;
  VoxWork w = vox_carve(scratch, gg, batch, cap_points);
  return vox_launch(gg, batch, cap_points, reinterpret_cast<const float4*>(points), n_points,
                    cell, cnt, pillar_of_cell, coord, npts, num_pillars,
                    reinterpret_cast<float4*>(pts), w, s);
}
