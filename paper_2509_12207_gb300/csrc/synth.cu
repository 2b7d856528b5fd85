// Synthetic GPU load for the robustness experiments (the paper's study of kernel utilisation and
// kernel execution time, Section 6.6): a frame of a synthetic chain runs n kernels of a
// vector-add style operation whose execution time and GPU utilisation are set by the chain.
//
// Utilisation = the fraction of the SMs a kernel occupies: it launches ctas = round(util x SMs)
// CTAs of 256 threads, each holding 116 KiB of (unused) shared memory so that no SM can take
// two of them: every CTA has an SM to itself.  Execution time: every CTA streams `iters` passes over its
// own 32 KiB slices of a, b and c (c = 0.5 c + a + s b, s the pass index, so that no pass can be
// dropped or merged by the compiler); the per-pass time is calibrated once per chain, so iters =
// kernel_us / (time per pass).  The slices stay in L2, so a synthetic kernel competes for SMs
// and L2, not for HBM.
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int kSlice = 2048;                 // float4 per CTA and array (32 KiB)
constexpr int kHoldSmem = 116 * 1024;        // > half of an SM's shared memory: one CTA per SM

__global__ void __launch_bounds__(256) synth_vadd(const float4* a, const float4* b, float4* c, int iters) {
  const size_t base = (size_t)blockIdx.x * kSlice;
  for (int it = 0; it < iters; ++it) {
    const float s = (float)it;
    for (int i = threadIdx.x; i < kSlice; i += blockDim.x) {
      const float4 x = a[base + i], y = b[base + i];
      float4 z = c[base + i];
      z.x = 0.5f * z.x + x.x + s * y.x;
      z.y = 0.5f * z.y + x.y + s * y.y;
      z.z = 0.5f * z.z + x.z + s * y.z;
      z.w = 0.5f * z.w + x.w + s * y.w;
      c[base + i] = z;
    }
  }
}

}  // namespace

int synth_alloc(SynthBuf* b, int units) {
  int dev = 0;
  int st = cuda_status(cudaGetDevice(&dev), "synthetic load: device");
  if (!st) st = cuda_status(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (st) return st;
  b->units = units;
  const size_t arr = (size_t)b->sms * kSlice * sizeof(float4);
  if (cudaMalloc(&b->ab, 2 * arr) != cudaSuccess || cudaMalloc(&b->c, (size_t)units * arr) != cudaSuccess) {
    cudaGetLastError();
    synth_free(b);
    return fail(PP_ENOMEM, "synthetic load: device buffers");
  }
  st = cuda_status(cudaFuncSetAttribute(synth_vadd, cudaFuncAttributeMaxDynamicSharedMemorySize, kHoldSmem),
                   "synthetic load: smem attribute");
  if (!st) st = cuda_status(cudaMemset(b->ab, 0, 2 * arr), "synthetic load: clear");
  if (!st) st = cuda_status(cudaMemset(b->c, 0, (size_t)units * arr), "synthetic load: clear");
  return st;
}

void synth_free(SynthBuf* b) {
  if (b->ab) cudaFree(b->ab);
  if (b->c) cudaFree(b->c);
  b->ab = nullptr;
  b->c = nullptr;
}

int synth_ctas(const SynthBuf& b, double util) {
  int n = (int)(util * b.sms + 0.5);
  return n < 1 ? 1 : (n > b.sms ? b.sms : n);
}

int synth_launch(const SynthBuf& b, int unit, int ctas, int iters, int n_kernels, cudaStream_t s) {
  if (unit < 0 || unit >= b.units || ctas < 1 || ctas > b.sms || iters < 1 || n_kernels < 1)
    return fail(PP_EINVAL, "synthetic load: bad launch");
  const float4* a = static_cast<const float4*>(b.ab);
  const float4* bb = a + (size_t)b.sms * kSlice;
  float4* c = static_cast<float4*>(b.c) + (size_t)unit * b.sms * kSlice;
  for (int k = 0; k < n_kernels; ++k) synth_vadd<<<ctas, 256, kHoldSmem, s>>>(a, bb, c, iters);
  return cuda_status(cudaGetLastError(), "synthetic load: launch");
}

// Times a launch at 8 and at 64 passes (after a warm-up) and solves t = t0 + k iters for the
// passes that take kernel_us.
int synth_calibrate(const SynthBuf& b, int ctas, double kernel_us, cudaStream_t s, int* iters) {
  cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
  int st = PP_OK;
  for (auto& x : e)
    if (!st) st = cuda_status(cudaEventCreate(&x), "synthetic load: event");
  if (!st) st = synth_launch(b, 0, ctas, 8, 1, s);
  if (!st) st = cuda_status(cudaEventRecord(e[0], s), "synthetic load: calibrate");
  if (!st) st = synth_launch(b, 0, ctas, 8, 1, s);
  if (!st) st = cuda_status(cudaEventRecord(e[1], s), "synthetic load: calibrate");
  if (!st) st = synth_launch(b, 0, ctas, 64, 1, s);
  if (!st) st = cuda_status(cudaEventRecord(e[2], s), "synthetic load: calibrate");
  if (!st) st = cuda_status(cudaEventSynchronize(e[2]), "synthetic load: calibrate");
  float t8 = 0, t64 = 0;
  if (!st) st = cuda_status(cudaEventElapsedTime(&t8, e[0], e[1]), "synthetic load: calibrate");
  if (!st) st = cuda_status(cudaEventElapsedTime(&t64, e[1], e[2]), "synthetic load: calibrate");
  for (auto& x : e)
    if (x) cudaEventDestroy(x);
  if (st) return st;
  const double k = (t64 - t8) * 1000.0 / 56.0;  // us per pass
  const double t0 = t8 * 1000.0 - 8.0 * k;
  double n = k > 0 ? (kernel_us - t0) / k : 1.0;
  n = n < 1.0 ? 1.0 : (n > 1e7 ? 1e7 : n);
  *iters = (int)(n + 0.5);
  return PP_OK;
}

}  // namespace pp
