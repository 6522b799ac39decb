// FMA-rate probe (include/dg_probe.h): independent fused multiply-add chains
// per thread, enough warps per SM to hide the pipe latency, timed with CUDA
// events.  Each chain computes a <- a * m + c with m and c kernel parameters,
// so the compiler can neither fold nor shorten the loop; the chains' sum is
// stored so that nothing is dead.
#include <cuda_runtime.h>

#include "../../include/dg_probe.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename R>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int iters, R m, R c, R* __restrict__ out) {
  R a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = R(threadIdx.x + 1) * R(1e-3) + R(i);
  // unrolled by 4 so that the loop's own instructions (counter, compare,
  // branch) are a small fraction of the issued ones
#pragma unroll 4
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
  }
  R s = R(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

template <typename R>
dg_status run(int repeats, void* scratch, cudaStream_t s, double* out) {
  const int sms = sm_count();
  if (sms <= 0) return DG_ERR_CUDA;
  const int blocks = sms * kBlocksPerSM;
  // about 5 GFLOP per launch in FP64 and 80 GFLOP in FP32 (a few ms each)
  const int iters = sizeof(R) == 8 ? 1024 : 16384;
  R* o = static_cast<R*>(scratch);
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return DG_ERR_CUDA;
  }
  const R m = R(0.9999999), c = R(1e-7);
  // untimed launches first, so that the clocks have left their idle state
  for (int w = 0; w < 5; ++w) fma_chains_kernel<R><<<blocks, kThreads, 0, s>>>(iters, m, c, o);
  cudaEventRecord(a, s);
  for (int r = 0; r < repeats; ++r) fma_chains_kernel<R><<<blocks, kThreads, 0, s>>>(iters, m, c, o);
  cudaEventRecord(b, s);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess || !(ms > 0.f)) return DG_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads * repeats;
  *out = flops / (ms * 1e-3);
  return DG_OK;
}

}  // namespace

extern "C" {

size_t dg_probe_scratch_bytes(void) {
  const int sms = sm_count();
  const size_t n = (size_t)(sms > 0 ? sms : 1) * kBlocksPerSM * kThreads * sizeof(double);
  return (n + 4095) & ~size_t(4095);
}

dg_status dg_probe_fma_rate(int precision, int repeats, void* scratch, void* stream, double* out_flops_per_second) {
  if (!out_flops_per_second || !scratch || repeats < 1 || repeats > 1000) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == DG_PREC_FP64) return run<double>(repeats, scratch, s, out_flops_per_second);
  if (precision == DG_PREC_FP32) return run<float>(repeats, scratch, s, out_flops_per_second);
  return DG_ERR_ARG;
}

}  // extern "C"
