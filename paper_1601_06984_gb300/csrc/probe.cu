// lbm_alu_peak: measured fused multiply-add rate of this GPU, the denominator
// of the ALU roofline of the FP64 stream-collide (the method itself is
// bandwidth bound in FP32 and BF16 storage; in FP64 storage GB300's FP64 pipe
// is the limit).  The paper has no counterpart: this is a diagnostic of the
// library.
//
// Every thread runs kChains independent multiply-add chains of kIters steps on
// values that stay finite (a x + b with |a| < 1), so the pipe is kept busy with
// no memory traffic; one value per thread is stored so the work is not
// removed.  Rate = 2 kChains kIters threads / time (a multiply-add counts as
// two floating-point operations), timed with CUDA events on a private stream
// around kReps launches after one warm-up launch.
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int kChains = 16;
constexpr int kIters = 2048;
constexpr int kReps = 5;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(T* out, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = T(threadIdx.x + c) * T(1e-3);
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <class T>
lbm_status run(void* scratch, uint64_t bytes, double* gflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LBM_ERR_CUDA;
  // whole waves of resident 256-thread blocks: FP64 (40 registers a thread)
  // fits six per SM, one wave of a few milliseconds on this part's narrow
  // FP64 pipe; FP32 (31 registers) eight per SM, two waves
  const int blocks = sms * (sizeof(T) == 8 ? 6 : 16);
  if (bytes < (uint64_t)blocks * kThreads * sizeof(T)) return LBM_ERR_ARG;
  T* out = static_cast<T*>(scratch);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  lbm_status s = LBM_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    s = LBM_ERR_CUDA;
  float ms = 0.f;
  if (s == LBM_OK) {
    k_fma_probe<T><<<blocks, kThreads, 0, st>>>(out, T(0.999), T(1e-4));
    cudaEventRecord(e0, st);
    for (int r = 0; r < kReps; ++r) k_fma_probe<T><<<blocks, kThreads, 0, st>>>(out, T(0.999), T(1e-4));
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
      s = LBM_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (s == LBM_OK) {
    const double flops = 2.0 * kChains * kIters * (double)blocks * kThreads * kReps;
    *gflops = flops / (ms * 1e-3) / 1e9;
  }
  return s;
}

}  // namespace

extern "C" lbm_status lbm_alu_peak(int32_t precision, void* device_scratch, uint64_t bytes, double* gflops) {
  if (!device_scratch || !gflops) return LBM_ERR_ARG;
  if (precision == LBM_FP64) return run<double>(device_scratch, bytes, gflops);
  if (precision == LBM_FP32DEV) return run<float>(device_scratch, bytes, gflops);
  return LBM_ERR_ARG;
}
