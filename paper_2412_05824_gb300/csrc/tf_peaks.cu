// turbofft_fma_peak: measured fused multiply-add throughput of the device
// (the roofline denominator of kernels bound by floating-point arithmetic).
//
// GB300 runs float64 at a small fraction of its float32 rate, so the float64
// transforms are bound by the FP64 pipe rather than by HBM; their roofline
// fraction needs the FP64 rate this device reaches, not a nominal figure.
// Every thread runs CHAINS independent FMA recurrences x <- x * a + b (a
// close to 1, b tiny, so values stay finite and normal) for `iters`
// iterations; the chains are independent, so the pipe, not the latency of one
// FMA, sets the time.  2 flops per FMA.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/turbofft.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop(T a, T b, int iters, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // the result is stored only if it is a value no input can produce, so the
  // loop cannot be removed and the store never happens in practice
  if (s == (T)-12345.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
turbofft_status run(double seconds, cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    return TURBOFFT_CUDA_ERROR;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_loop<T>, kThreads, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return TURBOFFT_CUDA_ERROR;
  }
  const int grid = sms * per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return TURBOFFT_CUDA_ERROR;
  }
  const T a = (T)0.9999999, b = (T)1e-7;
  turbofft_status status = TURBOFFT_SUCCESS;
  // calibrate the iteration count on a short launch, then time launches of
  // about 50 ms each until `seconds` have passed; keep the best rate
  int iters = 1 << 12;
  float ms = 0.f;
  double best = 0.0, total_ms = 0.0;
  for (int round = 0; round < 1000; ++round) {
    cudaEventRecord(e0, st);
    fma_loop<T><<<grid, kThreads, 0, st>>>(a, b, iters, (T*)nullptr);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      status = TURBOFFT_CUDA_ERROR;
      break;
    }
    const double flops = 2.0 * kChains * (double)iters * (double)grid * kThreads;
    if (ms > 10.f) {
      best = std::max(best, flops / (ms * 1e-3) / 1e12);
      total_ms += ms;
      if (total_ms >= seconds * 1e3) break;
    }
    if (ms < 40.f && iters < (1 << 28)) iters = (int)std::min<double>((double)(1 << 28), iters * std::max(2.0, 50.0 / std::max(ms, 0.01f)));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status == TURBOFFT_SUCCESS) *tflops = best;
  return status;
}

}  // namespace

extern "C" turbofft_status turbofft_fma_peak(turbofft_dtype dtype, double seconds, turbofft_stream stream,
                                             double* tflops) {
  if (!tflops || !(seconds > 0.0) || seconds > 60.0) return TURBOFFT_INVALID_VALUE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == TURBOFFT_C2C_F32) return run<float>(seconds, st, tflops);
  if (dtype == TURBOFFT_C2C_F64) return run<double>(seconds, st, tflops);
  return TURBOFFT_INVALID_VALUE;
}
