// Peak arithmetic rates of the device (measurement support for the rooflines): independent
// fused multiply-add chains on every SM, timed with CUDA events.  Nothing here changes a
// clock, power or any other device setting.
#include "dwf_internal.h"

namespace dwf {
namespace {

constexpr int kChains = 8;     // independent FMA chains per thread (covers the FMA latency)

// Each thread runs kChains independent chains x <- x * a + b for `iters` steps; the result is
// stored only if it equals an impossible value, so the compiler keeps the work and no store
// happens.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T a, T b, int iters, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = T(threadIdx.x + c);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  if (s == T(-12345.0)) sink[threadIdx.x] = s;
}

template <typename T>
dwf_status measure(cudaStream_t st, int iters, double* tflops) {
  int dev = 0, sms = 0;
  DWF_CUDA(cudaGetDevice(&dev));
  DWF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  // a = 1, b = 0 keep the chains finite; the values do not affect the FMA rate
  const T a = T(1), b = T(0);
  cudaEvent_t e0, e1;
  DWF_CUDA(cudaEventCreate(&e0));
  DWF_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  dwf_status status = DWF_OK;
  for (int rep = 0; rep < 4; rep++) {   // the first launch warms up and is not counted
    cudaEventRecord(e0, st);
    fma_peak_kernel<T><<<blocks, threads, 0, st>>>(a, b, iters, nullptr);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      status = cuda_error(e, "fma_peak_kernel");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != DWF_OK) return status;
  const double flops = 2.0 * (double)blocks * threads * kChains * iters;
  *tflops = flops / (best * 1e-3) / 1e12;
  return DWF_OK;
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_measure_peak(int which, void* stream, double* tflops) {
  if (!tflops) return set_error(DWF_ERR_ARG, "null tflops");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // FP64: ~20 GFLOP per launch (tens of ms at ~1 TFLOP/s); FP32: 16x the work
  if (which == 0) return measure<double>(st, 4096, tflops);
  if (which == 1) return measure<float>(st, 65536, tflops);
  return set_error(DWF_ERR_ARG, "which must be 0 (FP64) or 1 (FP32)");
}
