// Arithmetic throughput of the device for the roofline of the ALU-bound
// product kernels (the paper has no counterpart: a measurement aid).  Each
// thread runs eight independent fused multiply-add chains, so the issue rate
// of the FMA pipe, not its latency, bounds the loop.
#include <cuda_runtime.h>

#include <algorithm>

#include "problem.h"

namespace pie {

// Written only when the chains reach an impossible value, so that the
// compiler keeps the loop; never read.
static __device__ double g_peak_sink[2];

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, R b, R c) {
  R a0 = R(threadIdx.x), a1 = a0 + R(1), a2 = a0 + R(2), a3 = a0 + R(3);
  R a4 = a0 + R(4), a5 = a0 + R(5), a6 = a0 + R(6), a7 = a0 + R(7);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
    a4 = fma(a4, b, c);
    a5 = fma(a5, b, c);
    a6 = fma(a6, b, c);
    a7 = fma(a7, b, c);
  }
  const R s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == R(-1.2345e-30)) g_peak_sink[sizeof(R) == 8 ? 0 : 1] = double(s);
}

// Best of three timed launches (CUDA events) after ten untimed ones (the
// clocks ramp up from idle), in TFLOP/s (2 flop per FMA).
template <typename R>
static pie_status fma_peak(int nsm, int iters, cudaStream_t st, double* tflops) {
  const unsigned blocks = unsigned(nsm * 4);
  const double flops = 2.0 * 8.0 * double(iters) * double(blocks) * 256.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pie_status s = cuda_check(cudaEventCreate(&e0), "event");
  if (s == PIE_OK) s = cuda_check(cudaEventCreate(&e1), "event");
  for (int rep = 0; s == PIE_OK && rep < 10; ++rep)
    k_fma_chains<R><<<blocks, 256, 0, st>>>(iters, R(0.9999999), R(1e-7));
  double best = 0;
  for (int rep = 0; s == PIE_OK && rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_chains<R><<<blocks, 256, 0, st>>>(iters, R(0.9999999), R(1e-7));
    cudaEventRecord(e1, st);
    s = cuda_check(cudaEventSynchronize(e1), "peak probe");
    float ms = 0;
    if (s == PIE_OK) s = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "peak probe");
    if (s == PIE_OK && ms > 0) best = std::max(best, flops / (double(ms) * 1e-3) / 1e12);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *tflops = best;
  return s;
}

}  // namespace pie

using namespace pie;

extern "C" pie_status pie_measure_peaks(double* fp64_tflops, double* fp32_tflops, void* stream) {
  if (!fp64_tflops || !fp32_tflops) {
    set_error("pie_measure_peaks: NULL argument");
    return PIE_ERR_PARAM;
  }
  int dev = 0, nsm = 0;
  pie_status s = cuda_check(cudaGetDevice(&dev), "device");
  if (s == PIE_OK) s = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (s != PIE_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // about 20 ms per launch at GB300's nominal FP64 (1.25 TFLOP/s) and FP32 (80 TFLOP/s) rates
  s = fma_peak<double>(nsm, 10000, st, fp64_tflops);
  if (s == PIE_OK) s = fma_peak<float>(nsm, 600000, st, fp32_tflops);
  return s;
}
