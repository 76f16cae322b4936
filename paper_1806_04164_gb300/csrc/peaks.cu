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
// SM clock ticks and nanoseconds over one launch, read by thread 0 of block 0
static __device__ unsigned long long g_peak_clock[2];

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ACC = false: a_i = a_i b + c (the chain value is the multiplicand);
// ACC = true: a_i = x_i y + a_i (the chain value is the addend, the form of
// an accumulating complex multiply-add; x_i and y are loop invariants in
// registers).
template <typename R, bool ACC>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, R b, R c) {
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  const long long c0 = clock64();
  const unsigned long long t0 = timer ? global_ns() : 0;
  R a0 = R(threadIdx.x), a1 = a0 + R(1), a2 = a0 + R(2), a3 = a0 + R(3);
  R a4 = a0 + R(4), a5 = a0 + R(5), a6 = a0 + R(6), a7 = a0 + R(7);
  const R y = b * R(blockIdx.x & 7), x0 = c * a0, x1 = c * a1, x2 = c * a2, x3 = c * a3;
  const R x4 = c * a4, x5 = c * a5, x6 = c * a6, x7 = c * a7;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    if constexpr (ACC) {
      a0 = fma(x0, y, a0);
      a1 = fma(x1, y, a1);
      a2 = fma(x2, y, a2);
      a3 = fma(x3, y, a3);
      a4 = fma(x4, y, a4);
      a5 = fma(x5, y, a5);
      a6 = fma(x6, y, a6);
      a7 = fma(x7, y, a7);
    } else {
      a0 = fma(a0, b, c);
      a1 = fma(a1, b, c);
      a2 = fma(a2, b, c);
      a3 = fma(a3, b, c);
      a4 = fma(a4, b, c);
      a5 = fma(a5, b, c);
      a6 = fma(a6, b, c);
      a7 = fma(a7, b, c);
    }
  }
  const R s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == R(-1.2345e-30)) g_peak_sink[sizeof(R) == 8 ? 0 : 1] = double(s);
  if (timer) {
    g_peak_clock[0] = (unsigned long long)(clock64() - c0);
    g_peak_clock[1] = global_ns() - t0;
  }
}

// Best of three timed launches (CUDA events) after ten untimed ones (the
// clocks ramp up from idle), in TFLOP/s (2 flop per FMA), and the SM clock
// (MHz) block 0 saw during the best launch (clock64 ticks over globaltimer
// nanoseconds): long FMA streams can run below the maximum clock under the
// power limit, so the rate per clock is the hardware figure.  Raises
// *tflops (and sets *mhz) only when this form beats the value passed in.
template <typename R, bool ACC>
static pie_status fma_peak(int nsm, int blocks_per_sm, int iters, cudaStream_t st, double* tflops, double* mhz) {
  const unsigned blocks = unsigned(nsm * blocks_per_sm);
  const double flops = 2.0 * 8.0 * double(iters) * double(blocks) * 256.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pie_status s = cuda_check(cudaEventCreate(&e0), "event");
  if (s == PIE_OK) s = cuda_check(cudaEventCreate(&e1), "event");
  for (int rep = 0; s == PIE_OK && rep < 10; ++rep)
    k_fma_chains<R, ACC><<<blocks, 256, 0, st>>>(iters, R(0.9999999), R(1e-7));
  double best = *tflops;
  for (int rep = 0; s == PIE_OK && rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_chains<R, ACC><<<blocks, 256, 0, st>>>(iters, R(0.9999999), R(1e-7));
    cudaEventRecord(e1, st);
    s = cuda_check(cudaEventSynchronize(e1), "peak probe");
    float ms = 0;
    if (s == PIE_OK) s = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "peak probe");
    const double tf = flops / (double(ms) * 1e-3) / 1e12;
    if (s == PIE_OK && ms > 0 && tf > best) {
      best = tf;
      unsigned long long clk[2] = {0, 0};
      s = cuda_check(cudaMemcpyFromSymbol(clk, g_peak_clock, sizeof(clk)), "peak probe clock");
      *mhz = clk[1] > 0 ? double(clk[0]) / double(clk[1]) * 1e3 : 0.0;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *tflops = best;
  return s;
}

}  // namespace pie

using namespace pie;

extern "C" pie_status pie_measure_peaks(double* fp64_tflops, double* fp32_tflops, double* fp64_mhz, double* fp32_mhz,
                                        void* stream) {
  if (!fp64_tflops || !fp32_tflops || !fp64_mhz || !fp32_mhz) {
    set_error("pie_measure_peaks: NULL argument");
    return PIE_ERR_PARAM;
  }
  int dev = 0, nsm = 0;
  pie_status s = cuda_check(cudaGetDevice(&dev), "device");
  if (s == PIE_OK) s = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (s != PIE_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // about 20 ms per launch at GB300's nominal FP64 (1.25 TFLOP/s) and FP32
  // (80 TFLOP/s) rates; the best of both operand forms and of 4 and 8
  // blocks of 256 threads per SM
  *fp64_tflops = *fp32_tflops = 0;
  *fp64_mhz = *fp32_mhz = 0;
  for (int bps : {4, 8}) {
    if (s == PIE_OK) s = fma_peak<double, false>(nsm, bps, 40000 / bps, st, fp64_tflops, fp64_mhz);
    if (s == PIE_OK) s = fma_peak<double, true>(nsm, bps, 40000 / bps, st, fp64_tflops, fp64_mhz);
    if (s == PIE_OK) s = fma_peak<float, false>(nsm, bps, 2400000 / bps, st, fp32_tflops, fp32_mhz);
    if (s == PIE_OK) s = fma_peak<float, true>(nsm, bps, 2400000 / bps, st, fp32_tflops, fp32_mhz);
  }
  return s;
}
