// Device helpers: interleaved complex arithmetic in float or double.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "problem.h"

namespace pie {

template <typename R>
__device__ __forceinline__ C2<R> mk(R x, R y) {
  C2<R> c;
  c.x = x;
  c.y = y;
  return c;
}
template <typename R>
__device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
template <typename R>
__device__ __forceinline__ void cfma(C2<R>& acc, C2<R> a, C2<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cfma_conj(C2<R>& acc, C2<R> a, C2<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += r * b (r real)
template <typename R>
__device__ __forceinline__ void rfma(C2<R>& acc, R r, C2<R> b) {
  acc.x = fma(r, b.x, acc.x);
  acc.y = fma(r, b.y, acc.y);
}
template <typename R, typename S>
__device__ __forceinline__ C2<R> cvt(C2<S> a) {
  return mk<R>(R(a.x), R(a.y));
}
// Scales of half-precision near moments (PIE_FP32H): value = stored * s[plane].
struct MomScale {
  float s[kMom];
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Asynchronous copy of one 8- or 16-byte element from global to shared
// memory (cp.async: the thread does not wait for the load, so a staging
// loop keeps all its loads in flight).  Completed by cp_async_wait_all,
// after which the issuing thread sees the element; other threads see it
// after a barrier.
template <typename T>
__device__ __forceinline__ void cp_async(T* dst_shared, const T* src_global) {
  static_assert(sizeof(T) == 8 || sizeof(T) == 16, "cp.async element of 8 or 16 bytes");
  const unsigned d = unsigned(__cvta_generic_to_shared(dst_shared));
  if constexpr (sizeof(T) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src_global) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src_global) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

}  // namespace pie
