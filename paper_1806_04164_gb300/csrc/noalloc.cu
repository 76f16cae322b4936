// Near-part product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a product:
// code running inside a CUDA-graph capture they do not control, a host that
// forbids allocation after start-up (fixed memory budgets, real-time loops),
// or a framework whose allocator owns all device memory.  For them,
// pie_apply_near_noalloc computes the same y = Z_near x as pie_apply_near but
// takes its per-triangle scratch (local coefficients and potentials) from the
// file-scope device array below instead of the problem's own buffers, and it
// calls no allocating routine.
#include "handles.h"

namespace pie {

// 24 MiB: coefficients + potentials, 2 x 6 complex per triangle, i.e. at most
// 131072 triangles for complex double and 262144 for complex float.  Every
// GPU that loads the library holds this array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(24) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the problem's device, looked up
// when the problem is created (pie_problem_create runs outside any stream
// capture, with that device current) and kept in the problem.  In host code
// the array's name is only a host-side stand-in, never a device address.
pie_status noalloc_bind(Problem& pr) {
  void* p = nullptr;
  pie_status s = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
  if (s == PIE_OK) pr.noalloc_scratch = p;
  return s;
}

}  // namespace pie


using namespace pie;

extern "C" pie_status pie_apply_near_noalloc(pie_problem* h, const void* x, void* y, int dtype, void* stream) {
  if (!h || !x || !y) {
    set_error("pie_apply_near_noalloc: NULL argument");
    return PIE_ERR_PARAM;
  }
  Problem& pr = h->p;
  const int want = pr.io_f32() ? PIE_C64 : PIE_C128;
  if (dtype != want) {
    set_error("pie_apply_near_noalloc: dtype does not match the problem precision");
    return PIE_ERR_PARAM;
  }
  const size_t es = pr.io_f32() ? sizeof(cf) : sizeof(cd);
  const size_t half = size_t(6) * es * size_t(pr.T);
  const size_t need = 2 * ((half + 255) / 256) * 256;
  if (need > kNoAllocScratchBytes) {
    set_error("pie_apply_near_noalloc: mesh too large for the fixed scratch (" + std::to_string(pr.T) +
              " triangles; the limit is " + std::to_string(kNoAllocScratchBytes / (12 * es)) + ")");
    return PIE_ERR_PARAM;
  }
  pie_status s = check_device(pr, "pie_apply_near_noalloc");
  if (s != PIE_OK) return s;
  char* coef = static_cast<char*>(pr.noalloc_scratch);
  char* pot = coef + need / 2;
  return apply_near_scratch(pr, x, y, coef, pot, static_cast<cudaStream_t>(stream));
}
