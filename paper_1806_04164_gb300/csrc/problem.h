// Problem state shared by the host orchestration and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace pie {

template <typename R>
struct alignas(2 * sizeof(R)) C2 {
  R x, y;
};
typedef C2<double> cd;
typedef C2<float> cf;

constexpr int kComp = 5;      // radiated densities per box: mu0 J (3), sigma, d
constexpr int kNoffs = 316;   // one-box-buffer translation offsets
constexpr int kMom = 8;       // moments per triangle pair: m0, mt(3), ms(3), mts
constexpr int kStages = 8;    // coef, near, aggregation, interpolation, translation, anterpolation, disaggregation, assembly

struct LevelDev {
  int64_t nb = 0;
  int32_t* il_ptr = nullptr;   // [nb+1]
  int32_t* il_idx = nullptr;   // [nnz]
  int32_t* il_off = nullptr;   // [nnz]
  int32_t* child_start = nullptr;  // [nb+1] children at level l+1 (l < L)
  int32_t* parent = nullptr;   // [nb] parent box number at level l-1
  int8_t* octant = nullptr;    // [nb] octant of the box within its parent
  void* trans = nullptr;       // [316][P] translation operator (far precision)
  void* S = nullptr;           // [max_nrhs][nb][5][P]
  void* G = nullptr;           // [max_nrhs][nb][5][P]
  void* phase = nullptr;       // [8][P] interpolation phase for children (l < L)
  void* F = nullptr;           // [P][P] filter from level l+1 to l (l < L), F[p][p']
  void* Ft = nullptr;          // [P][P] its transpose
  void* Kf = nullptr;          // [2 ntheta][ntheta][ntheta] azimuthal blocks of F
  double kappa = 0;            // kappa_l = k0 / s_l
};

struct Problem {
  Mesh mesh;
  Tree tree;
  double k0 = 0, w = 0;
  pie_params par{};
  int P = 0;
  int64_t T = 0, E = 0, N = 0;
  int64_t nnz = 0;      // near pair entries
  int64_t nleaf = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;

  // tree-ordered triangle data
  int32_t* tri_edge = nullptr;   // [T*3]
  double* tri_c = nullptr;       // [T*3]  s l / (2A)
  double* tri_dcp = nullptr;     // [T*9]  c_t - p
  int64_t* perm = nullptr;       // [T] tree -> mesh
  int64_t* inv_perm = nullptr;   // [T] mesh -> tree
  int32_t* edge_tt = nullptr;    // [E*2] tree positions of T+, T-
  int8_t* edge_k = nullptr;      // [E*2] local edge slot in those triangles
  double* vert = nullptr;        // [T*9] vertices (tree order)
  double* cent = nullptr;        // [T*3]
  double* h2 = nullptr;          // [T]
  double* area = nullptr;        // [T]
  int32_t* leaf_of = nullptr;    // [T]
  int32_t* leaf_start = nullptr; // [nleaf+1]
  double* leaf_center = nullptr; // [nleaf*3]
  int32_t* near_ptr = nullptr;   // [nleaf+1]
  int32_t* near_idx = nullptr;
  int32_t* near_off = nullptr;   // per near-list entry: position of that box's sources in the test rows
  int64_t* row_ptr = nullptr;    // [T+1]

  // angular grid
  double* khat = nullptr;        // [P*3]
  double* wgt = nullptr;         // [P]
  double* rule7 = nullptr;       // [7][4] barycentric (3) + weight, 7-point rule
  std::vector<double> rule7_host;  // the same rule on the host
  double* rule64 = nullptr;      // [64][4] collapsed Gauss 8 x 8

  // operator tables
  void* mom = nullptr;           // [8][nnz] complex (near precision)
  void* Pi = nullptr;            // [T][P/2]
  void* M = nullptr;             // [T][3][P/2] radiation tables (half grid), triangle-major
  void* PiR = nullptr;           // [P/2][T]    the same tables, sample-major (receiving side)
  void* MR = nullptr;            // [3][P/2][T]
  std::vector<LevelDev> lev;     // [L+1]

  // per-stage CUDA-event profiling (pie_profile_begin / pie_profile_end)
  std::vector<cudaEvent_t> prof_ev;  // [max_applies][kStages][2]
  int prof_cap = 0, prof_n = 0;

  // work buffers
  void* coef = nullptr;          // [max_nrhs][T][6] complex (io precision)
  void* coef32 = nullptr;        // [T][6] complex float copy for the MIXED near part
  void* gsgd = nullptr;          // 2 x [max_nrhs][nleaf][5][P/2] antipodal sum / difference leaf patterns
  void* vec = nullptr;           // [N] complex (io precision), adjoint scratch
  void* vec2 = nullptr;          // [N] complex (io precision), single-layer scratch
  void* pot = nullptr;           // [max_nrhs][T][6] far-part potentials (near part too when pot2 is unused)
  void* pot2 = nullptr;          // [max_nrhs][T][6] near-part potentials of the full product
  // when tune.overlap is set the near part runs on `side` (default
  // priority) and the far part on `far`, a stream of the device's highest
  // priority, both forked from and joined back into the caller's stream: the
  // far part's short, latency-bound kernels then take SM slots ahead of the
  // near part's many blocks instead of queueing behind them
  cudaStream_t side = nullptr, far = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_far = nullptr;
  int nsm = 0;                   // SMs of the device
  int device = 0;                // the device the problem was built on (current at pie_problem_create)
  void* noalloc_scratch = nullptr;  // device address of the fixed scratch of pie_apply_near_noalloc
  pie_tuning tune{1, 2, 1, 0, 0, 0};
  // parts of the product that run (pie_apply_levels): translations at the
  // levels whose bit is set, and the near part
  uint32_t far_mask = 0xffffffffu;
  bool with_near = true;

  // PIE_FP32H: moments stored as half pairs, value = stored * mom_scale[plane]
  float mom_scale[kMom] = {1, 1, 1, 1, 1, 1, 1, 1};

  bool near_f32() const { return par.precision != PIE_FP64; }
  bool near_h16() const { return par.precision == PIE_FP32H; }
  bool far_f32() const { return par.precision == PIE_FP32 || par.precision == PIE_FP32H; }
  bool io_f32() const { return far_f32(); }
};

// setup kernels (setup.cu)
pie_status setup_device(Problem& pr, cudaStream_t st);
// apply (apply.cu)
pie_status apply_one(Problem& pr, const void* x, void* y, cudaStream_t st);
pie_status apply_batch(Problem& pr, const void* x, void* y, int nrhs, cudaStream_t st);
// x, y: N x nrhs columns, passes of tune.rhs_chunk columns
pie_status apply_cols(Problem& pr, const void* x, void* y, int nrhs, cudaStream_t st);
// one-time kernel attributes of the product (not allowed inside a stream capture)
pie_status prepare_apply(Problem& pr);
// records the start (end = false) or end of stage `stage` of the current apply when profiling
void prof_mark(Problem& pr, int stage, bool end, cudaStream_t st);
pie_status apply_near_one(Problem& pr, const void* x, void* y, cudaStream_t st);
pie_status apply_near_scratch(Problem& pr, const void* x, void* y, void* coef, void* pot, cudaStream_t st);
pie_status rhs_planewave(Problem& pr, const double* khat, const double* pol, double E0, void* b,
                         cudaStream_t st);
pie_status rhs_potentials(Problem& pr, const void* Aq, const void* Pq, void* b, cudaStream_t st);
pie_status farfield(Problem& pr, const void* x, const double* rhat, int64_t ndir, void* E,
                    cudaStream_t st);
pie_status apply_t_one(Problem& pr, const void* x, void* y, bool conj, cudaStream_t st);
pie_status single_layer_one(Problem& pr, const void* q, void* y, cudaStream_t st);
pie_status solve_single_layer(Problem& pr, const void* b, void* x, double tol, int maxit, int restart,
                              pie_solve_stats* stats, cudaStream_t st);
pie_status rhs_potential(Problem& pr, const double* khat, const double* pol, double E0, void* b, cudaStream_t st);
pie_status nearzone(Problem& pr, const void* x, const void* rho, const double* pts, int64_t npts, void* E,
                    cudaStream_t st);
pie_status farfield_adjoint(Problem& pr, const double* rhat, int64_t ndir, const void* E, void* u,
                            cudaStream_t st);
pie_status solve(Problem& pr, const void* b, void* x, double tol, int maxit, int restart,
                 pie_solve_stats* stats, cudaStream_t st, bool guess = false);
pie_status solve_nested(Problem& outer, Problem& inner, const void* b, void* x, const pie_nested_params& np,
                        pie_nested_stats* stats, cudaStream_t st);

pie_status cuda_check(cudaError_t e, const char* what);
// looks up the fixed scratch of pie_apply_near_noalloc on the current device (noalloc.cu)
pie_status noalloc_bind(Problem& pr);
// PIE_ERR_PARAM unless the current device is the one the problem was built on
pie_status check_device(const Problem& pr, const char* who);
void* dalloc(Problem& pr, size_t bytes);

}  // namespace pie
