// Restarted GMRES on the PIE system (Section 4 solves with GMRES).
//
// The system is scaled symmetrically, A = D Z D with D = |diag Z|^{-1/2}
// (the diagonal comes from the near-part self and neighbour pair moments), so
// that the RWG and pulse blocks, whose physical units differ, are balanced.
// Arnoldi runs on the device in complex double with classical Gram-Schmidt,
// repeated when the first pass cancels most of the vector (DGKS criterion);
// dot products use fixed-order two-pass reductions (results do not depend on
// scheduling).  The small Hessenberg problem (Givens rotations)
// is solved on the host.  Stopping test: ||b - Z x|| / ||b|| <= tol on the
// unscaled system, recomputed from the true residual at every restart.
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "device.cuh"

namespace pie {

typedef std::complex<double> zc;
constexpr int kRedThreads = 256;

static inline unsigned nb_(int64_t n, int b) { return unsigned((n + b - 1) / b); }

// Entry index of the pair (test t, source s) in the near moment planes, or -1.
__device__ int64_t near_entry(int64_t t, int64_t s, const int32_t* leaf_of, const int32_t* leaf_start,
                              const int32_t* near_ptr, const int32_t* near_idx, const int64_t* row_ptr) {
  int bt = leaf_of[t], bs = leaf_of[s];
  int64_t e = row_ptr[t];
  for (int qi = near_ptr[bt]; qi < near_ptr[bt + 1]; ++qi) {
    int q = near_idx[qi];
    if (q == bs) return e + (s - leaf_start[q]);
    e += leaf_start[q + 1] - leaf_start[q];
  }
  return -1;
}

// |Z_ii|^{-1/2} for every unknown (mesh order), from the near pair moments.
template <typename Rm>
__global__ void k_diag_scale(int64_t N, int64_t E, int64_t nnz, const int32_t* __restrict__ edge_tt,
                             const int8_t* __restrict__ edge_k, const double* __restrict__ tri_c,
                             const double* __restrict__ tri_dcp, const int64_t* __restrict__ inv_perm,
                             const int32_t* __restrict__ leaf_of, const int32_t* __restrict__ leaf_start,
                             const int32_t* __restrict__ near_ptr, const int32_t* __restrict__ near_idx,
                             const int64_t* __restrict__ row_ptr, const C2<Rm>* __restrict__ mom, double w2e,
                             double* __restrict__ dscale) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double zr = 0, zi = 0;
  if (i < E) {
    for (int s1 = 0; s1 < 2; ++s1)
      for (int s2 = 0; s2 < 2; ++s2) {
        int64_t t1 = edge_tt[2 * i + s1], t2 = edge_tt[2 * i + s2];
        int k1 = edge_k[2 * i + s1], k2 = edge_k[2 * i + s2];
        int64_t e = near_entry(t1, t2, leaf_of, leaf_start, near_ptr, near_idx, row_ptr);
        if (e < 0) continue;
        const double* d1 = tri_dcp + 9 * t1 + 3 * k1;
        const double* d2 = tri_dcp + 9 * t2 + 3 * k2;
        double cc = kMu0 * tri_c[3 * t1 + k1] * tri_c[3 * t2 + k2];
        C2<Rm> m0 = mom[e], mts = mom[7 * nnz + e];
        double vr = double(mts.x), vi = double(mts.y), dd = 0;
        for (int d = 0; d < 3; ++d) {
          C2<Rm> mt = mom[(1 + d) * nnz + e], ms = mom[(4 + d) * nnz + e];
          vr += d1[d] * double(ms.x) + double(mt.x) * d2[d];
          vi += d1[d] * double(ms.y) + double(mt.y) * d2[d];
          dd += d1[d] * d2[d];
        }
        vr += dd * double(m0.x);
        vi += dd * double(m0.y);
        zr += cc * vr;
        zi += cc * vi;
      }
  } else {
    int64_t t = inv_perm[i - E];
    int64_t e = near_entry(t, t, leaf_of, leaf_start, near_ptr, near_idx, row_ptr);
    C2<Rm> m0 = mom[e];
    zr = w2e * double(m0.x);
    zi = w2e * double(m0.y);
  }
  double a = sqrt(zr * zr + zi * zi);
  dscale[i] = a > 0 ? 1.0 / sqrt(a) : 1.0;
}

// |S_tt|^{-1/2} for the single layer of Eq. (3) (pulse t in mesh order):
// S_tt = int_t int_t g, the self-pair moment m0.
template <typename Rm>
__global__ void k_diag_single(int64_t T, const int64_t* __restrict__ inv_perm, const int32_t* __restrict__ leaf_of,
                              const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ near_ptr,
                              const int32_t* __restrict__ near_idx, const int64_t* __restrict__ row_ptr,
                              const C2<Rm>* __restrict__ mom, double* __restrict__ dscale) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= T) return;
  int64_t t = inv_perm[i];
  int64_t e = near_entry(t, t, leaf_of, leaf_start, near_ptr, near_idx, row_ptr);
  C2<Rm> m0 = mom[e];
  double a = sqrt(double(m0.x) * double(m0.x) + double(m0.y) * double(m0.y));
  dscale[i] = a > 0 ? 1.0 / sqrt(a) : 1.0;
}

// y = d x, converting between the Krylov basis type and complex double.
template <typename A, typename B>
__global__ void k_scale(int64_t N, const double* __restrict__ d, const C2<A>* __restrict__ x, C2<B>* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) y[i] = mk<B>(B(d[i] * double(x[i].x)), B(d[i] * double(x[i].y)));
}

// y = a - b (elementwise, complex double)
__global__ void k_sub(int64_t N, const cd* __restrict__ a, const cd* __restrict__ b, cd* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) y[i] = mk<double>(a[i].x - b[i].x, a[i].y - b[i].y);
}

// y = alpha x (real alpha)
template <typename B>
__global__ void k_axs(int64_t N, double alpha, const C2<B>* __restrict__ x, C2<B>* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) y[i] = mk<B>(B(alpha * double(x[i].x)), B(alpha * double(x[i].y)));
}

// partial[v][tile] = sum over the tile's entries of conj(V[v][n]) w[n]
// (accumulated in the basis type per lane, then in double).  Pass 1 of a
// fixed-order reduction.  A block stages one tile of w in shared memory;
// each warp runs it against its share of a chunk of kDotVecs vectors, every
// lane streaming kDotTile / 32 entries of a vector before one warp
// reduction; grid = (tiles, vector chunks).
constexpr int kTile = 2048;     // largest tile (entries of w per block)
constexpr int kMinTile = 256;   // smallest, for short vectors
constexpr int kDotVecs = 64;
template <typename B>
__global__ void __launch_bounds__(kRedThreads) k_mdot(int64_t N, int nv, const C2<B>* __restrict__ V, int64_t ldv,
                                                      const C2<B>* __restrict__ w, cd* __restrict__ partial,
                                                      int tile) {
  __shared__ C2<B> ws[kTile];
  const int64_t n0 = int64_t(blockIdx.x) * tile;
  const int lim = int(min(int64_t(tile), N - n0));
  for (int k = threadIdx.x; k < tile; k += kRedThreads) ws[k] = k < lim ? w[n0 + k] : mk<B>(0, 0);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < kDotVecs; c += kRedThreads / 32) {
    const int v = blockIdx.y * kDotVecs + c;
    if (v >= nv) break;
    const C2<B>* vv = V + int64_t(v) * ldv + n0;
    B ar = 0, ai = 0;
#pragma unroll 8
    for (int k = lane; k < lim; k += 32) {
      const C2<B> a = vv[k], b = ws[k];
      ar += a.x * b.x + a.y * b.y;
      ai += a.x * b.y - a.y * b.x;
    }
    const double dr = warp_sum(double(ar)), di = warp_sum(double(ai));
    if (lane == 0) partial[int64_t(v) * gridDim.x + blockIdx.x] = mk<double>(dr, di);
  }
}

// Pass 2: out[v] = sum over tiles of partial[v][.], one warp per vector,
// lanes over tiles in a fixed order, then a fixed shuffle tree.
__global__ void k_mdot_finish(int nv, int nblk, const cd* __restrict__ partial, cd* __restrict__ out) {
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (v >= nv) return;
  double r = 0, i = 0;
  for (int b = lane; b < nblk; b += 32) {
    r += partial[(int64_t)v * nblk + b].x;
    i += partial[(int64_t)v * nblk + b].y;
  }
  r = warp_sum(r);
  i = warp_sum(i);
  if (lane == 0) out[v] = mk<double>(r, i);
}

// w -= sum_v h[v] V[v] (in the basis type, h staged in shared memory),
// followed by the squared norm of the updated w: per-block
// partial sums (fixed order) in partial[blockIdx.x], finished by
// k_mdot_finish.  Block size kRedThreads.
template <typename B>
__global__ void __launch_bounds__(kRedThreads) k_mupdate_norm(int64_t N, int nv, const C2<B>* __restrict__ V,
                                                              int64_t ldv, const cd* __restrict__ h,
                                                              C2<B>* __restrict__ w, cd* __restrict__ partial) {
  extern __shared__ unsigned char hraw[];
  C2<B>* hs = reinterpret_cast<C2<B>*>(hraw);
  __shared__ double sn[kRedThreads / 32];
  for (int v = threadIdx.x; v < nv; v += blockDim.x) hs[v] = mk<B>(B(h[v].x), B(h[v].y));
  __syncthreads();
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double nrm = 0;
  if (n < N) {
    // four independent partial sums (vectors v = 4q + u), 16 loads in flight
    B r[4] = {0, 0, 0, 0}, i[4] = {0, 0, 0, 0};
    int v = 0;
#pragma unroll 4
    for (; v + 3 < nv; v += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const C2<B> a = V[(v + u) * ldv + n], c = hs[v + u];
        r[u] += c.x * a.x - c.y * a.y;
        i[u] += c.x * a.y + c.y * a.x;
      }
    }
    for (; v < nv; ++v) {
      const C2<B> a = V[v * ldv + n], c = hs[v];
      r[0] += c.x * a.x - c.y * a.y;
      i[0] += c.x * a.y + c.y * a.x;
    }
    const B rs = (r[0] + r[1]) + (r[2] + r[3]), is = (i[0] + i[1]) + (i[2] + i[3]);
    const C2<B> o = mk<B>(w[n].x - rs, w[n].y - is);
    w[n] = o;
    nrm = double(o.x) * double(o.x) + double(o.y) * double(o.y);
  }
  nrm = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) sn[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kRedThreads / 32; ++k) t += sn[k];
    partial[blockIdx.x] = mk<double>(t, 0.0);
  }
}

// x += d (sum_v y[v] V[v]) in complex double (the solution stays FP64).
template <typename B>
__global__ void k_xupdate(int64_t N, int nv, const C2<B>* __restrict__ V, int64_t ldv, const cd* __restrict__ y,
                          const double* __restrict__ d, cd* __restrict__ x) {
  extern __shared__ cd ys[];
  for (int v = threadIdx.x; v < nv; v += blockDim.x) ys[v] = y[v];
  __syncthreads();
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  double r = 0, i = 0;
  for (int v = 0; v < nv; ++v) {
    C2<B> a = V[v * ldv + n];
    cd c = ys[v];
    r += c.x * double(a.x) - c.y * double(a.y);
    i += c.x * double(a.y) + c.y * double(a.x);
  }
  x[n] = mk<double>(x[n].x + d[n] * r, x[n].y + d[n] * i);
}

// out = sum_v y[v] V[v] in complex double (no scaling, overwrites out).
template <typename B>
__global__ void k_combine(int64_t N, int nv, const C2<B>* __restrict__ V, int64_t ldv, const cd* __restrict__ y,
                          cd* __restrict__ out) {
  extern __shared__ cd yc[];
  for (int v = threadIdx.x; v < nv; v += blockDim.x) yc[v] = y[v];
  __syncthreads();
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  double r = 0, i = 0;
  for (int v = 0; v < nv; ++v) {
    C2<B> a = V[v * ldv + n];
    cd c = yc[v];
    r += c.x * double(a.x) - c.y * double(a.y);
    i += c.x * double(a.y) + c.y * double(a.x);
  }
  out[n] = mk<double>(r, i);
}

// partial[block] = sum over the block's entries of |(sum_v c[v] V[v][n]) / d[n]|^2:
// pass 1 of ||D^-1 V c||^2 (finished by k_mdot_finish).  Block size kRedThreads.
template <typename B>
__global__ void __launch_bounds__(kRedThreads) k_resnorm(int64_t N, int nv, const C2<B>* __restrict__ V, int64_t ldv,
                                                         const cd* __restrict__ c, const double* __restrict__ d,
                                                         cd* __restrict__ partial) {
  extern __shared__ cd cc[];
  __shared__ double sn[kRedThreads / 32];
  for (int v = threadIdx.x; v < nv; v += blockDim.x) cc[v] = c[v];
  __syncthreads();
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double nrm = 0;
  if (n < N) {
    double r = 0, i = 0;
    for (int v = 0; v < nv; ++v) {
      const C2<B> a = V[v * ldv + n];
      r += cc[v].x * double(a.x) - cc[v].y * double(a.y);
      i += cc[v].x * double(a.y) + cc[v].y * double(a.x);
    }
    r /= d[n];
    i /= d[n];
    nrm = r * r + i * i;
  }
  nrm = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) sn[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kRedThreads / 32; ++k) t += sn[k];
    partial[blockIdx.x] = mk<double>(t, 0.0);
  }
}

// y = x converted between complex double and the Krylov basis type.
template <typename A, typename B>
__global__ void k_cvt(int64_t N, const C2<A>* __restrict__ x, C2<B>* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) y[i] = mk<B>(B(x[i].x), B(x[i].y));
}

// ---------------------------------------------------------------- host loop

struct Work {
  std::vector<void*> ptrs;
  ~Work() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t n, pie_status& s) {
    if (s != PIE_OK) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      set_error("pie_solve: device allocation failed");
      s = PIE_ERR_OOM;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

// Shared scratch of the Krylov loop.
struct Ctx {
  Problem& pr;      // the problem whose operator the products apply
  cudaStream_t st;
  int op;           // 0: the PIE operator Z (N unknowns); 1: the single layer of Eq. (3) (T unknowns)
  int64_t N;
  double* d;        // symmetric scaling
  cd* u;            // operator input (double)
  cd* wd;           // operator output (double)
  cd* partial;      // reduction partials
  cd* hdev;         // small device vector
  int hcap = 0;     // its length (the last entry holds norms)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last operator product
  bool pending = false;                      // ev0 / ev1 hold a product not yet counted
  double op_ms = 0;                          // time in operator products
  int reorth = 0;                            // second Gram-Schmidt passes
  cf* u32 = nullptr;                         // operator input / output of a problem with
  cf* w32 = nullptr;                         // complex-float vectors (PIE_FP32)
};

// Adds the last product's time (its events have completed: every product is
// followed by a synchronising reduction before the next one).
static void op_time_flush(Ctx& c) {
  if (!c.pending || !c.ev0) return;
  float ms = 0;
  if (cudaEventElapsedTime(&ms, c.ev0, c.ev1) == cudaSuccess)
    c.op_ms += ms;
  else
    cudaGetLastError();
  c.pending = false;
}

// out = Z in, or out = S in for the single-layer operator of Eq. (3)
// (vectors in the io precision of the context's problem).
static pie_status op_apply(Ctx& c, const void* in, void* out) {
  op_time_flush(c);
  if (c.ev0) cudaEventRecord(c.ev0, c.st);
  pie_status s = c.op == 0 ? apply_one(c.pr, in, out, c.st) : single_layer_one(c.pr, in, out, c.st);
  if (c.ev1) {
    cudaEventRecord(c.ev1, c.st);
    c.pending = true;
  }
  return s;
}

// out = D Op D in for a Krylov vector in type B; the product runs on complex
// double vectors, or on complex float ones for a PIE_FP32 problem.
template <typename B>
static pie_status op_scaled(Ctx& c, const C2<B>* in, C2<B>* out) {
  const int64_t N = c.N;
  pie_status s;
  if (c.pr.io_f32()) {
    k_scale<B, float><<<nb_(N, 256), 256, 0, c.st>>>(N, c.d, in, c.u32);
    if ((s = op_apply(c, c.u32, c.w32)) != PIE_OK) return s;
    k_scale<float, B><<<nb_(N, 256), 256, 0, c.st>>>(N, c.d, c.w32, out);
  } else {
    k_scale<B, double><<<nb_(N, 256), 256, 0, c.st>>>(N, c.d, in, c.u);
    if ((s = op_apply(c, c.u, c.wd)) != PIE_OK) return s;
    k_scale<double, B><<<nb_(N, 256), 256, 0, c.st>>>(N, c.d, c.wd, out);
  }
  return PIE_OK;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      a = b = nullptr;  // timing of the products is then left out
    }
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// conj(a) . b over N entries, deterministic; result on the host.
template <typename B>
static pie_status dotc(Ctx& c, int nv, const C2<B>* V, const C2<B>* w, zc* out_host) {
  // tiles of kTile entries, smaller (down to kMinTile) when that leaves fewer
  // than two blocks per SM
  int tile = kTile;
  if ((c.N + kTile - 1) / kTile < 2 * int64_t(c.pr.nsm))
    tile = int(std::max<int64_t>(kMinTile, ((c.N / (2 * std::max(c.pr.nsm, 1)) + 31) / 32) * 32));
  tile = std::min(tile, kTile);
  const unsigned tiles = unsigned((c.N + tile - 1) / tile);
  k_mdot<B><<<dim3(tiles, unsigned((nv + kDotVecs - 1) / kDotVecs)), kRedThreads, 0, c.st>>>(c.N, nv, V, c.N, w,
                                                                                            c.partial, tile);
  k_mdot_finish<<<nb_(int64_t(nv) * 32, 128), 128, 0, c.st>>>(nv, int(tiles), c.partial, c.hdev);
  pie_status s = cuda_check(cudaMemcpyAsync(out_host, c.hdev, sizeof(cd) * nv, cudaMemcpyDeviceToHost, c.st), "dot");
  if (s == PIE_OK) s = cuda_check(cudaStreamSynchronize(c.st), "dot sync");
  return s;
}

// w -= sum_{v<nv} hdev[v] V[v]; returns ||w|| (host) after the update.
template <typename B>
static pie_status update_norm(Ctx& c, int nv, const C2<B>* V, C2<B>* w, double* norm) {
  const unsigned blocks = nb_(c.N, kRedThreads);
  k_mupdate_norm<B><<<blocks, kRedThreads, sizeof(C2<B>) * nv, c.st>>>(c.N, nv, V, c.N, c.hdev, w, c.partial);
  k_mdot_finish<<<1, 32, 0, c.st>>>(1, int(blocks), c.partial, c.hdev + c.hcap - 1);
  cd out;
  pie_status s = cuda_check(cudaMemcpyAsync(&out, c.hdev + c.hcap - 1, sizeof(cd), cudaMemcpyDeviceToHost, c.st),
                            "norm");
  if (s == PIE_OK) s = cuda_check(cudaStreamSynchronize(c.st), "norm sync");
  *norm = std::sqrt(out.x);
  return s;
}

static pie_status to_dev(Ctx& c, const std::vector<zc>& v, int n) {
  std::vector<cd> h(n);
  for (int i = 0; i < n; ++i) h[i] = cd{v[i].real(), v[i].imag()};
  pie_status s = cuda_check(cudaMemcpyAsync(c.hdev, h.data(), sizeof(cd) * n, cudaMemcpyHostToDevice, c.st), "copy");
  if (s == PIE_OK) s = cuda_check(cudaStreamSynchronize(c.st), "copy sync");  // h must outlive the copy
  return s;
}

struct Cycle {
  std::vector<zc> H, cs, sn, g, h, h2;
  int m;
  explicit Cycle(int m_) : H(size_t(m_ + 1) * m_), cs(m_), sn(m_), g(m_ + 1), h(m_ + 1), h2(m_ + 1), m(m_) {}
  void reset(double beta) {
    std::fill(H.begin(), H.end(), zc(0));
    std::fill(g.begin(), g.end(), zc(0));
    g[0] = beta;
  }
};

// Classical Gram-Schmidt of w (basis slot j + 1) against V[0..j]; a second
// pass only when the first one cancelled most of w (Daniel-Gragg-Kaufman-
// Stewart criterion).  One reduction gives (v_i, w) for i <= j and (w, w);
// the update returns the new norm.  cy.h[0..j] gets the projections, *hn
// the norm of the orthogonalised w.
template <typename B>
static pie_status orthogonalize(Ctx& c, const C2<B>* V, int j, C2<B>* w, Cycle& cy, double* hn) {
  pie_status s;
  if ((s = dotc<B>(c, j + 2, V, w, cy.h.data())) != PIE_OK) return s;
  const double wn0 = std::sqrt(cy.h[j + 1].real());
  if ((s = update_norm<B>(c, j + 1, V, w, hn)) != PIE_OK) return s;
  if (*hn < 0.7 * wn0) {
    ++c.reorth;
    if ((s = dotc<B>(c, j + 1, V, w, cy.h2.data())) != PIE_OK) return s;
    if ((s = update_norm<B>(c, j + 1, V, w, hn)) != PIE_OK) return s;
    for (int i = 0; i <= j; ++i) cy.h[i] += cy.h2[i];
  }
  for (int i = 0; i <= j; ++i)
    if (!std::isfinite(cy.h[i].real()) || !std::isfinite(cy.h[i].imag()) || !std::isfinite(*hn)) {
      set_error("pie_solve: non-finite Arnoldi coefficient");
      return PIE_ERR_NAN;
    }
  return PIE_OK;
}

// Column j of the Hessenberg matrix (cy.h[0..j] and hn below the diagonal):
// previous rotations, then a new one G = [[conj c, conj s], [-s, c]].
// Returns the rotated diagonal entry.
static double hessenberg_column(Cycle& cy, int j, double hn) {
  const int m = cy.m;
  for (int i = 0; i <= j; ++i) cy.H[size_t(i) * m + j] = cy.h[i];
  for (int i = 0; i < j; ++i) {
    zc a = cy.H[size_t(i) * m + j], b = cy.H[size_t(i + 1) * m + j];
    cy.H[size_t(i) * m + j] = std::conj(cy.cs[i]) * a + std::conj(cy.sn[i]) * b;
    cy.H[size_t(i + 1) * m + j] = -cy.sn[i] * a + cy.cs[i] * b;
  }
  zc a = cy.H[size_t(j) * m + j];
  double den = std::sqrt(std::norm(a) + hn * hn);
  cy.cs[j] = a / den;
  cy.sn[j] = zc(hn / den);
  cy.H[size_t(j) * m + j] = den;
  cy.g[j + 1] = -cy.sn[j] * cy.g[j];
  cy.g[j] = std::conj(cy.cs[j]) * cy.g[j];
  return den;
}

// y = R^{-1} g over the first j columns (back substitution).
static void back_substitute(const Cycle& cy, int j, std::vector<zc>& y) {
  const int m = cy.m;
  y.assign(j, zc(0));
  for (int i = j - 1; i >= 0; --i) {
    zc acc = cy.g[i];
    for (int k = i + 1; k < j; ++k) acc -= cy.H[size_t(i) * m + k] * y[k];
    y[i] = acc / cy.H[size_t(i) * m + i];
  }
}

// The unscaled residual ||b - Z x_j|| of the cycle's current iterate, from
// the small problem: its residual in the rotated frame is g_{j+1} e_{j+1};
// rotated back (G_j^H .. G_0^H) it gives coefficients a over V[0..j+1], the
// scaled residual is V a and the residual D^-1 V a (exact in exact
// arithmetic; each cycle's true residual is recomputed with a product).
template <typename B>
static pie_status unscaled_residual(Ctx& c, const C2<B>* V, const Cycle& cy, int j, double* out) {
  std::vector<zc> a(j + 2, zc(0));
  a[j + 1] = cy.g[j + 1];
  for (int i = j; i >= 0; --i) {
    const zc ai = a[i], aj = a[i + 1];
    a[i] = cy.cs[i] * ai - std::conj(cy.sn[i]) * aj;
    a[i + 1] = cy.sn[i] * ai + std::conj(cy.cs[i]) * aj;
  }
  pie_status s = to_dev(c, a, j + 2);
  if (s != PIE_OK) return s;
  const unsigned blocks = nb_(c.N, kRedThreads);
  k_resnorm<B><<<blocks, kRedThreads, sizeof(cd) * (j + 2), c.st>>>(c.N, j + 2, V, c.N, c.hdev, c.d, c.partial);
  k_mdot_finish<<<1, 32, 0, c.st>>>(1, int(blocks), c.partial, c.hdev + c.hcap - 1);
  cd r;
  s = cuda_check(cudaMemcpyAsync(&r, c.hdev + c.hcap - 1, sizeof(cd), cudaMemcpyDeviceToHost, c.st), "residual");
  if (s == PIE_OK) s = cuda_check(cudaStreamSynchronize(c.st), "residual sync");
  *out = std::sqrt(r.x);
  return s;
}

// One GMRES cycle (no restart) on the scaled operator D Op D, x0 = 0, with
// V[0] = D r / ||D r|| given: Arnoldi up to m steps, or until the rotated
// (scaled) residual falls below stop_abs, or -- with hint_every > 0 -- the
// unscaled residual of the iterate, formed from the small problem every
// hint_every steps (unscaled_residual), falls to stop_unscaled.  These
// estimates end the cycle only after min_steps steps.  On return y (host)
// holds the coefficients, j the number of steps, *early whether an estimate
// ended the cycle.
template <typename B>
static pie_status arnoldi_cycle(Ctx& c, C2<B>* V, Cycle& cy, double beta, double stop_abs, int max_steps,
                                int& j_out, std::vector<zc>& y, bool& breakdown, int& steps_done,
                                int hint_every = 0, double stop_unscaled = 0, int min_steps = 0,
                                bool* early = nullptr) {
  if (early) *early = false;
  const int64_t N = c.N;
  const int m = cy.m;
  pie_status s = PIE_OK;
  cy.reset(beta);
  int j = 0;
  breakdown = false;
  for (; j < m && j < max_steps; ++j) {
    // the new vector is built in its own basis slot: w = D Op D v_j
    C2<B>* w = V + size_t(j + 1) * N;
    if ((s = op_scaled<B>(c, V + size_t(j) * N, w)) != PIE_OK) return s;
    double hn = 0;
    if ((s = orthogonalize<B>(c, V, j, w, cy, &hn)) != PIE_OK) return s;
    const double den = hessenberg_column(cy, j, hn);
    ++steps_done;
    if (hn <= 1e-14 * den) {
      breakdown = true;
      ++j;
      break;
    }
    k_axs<B><<<nb_(N, 256), 256, 0, c.st>>>(N, 1.0 / hn, w, w);
    if (j + 1 < min_steps) continue;
    bool stop = std::abs(cy.g[j + 1]) <= stop_abs;
    if (!stop && hint_every > 0 && (j + 1) % hint_every == 0) {
      double ru = 0;
      if ((s = unscaled_residual<B>(c, V, cy, j, &ru)) != PIE_OK) return s;
      stop = ru <= stop_unscaled;
    }
    if (stop) {
      if (early) *early = true;
      ++j;
      break;
    }
  }
  back_substitute(cy, j, y);
  j_out = j;
  return cuda_check(cudaGetLastError(), "arnoldi");
}

// |Z_ii|^{-1/2} (op 0) or |S_tt|^{-1/2} (op 1) from the near pair moments.
static void diag_scaling(Problem& pr, int op, int64_t N, double* d, cudaStream_t st) {
  const double w2e = pr.w * pr.w * eps0();
  if (op == 1) {
    if (pr.near_f32())
      k_diag_single<float><<<nb_(N, 256), 256, 0, st>>>(N, pr.inv_perm, pr.leaf_of, pr.leaf_start, pr.near_ptr,
                                                        pr.near_idx, pr.row_ptr, static_cast<const cf*>(pr.mom), d);
    else
      k_diag_single<double><<<nb_(N, 256), 256, 0, st>>>(N, pr.inv_perm, pr.leaf_of, pr.leaf_start, pr.near_ptr,
                                                         pr.near_idx, pr.row_ptr, static_cast<const cd*>(pr.mom), d);
  } else if (pr.near_f32())
    k_diag_scale<float><<<nb_(N, 256), 256, 0, st>>>(N, pr.E, pr.nnz, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                     pr.inv_perm, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx,
                                                     pr.row_ptr, static_cast<const cf*>(pr.mom), w2e, d);
  else
    k_diag_scale<double><<<nb_(N, 256), 256, 0, st>>>(N, pr.E, pr.nnz, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                      pr.inv_perm, pr.leaf_of, pr.leaf_start, pr.near_ptr,
                                                      pr.near_idx, pr.row_ptr, static_cast<const cd*>(pr.mom), w2e, d);
}

// Restarted GMRES with the Krylov basis in type B (double for PIE_FP64,
// float for PIE_MIXED) and the solution, the true residual and the stopping
// test in complex double: each restart recomputes r = b - Z x in FP64, so
// the basis precision limits only the progress of a cycle, not the accuracy
// reached (iterative refinement with a GMRES inner solver).
template <typename B>
static pie_status solve_t(Problem& pr, int op, const void* bv, void* xv, double tol, int maxit, int restart,
                          pie_solve_stats* stats, cudaStream_t st, bool guess = false) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t N = op == 0 ? pr.N : pr.T;
  const int m = std::min(restart, maxit);
  pie_status s = PIE_OK;
  Work wk;
  double* d = wk.get<double>(N, s);
  C2<B>* V = wk.get<C2<B>>(size_t(N) * (m + 1), s);
  cd* u = wk.get<cd>(N, s);
  cd* wd = wk.get<cd>(N, s);
  cd* r = wk.get<cd>(N, s);
  cd* partial = wk.get<cd>(std::max(size_t((N + kMinTile - 1) / kMinTile) * (m + 2), size_t(nb_(N, kRedThreads))), s);
  cd* hdev = wk.get<cd>(m + 3, s);
  if (s != PIE_OK) return s;
  EventPair evp;
  Ctx c{pr, st, op, N, d, u, wd, partial, hdev};
  c.hcap = m + 3;
  if (evp.a && evp.b) {
    c.ev0 = evp.a;
    c.ev1 = evp.b;
  }
  const cd* b = static_cast<const cd*>(bv);
  cd* x = static_cast<cd*>(xv);
  diag_scaling(pr, op, N, d, st);
  if (guess) {  // start from the caller's x: r = b - Z x
    if ((s = op_apply(c, x, wd)) != PIE_OK) return s;
    k_sub<<<nb_(N, 256), 256, 0, st>>>(N, b, wd, r);
  } else {
    cudaMemsetAsync(x, 0, sizeof(cd) * N, st);
    cudaMemcpyAsync(r, b, sizeof(cd) * N, cudaMemcpyDeviceToDevice, st);
  }
  zc tmp[1];
  if ((s = dotc<double>(c, 1, b, b, tmp)) != PIE_OK) return s;
  const double bn = std::sqrt(tmp[0].real());
  int it = 0;
  double rel = bn == 0 ? 0.0 : 1.0;
  pie_status result = bn == 0 ? PIE_OK : PIE_ERR_NOCONV;
  if (bn == 0) cudaMemsetAsync(x, 0, sizeof(cd) * N, st);  // b = 0: the solution is x = 0, whatever the guess
  Cycle cy(m);
  std::vector<zc> y;
  // A cycle ends when the rotated residual falls to tol / 2 (scaled
  // system) or the unscaled residual of its iterate, formed every 4 steps
  // from the small problem, to tol; the true residual b - Z x then decides.
  // Near 1e-6 the true residual of the large problems fluctuates with the
  // far part's rounding (a ~2.5e-6 nonlinearity of the product) and the
  // estimates drift from it in either direction; short cycles that restart
  // from the true residual then often meet tol.  Only after twelve cycles in
  // a row that an estimate ended but whose true residual missed tol do the
  // next cycles run at least min_steps steps (25, then doubling, up to
  // restart): the case where the rounding floor lies above tol.
  int min_steps = 0, overruled = 0;
  bool early = false;
  while (result != PIE_OK && it < maxit) {
    if ((s = dotc<double>(c, 1, r, r, tmp)) != PIE_OK) return s;
    rel = std::sqrt(tmp[0].real()) / bn;
    if (!std::isfinite(rel)) {
      set_error("pie_solve: non-finite residual");
      return PIE_ERR_NAN;
    }
    if (rel <= tol) {
      result = PIE_OK;
      break;
    }
    // first Krylov vector: the scaled residual D r, normalised
    k_scale<double, double><<<nb_(N, 256), 256, 0, st>>>(N, d, r, u);
    if ((s = dotc<double>(c, 1, u, u, tmp)) != PIE_OK) return s;
    const double beta = std::sqrt(tmp[0].real());
    k_scale<double, B><<<nb_(N, 256), 256, 0, st>>>(N, d, r, V);
    k_axs<B><<<nb_(N, 256), 256, 0, st>>>(N, 1.0 / beta, V, V);
    int j = 0;
    bool breakdown = false;
    const double dbn = beta / rel;  // scale of ||D b|| for the cycle's stopping estimate
    if ((s = arnoldi_cycle<B>(c, V, cy, beta, 0.5 * tol * dbn, maxit - it, j, y, breakdown, it, 4, tol * bn,
                              min_steps, &early)) != PIE_OK)
      return s;
    // x += D (sum_j y_j V_j), in complex double
    if ((s = to_dev(c, y, j)) != PIE_OK) return s;
    k_xupdate<B><<<nb_(N, 256), 256, sizeof(cd) * std::max(j, 1), st>>>(N, j, V, N, hdev, d, x);
    // true residual r = b - Z x (FP64 vectors)
    if ((s = op_apply(c, x, wd)) != PIE_OK) return s;
    k_sub<<<nb_(N, 256), 256, 0, st>>>(N, b, wd, r);
    if ((s = cuda_check(cudaGetLastError(), "gmres launch")) != PIE_OK) return s;
    if (early) {
      if ((s = dotc<double>(c, 1, r, r, tmp)) != PIE_OK) return s;
      overruled = std::sqrt(tmp[0].real()) > tol * bn ? overruled + 1 : 0;
      if (overruled >= 12) min_steps = std::min(m, std::max(25, 2 * min_steps));
    } else {
      overruled = 0;
    }
    if (breakdown) {
      if ((s = dotc<double>(c, 1, r, r, tmp)) != PIE_OK) return s;
      rel = std::sqrt(tmp[0].real()) / bn;
      result = rel <= tol ? PIE_OK : PIE_ERR_BREAKDOWN;
      if (result != PIE_OK) set_error("pie_solve: Arnoldi breakdown before convergence");
      break;
    }
  }
  if (result != PIE_OK && result != PIE_ERR_BREAKDOWN) {
    if ((s = dotc<double>(c, 1, r, r, tmp)) != PIE_OK) return s;
    rel = std::sqrt(tmp[0].real()) / bn;
    if (rel <= tol)
      result = PIE_OK;
    else
      set_error("pie_solve: tolerance not reached in maxit iterations");
  }
  if ((s = cuda_check(cudaStreamSynchronize(st), "gmres sync")) != PIE_OK) return s;
  op_time_flush(c);
  if (stats) {
    stats->iterations = it;
    stats->rel_residual = rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->reorthogonalizations = c.reorth;
    stats->product_seconds = c.op_ms * 1e-3;
  }
  return result;
}

pie_status solve(Problem& pr, const void* b, void* x, double tol, int maxit, int restart, pie_solve_stats* stats,
                 cudaStream_t st, bool guess) {
  if (pr.io_f32()) {
    set_error("pie_solve: needs a PIE_FP64 or PIE_MIXED problem (complex double vectors)");
    return PIE_ERR_PARAM;
  }
  if (pr.par.precision == PIE_MIXED) return solve_t<float>(pr, 0, b, x, tol, maxit, restart, stats, st, guess);
  return solve_t<double>(pr, 0, b, x, tol, maxit, restart, stats, st, guess);
}

pie_status solve_single_layer(Problem& pr, const void* b, void* x, double tol, int maxit, int restart,
                              pie_solve_stats* stats, cudaStream_t st) {
  if (pr.io_f32()) {
    set_error("pie_solve_single_layer: needs a PIE_FP64 or PIE_MIXED problem (complex double vectors)");
    return PIE_ERR_PARAM;
  }
  if (pr.par.precision == PIE_MIXED) return solve_t<float>(pr, 1, b, x, tol, maxit, restart, stats, st);
  return solve_t<double>(pr, 1, b, x, tol, maxit, restart, stats, st);
}

// ---------------------------------------------------------------- nested solve

// Flexible GMRES (Saad 1993) on the outer operator D Z D, right-preconditioned
// by a few GMRES steps on the inner operator D Z' D: z_j = M_j(v_j) is one
// inner cycle from zero on the outer Krylov vector v_j, the outer product is
// w = D Z D z_j, and the solution is x += D sum_j y_j z_j.  Z' is the same
// discrete PIE operator with its far part at (tau, kappa a, N_theta) chosen for
// complex float (Eqs. (4)-(5): the rounding amplification of the scaled
// Hankel terms is small there), so its products are far cheaper than those of
// the outer FP64-far operator; the outer operator, the solution and the true
// residual at every restart stay in complex double.  outer_restart = 0 is
// plain iterative refinement: x += D z with z = M(D r / ||D r||) ||D r||.
template <typename Bi>
static pie_status nested_t(Problem& po, Problem& pi, const cd* b, cd* x, const pie_nested_params& np,
                           pie_nested_stats* stats, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t N = po.N;
  const int mi = np.inner_restart;
  const int mo = std::max(np.outer_restart, 1);
  const bool ir = np.outer_restart == 0;
  const int mmax = std::max(mi, mo);
  pie_status s = PIE_OK;
  Work wk;
  double* d = wk.get<double>(N, s);
  C2<Bi>* Vi = wk.get<C2<Bi>>(size_t(N) * (mi + 1), s);  // inner basis
  cd* Vo = wk.get<cd>(size_t(N) * (mo + 1), s);           // outer basis
  cd* Zo = wk.get<cd>(size_t(N) * mo, s);                 // preconditioned outer vectors
  cd* u = wk.get<cd>(N, s);
  cd* wd = wk.get<cd>(N, s);
  cd* r = wk.get<cd>(N, s);
  cf* u32 = pi.io_f32() ? wk.get<cf>(N, s) : nullptr;
  cf* w32 = pi.io_f32() ? wk.get<cf>(N, s) : nullptr;
  cd* partial = wk.get<cd>(std::max(size_t((N + kMinTile - 1) / kMinTile) * (mmax + 2), size_t(nb_(N, kRedThreads))),
                           s);
  cd* hdev = wk.get<cd>(mmax + 3, s);
  if (s != PIE_OK) return s;
  EventPair evo, evi;
  Ctx co{po, st, 0, N, d, u, wd, partial, hdev};
  Ctx ci{pi, st, 0, N, d, u, wd, partial, hdev};
  co.hcap = ci.hcap = mmax + 3;
  ci.u32 = u32;
  ci.w32 = w32;
  if (evo.a && evo.b) co.ev0 = evo.a, co.ev1 = evo.b;
  if (evi.a && evi.b) ci.ev0 = evi.a, ci.ev1 = evi.b;
  diag_scaling(po, 0, N, d, st);
  cudaMemsetAsync(x, 0, sizeof(cd) * N, st);
  cudaMemcpyAsync(r, b, sizeof(cd) * N, cudaMemcpyDeviceToDevice, st);
  zc tmp[1];
  if ((s = dotc<double>(co, 1, b, b, tmp)) != PIE_OK) return s;
  const double bn = std::sqrt(tmp[0].real());
  int inner_steps = 0, outer_steps = 0, outer_products = 0;
  double rel = bn == 0 ? 0.0 : 1.0;
  pie_status result = bn == 0 ? PIE_OK : PIE_ERR_NOCONV;
  Cycle cyi(mi), cyo(mo);
  std::vector<zc> y, yo;
  // z = M(v): one inner GMRES cycle on D Z' D from zero for the unit vector v
  // (complex double), at most mi steps, stopping at relative residual
  // inner_tol; z in complex double.
  auto precondition = [&](const cd* v, cd* z) -> pie_status {
    k_cvt<double, Bi><<<nb_(N, 256), 256, 0, st>>>(N, v, Vi);
    int j = 0;
    bool brk = false;
    pie_status e = arnoldi_cycle<Bi>(ci, Vi, cyi, 1.0, np.inner_tol, std::min(mi, np.maxit - inner_steps), j, y,
                                     brk, inner_steps);
    if (e != PIE_OK) return e;
    if (j == 0) return cuda_check(cudaMemcpyAsync(z, v, sizeof(cd) * N, cudaMemcpyDeviceToDevice, st), "copy");
    if ((e = to_dev(ci, y, j)) != PIE_OK) return e;
    k_combine<Bi><<<nb_(N, 256), 256, sizeof(cd) * j, st>>>(N, j, Vi, N, hdev, z);
    return cuda_check(cudaGetLastError(), "precondition");
  };
  // An outer cycle ends when the rotated (scaled) residual or the unscaled
  // residual of its iterate, formed every step from the small problem,
  // reaches tol; the true residual then decides.  After twelve cycles in a
  // row so ended whose true residual missed tol, the next cycles run at least
  // min_steps steps (5, then doubling, up to outer_restart).
  int min_steps = 0, overruled = 0;
  bool early = false;
  while (result != PIE_OK && inner_steps < np.maxit && outer_products < np.max_outer) {
    if ((s = dotc<double>(co, 1, r, r, tmp)) != PIE_OK) return s;
    rel = std::sqrt(tmp[0].real()) / bn;
    if (!std::isfinite(rel)) {
      set_error("pie_solve_nested: non-finite residual");
      return PIE_ERR_NAN;
    }
    if (rel <= np.tol) {
      result = PIE_OK;
      break;
    }
    // first outer vector: the scaled residual D r, normalised
    k_scale<double, double><<<nb_(N, 256), 256, 0, st>>>(N, d, r, Vo);
    if ((s = dotc<double>(co, 1, Vo, Vo, tmp)) != PIE_OK) return s;
    const double beta = std::sqrt(tmp[0].real());
    k_axs<double><<<nb_(N, 256), 256, 0, st>>>(N, 1.0 / beta, Vo, Vo);
    int j = 0;
    if (ir) {
      // x += beta D M(v0)
      if ((s = precondition(Vo, Zo)) != PIE_OK) return s;
      ++outer_steps;
      yo.assign(1, zc(beta));
      j = 1;
    } else {
      const double dbn = beta / rel;  // scale of ||D b||
      early = false;
      cyo.reset(beta);
      bool brk = false;
      for (; j < mo && inner_steps < np.maxit && outer_products < np.max_outer; ++j) {
        cd* zj = Zo + size_t(j) * N;
        if ((s = precondition(Vo + size_t(j) * N, zj)) != PIE_OK) return s;
        cd* w = Vo + size_t(j + 1) * N;
        if ((s = op_scaled<double>(co, zj, w)) != PIE_OK) return s;
        ++outer_products;
        double hn = 0;
        if ((s = orthogonalize<double>(co, Vo, j, w, cyo, &hn)) != PIE_OK) return s;
        const double den = hessenberg_column(cyo, j, hn);
        ++outer_steps;
        if (hn <= 1e-14 * den) {
          brk = true;
          ++j;
          break;
        }
        k_axs<double><<<nb_(N, 256), 256, 0, st>>>(N, 1.0 / hn, w, w);
        if (j + 1 < min_steps) continue;
        bool stop = std::abs(cyo.g[j + 1]) <= np.tol * dbn;
        if (!stop) {
          double ru = 0;
          if ((s = unscaled_residual<double>(co, Vo, cyo, j, &ru)) != PIE_OK) return s;
          stop = ru <= np.tol * bn;
        }
        if (stop) {
          early = true;
          ++j;
          break;
        }
      }
      (void)brk;
      back_substitute(cyo, j, yo);
    }
    // x += D (sum_j y_j z_j), complex double
    if ((s = to_dev(co, yo, j)) != PIE_OK) return s;
    k_xupdate<double><<<nb_(N, 256), 256, sizeof(cd) * std::max(j, 1), st>>>(N, j, Zo, N, hdev, d, x);
    // true residual r = b - Z x with the outer operator
    if ((s = op_apply(co, x, wd)) != PIE_OK) return s;
    ++outer_products;
    k_sub<<<nb_(N, 256), 256, 0, st>>>(N, b, wd, r);
    if ((s = cuda_check(cudaGetLastError(), "nested launch")) != PIE_OK) return s;
    if (early) {
      if ((s = dotc<double>(co, 1, r, r, tmp)) != PIE_OK) return s;
      overruled = std::sqrt(tmp[0].real()) > np.tol * bn ? overruled + 1 : 0;
      if (overruled >= 12) min_steps = std::min(mo, std::max(5, 2 * min_steps));
    } else {
      overruled = 0;
    }
  }
  if (result != PIE_OK) {
    if ((s = dotc<double>(co, 1, r, r, tmp)) != PIE_OK) return s;
    rel = std::sqrt(tmp[0].real()) / bn;
    if (rel <= np.tol)
      result = PIE_OK;
    else
      set_error("pie_solve_nested: tolerance not reached within maxit inner steps / max_outer outer products");
  }
  if ((s = cuda_check(cudaStreamSynchronize(st), "nested sync")) != PIE_OK) return s;
  op_time_flush(co);
  op_time_flush(ci);
  if (stats) {
    stats->inner_iterations = inner_steps;
    stats->outer_iterations = outer_steps;
    stats->outer_products = outer_products;
    stats->rel_residual = rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->inner_product_seconds = ci.op_ms * 1e-3;
    stats->outer_product_seconds = co.op_ms * 1e-3;
  }
  return result;
}

pie_status solve_nested(Problem& outer, Problem& inner, const void* b, void* x, const pie_nested_params& np,
                        pie_nested_stats* stats, cudaStream_t st) {
  // the inner Krylov basis is complex float unless the inner operator is FP64
  if (inner.par.precision == PIE_FP64)
    return nested_t<double>(outer, inner, static_cast<const cd*>(b), static_cast<cd*>(x), np, stats, st);
  return nested_t<float>(outer, inner, static_cast<const cd*>(b), static_cast<cd*>(x), np, stats, st);
}

}  // namespace pie
