// One MLFMA matrix-vector product y = Z x for the PIEs (Section 3):
// local coefficients, near pair products, leaf aggregation, interpolation,
// translation (Eq. (5) operators), anterpolation, leaf disaggregation and
// Galerkin assembly (Section 2).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <type_traits>

#include "device.cuh"

namespace pie {

// a0: affine restriction of J to every triangle (tree order),
// J|_t = a (r - c_t) + beta, and the pulse densities sigma, d = 2a + w^2 eps0 sigma.
template <typename Rio>
__global__ void k_coef(int64_t T, int64_t E, const C2<Rio>* __restrict__ x, const int64_t* __restrict__ perm,
                       const int32_t* __restrict__ tri_edge, const double* __restrict__ tri_c,
                       const double* __restrict__ tri_dcp, double w2e, C2<Rio>* __restrict__ coef,
                       cf* __restrict__ coef32, int64_t sx = 0, int64_t sc = 0) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
  // right-hand side blockIdx.y (strides sx, sc between right-hand sides)
  x += blockIdx.y * sx;
  if (coef) coef += blockIdx.y * sc;
  if (coef32) coef32 += blockIdx.y * sc;
  double ar = 0, ai = 0, br[3] = {0, 0, 0}, bi[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int32_t n = tri_edge[3 * t + k];
    if (n < 0) continue;
    double c = tri_c[3 * t + k];
    double xr = double(x[n].x), xi = double(x[n].y);
    ar += c * xr;
    ai += c * xi;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double cd_ = c * tri_dcp[9 * t + 3 * k + d];
      br[d] += cd_ * xr;
      bi[d] += cd_ * xi;
    }
  }
  C2<Rio> s = x[E + perm[t]];
  double sr = double(s.x), si = double(s.y);
  double v[12] = {ar, ai, br[0], bi[0], br[1], bi[1], br[2], bi[2], sr, si, 2.0 * ar + w2e * sr, 2.0 * ai + w2e * si};
  if (coef) {
    C2<Rio>* o = coef + 6 * t;
    for (int q = 0; q < 6; ++q) o[q] = mk<Rio>(Rio(v[2 * q]), Rio(v[2 * q + 1]));
  }
  if (coef32) {  // float copy for a float near part: converted once per triangle
    cf* o = coef32 + 6 * t;
    for (int q = 0; q < 6; ++q) o[q] = mk<float>(float(v[2 * q]), float(v[2 * q + 1]));
  }
}

// PIE_FP32H pair record: eight half pairs (m0, mt_xyz, ms_xyz, mts) at
// momh[8 e .. 8 e + 7], 32 bytes, read as two streaming 16-byte loads.
__device__ __forceinline__ void load_half_record(const __half2* __restrict__ momh, int64_t e, uint4& lo, uint4& hi) {
  const uint4* p = reinterpret_cast<const uint4*>(momh) + 2 * e;
  lo = __ldcs(p);
  hi = __ldcs(p + 1);
}

// The record's moments in float: each half pair times its plane's scale.
template <typename Rm>
__device__ __forceinline__ void unpack_half(const uint4& lo, const uint4& hi, const MomScale& msc, C2<Rm>* m) {
  const uint32_t w[kMom] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
  for (int q = 0; q < kMom; ++q) {
    __half2 h;
    memcpy(&h, &w[q], sizeof(h));
    const float2 v = __half22float2(h);
    m[q] = mk<Rm>(Rm(v.x * msc.s[q]), Rm(v.y * msc.s[q]));
  }
}

template <typename Rm>
__device__ __forceinline__ void unpack_half_record(const __half2* __restrict__ momh, int64_t e, const MomScale& msc,
                                                   C2<Rm>* m) {
  uint4 lo, hi;
  load_half_record(momh, e, lo, hi);
  unpack_half<Rm>(lo, hi, msc, m);
}

// a1: near part.  One warp per test triangle t; lanes run over the source
// triangles of the neighbouring leaf boxes (contiguous in tree order), whose
// eight pair moments are stored plane by plane ([8][nnz]), so a warp reads
// 32 consecutive entries of each plane (measured faster than per-pair
// records with vector loads).  Writes pot[t] (initialises it).  H16: the
// moments come from momh (PIE_FP32H: one record of eight half pairs per
// pair, 32 bytes, two 16-byte loads) times their plane's scale.
template <typename Rm, typename Rio, int RB = 1, bool H16 = false>
__global__ void __launch_bounds__(256) k_near(int64_t T, int64_t nnz, const int32_t* __restrict__ leaf_of,
                                              const int32_t* __restrict__ leaf_start,
                                              const int32_t* __restrict__ near_ptr,
                                              const int32_t* __restrict__ near_idx,
                                              const int32_t* __restrict__ near_off,
                                              const int64_t* __restrict__ row_ptr, const C2<Rm>* __restrict__ mom,
                                              const __half2* __restrict__ momh, MomScale msc,
                                              const C2<Rm>* __restrict__ coef, Rm mu0, C2<Rio>* __restrict__ pot,
                                              int nrhs = 1, int64_t sc = 0, int64_t sp = 0) {
  const int lane = threadIdx.x & 31;
  // right-hand sides r0 .. r0 + RB - 1 share every moment load
  const int r0 = blockIdx.y * RB;
  // one warp per test triangle, with a grid stride when the grid is smaller
  // than T warps (a bounded share of the SMs beside the far part)
  const int64_t wstride = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < T; t += wstride) {
    const int b = leaf_of[t];
    const int q0 = near_ptr[b], q1 = near_ptr[b + 1];
    const int64_t e0 = row_ptr[t];
    const int len = int(row_ptr[t + 1] - e0);
    C2<Rm> acc[RB][6];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[r][i] = mk<Rm>(0, 0);
    // the row is the concatenation of the near boxes' source ranges; lanes walk
    // it flat (32 consecutive entries per step), each lane keeping a cursor on
    // the near box that holds its position
    int qi = q0;
    for (int j = lane; j < len; j += 32) {
      while (qi + 1 < q1 && near_off[qi + 1] <= j) ++qi;
      const int64_t s = leaf_start[near_idx[qi]] + (j - near_off[qi]);
      const int64_t ee = e0 + j;
      C2<Rm> m0, mt0, mt1, mt2, ms0, ms1, ms2, mts;
      if constexpr (H16) {
        C2<Rm> m[kMom];
        unpack_half_record(momh, ee, msc, m);
        m0 = m[0], mt0 = m[1], mt1 = m[2], mt2 = m[3], ms0 = m[4], ms1 = m[5], ms2 = m[6], mts = m[7];
      } else {
        m0 = mom[ee];
        mt0 = mom[nnz + ee], mt1 = mom[2 * nnz + ee], mt2 = mom[3 * nnz + ee];
        ms0 = mom[4 * nnz + ee], ms1 = mom[5 * nnz + ee], ms2 = mom[6 * nnz + ee];
        mts = mom[7 * nnz + ee];
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r0 + r >= nrhs) break;
        const C2<Rm>* c = coef + (r0 + r) * sc + 6 * s;
        C2<Rm> a = c[0], b0 = c[1], b1 = c[2], b2 = c[3], sg = c[4], dd = c[5];
        cfma(acc[r][0], a, mts);
        cfma(acc[r][0], b0, mt0);
        cfma(acc[r][0], b1, mt1);
        cfma(acc[r][0], b2, mt2);
        cfma(acc[r][1], a, ms0);
        cfma(acc[r][1], b0, m0);
        cfma(acc[r][2], a, ms1);
        cfma(acc[r][2], b1, m0);
        cfma(acc[r][3], a, ms2);
        cfma(acc[r][3], b2, m0);
        cfma(acc[r][4], sg, m0);
        cfma(acc[r][5], dd, m0);
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r0 + r >= nrhs) break;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        acc[r][i].x = warp_sum(acc[r][i].x);
        acc[r][i].y = warp_sum(acc[r][i].y);
      }
      if (lane == 0) {
        C2<Rio>* o = pot + (r0 + r) * sp + 6 * t;
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = mk<Rio>(Rio(mu0 * acc[r][i].x), Rio(mu0 * acc[r][i].y));
        o[4] = cvt<Rio>(acc[r][4]);
        o[5] = cvt<Rio>(acc[r][5]);
      }
    }
  }
}

// a1, float near part: one block per leaf box (grid stride over boxes) and
// per group of RB right-hand sides (blockIdx.y).  Every test triangle of a
// box runs over the same source list (the concatenated source ranges of its
// near boxes), so the block stages those sources' coefficients in shared
// memory once per right-hand side, plane by plane ([RB][6][len], dynamic
// shared memory), and its warps take the box's test triangles in turn,
// lanes over the row as in k_near (lane j, j + 32, ...): each moment is read
// once for the RB right-hand sides, and every right-hand side sees the same
// operations in the same order as in k_near, so the same result to the last
// bit.  Rows longer than kNearStage read the coefficients from global
// memory instead.
constexpr int kNearStage = 512;
constexpr int kNearBoxThreads = 128;  // threads per block (per leaf box); 256 measured 8 % slower (FP32H)
template <int RB>
constexpr size_t near_box_smem() {
  return size_t(RB) * 6 * kNearStage * sizeof(cf);
}
template <typename Rio, bool H16, int RB>
__global__ void __launch_bounds__(kNearBoxThreads, RB == 1 ? 6 : (RB == 2 ? 4 : 2))
    k_near_box(int64_t nleaf, int64_t nnz, const int32_t* __restrict__ leaf_start,
               const int32_t* __restrict__ near_ptr, const int32_t* __restrict__ near_idx,
               const int32_t* __restrict__ near_off, const int64_t* __restrict__ row_ptr,
               const cf* __restrict__ mom, const __half2* __restrict__ momh, MomScale msc,
               const cf* __restrict__ coef, float mu0, C2<Rio>* __restrict__ pot, int nrhs = 1, int64_t sc = 0,
               int64_t sp = 0) {
  extern __shared__ __align__(16) unsigned char near_smem[];
  cf* cs = reinterpret_cast<cf*>(near_smem);  // [RB][6][kNearStage]
  const int r0 = blockIdx.y * RB;             // right-hand sides r0 .. r0 + nr - 1
  const int nr = min(RB, nrhs - r0);
  coef += r0 * sc;
  pot += r0 * sp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int64_t b = blockIdx.x; b < nleaf; b += gridDim.x) {
    const int q0 = near_ptr[b], q1 = near_ptr[b + 1];
    const int t0 = leaf_start[b], t1 = leaf_start[b + 1];
    const int len = int(row_ptr[t0 + 1] - row_ptr[t0]);
    const bool staged = len <= kNearStage;
    __syncthreads();  // the previous box's readers are done with cs
    if (staged) {
      int qi = q0;  // j grows: the cursor only moves forward
      for (int j = threadIdx.x; j < len; j += blockDim.x) {
        while (qi + 1 < q1 && near_off[qi + 1] <= j) ++qi;
        const int64_t src = 6 * (int64_t(leaf_start[near_idx[qi]]) + (j - near_off[qi]));
        for (int r = 0; r < nr; ++r)
#pragma unroll
          for (int k = 0; k < 6; ++k) cp_async(&cs[(r * 6 + k) * kNearStage + j], coef + r * sc + src + k);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    for (int t = t0 + warp; t < t1; t += nwarp) {
      const int64_t e0 = row_ptr[t];
      cf acc[RB][6];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[r][i] = mk<float>(0, 0);
      int qi = q0;
      // entry j's six source coefficients of right-hand side r (a cursor on
      // the near box that holds j when they are not staged; j never
      // decreases from one call to the next)
      auto coefs = [&](int r, int j, cf* c) {
        if (staged) {
#pragma unroll
          for (int k = 0; k < 6; ++k) c[k] = cs[(r * 6 + k) * kNearStage + j];
        } else {
          while (qi + 1 < q1 && near_off[qi + 1] <= j) ++qi;
          const cf* src = coef + r * sc + 6 * (int64_t(leaf_start[near_idx[qi]]) + (j - near_off[qi]));
#pragma unroll
          for (int k = 0; k < 6; ++k) c[k] = src[k];
        }
      };
      // m: m0, mt(3), ms(3), mts; c: a, beta(3), sigma, d
      auto accumulate = [](cf* a, const cf* m, const cf* c) {
        cfma(a[0], c[0], m[7]);
        cfma(a[0], c[1], m[1]);
        cfma(a[0], c[2], m[2]);
        cfma(a[0], c[3], m[3]);
        cfma(a[1], c[0], m[4]);
        cfma(a[1], c[1], m[0]);
        cfma(a[2], c[0], m[5]);
        cfma(a[2], c[2], m[0]);
        cfma(a[3], c[0], m[6]);
        cfma(a[3], c[3], m[0]);
        cfma(a[4], c[4], m[0]);
        cfma(a[5], c[5], m[0]);
      };
      // one entry's moments against every right-hand side's coefficients
      auto entry = [&](int j, const cf* m) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
          if (r < nr) {
            cf c[6];
            coefs(r, j, c);
            accumulate(acc[r], m, c);
          }
      };
      if constexpr (H16) {
        // entries j, j + 32, ... (U of them): their 32-byte records loaded
        // together, then accumulated in that order, the order of the
        // one-entry loop
        constexpr int U = RB == 1 ? 4 : 2;
        for (int j = lane; j < len; j += 32 * U) {
          uint4 lo[U], hi[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (j + 32 * u < len) load_half_record(momh, e0 + j + 32 * u, lo[u], hi[u]);
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (j + 32 * u < len) {
              cf m[kMom];
              unpack_half<float>(lo[u], hi[u], msc, m);
              entry(j + 32 * u, m);
            }
        }
      } else {
        // entries j and j + 32 loaded together (twice the loads in flight),
        // accumulated in the order j, j + 32 of the one-entry loop
        for (int j = lane; j < len; j += 64) {
          cf ma[kMom], mb[kMom];
          const bool two = j + 32 < len;
#pragma unroll
          for (int q = 0; q < kMom; ++q) ma[q] = mom[q * nnz + e0 + j];
          if (two)
#pragma unroll
            for (int q = 0; q < kMom; ++q) mb[q] = mom[q * nnz + e0 + j + 32];
          entry(j, ma);
          if (two) entry(j + 32, mb);
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r >= nr) break;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          acc[r][i].x = warp_sum(acc[r][i].x);
          acc[r][i].y = warp_sum(acc[r][i].y);
        }
        if (lane == 0) {
          C2<Rio>* o = pot + r * sp + 6 * int64_t(t);
#pragma unroll
          for (int i = 0; i < 4; ++i) o[i] = mk<Rio>(Rio(mu0 * acc[r][i].x), Rio(mu0 * acc[r][i].y));
          o[4] = cvt<Rio>(acc[r][4]);
          o[5] = cvt<Rio>(acc[r][5]);
        }
      }
    }
  }
}

// The RB = 4 instance takes more than the 48 KB of shared memory a kernel
// gets without asking: raise its limit once per instance and device (the
// attribute belongs to the current device's copy of the kernel).
static bool device_done(std::atomic<uint64_t>& mask, int* bit) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    *bit = -1;
    return false;
  }
  *bit = dev;
  return (mask.load() >> dev) & 1u;
}

template <typename Rio, bool H16, int RB>
static pie_status near_box_prepare() {
  static std::atomic<uint64_t> done{0};
  int bit = -1;
  if (near_box_smem<RB>() <= 49152 || device_done(done, &bit)) return PIE_OK;
  pie_status s = cuda_check(cudaFuncSetAttribute(k_near_box<Rio, H16, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(near_box_smem<RB>())),
                            "near smem attribute");
  if (s == PIE_OK && bit >= 0) done.fetch_or(uint64_t(1) << bit);
  return s;
}

// Antipode of half-grid sample q (theta rows 0..ntheta/2-1): -khat_q is
// the sample (ntheta-1-i, j+ntheta mod 2 ntheta).
__device__ __forceinline__ int antipode(int q, int ntheta) {
  int nphi = 2 * ntheta;
  int i = q / nphi, j = q % nphi;
  return (ntheta - 1 - i) * nphi + (j + ntheta) % nphi;
}

// a2: leaf aggregation.  One block per leaf box, one thread per half-grid
// sample q.  The radiation tables are stored for the half grid only, since
// Pi(-khat) = conj(Pi(khat)) and M(-khat) = conj(M(khat)); with c X = c Xr +
// i c Xi the pair of samples is S(q) = A + iB, S(-q) = A - iB, where
// A = sum c Xr and B = sum c Xi.
// Small angular grids pack several boxes into one block (threadIdx.y).
template <typename Rf>
__global__ void k_agg(int P, int ntheta, int64_t nb, const int32_t* __restrict__ leaf_start,
                      const C2<Rf>* __restrict__ Pi, const C2<Rf>* __restrict__ M, const C2<Rf>* __restrict__ coef,
                      Rf mu0, C2<Rf>* __restrict__ S, int64_t sc = 0, int64_t sS = 0) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.y + threadIdx.y;
  if (b >= nb) return;
  coef += blockIdx.y * sc;
  S += blockIdx.y * sS;
  const int Ph = P / 2;
  const int t0 = leaf_start[b], t1 = leaf_start[b + 1];
  for (int q = threadIdx.x; q < Ph; q += blockDim.x) {
    C2<Rf> A[kComp], B[kComp];
#pragma unroll
    for (int c = 0; c < kComp; ++c) A[c] = B[c] = mk<Rf>(0, 0);
    // triangle t's coefficients and table entries, then its multiply-adds;
    // in float two triangles' loads are issued together (latency-bound
    // small grids), the multiply-adds still in triangle order
    constexpr int U = sizeof(Rf) == 4 ? 2 : 1;
    struct Tri {
      C2<Rf> c[6], pi, m[3];
    };
    auto load = [&](int t, Tri& r) {
      const C2<Rf>* cf_ = coef + 6 * (int64_t)t;
#pragma unroll
      for (int k = 0; k < 6; ++k) r.c[k] = cf_[k];
      r.pi = Pi[(int64_t)t * Ph + q];
#pragma unroll
      for (int d = 0; d < 3; ++d) r.m[d] = M[((int64_t)t * 3 + d) * Ph + q];
    };
    auto accumulate = [&](const Tri& r) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        rfma(A[d], r.m[d].x, r.c[0]);
        rfma(A[d], r.pi.x, r.c[1 + d]);
        rfma(B[d], r.m[d].y, r.c[0]);
        rfma(B[d], r.pi.y, r.c[1 + d]);
      }
      rfma(A[3], r.pi.x, r.c[4]);
      rfma(B[3], r.pi.y, r.c[4]);
      rfma(A[4], r.pi.x, r.c[5]);
      rfma(B[4], r.pi.y, r.c[5]);
    };
    int t = t0;
    if constexpr (U > 1)
      for (; t + U <= t1; t += U) {
        Tri r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) load(t + u, r[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) accumulate(r[u]);
      }
    for (; t < t1; ++t) {
      Tri r;
      load(t, r);
      accumulate(r);
    }
    const int qa = antipode(q, ntheta);
    C2<Rf>* o = S + (int64_t)b * kComp * P;
#pragma unroll
    for (int c = 0; c < kComp; ++c) {
      Rf f = c < 3 ? mu0 : Rf(1);
      o[c * P + q] = mk<Rf>(f * (A[c].x - B[c].y), f * (A[c].y + B[c].x));
      o[c * P + qa] = mk<Rf>(f * (A[c].x + B[c].y), f * (A[c].y - B[c].x));
    }
  }
}

// a3: interpolation from level l+1 to its parents at level l:
// S_l[b] = sum_children phase_o (F S_child); one block per parent, one thread
// per sample.  The children's patterns are staged in shared memory cg at a
// time (all eight when they fit: one load latency per parent instead of one
// per child), and with fs the filter F^T too (else it is read from global
// memory); children are summed in order, whatever cg.
template <typename Rf>
__global__ void k_interp(int P, int64_t nb, const int32_t* __restrict__ child_start,
                         const int8_t* __restrict__ oct_child, const C2<Rf>* __restrict__ Sc,
                         const Rf* __restrict__ Ft, const C2<Rf>* __restrict__ phase, C2<Rf>* __restrict__ Sp,
                         int64_t sSc = 0, int64_t sSp = 0, int cg = 1, bool fs = false) {
  Sc += blockIdx.y * sSc;
  Sp += blockIdx.y * sSp;
  extern __shared__ unsigned char smem_raw[];
  // the filter (P x P, when fs) first, then one staging region of cg
  // children per threadIdx.y row (small angular grids: one parent per row)
  Rf* fsm = reinterpret_cast<Rf*>(smem_raw);
  const size_t fbytes = fs ? ((sizeof(Rf) * P * P + 15) / 16) * 16 : 0;
  C2<Rf>* sm = reinterpret_cast<C2<Rf>*>(smem_raw + fbytes) + threadIdx.y * cg * kComp * P;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  if (fs)  // P x P reals as 8-byte words (P = 2 N_theta^2 is even)
    for (int i = tid; i < P * P * int(sizeof(Rf)) / 8; i += nth)
      cp_async(reinterpret_cast<uint2*>(fsm) + i, reinterpret_cast<const uint2*>(Ft) + i);
  const Rf* F = fs ? fsm : Ft;
  const int64_t b = int64_t(blockIdx.x) * blockDim.y + threadIdx.y;
  const bool live = b < nb;
  const int c0 = live ? child_start[b] : 0, c1 = live ? child_start[b + 1] : 0;
  const int p = threadIdx.x;
  C2<Rf> acc[kComp];
#pragma unroll
  for (int c = 0; c < kComp; ++c) acc[c] = mk<Rf>(0, 0);
  for (int k0 = c0;; k0 += cg) {
    const int nk = k0 < c1 ? min(cg, c1 - k0) : 0;
    if (!__syncthreads_or(nk > 0)) {  // every row of the block done
      cp_async_wait_all();            // (nothing may stay in flight at exit)
      break;
    }
    // the nk children are consecutive at level l+1: one contiguous copy
    for (int i = threadIdx.x; i < nk * kComp * P; i += blockDim.x) cp_async(sm + i, Sc + (int64_t)k0 * kComp * P + i);
    cp_async_wait_all();  // (also completes the filter's copy)
    __syncthreads();
    for (int k = 0; k < nk && p < P; ++k) {
      const C2<Rf>* sk = sm + k * kComp * P;
      C2<Rf> sum[kComp];
#pragma unroll
      for (int c = 0; c < kComp; ++c) sum[c] = mk<Rf>(0, 0);
#pragma unroll 4
      for (int q = 0; q < P; ++q) {
        Rf f = F[(int64_t)q * P + p];
#pragma unroll
        for (int c = 0; c < kComp; ++c) rfma(sum[c], f, sk[c * P + q]);
      }
      C2<Rf> ph = phase[oct_child[k0 + k] * P + p];
#pragma unroll
      for (int c = 0; c < kComp; ++c) cfma(acc[c], ph, sum[c]);
    }
  }
  if (live && p < P) {
#pragma unroll
    for (int c = 0; c < kComp; ++c) Sp[((int64_t)b * kComp + c) * P + p] = acc[c];
  }
}

// ---- factorised filter: F is block-circulant in azimuth (its entries depend
// on phi_j - phi_j' only), so the length-NPHI DFT along phi turns it into
// one real NT x NT block K_m per azimuthal frequency m:
//   (F s)[i][j] = sum_m e^{i m phi_j} sum_i' K_m[i][i'] shat[i'][m],
//   shat[i'][m] = sum_j e^{-i m phi_j} s[i'][j],  K_m = (1/NPHI) DFT_d f_ii'(d).
// F^T uses K_m transposed.

// Structure used below (N_theta = 8, so NPHI = 16 and degrees up to 7):
//  * K_m = K_{-m}, and K_8 = 0: azimuthal order |m| <= degree <= 7, so the
//    Nyquist frequency m = 8 carries nothing;
//  * the Gauss-Legendre theta nodes are symmetric about the equator and
//    P_l^m(-x) = (-1)^(l+m) P_l^m(x), so every K_m commutes with the row
//    reflection i -> NT-1-i.  In the sums and differences of mirrored rows,
//    se_k = s_k + s_{NT-1-k}, so_k = s_k - s_{NT-1-k} (k < NT/2), K_m is two
//    (NT/2) x (NT/2) blocks:  y_i = ye_i + yo_i, y_{NT-1-i} = ye_i - yo_i with
//    ye = KE se, yo = KO so, KE_ik = (K_ik + K_i,NT-1-k)/2,
//    KO_ik = (K_ik - K_i,NT-1-k)/2.  Half the multiply-adds of the full block.

// 4-point DFT in place, X_k = sum_n x_n w^(nk), w = -i (forward) or +i.
template <bool INV, typename R>
__device__ __forceinline__ void dft4(C2<R>& a, C2<R>& b, C2<R>& c, C2<R>& d) {
  const C2<R> t0 = mk<R>(a.x + c.x, a.y + c.y), t1 = mk<R>(a.x - c.x, a.y - c.y);
  const C2<R> t2 = mk<R>(b.x + d.x, b.y + d.y), t3 = mk<R>(b.x - d.x, b.y - d.y);
  a = mk<R>(t0.x + t2.x, t0.y + t2.y);
  c = mk<R>(t0.x - t2.x, t0.y - t2.y);
  // forward: X1 = t1 - i t3, X3 = t1 + i t3 (inverse: signs swapped)
  const C2<R> p = mk<R>(t1.x + t3.y, t1.y - t3.x), q = mk<R>(t1.x - t3.y, t1.y + t3.x);
  b = INV ? q : p;
  d = INV ? p : q;
}

// v * exp(-/+ 2 pi i E / 16) for the exponents of the 16 = 4 x 4 split.
// cos(pi/8) = sqrt(2 + sqrt 2) / 2, sin(pi/8) = sqrt(2 - sqrt 2) / 2.
template <bool INV, int E, typename R>
__device__ __forceinline__ C2<R> twiddle16(C2<R> v) {
  constexpr double c8 = 0.92387953251128675613, s8 = 0.38268343236508977173, h = 0.70710678118654752440;
  constexpr double c = E == 1 ? c8 : E == 3 ? s8 : E == 9 ? -c8 : 0.0;
  constexpr double s = E == 1 ? s8 : E == 3 ? c8 : E == 9 ? -s8 : 0.0;
  const R x = v.x, y = v.y;
  if constexpr (E == 2) {  // (1 -/+ i) h
    return INV ? mk<R>(R(h) * (x - y), R(h) * (x + y)) : mk<R>(R(h) * (x + y), R(h) * (y - x));
  } else if constexpr (E == 4) {  // -/+ i
    return INV ? mk<R>(-y, x) : mk<R>(y, -x);
  } else if constexpr (E == 6) {  // (-1 -/+ i) h
    return INV ? mk<R>(-R(h) * (x + y), R(h) * (x - y)) : mk<R>(R(h) * (y - x), -R(h) * (x + y));
  } else {  // c -/+ i s
    return INV ? mk<R>(fma(x, R(c), -y * R(s)), fma(y, R(c), x * R(s)))
               : mk<R>(fma(x, R(c), y * R(s)), fma(y, R(c), -x * R(s)));
  }
}

// 16-point DFT in registers, X_k = sum_n x_n exp(-/+ 2 pi i n k / 16) (no
// scaling): n = 4 q + r, k = k1 + 4 k2; 4-point DFTs over q, twiddles
// exp(-/+ 2 pi i r k1 / 16), 4-point DFTs over r.  X is returned in out.
template <bool INV, typename R>
__device__ __forceinline__ void fft16(C2<R>* x, C2<R>* out) {
#pragma unroll
  for (int r = 0; r < 4; ++r) dft4<INV>(x[r], x[r + 4], x[r + 8], x[r + 12]);  // x[r + 4 k1] = Y_r[k1]
  x[5] = twiddle16<INV, 1>(x[5]);
  x[9] = twiddle16<INV, 2>(x[9]);
  x[13] = twiddle16<INV, 3>(x[13]);
  x[6] = twiddle16<INV, 2>(x[6]);
  x[10] = twiddle16<INV, 4>(x[10]);
  x[14] = twiddle16<INV, 6>(x[14]);
  x[7] = twiddle16<INV, 3>(x[7]);
  x[11] = twiddle16<INV, 6>(x[11]);
  x[15] = twiddle16<INV, 9>(x[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) out[k1 + 4 * k2] = x[4 * k1 + k2];
}

constexpr int kFftBatch = 4;  // children per batch in the factorised filter kernels

// Mirror-split blocks of K_m (or of K_m^T when TR) in shared memory:
// KE[m][i][k], KO[m][i][k], i, k < NT/2.
template <int NT, bool TR, typename Rf>
__device__ __forceinline__ void load_split_blocks(const Rf* __restrict__ Kf, Rf* KE, Rf* KO, int tid, int nth) {
  constexpr int NPHI = 2 * NT, H = NT / 2;
  for (int it = tid; it < NPHI * H * H; it += nth) {
    const int m = it / (H * H), i = (it / H) % H, k = it % H;
    const Rf* Km = Kf + m * NT * NT;
    const Rf a = TR ? Km[k * NT + i] : Km[i * NT + k];
    const Rf b = TR ? Km[(NT - 1 - k) * NT + i] : Km[i * NT + NT - 1 - k];
    KE[it] = Rf(0.5) * (a + b);
    KO[it] = Rf(0.5) * (a - b);
  }
}

// One azimuthal frequency m of one (child, component): y = K_m a over the NT
// theta rows (a strided by one in shared memory), written to out[i * BP].
template <int NT, int BP, typename Rf>
__device__ __forceinline__ void apply_split_block(const C2<Rf>* a, const Rf* KE, const Rf* KO, C2<Rf>* out) {
  constexpr int H = NT / 2;
  C2<Rf> se[H], so[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const C2<Rf> u = a[k], v = a[NT - 1 - k];
    se[k] = mk<Rf>(u.x + v.x, u.y + v.y);
    so[k] = mk<Rf>(u.x - v.x, u.y - v.y);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    C2<Rf> ye = mk<Rf>(0, 0), yo = mk<Rf>(0, 0);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      rfma(ye, KE[i * H + k], se[k]);
      rfma(yo, KO[i * H + k], so[k]);
    }
    out[i * BP] = mk<Rf>(ye.x + yo.x, ye.y + yo.y);
    out[(NT - 1 - i) * BP] = mk<Rf>(ye.x - yo.x, ye.y - yo.y);
  }
}

template <int NT, typename Rf>
__host__ __device__ constexpr size_t fft_smem_bytes(bool interp) {
  constexpr int NPHI = 2 * NT, P = NT * NPHI;
  return sizeof(C2<Rf>) * (size_t(kFftBatch) * kComp * NPHI * (NT + 1) + (interp ? size_t(kComp) * P : 0)) +
         sizeof(Rf) * 2 * NPHI * (NT / 2) * (NT / 2);
}

// One K_m block in place on a spectrum column (NT theta rows, stride 1):
// K_8 = 0, the others through their mirror-split halves.
template <int NT, typename Rf>
__device__ __forceinline__ void filter_column(C2<Rf>* col, int m, const Rf* KE, const Rf* KO) {
  constexpr int NPHI = 2 * NT, H = NT / 2;
  if (m == NPHI / 2) {
#pragma unroll
    for (int i = 0; i < NT; ++i) col[i] = mk<Rf>(0, 0);
    return;
  }
  C2<Rf> a[NT];
#pragma unroll
  for (int i = 0; i < NT; ++i) a[i] = col[i];
  apply_split_block<NT, 1>(a, KE + m * H * H, KO + m * H * H, col);
}

// a3 (factorised): one block per parent box, kFftBatch children at a time.
// Per (child, component) one shared-memory region of NPHI x (NT+1) complex
// holds, in turn, the row spectra [m][i], the filtered spectra (the K_m
// blocks act in place on each column m), and the shifted child pattern, row
// i written over the row's own spectra ([j][i]) before it is added to the
// parent's.  Threads:
// one per (child, component, theta row) for the DFTs, one per (child,
// component, azimuthal frequency) for the K_m blocks.
template <int NT, typename Rf>
__global__ void __launch_bounds__(kFftBatch * kComp * NT, 3) k_interp_fft(
    const int32_t* __restrict__ child_start, const int8_t* __restrict__ oct_child, const C2<Rf>* __restrict__ Sc,
    const Rf* __restrict__ Kf, const C2<Rf>* __restrict__ phase, C2<Rf>* __restrict__ Sp, int64_t sSc = 0,
    int64_t sSp = 0) {
  static_assert(NT == 8, "the register DFT is the 16-point one");
  Sc += blockIdx.y * sSc;
  Sp += blockIdx.y * sSp;
  constexpr int NPHI = 2 * NT, P = NT * NPHI, NB = kFftBatch, H = NT / 2;
  // AP: column stride of the spectra (padded by one so that lanes striding
  // over columns hit distinct banks)
  constexpr int AP = NT + 1, REG = NPHI * AP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<Rf>* A = reinterpret_cast<C2<Rf>*>(smem_raw);  // [slot][c] regions of REG complex
  C2<Rf>* acc = A + NB * kComp * REG;                 // parent pattern [c][p]
  Rf* KE = reinterpret_cast<Rf*>(acc + kComp * P);    // mirror-split K_m blocks
  Rf* KO = KE + NPHI * H * H;
  const int tid = threadIdx.x, nth = blockDim.x;
  load_split_blocks<NT, false>(Kf, KE, KO, tid, nth);
  for (int i = tid; i < kComp * P; i += nth) acc[i] = mk<Rf>(0, 0);
  const int b = blockIdx.x, c0 = child_start[b], c1 = child_start[b + 1];
  const int slot = tid / (kComp * NT), c = (tid / NT) % kComp, i = tid % NT;
  for (int base = c0; base < c1; base += NB) {
    const int nb = min(NB, c1 - base);
    C2<Rf>* R = A + (slot * kComp + c) * REG;
    __syncthreads();
    if (slot < nb) {  // forward DFT of every row
      C2<Rf> x[NPHI], X[NPHI];
      const C2<Rf>* src = Sc + ((int64_t)(base + slot) * kComp + c) * P + i * NPHI;
#pragma unroll
      for (int j = 0; j < NPHI; ++j) x[j] = src[j];
      fft16<false>(x, X);
#pragma unroll
      for (int m = 0; m < NPHI; ++m) R[m * AP + i] = X[m];
    }
    __syncthreads();
    for (int it = tid; it < nb * kComp * NPHI; it += nth)  // K_m blocks, in place
      filter_column<NT>(A + (it / NPHI) * REG + (it % NPHI) * AP, it % NPHI, KE, KO);
    __syncthreads();
    if (slot < nb) {  // inverse DFT, phase shift to the parent centre, in the row's own column
      C2<Rf> x[NPHI], X[NPHI];
#pragma unroll
      for (int m = 0; m < NPHI; ++m) x[m] = R[m * AP + i];
      fft16<true>(x, X);
      const C2<Rf>* ph = phase + oct_child[base + slot] * P + i * NPHI;
#pragma unroll
      for (int j = 0; j < NPHI; ++j) R[j * AP + i] = cmul(ph[j], X[j]);
    }
    __syncthreads();
    for (int k = tid; k < kComp * P; k += nth) {
      const int cc = k / P, row = (k / NPHI) % NT, j = k % NPHI;
      C2<Rf> v = acc[k];
      for (int s = 0; s < nb; ++s) {
        const C2<Rf> u = A[(s * kComp + cc) * REG + j * AP + row];
        v.x += u.x;
        v.y += u.y;
      }
      acc[k] = v;
    }
  }
  __syncthreads();
  for (int k = tid; k < kComp * P; k += nth) Sp[(int64_t)b * kComp * P + k] = acc[k];
}

// a5 (factorised): one block per parent box; its children take
// F^T (conj(phase_o) G_parent), added to their incoming patterns.  Same
// shared-memory regions as k_interp_fft, without the parent accumulator.
template <int NT, typename Rf>
__global__ void __launch_bounds__(kFftBatch * kComp * NT, 4) k_anterp_fft(
    const int32_t* __restrict__ child_start, const int8_t* __restrict__ oct_child, const C2<Rf>* __restrict__ Gp,
    const Rf* __restrict__ Kf, const C2<Rf>* __restrict__ phase, C2<Rf>* __restrict__ Gc, int64_t sGp = 0,
    int64_t sGc = 0) {
  static_assert(NT == 8, "the register DFT is the 16-point one");
  Gp += blockIdx.y * sGp;
  Gc += blockIdx.y * sGc;
  constexpr int NPHI = 2 * NT, P = NT * NPHI, NB = kFftBatch, H = NT / 2;
  constexpr int AP = NT + 1, REG = NPHI * AP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<Rf>* A = reinterpret_cast<C2<Rf>*>(smem_raw);
  Rf* KE = reinterpret_cast<Rf*>(A + NB * kComp * REG);
  Rf* KO = KE + NPHI * H * H;
  const int tid = threadIdx.x, nth = blockDim.x;
  load_split_blocks<NT, true>(Kf, KE, KO, tid, nth);
  const int b = blockIdx.x, c0 = child_start[b], c1 = child_start[b + 1];
  const int slot = tid / (kComp * NT), c = (tid / NT) % kComp, i = tid % NT;
  for (int base = c0; base < c1; base += NB) {
    const int nb = min(NB, c1 - base);
    C2<Rf>* R = A + (slot * kComp + c) * REG;
    __syncthreads();
    if (slot < nb) {
      C2<Rf> x[NPHI], X[NPHI];
      const C2<Rf>* src = Gp + ((int64_t)b * kComp + c) * P + i * NPHI;
      const C2<Rf>* ph = phase + oct_child[base + slot] * P + i * NPHI;
#pragma unroll
      for (int j = 0; j < NPHI; ++j) {
        C2<Rf> g = src[j], w = ph[j];
        x[j] = mk<Rf>(w.x * g.x + w.y * g.y, w.x * g.y - w.y * g.x);  // conj(w) g
      }
      fft16<false>(x, X);
#pragma unroll
      for (int m = 0; m < NPHI; ++m) R[m * AP + i] = X[m];
    }
    __syncthreads();
    for (int it = tid; it < nb * kComp * NPHI; it += nth)  // transposed K_m blocks, in place
      filter_column<NT>(A + (it / NPHI) * REG + (it % NPHI) * AP, it % NPHI, KE, KO);
    __syncthreads();
    if (slot < nb) {
      C2<Rf> x[NPHI], X[NPHI];
#pragma unroll
      for (int m = 0; m < NPHI; ++m) x[m] = R[m * AP + i];
      fft16<true>(x, X);
      C2<Rf>* dst = Gc + ((int64_t)(base + slot) * kComp + c) * P + i * NPHI;
#pragma unroll
      for (int j = 0; j < NPHI; ++j) {
        C2<Rf> g = dst[j];
        dst[j] = mk<Rf>(g.x + X[j].x, g.y + X[j].y);
      }
    }
  }
}

// a4: translation at one level: G[d] = sum_{s in IL(d)} T[off] * S[s];
// one destination box per threadIdx.y row of a block (several rows for small
// angular grids), one thread per sample, five components.  In float the
// list is walked U = 4 entries at a time: their loads are issued together
// and the multiply-adds follow in list order (the order of the one-entry
// loop), so a thread waits for one load latency per four entries instead of
// per entry (the small-grid float levels are latency-bound).  In double the
// FP64 pipe bounds the kernel and U = 1 (measured: U = 2 was 0.5 % slower).
template <typename Rf>
__global__ void k_trans(int P, int64_t nb, const int32_t* __restrict__ il_ptr, const int32_t* __restrict__ il_idx,
                        const int32_t* __restrict__ il_off, const C2<Rf>* __restrict__ Tt,
                        const C2<Rf>* __restrict__ S, C2<Rf>* __restrict__ G, int64_t sS = 0) {
  constexpr int U = sizeof(Rf) == 4 ? 4 : 1;
  const int64_t d = int64_t(blockIdx.x) * blockDim.y + threadIdx.y;
  if (d >= nb) return;
  S += blockIdx.y * sS;
  G += blockIdx.y * sS;
  const int j0 = il_ptr[d], j1 = il_ptr[d + 1];
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    C2<Rf> acc[kComp];
#pragma unroll
    for (int c = 0; c < kComp; ++c) acc[c] = mk<Rf>(0, 0);
    int j = j0;
    for (; j + U <= j1; j += U) {
      C2<Rf> tv[U], sv[U][kComp];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        tv[u] = Tt[(int64_t)il_off[j + u] * P + p];
        const C2<Rf>* src = S + (int64_t)il_idx[j + u] * kComp * P + p;
#pragma unroll
        for (int c = 0; c < kComp; ++c) sv[u][c] = src[c * P];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < kComp; ++c) cfma(acc[c], tv[u], sv[u][c]);
    }
    for (; j < j1; ++j) {
      int s = il_idx[j];
      C2<Rf> tv = Tt[(int64_t)il_off[j] * P + p];
      const C2<Rf>* src = S + (int64_t)s * kComp * P + p;
#pragma unroll
      for (int c = 0; c < kComp; ++c) cfma(acc[c], tv, src[c * P]);
    }
#pragma unroll
    for (int c = 0; c < kComp; ++c) G[((int64_t)d * kComp + c) * P + p] = acc[c];
  }
}

// a4 for float patterns of at most 128 samples (the inner operator of the
// nested solve): the interaction list of a box is cut into kTransSplit
// contiguous chunks, one per threadIdx.y sub-row, walked as in k_trans (four
// entries at a time), and the chunks' partial sums are added in chunk order
// through shared memory.  A coarse level has few boxes and long lists, so
// this shortens the chain of dependent loads a thread waits through.  The
// order of operations depends on the list alone, never on the launch shape.
constexpr int kTransSplit = 4;
template <typename Rf>
__global__ void k_trans_split(int P, int64_t nb, const int32_t* __restrict__ il_ptr,
                              const int32_t* __restrict__ il_idx, const int32_t* __restrict__ il_off,
                              const C2<Rf>* __restrict__ Tt, const C2<Rf>* __restrict__ S, C2<Rf>* __restrict__ G,
                              int64_t sS = 0) {
  constexpr int U = 4;
  extern __shared__ unsigned char smem_raw[];
  C2<Rf>* part = reinterpret_cast<C2<Rf>*>(smem_raw);  // [row][chunk][component][P]
  const int r = threadIdx.y / kTransSplit, k = threadIdx.y % kTransSplit, p = threadIdx.x;
  const int64_t d = int64_t(blockIdx.x) * (blockDim.y / kTransSplit) + r;
  const bool live = d < nb && p < P;
  S += blockIdx.y * sS;
  G += blockIdx.y * sS;
  C2<Rf> acc[kComp];
#pragma unroll
  for (int c = 0; c < kComp; ++c) acc[c] = mk<Rf>(0, 0);
  if (live) {
    const int j0 = il_ptr[d], len = il_ptr[d + 1] - j0;
    const int q = (len + kTransSplit - 1) / kTransSplit;
    const int a = j0 + min(len, k * q), b = j0 + min(len, (k + 1) * q);
    int j = a;
    for (; j + U <= b; j += U) {
      C2<Rf> tv[U], sv[U][kComp];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        tv[u] = Tt[(int64_t)il_off[j + u] * P + p];
        const C2<Rf>* src = S + (int64_t)il_idx[j + u] * kComp * P + p;
#pragma unroll
        for (int c = 0; c < kComp; ++c) sv[u][c] = src[c * P];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < kComp; ++c) cfma(acc[c], tv[u], sv[u][c]);
    }
    for (; j < b; ++j) {
      C2<Rf> tv = Tt[(int64_t)il_off[j] * P + p];
      const C2<Rf>* src = S + (int64_t)il_idx[j] * kComp * P + p;
#pragma unroll
      for (int c = 0; c < kComp; ++c) cfma(acc[c], tv, src[c * P]);
    }
  }
  C2<Rf>* mine = part + ((int64_t)(r * kTransSplit + k) * kComp) * P;
  if (p < P && k > 0)
#pragma unroll
    for (int c = 0; c < kComp; ++c) mine[c * P + p] = acc[c];
  __syncthreads();
  if (!live || k > 0) return;
#pragma unroll
  for (int kk = 1; kk < kTransSplit; ++kk) {
    const C2<Rf>* o = part + ((int64_t)(r * kTransSplit + kk) * kComp) * P;
#pragma unroll
    for (int c = 0; c < kComp; ++c) {
      acc[c].x += o[c * P + p].x;
      acc[c].y += o[c * P + p].y;
    }
  }
#pragma unroll
  for (int c = 0; c < kComp; ++c) G[((int64_t)d * kComp + c) * P + p] = acc[c];
}

// a5: anterpolation from level l to level l+1:
// G_child += F^T (conj(phase_o) G_parent); one child box per threadIdx.y
// row of a block (several rows for small angular grids).  With fs the
// filter F is staged in shared memory first (else read from global memory).
template <typename Rf>
__global__ void k_anterp(int P, int64_t nc, const int32_t* __restrict__ parent, const int8_t* __restrict__ oct_child,
                         const C2<Rf>* __restrict__ Gp, const Rf* __restrict__ Fg, const C2<Rf>* __restrict__ phase,
                         C2<Rf>* __restrict__ Gc, int64_t sGp = 0, int64_t sGc = 0, bool fs = false) {
  Gp += blockIdx.y * sGp;
  Gc += blockIdx.y * sGc;
  extern __shared__ unsigned char smem_raw[];
  Rf* fsm = reinterpret_cast<Rf*>(smem_raw);
  const size_t fbytes = fs ? ((sizeof(Rf) * P * P + 15) / 16) * 16 : 0;
  C2<Rf>* sm = reinterpret_cast<C2<Rf>*>(smem_raw + fbytes) + threadIdx.y * kComp * P;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  if (fs)  // P x P reals as 8-byte words (P = 2 N_theta^2 is even)
    for (int i = tid; i < P * P * int(sizeof(Rf)) / 8; i += nth)
      cp_async(reinterpret_cast<uint2*>(fsm) + i, reinterpret_cast<const uint2*>(Fg) + i);
  const Rf* F = fs ? fsm : Fg;
  const int64_t ch = int64_t(blockIdx.x) * blockDim.y + threadIdx.y;
  const bool live = ch < nc;
  const int par = live ? parent[ch] : 0;
  const int o = live ? oct_child[ch] : 0;
  // the parent's pattern copied in, then turned in place by the thread
  // that copied each entry: conj(phase_o) G_parent
  for (int i = threadIdx.x; live && i < kComp * P; i += blockDim.x) cp_async(sm + i, Gp + (int64_t)par * kComp * P + i);
  cp_async_wait_all();
  for (int i = threadIdx.x; live && i < kComp * P; i += blockDim.x) {
    const int q = i % P;
    const C2<Rf> g = sm[i], ph = phase[o * P + q];
    C2<Rf> h;
    h.x = ph.x * g.x + ph.y * g.y;   // conj(ph) * g
    h.y = ph.x * g.y - ph.y * g.x;
    sm[i] = h;
  }
  __syncthreads();
  if (!live) return;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    C2<Rf> sum[kComp];
#pragma unroll
    for (int c = 0; c < kComp; ++c) sum[c] = mk<Rf>(0, 0);
#pragma unroll 4
    for (int q = 0; q < P; ++q) {
      Rf f = F[(int64_t)q * P + p];
#pragma unroll
      for (int c = 0; c < kComp; ++c) rfma(sum[c], f, sm[c * P + q]);
    }
#pragma unroll
    for (int c = 0; c < kComp; ++c) {
      C2<Rf>& g = Gc[((int64_t)ch * kComp + c) * P + p];
      g.x += sum[c].x;
      g.y += sum[c].y;
    }
  }
}

// Sum and difference of the incoming leaf patterns over antipodal sample
// pairs, once per box: GS[b][c][q] = G(q) + G(-q), GD[b][c][q] = G(q) - G(-q)
// (half grid q), shared by all triangles of the box in the disaggregation.
template <typename Rf>
__global__ void k_gsgd(int P, int ntheta, const C2<Rf>* __restrict__ G, C2<Rf>* __restrict__ GS,
                       C2<Rf>* __restrict__ GD, int64_t sG = 0, int64_t sH = 0) {
  const int b = blockIdx.x;
  const int Ph = P / 2;
  G += blockIdx.y * sG;
  GS += blockIdx.y * sH;
  GD += blockIdx.y * sH;
  for (int i = threadIdx.x; i < kComp * Ph; i += blockDim.x) {
    const int c = i / Ph, q = i % Ph;
    const C2<Rf> u = G[((int64_t)b * kComp + c) * P + q];
    const C2<Rf> v = G[((int64_t)b * kComp + c) * P + antipode(q, ntheta)];
    GS[((int64_t)b * kComp + c) * Ph + q] = mk<Rf>(u.x + v.x, u.y + v.y);
    GD[((int64_t)b * kComp + c) * Ph + q] = mk<Rf>(u.x - v.x, u.y - v.y);
  }
}

// a6: leaf disaggregation with the receiving (conjugate) patterns.  One
// thread per triangle; the receiving tables are stored sample-major
// ([Ph][T], [3][Ph][T]) so that consecutive threads read consecutive
// triangles, and the box's sum / difference patterns are shared through the
// cache.  Over a sample pair (q, -q):
// conj(X(q)) G(q) + X(q) G(-q) = Xr (G(q) + G(-q)) - i Xi (G(q) - G(-q)).
// Adds to pot[t].
template <typename Rf, typename Rio>
__global__ void __launch_bounds__(256) k_disagg(int64_t T, int P, const int32_t* __restrict__ leaf_of,
                                                const C2<Rf>* __restrict__ PiR, const C2<Rf>* __restrict__ MR,
                                                const C2<Rf>* __restrict__ GS, const C2<Rf>* __restrict__ GD,
                                                C2<Rio>* __restrict__ pot, int64_t sH = 0, int64_t sp = 0) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int Ph = P / 2;
  GS += blockIdx.y * sH + (int64_t)leaf_of[t] * kComp * Ph;
  GD += blockIdx.y * sH + (int64_t)leaf_of[t] * kComp * Ph;
  pot += blockIdx.y * sp;
  C2<Rf> acc[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) acc[i] = mk<Rf>(0, 0);
  // sample pair q's patterns and table entries, then its multiply-adds
  // (issuing two sample pairs' loads together was measured slower at
  // N = 819,200 in float: 0.096 against 0.085 ms)
  struct Sample {
    C2<Rf> gs[kComp], gd[kComp], pi, m[3];
  };
  auto load = [&](int q, Sample& r) {
#pragma unroll
    for (int c = 0; c < kComp; ++c) {
      r.gs[c] = GS[c * Ph + q];
      r.gd[c] = GD[c * Ph + q];
    }
    r.pi = PiR[(int64_t)q * T + t];
#pragma unroll
    for (int d = 0; d < 3; ++d) r.m[d] = MR[((int64_t)d * Ph + q) * T + t];
  };
  auto accumulate = [&](const Sample& r) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const C2<Rf> m = r.m[d];
      // U += Mr gs - i Mi gd
      rfma(acc[0], m.x, r.gs[d]);
      acc[0].x = fma(m.y, r.gd[d].y, acc[0].x);
      acc[0].y = fma(-m.y, r.gd[d].x, acc[0].y);
      // V_d += Pr gs - i Pi gd
      rfma(acc[1 + d], r.pi.x, r.gs[d]);
      acc[1 + d].x = fma(r.pi.y, r.gd[d].y, acc[1 + d].x);
      acc[1 + d].y = fma(-r.pi.y, r.gd[d].x, acc[1 + d].y);
    }
#pragma unroll
    for (int c = 3; c < 5; ++c) {
      rfma(acc[1 + c], r.pi.x, r.gs[c]);
      acc[1 + c].x = fma(r.pi.y, r.gd[c].y, acc[1 + c].x);
      acc[1 + c].y = fma(-r.pi.y, r.gd[c].x, acc[1 + c].y);
    }
  };
  for (int q = 0; q < Ph; ++q) {
    Sample r;
    load(q, r);
    accumulate(r);
  }
  C2<Rio>* o = pot + 6 * t;
#pragma unroll
  for (int i = 0; i < 6; ++i) o[i] = mk<Rio>(Rio(acc[i].x), Rio(acc[i].y));
}

// Per-triangle potential j of the product: near + far (each rounded to the
// io precision, summed in double, rounded again), or pot alone.
template <typename Rio>
__device__ __forceinline__ C2<Rio> pot_sum(const C2<Rio>* pot, const C2<Rio>* pot2, int64_t j) {
  if (!pot2) return pot[j];
  const C2<Rio> a = pot2[j], b = pot[j];
  return mk<Rio>(Rio(double(a.x) + double(b.x)), Rio(double(a.y) + double(b.y)));
}

// a7: Galerkin testing of the per-triangle potentials (Section 2):
// RWG m: sum over its two triangles of c [U + (c_t - p).V] + 2c T1; pulse t: T2.
// pot2 (may be null): near-part potentials, added to pot first.
template <typename Rio>
__global__ void k_assemble(int64_t N, int64_t E, const int32_t* __restrict__ edge_tt,
                           const int8_t* __restrict__ edge_k, const double* __restrict__ tri_c,
                           const double* __restrict__ tri_dcp, const int64_t* __restrict__ inv_perm,
                           const C2<Rio>* __restrict__ pot, C2<Rio>* __restrict__ y, int64_t sp = 0, int64_t sy = 0,
                           const C2<Rio>* __restrict__ pot2 = nullptr) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  pot += blockIdx.y * sp;
  if (pot2) pot2 += blockIdx.y * sp;
  y += blockIdx.y * sy;
  if (i < E) {
    double yr = 0, yi = 0;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int64_t t = edge_tt[2 * i + side];
      int k = edge_k[2 * i + side];
      double c = tri_c[3 * t + k];
      const double* dcp = tri_dcp + 9 * t + 3 * k;
      C2<Rio> p[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) p[j] = pot_sum(pot, pot2, 6 * t + j);
      double ur = double(p[0].x) + dcp[0] * double(p[1].x) + dcp[1] * double(p[2].x) + dcp[2] * double(p[3].x);
      double ui = double(p[0].y) + dcp[0] * double(p[1].y) + dcp[1] * double(p[2].y) + dcp[2] * double(p[3].y);
      yr += c * (ur + 2.0 * double(p[4].x));
      yi += c * (ui + 2.0 * double(p[4].y));
    }
    y[i] = mk<Rio>(Rio(yr), Rio(yi));
  } else {
    int64_t t = inv_perm[i - E];
    y[i] = pot_sum(pot, pot2, 6 * t + 5);
  }
}

// ---------------------------------------------------------------- orchestration

static inline unsigned nblk(int64_t n, int b) { return unsigned((n + b - 1) / b); }

static inline MomScale mom_scale(const Problem& pr) {
  MomScale m;
  for (int q = 0; q < kMom; ++q) m.s[q] = pr.mom_scale[q];
  return m;
}

void prof_mark(Problem& pr, int stage, bool end, cudaStream_t st) {
  if (pr.prof_n >= pr.prof_cap) return;
  cudaEventRecord(pr.prof_ev[(size_t(pr.prof_n) * kStages + stage) * 2 + (end ? 1 : 0)], st);
}

template <int NT, typename Rf>
static size_t fft_smem(bool interp) {
  return fft_smem_bytes<NT, Rf>(interp);
}

// Opt the factorised filter kernels into their (above 48 KB) dynamic shared memory.
template <int NT, typename Rf>
static pie_status fft_prepare() {
  static std::atomic<uint64_t> done{0};  // per device, as near_box_prepare
  int bit = -1;
  if (device_done(done, &bit)) return PIE_OK;
  pie_status s = cuda_check(cudaFuncSetAttribute(k_interp_fft<NT, Rf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(fft_smem<NT, Rf>(true))),
                            "smem attribute");
  if (s == PIE_OK)
    s = cuda_check(cudaFuncSetAttribute(k_anterp_fft<NT, Rf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(fft_smem<NT, Rf>(false))),
                   "smem attribute");
  if (s == PIE_OK && bit >= 0) done.fetch_or(uint64_t(1) << bit);
  return s;
}

template <typename Rm, typename Rf, typename Rio, bool H16 = false>
static pie_status apply_t(Problem& pr, const void* xv, void* yv, int nrhs, cudaStream_t st) {
  const int P = pr.P;
  const int L = pr.tree.L;
  const C2<Rio>* x = static_cast<const C2<Rio>*>(xv);
  C2<Rio>* y = static_cast<C2<Rio>*>(yv);
  C2<Rio>* coef = static_cast<C2<Rio>*>(pr.coef);
  C2<Rio>* pot = static_cast<C2<Rio>*>(pr.pot);
  const double w2e = pr.w * pr.w * eps0();
  const unsigned nr = unsigned(nrhs);
  const int64_t sN = pr.N, sT = 6 * pr.T;  // right-hand-side strides of x / y and of coef / pot
  constexpr bool split = sizeof(Rm) < sizeof(Rio);  // float near part, double coefficients
  cf* coef32 = split ? static_cast<cf*>(pr.coef32) : nullptr;
  const C2<Rm>* ncoef = split ? reinterpret_cast<const C2<Rm>*>(coef32) : reinterpret_cast<const C2<Rm>*>(coef);
  prof_mark(pr, 0, false, st);
  k_coef<Rio><<<dim3(nblk(pr.T, 256), nr), 256, 0, st>>>(pr.T, pr.E, x, pr.perm, pr.tri_edge, pr.tri_c, pr.tri_dcp,
                                                         w2e, coef, coef32, sN, sT);
  prof_mark(pr, 0, true, st);
  // near part into pot2, far part into pot.  With tune.overlap the near part
  // runs on the side stream (HBM-bound, a bounded grid) and the far part on
  // the problem's high-priority stream, concurrently; per-stage profiling
  // keeps them in order on the caller's stream.
  const bool profiling = pr.prof_n < pr.prof_cap;
  const bool with_near = pr.with_near;
  const bool overlap = pr.tune.overlap && !profiling && with_near;
  C2<Rio>* pot2 = static_cast<C2<Rio>*>(pr.pot2);
  cudaStream_t sn = st, sf = st;
  unsigned near_grid = nblk(pr.T * 32, 256);
  if (overlap) {
    // inside a stream capture (a multi-mesh group's graph) the far part
    // stays on the capturing stream: with every member's far part at the
    // highest priority the members' near parts waited for all of them
    // (group launch 131.4 -> 137.6 ms for the four configuration-3 meshes)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    pie_status s = cuda_check(cudaStreamIsCapturing(st, &cap), "capture status");
    if (s == PIE_OK) s = cuda_check(cudaEventRecord(pr.ev_fork, st), "fork");
    if (s == PIE_OK) s = cuda_check(cudaStreamWaitEvent(pr.side, pr.ev_fork, 0), "fork");
    if (s == PIE_OK && cap == cudaStreamCaptureStatusNone)
      s = cuda_check(cudaStreamWaitEvent(pr.far, pr.ev_fork, 0), "fork");
    if (s != PIE_OK) return s;
    sn = pr.side;
    if (cap == cudaStreamCaptureStatusNone) sf = pr.far;
    if (pr.tune.near_ctas_per_sm > 0)
      near_grid = std::min<unsigned>(near_grid, unsigned(pr.nsm * pr.tune.near_ctas_per_sm));
  }
  prof_mark(pr, 1, false, st);
  // the near part reads each pair's moments once for RB right-hand sides
  // (RB chosen per call: a wide accumulator set costs occupancy when unused)
  auto near_launch = [&](auto rb) {
    constexpr int RB = decltype(rb)::value;
    k_near<Rm, Rio, RB, H16><<<dim3(near_grid, unsigned((nrhs + RB - 1) / RB)), 256, 0, sn>>>(
        pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr,
        static_cast<const C2<Rm>*>(pr.mom), static_cast<const __half2*>(pr.mom), mom_scale(pr), ncoef, Rm(kMu0),
        pot2, nrhs, sT, sT);
  };
  // float near part: the box-staged kernel (RB 1, 2 or 4) for one column,
  // or for any pass when tune.near_kernel is 2; otherwise one warp per test
  // triangle (RB 1, 2, 4 or 8).  The box kernel measured slower on passes of
  // many columns of small meshes whose rows outgrow its staging buffer.
  int rb = pr.tune.near_rhs_block;
  if (rb == 0) rb = nrhs == 1 ? 1 : (nrhs == 2 || sizeof(Rm) == 8) ? 2 : nrhs <= 4 ? 4 : 8;
  const bool boxed = sizeof(Rm) == 4 && (pr.tune.near_kernel == 2 || (pr.tune.near_kernel == 0 && rb == 1));
  auto box_launch = [&](auto rbc) -> pie_status {
    if constexpr (sizeof(Rm) == 4) {
      constexpr int RB = decltype(rbc)::value;
      pie_status s = near_box_prepare<Rio, H16, RB>();
      if (s != PIE_OK) return s;
      unsigned grid = unsigned(pr.nleaf);
      if (overlap && pr.tune.near_ctas_per_sm > 0)  // in CTAs of 256 threads per SM
        grid = std::min<unsigned>(grid, unsigned(pr.nsm * pr.tune.near_ctas_per_sm * (256 / kNearBoxThreads)));
      k_near_box<Rio, H16, RB><<<dim3(grid, unsigned((nrhs + RB - 1) / RB)), kNearBoxThreads, near_box_smem<RB>(),
                                 sn>>>(pr.nleaf, pr.nnz, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off,
                                       pr.row_ptr, static_cast<const cf*>(pr.mom),
                                       static_cast<const __half2*>(pr.mom), mom_scale(pr),
                                       reinterpret_cast<const cf*>(ncoef), float(kMu0), pot2, nrhs, sT, sT);
    }
    return PIE_OK;
  };
  if (!with_near) {
    pot2 = nullptr;
  } else if (boxed && (rb == 1 || rb == 2 || rb == 4)) {
    pie_status s = rb == 1   ? box_launch(std::integral_constant<int, 1>())
                   : rb == 2 ? box_launch(std::integral_constant<int, 2>())
                             : box_launch(std::integral_constant<int, 4>());
    if (s != PIE_OK) return s;
  } else if (rb == 1)
    near_launch(std::integral_constant<int, 1>());
  else if (rb == 2)
    near_launch(std::integral_constant<int, 2>());
  else if (rb == 4)
    near_launch(std::integral_constant<int, 4>());
  else
    near_launch(std::integral_constant<int, 8>());
  if (overlap) {
    pie_status s = cuda_check(cudaEventRecord(pr.ev_join, sn), "join");
    if (s != PIE_OK) return s;
  }
  prof_mark(pr, 1, true, st);
  const int tpb = P < 1024 ? ((P + 31) / 32) * 32 : 1024;
  const C2<Rf>* Pi = static_cast<const C2<Rf>*>(pr.Pi);
  const C2<Rf>* M = static_cast<const C2<Rf>*>(pr.M);
  auto sl = [&](int l) { return int64_t(pr.lev[l].nb) * kComp * P; };  // pattern stride per right-hand side
  prof_mark(pr, 2, false, st);
  // far coefficients in the far precision (MIXED and FP64: the io buffer)
  const C2<Rf>* fcoef = reinterpret_cast<const C2<Rf>*>(coef);
  // boxes per block of the per-box far kernels (threads: one per sample):
  // tune.far_rows, or enough to fill 128 threads; at most 1024 threads
  auto far_rows = [&](int threads) {
    const int r = pr.tune.far_rows > 0 ? pr.tune.far_rows : (threads < 64 ? 128 / threads : 1);
    return std::max(1, std::min(r, 1024 / threads));
  };
  {
    // half-grid threads per box
    const int ath = P / 2 < 32 ? P / 2 : ((P / 2 + 31) / 32) * 32;
    const int abp = far_rows(ath);
    k_agg<Rf><<<dim3(nblk(pr.lev[L].nb, abp), nr), dim3(ath, abp), 0, sf>>>(
        P, pr.par.ntheta, pr.lev[L].nb, pr.leaf_start, Pi, M, fcoef, Rf(kMu0), static_cast<C2<Rf>*>(pr.lev[L].S),
        sT, sl(L));
  }
  prof_mark(pr, 2, true, st);
  const size_t sm = sizeof(C2<Rf>) * kComp * P;
  // dense-filter kernels: the P x P filter in shared memory when it is at
  // most 16 KB; boxes per block within 48 KB of shared memory; interpolation
  // stages up to eight children per parent in what is left
  const size_t fsb = ((sizeof(Rf) * size_t(P) * P + 15) / 16) * 16;
  const bool fsh = fsb <= 16384;
  const size_t fsm_bytes = fsh ? fsb : 0;
  const int fbp = std::max(1, std::min(far_rows(tpb), int((49152 - fsm_bytes) / sm)));
  const int cg = int(std::max<size_t>(1, std::min<size_t>(8, (49152 - fsm_bytes) / (sm * fbp))));
  const bool fft8 = pr.par.ntheta == 8;
  if (fft8) {
    pie_status s = fft_prepare<8, Rf>();
    if (s != PIE_OK) return s;
  }
  prof_mark(pr, 3, false, st);
  for (int l = L - 1; l >= 3 && fft8; --l) {
    k_interp_fft<8, Rf><<<dim3(unsigned(pr.lev[l].nb), nr), kFftBatch * kComp * 8, fft_smem<8, Rf>(true), sf>>>(
        pr.lev[l].child_start, pr.lev[l + 1].octant, static_cast<const C2<Rf>*>(pr.lev[l + 1].S),
        static_cast<const Rf*>(pr.lev[l].Kf), static_cast<const C2<Rf>*>(pr.lev[l].phase),
        static_cast<C2<Rf>*>(pr.lev[l].S), sl(l + 1), sl(l));
  }
  for (int l = L - 1; l >= 3 && !fft8; --l) {
    k_interp<Rf><<<dim3(nblk(pr.lev[l].nb, fbp), nr), dim3(tpb, fbp), fsm_bytes + sm * fbp * cg, sf>>>(
        P, pr.lev[l].nb, pr.lev[l].child_start, pr.lev[l + 1].octant, static_cast<const C2<Rf>*>(pr.lev[l + 1].S),
        static_cast<const Rf*>(pr.lev[l].Ft), static_cast<const C2<Rf>*>(pr.lev[l].phase),
        static_cast<C2<Rf>*>(pr.lev[l].S), sl(l + 1), sl(l), cg, fsh);
  }
  prof_mark(pr, 3, true, st);
  prof_mark(pr, 4, false, st);
  for (int l = 3; l <= L; ++l) {
    if (!((pr.far_mask >> l) & 1u)) {  // level left out: no incoming pattern of its own
      pie_status s = cuda_check(cudaMemsetAsync(pr.lev[l].G, 0, sizeof(C2<Rf>) * sl(l) * nr, sf), "memset");
      if (s != PIE_OK) return s;
      continue;
    }
    bool split_done = false;
    if constexpr (sizeof(Rf) == 4) {
      if (tpb <= 128) {  // float, small grid: each list cut into kTransSplit chunks
        const int tbp = far_rows(tpb * kTransSplit);
        k_trans_split<Rf><<<dim3(nblk(pr.lev[l].nb, tbp), nr), dim3(tpb, tbp * kTransSplit),
                            sizeof(C2<Rf>) * kComp * P * kTransSplit * tbp, sf>>>(
            P, pr.lev[l].nb, pr.lev[l].il_ptr, pr.lev[l].il_idx, pr.lev[l].il_off,
            static_cast<const C2<Rf>*>(pr.lev[l].trans), static_cast<const C2<Rf>*>(pr.lev[l].S),
            static_cast<C2<Rf>*>(pr.lev[l].G), sl(l));
        split_done = true;
      }
    }
    if (!split_done) {
      const int tbp = far_rows(tpb);  // destination boxes per block
      k_trans<Rf><<<dim3(nblk(pr.lev[l].nb, tbp), nr), dim3(tpb, tbp), 0, sf>>>(
          P, pr.lev[l].nb, pr.lev[l].il_ptr, pr.lev[l].il_idx, pr.lev[l].il_off,
          static_cast<const C2<Rf>*>(pr.lev[l].trans), static_cast<const C2<Rf>*>(pr.lev[l].S),
          static_cast<C2<Rf>*>(pr.lev[l].G), sl(l));
    }
  }
  prof_mark(pr, 4, true, st);
  prof_mark(pr, 5, false, st);
  for (int l = 3; l < L && fft8; ++l) {
    k_anterp_fft<8, Rf><<<dim3(unsigned(pr.lev[l].nb), nr), kFftBatch * kComp * 8, fft_smem<8, Rf>(false), sf>>>(
        pr.lev[l].child_start, pr.lev[l + 1].octant, static_cast<const C2<Rf>*>(pr.lev[l].G),
        static_cast<const Rf*>(pr.lev[l].Kf), static_cast<const C2<Rf>*>(pr.lev[l].phase),
        static_cast<C2<Rf>*>(pr.lev[l + 1].G), sl(l), sl(l + 1));
  }
  for (int l = 3; l < L && !fft8; ++l) {
    k_anterp<Rf><<<dim3(nblk(pr.lev[l + 1].nb, fbp), nr), dim3(tpb, fbp), fsm_bytes + sm * fbp, sf>>>(
        P, pr.lev[l + 1].nb, pr.lev[l + 1].parent, pr.lev[l + 1].octant, static_cast<const C2<Rf>*>(pr.lev[l].G),
        static_cast<const Rf*>(pr.lev[l].F), static_cast<const C2<Rf>*>(pr.lev[l].phase),
        static_cast<C2<Rf>*>(pr.lev[l + 1].G), sl(l), sl(l + 1), fsh);
  }
  prof_mark(pr, 5, true, st);
  prof_mark(pr, 6, false, st);
  {
    C2<Rf>* GS = static_cast<C2<Rf>*>(pr.gsgd);
    C2<Rf>* GD = GS + int64_t(pr.par.max_nrhs) * pr.lev[L].nb * kComp * (P / 2);
    const int64_t sH = int64_t(pr.lev[L].nb) * kComp * (P / 2);
    k_gsgd<Rf><<<dim3(unsigned(pr.lev[L].nb), nr), 128, 0, sf>>>(P, pr.par.ntheta,
                                                                 static_cast<const C2<Rf>*>(pr.lev[L].G), GS, GD,
                                                                 sl(L), sH);
    k_disagg<Rf, Rio><<<dim3(nblk(pr.T, 256), nr), 256, 0, sf>>>(
        pr.T, P, pr.leaf_of, static_cast<const C2<Rf>*>(pr.PiR), static_cast<const C2<Rf>*>(pr.MR), GS, GD, pot, sH,
        sT);
  }
  prof_mark(pr, 6, true, st);
  if (overlap) {
    pie_status s = PIE_OK;
    if (sf != st) {
      s = cuda_check(cudaEventRecord(pr.ev_far, sf), "join");
      if (s == PIE_OK) s = cuda_check(cudaStreamWaitEvent(st, pr.ev_far, 0), "join");
    }
    if (s == PIE_OK) s = cuda_check(cudaStreamWaitEvent(st, pr.ev_join, 0), "join");
    if (s != PIE_OK) return s;
  }
  prof_mark(pr, 7, false, st);
  k_assemble<Rio><<<dim3(nblk(pr.N, 256), nr), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c,
                                                             pr.tri_dcp, pr.inv_perm, pot, y, sT, sN, pot2);
  prof_mark(pr, 7, true, st);
  if (pr.prof_n < pr.prof_cap) ++pr.prof_n;
  return cuda_check(cudaGetLastError(), "apply launch");
}

// Near part alone: y = Z_near x (pairs of triangles in neighbouring leaf boxes).
template <typename Rm, typename Rio, bool H16 = false>
static pie_status apply_near_t(Problem& pr, const void* xv, void* yv, cudaStream_t st) {
  C2<Rio>* coef = static_cast<C2<Rio>*>(pr.coef);
  C2<Rio>* pot = static_cast<C2<Rio>*>(pr.pot);
  constexpr bool split = sizeof(Rm) < sizeof(Rio);
  cf* coef32 = split ? static_cast<cf*>(pr.coef32) : nullptr;
  const C2<Rm>* ncoef = split ? reinterpret_cast<const C2<Rm>*>(coef32) : reinterpret_cast<const C2<Rm>*>(coef);
  k_coef<Rio><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const C2<Rio>*>(xv), pr.perm, pr.tri_edge,
                                               pr.tri_c, pr.tri_dcp, pr.w * pr.w * eps0(), coef, coef32);
  bool boxed = false;  // the box-staged kernel (float near part, unless tuned off)
  if constexpr (sizeof(Rm) == 4) {
    if (pr.tune.near_kernel != 1) {
      k_near_box<Rio, H16, 1><<<unsigned(pr.nleaf), kNearBoxThreads, near_box_smem<1>(), st>>>(
          pr.nleaf, pr.nnz, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr,
          static_cast<const cf*>(pr.mom), static_cast<const __half2*>(pr.mom), mom_scale(pr), ncoef, float(kMu0),
          pot);
      boxed = true;
    }
  }
  if (!boxed)
    k_near<Rm, Rio, 1, H16><<<nblk(pr.T * 32, 256), 256, 0, st>>>(
        pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr,
        static_cast<const C2<Rm>*>(pr.mom), static_cast<const __half2*>(pr.mom), mom_scale(pr), ncoef, Rm(kMu0),
        pot);
  k_assemble<Rio><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                   pr.inv_perm, pot, static_cast<C2<Rio>*>(yv));
  return cuda_check(cudaGetLastError(), "apply_near launch");
}

pie_status apply_near_one(Problem& pr, const void* x, void* y, cudaStream_t st) {
  switch (pr.par.precision) {
    case PIE_FP64:
      return apply_near_t<double, double>(pr, x, y, st);
    case PIE_FP32:
      return apply_near_t<float, float>(pr, x, y, st);
    case PIE_FP32H:
      return apply_near_t<float, float, true>(pr, x, y, st);
    default:
      return apply_near_t<float, double>(pr, x, y, st);
  }
}

pie_status apply_batch(Problem& pr, const void* x, void* y, int nrhs, cudaStream_t st) {
  if (nrhs < 1 || nrhs > pr.par.max_nrhs) {
    set_error("batch larger than max_nrhs");
    return PIE_ERR_PARAM;
  }
  switch (pr.par.precision) {
    case PIE_FP64:
      return apply_t<double, double, double>(pr, x, y, nrhs, st);
    case PIE_FP32:
      return apply_t<float, float, float>(pr, x, y, nrhs, st);
    case PIE_MIXED:
      return apply_t<float, double, double>(pr, x, y, nrhs, st);
    case PIE_FP32H:
      return apply_t<float, float, float, true>(pr, x, y, nrhs, st);
  }
  set_error("unknown precision");
  return PIE_ERR_PARAM;
}

pie_status apply_one(Problem& pr, const void* x, void* y, cudaStream_t st) { return apply_batch(pr, x, y, 1, st); }

pie_status prepare_apply(Problem& pr) {
  if (pr.par.ntheta != 8) return PIE_OK;
  return pr.far_f32() ? fft_prepare<8, float>() : fft_prepare<8, double>();
}

pie_status apply_cols(Problem& pr, const void* x, void* y, int nrhs, cudaStream_t st) {
  const size_t col = (pr.io_f32() ? sizeof(cf) : sizeof(cd)) * size_t(pr.N);
  const int chunk = std::max(1, std::min(pr.tune.rhs_chunk, pr.par.max_nrhs));
  for (int j = 0; j < nrhs; j += chunk) {
    pie_status s = apply_batch(pr, static_cast<const char*>(x) + col * j, static_cast<char*>(y) + col * j,
                               std::min(chunk, nrhs - j), st);
    if (s != PIE_OK) return s;
  }
  return PIE_OK;
}

// ---------------------------------------------------------------- right-hand side

// Per triangle (tree order) the integrals of the plane-wave potentials with
// the 7-point rule, stored in the potential layout so that k_assemble forms
// b_J = -<f_m, A> and b_sigma = -i w eps0 <p_t, Phi>:
//   U = -int (r - c_t).A,  V = -int A,  T1 = 0,  T2 = -i w eps0 int Phi.
template <typename Rio>
__global__ void k_rhs(int64_t T, const double* __restrict__ vert, const double* __restrict__ cent,
                      const double* __restrict__ area, double k0, double kx, double ky, double kz, double ex,
                      double ey, double ez, double E0, double weps, const double* __restrict__ rule,
                      C2<Rio>* __restrict__ pot) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
  const double* v = vert + 9 * t;
  double Ur = 0, Ui = 0, Vr[3] = {0, 0, 0}, Vi[3] = {0, 0, 0}, Pr = 0, Pim = 0;
  for (int q = 0; q < 7; ++q) {
    double b0 = rule[4 * q], b1 = rule[4 * q + 1], b2 = rule[4 * q + 2], wq = rule[4 * q + 3] * area[t];
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = b0 * v[d] + b1 * v[3 + d] + b2 * v[6 + d];
    double s, c;
    sincos(k0 * (kx * r[0] + ky * r[1] + kz * r[2]), &s, &c);
    double er = ex * r[0] + ey * r[1] + ez * r[2];
    // Phi = -E0 (e.r) e^{i phase};  A = -(E0/c0)(e.r) khat e^{i phase}
    double phr = -E0 * er * c, phi = -E0 * er * s;
    Pr += wq * phr;
    Pim += wq * phi;
    double ar = phr / kC0, ai = phi / kC0;
    double kh[3] = {kx, ky, kz};
    double ud = 0;
    for (int d = 0; d < 3; ++d) ud += (r[d] - cent[3 * t + d]) * kh[d];
    Ur += wq * ud * ar;
    Ui += wq * ud * ai;
    for (int d = 0; d < 3; ++d) {
      Vr[d] += wq * kh[d] * ar;
      Vi[d] += wq * kh[d] * ai;
    }
  }
  C2<Rio>* o = pot + 6 * t;
  o[0] = mk<Rio>(Rio(-Ur), Rio(-Ui));
  for (int d = 0; d < 3; ++d) o[1 + d] = mk<Rio>(Rio(-Vr[d]), Rio(-Vi[d]));
  o[4] = mk<Rio>(0, 0);
  // -i weps (Pr + i Pim) = weps Pim - i weps Pr
  o[5] = mk<Rio>(Rio(weps * Pim), Rio(-weps * Pr));
}

pie_status rhs_planewave(Problem& pr, const double* khat, const double* pol, double E0, void* b, cudaStream_t st) {
  const double* rule = pr.rule7;
  const double weps = pr.w * eps0();
  if (pr.io_f32()) {
    k_rhs<float><<<nblk(pr.T, 128), 128, 0, st>>>(pr.T, pr.vert, pr.cent, pr.area, pr.k0, khat[0], khat[1], khat[2],
                                                  pol[0], pol[1], pol[2], E0, weps, rule, static_cast<cf*>(pr.pot));
    k_assemble<float><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                       pr.inv_perm, static_cast<cf*>(pr.pot), static_cast<cf*>(b));
  } else {
    k_rhs<double><<<nblk(pr.T, 128), 128, 0, st>>>(pr.T, pr.vert, pr.cent, pr.area, pr.k0, khat[0], khat[1], khat[2],
                                                   pol[0], pol[1], pol[2], E0, weps, rule, static_cast<cd*>(pr.pot));
    k_assemble<double><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                        pr.inv_perm, static_cast<cd*>(pr.pot), static_cast<cd*>(b));
  }
  return cuda_check(cudaGetLastError(), "rhs launch");
}

// Right-hand side for potentials given at the 7 quadrature points of every
// triangle (Eqs. (1)-(2)): U = -int (r - c_t).A, V = -int A, T1 = 0,
// T2 = -i w eps0 int Phi, tested by k_assemble into b_J = -<f_m, A>,
// b_sigma = -i w eps0 <p_t, Phi>.  Aq [T][7][3], Pq [T][7] in mesh order.
template <typename Rio>
__global__ void k_rhs_q(int64_t T, const int64_t* __restrict__ perm, const double* __restrict__ vert,
                        const double* __restrict__ cent, const double* __restrict__ area, const cd* __restrict__ Aq,
                        const cd* __restrict__ Pq, double weps, const double* __restrict__ rule,
                        C2<Rio>* __restrict__ pot) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int64_t m = perm[t];
  const double* v = vert + 9 * t;
  double Ur = 0, Ui = 0, Vr[3] = {0, 0, 0}, Vi[3] = {0, 0, 0}, Pr = 0, Pim = 0;
  for (int q = 0; q < 7; ++q) {
    const double b0 = rule[4 * q], b1 = rule[4 * q + 1], b2 = rule[4 * q + 2], wq = rule[4 * q + 3] * area[t];
    const cd* A = Aq + (m * 7 + q) * 3;
    const cd P = Pq[m * 7 + q];
    for (int d = 0; d < 3; ++d) {
      const double u = b0 * v[d] + b1 * v[3 + d] + b2 * v[6 + d] - cent[3 * t + d];
      Ur += wq * u * A[d].x;
      Ui += wq * u * A[d].y;
      Vr[d] += wq * A[d].x;
      Vi[d] += wq * A[d].y;
    }
    Pr += wq * P.x;
    Pim += wq * P.y;
  }
  C2<Rio>* o = pot + 6 * t;
  o[0] = mk<Rio>(Rio(-Ur), Rio(-Ui));
  for (int d = 0; d < 3; ++d) o[1 + d] = mk<Rio>(Rio(-Vr[d]), Rio(-Vi[d]));
  o[4] = mk<Rio>(0, 0);
  o[5] = mk<Rio>(Rio(weps * Pim), Rio(-weps * Pr));
}

pie_status rhs_potentials(Problem& pr, const void* Aq, const void* Pq, void* b, cudaStream_t st) {
  const double weps = pr.w * eps0();
  const cd* A = static_cast<const cd*>(Aq);
  const cd* P = static_cast<const cd*>(Pq);
  if (pr.io_f32()) {
    k_rhs_q<float><<<nblk(pr.T, 128), 128, 0, st>>>(pr.T, pr.perm, pr.vert, pr.cent, pr.area, A, P, weps, pr.rule7,
                                                    static_cast<cf*>(pr.pot));
    k_assemble<float><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                       pr.inv_perm, static_cast<cf*>(pr.pot), static_cast<cf*>(b));
  } else {
    k_rhs_q<double><<<nblk(pr.T, 128), 128, 0, st>>>(pr.T, pr.perm, pr.vert, pr.cent, pr.area, A, P, weps, pr.rule7,
                                                     static_cast<cd*>(pr.pot));
    k_assemble<double><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                        pr.inv_perm, static_cast<cd*>(pr.pot), static_cast<cd*>(b));
  }
  return cuda_check(cudaGetLastError(), "rhs launch");
}

// ---------------------------------------------------------------- far field

// One block per direction: sum over triangles and quadrature points of
// J(r) exp(-i k0 rhat.r) w, then E = i w mu0/(4 pi) (I - rr) F.
template <typename Rio>
__global__ void k_farfield(int64_t T, const double* __restrict__ vert, const double* __restrict__ cent,
                           const double* __restrict__ area, const C2<Rio>* __restrict__ coef,
                           const double* __restrict__ rhat, double k0, double pref, const double* __restrict__ rule,
                           cd* __restrict__ E) {
  __shared__ double red[6][32];
  int dir = blockIdx.x;
  double rx = rhat[3 * dir], ry = rhat[3 * dir + 1], rz = rhat[3 * dir + 2];
  double Fr[3] = {0, 0, 0}, Fi[3] = {0, 0, 0};
  for (int64_t t = threadIdx.x; t < T; t += blockDim.x) {
    const double* v = vert + 9 * t;
    const C2<Rio>* c = coef + 6 * t;
    double ar = double(c[0].x), ai = double(c[0].y);
    for (int q = 0; q < 7; ++q) {
      double b0 = rule[4 * q], b1 = rule[4 * q + 1], b2 = rule[4 * q + 2], wq = rule[4 * q + 3] * area[t];
      double r[3];
      for (int d = 0; d < 3; ++d) r[d] = b0 * v[d] + b1 * v[3 + d] + b2 * v[6 + d];
      double s, cs;
      sincos(-k0 * (rx * r[0] + ry * r[1] + rz * r[2]), &s, &cs);
      for (int d = 0; d < 3; ++d) {
        double u = r[d] - cent[3 * t + d];
        double jr = ar * u + double(c[1 + d].x), ji = ai * u + double(c[1 + d].y);
        Fr[d] += wq * (jr * cs - ji * s);
        Fi[d] += wq * (jr * s + ji * cs);
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
    Fr[d] = warp_sum(Fr[d]);
    Fi[d] = warp_sum(Fi[d]);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int d = 0; d < 3; ++d) {
      red[d][wid] = Fr[d];
      red[3 + d][wid] = Fi[d];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int i = 0; i < 6; ++i) S[i] += red[i][w];
    double rr[3] = {rx, ry, rz};
    double dr = rx * S[0] + ry * S[1] + rz * S[2], di = rx * S[3] + ry * S[4] + rz * S[5];
    for (int d = 0; d < 3; ++d) {
      double tr_ = S[d] - rr[d] * dr, ti = S[3 + d] - rr[d] * di;
      // i pref (tr + i ti) = -pref ti + i pref tr
      E[3 * dir + d].x = -pref * ti;
      E[3 * dir + d].y = pref * tr_;
    }
  }
}

pie_status farfield(Problem& pr, const void* x, const double* rhat, int64_t ndir, void* E, cudaStream_t st) {
  const double* rule = pr.rule7;
  double* d_rhat = nullptr;
  pie_status s = cuda_check(cudaMallocAsync((void**)&d_rhat, sizeof(double) * 3 * ndir, st), "farfield alloc");
  if (s != PIE_OK) return s;
  s = cuda_check(cudaMemcpyAsync(d_rhat, rhat, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, st), "copy");
  if (s != PIE_OK) return s;
  const double w2e = pr.w * pr.w * eps0();
  const double pref = pr.w * kMu0 / (4.0 * kPi);
  if (pr.io_f32()) {
    k_coef<float><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const cf*>(x), pr.perm, pr.tri_edge,
                                                   pr.tri_c, pr.tri_dcp, w2e, static_cast<cf*>(pr.coef), nullptr);
    k_farfield<float><<<unsigned(ndir), 256, 0, st>>>(pr.T, pr.vert, pr.cent, pr.area, static_cast<cf*>(pr.coef),
                                                      d_rhat, pr.k0, pref, rule, static_cast<cd*>(E));
  } else {
    k_coef<double><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const cd*>(x), pr.perm, pr.tri_edge,
                                                    pr.tri_c, pr.tri_dcp, w2e, static_cast<cd*>(pr.coef), nullptr);
    k_farfield<double><<<unsigned(ndir), 256, 0, st>>>(pr.T, pr.vert, pr.cent, pr.area, static_cast<cd*>(pr.coef),
                                                       d_rhat, pr.k0, pref, rule, static_cast<cd*>(E));
  }
  s = cuda_check(cudaGetLastError(), "farfield launch");
  cudaFreeAsync(d_rhat, st);
  return s;
}

}  // namespace pie

namespace pie {

// Near part with caller-chosen scratch for the per-triangle coefficients and
// potentials (each [T][6] complex of the problem's io type).
pie_status apply_near_scratch(Problem& pr, const void* x, void* y, void* coef, void* pot, cudaStream_t st) {
  const double w2e = pr.w * pr.w * eps0();
  if (pr.io_f32()) {
    k_coef<float><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const cf*>(x), pr.perm, pr.tri_edge,
                                                   pr.tri_c, pr.tri_dcp, w2e, static_cast<cf*>(coef), nullptr);
    if (pr.near_h16())
      k_near<float, float, 1, true><<<nblk(pr.T * 32, 256), 256, 0, st>>>(
          pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr, nullptr,
          static_cast<const __half2*>(pr.mom), mom_scale(pr), static_cast<const cf*>(coef), float(kMu0),
          static_cast<cf*>(pot));
    else
      k_near<float, float><<<nblk(pr.T * 32, 256), 256, 0, st>>>(
          pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr,
          static_cast<const cf*>(pr.mom), nullptr, mom_scale(pr), static_cast<const cf*>(coef), float(kMu0),
          static_cast<cf*>(pot));
    k_assemble<float><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                       pr.inv_perm, static_cast<const cf*>(pot), static_cast<cf*>(y));
  } else {
    const bool split = pr.near_f32();
    k_coef<double><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const cd*>(x), pr.perm, pr.tri_edge,
                                                    pr.tri_c, pr.tri_dcp, w2e, split ? nullptr : static_cast<cd*>(coef),
                                                    split ? static_cast<cf*>(coef) : nullptr);
    if (split)
      k_near<float, double><<<nblk(pr.T * 32, 256), 256, 0, st>>>(
          pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr,
          static_cast<const cf*>(pr.mom), nullptr, mom_scale(pr), static_cast<const cf*>(coef), float(kMu0),
          static_cast<cd*>(pot));
    else
      k_near<double, double><<<nblk(pr.T * 32, 256), 256, 0, st>>>(
          pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr,
          static_cast<const cd*>(pr.mom), nullptr, mom_scale(pr), static_cast<const cd*>(coef), kMu0,
          static_cast<cd*>(pot));
    k_assemble<double><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                        pr.inv_perm, static_cast<const cd*>(pot), static_cast<cd*>(y));
  }
  return cuda_check(cudaGetLastError(), "apply_near_noalloc launch");
}

}  // namespace pie

namespace pie {

// ---------------------------------------------------------------- adjoint

template <typename R>
__global__ void k_conj(int64_t n, const C2<R>* __restrict__ x, C2<R>* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = mk<R>(x[i].x, -x[i].y);
}

// y = Z^T x (conj = false) or Z^H x = conj(Z conj x) (conj = true).  The
// discrete operator is complex symmetric -- the near pair moments by the
// two-sided near-singular rule, the far part by the antipodal angular grid
// (aggregation and disaggregation are each other's transposes, F^T is the
// anterpolation of F, T_{-w}(k) = T_w(-k)) -- so Z^T x runs the same stages.
pie_status apply_t_one(Problem& pr, const void* x, void* y, bool conj, cudaStream_t st) {
  if (!conj) return apply_one(pr, x, y, st);
  const int64_t N = pr.N;
  if (pr.io_f32()) {
    k_conj<float><<<nblk(N, 256), 256, 0, st>>>(N, static_cast<const cf*>(x), static_cast<cf*>(pr.vec));
    pie_status s = apply_one(pr, pr.vec, y, st);
    if (s != PIE_OK) return s;
    k_conj<float><<<nblk(N, 256), 256, 0, st>>>(N, static_cast<const cf*>(y), static_cast<cf*>(y));
  } else {
    k_conj<double><<<nblk(N, 256), 256, 0, st>>>(N, static_cast<const cd*>(x), static_cast<cd*>(pr.vec));
    pie_status s = apply_one(pr, pr.vec, y, st);
    if (s != PIE_OK) return s;
    k_conj<double><<<nblk(N, 256), 256, 0, st>>>(N, static_cast<const cd*>(y), static_cast<cd*>(y));
  }
  return cuda_check(cudaGetLastError(), "adjoint launch");
}

// Adjoint of the far-field map x -> E (Section 2 far zone): with
// h(r) = sum_d conj(i w mu0 / 4 pi) exp(+i k rhat_d . r) (I - rhat_d rhat_d) E_d,
// (F^H E)_m = sum_{t in m} c_t,m int_t (r - p_m) . h(r) dr, i.e. the Galerkin
// testing of the potentials U = int (r - c_t).h, V = int h (T1 = T2 = 0).
template <typename Rio>
__global__ void k_farfield_adj(int64_t T, int64_t ndir, const double* __restrict__ vert,
                               const double* __restrict__ cent, const double* __restrict__ area,
                               const double* __restrict__ rhat, const cd* __restrict__ E, double k0, double pref,
                               const double* __restrict__ rule, C2<Rio>* __restrict__ pot) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
  const double* v = vert + 9 * t;
  double Ur = 0, Ui = 0, Vr[3] = {0, 0, 0}, Vi[3] = {0, 0, 0};
  for (int q = 0; q < 7; ++q) {
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = rule[4 * q] * v[d] + rule[4 * q + 1] * v[3 + d] + rule[4 * q + 2] * v[6 + d];
    const double wq = rule[4 * q + 3] * area[t];
    double hr[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int64_t dd = 0; dd < ndir; ++dd) {
      const double* rh = rhat + 3 * dd;
      const cd* e = E + 3 * dd;
      double er_ = rh[0] * e[0].x + rh[1] * e[1].x + rh[2] * e[2].x;
      double ei_ = rh[0] * e[0].y + rh[1] * e[1].y + rh[2] * e[2].y;
      double s, c;
      sincos(k0 * (rh[0] * r[0] + rh[1] * r[1] + rh[2] * r[2]), &s, &c);
      for (int d = 0; d < 3; ++d) {
        double pr_ = e[d].x - rh[d] * er_, pi_ = e[d].y - rh[d] * ei_;  // (I - rr) E
        hr[d] += c * pr_ - s * pi_;
        hi[d] += c * pi_ + s * pr_;
      }
    }
    // times conj(i pref) = -i pref
    for (int d = 0; d < 3; ++d) {
      double a = pref * hi[d], b = -pref * hr[d];
      double u = r[d] - cent[3 * t + d];
      Ur += wq * u * a;
      Ui += wq * u * b;
      Vr[d] += wq * a;
      Vi[d] += wq * b;
    }
  }
  C2<Rio>* o = pot + 6 * t;
  o[0] = mk<Rio>(Rio(Ur), Rio(Ui));
  for (int d = 0; d < 3; ++d) o[1 + d] = mk<Rio>(Rio(Vr[d]), Rio(Vi[d]));
  o[4] = mk<Rio>(0, 0);
  o[5] = mk<Rio>(0, 0);
}

pie_status farfield_adjoint(Problem& pr, const double* rhat, int64_t ndir, const void* E, void* u, cudaStream_t st) {
  double* d_rhat = nullptr;
  pie_status s = cuda_check(cudaMallocAsync((void**)&d_rhat, sizeof(double) * 3 * ndir, st), "farfield alloc");
  if (s != PIE_OK) return s;
  s = cuda_check(cudaMemcpyAsync(d_rhat, rhat, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, st), "copy");
  if (s != PIE_OK) return s;
  const double pref = pr.w * kMu0 / (4.0 * kPi);
  if (pr.io_f32()) {
    k_farfield_adj<float><<<nblk(pr.T, 128), 128, 0, st>>>(pr.T, ndir, pr.vert, pr.cent, pr.area, d_rhat,
                                                           static_cast<const cd*>(E), pr.k0, pref, pr.rule7,
                                                           static_cast<cf*>(pr.pot));
    k_assemble<float><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                       pr.inv_perm, static_cast<cf*>(pr.pot), static_cast<cf*>(u));
  } else {
    k_farfield_adj<double><<<nblk(pr.T, 128), 128, 0, st>>>(pr.T, ndir, pr.vert, pr.cent, pr.area, d_rhat,
                                                            static_cast<const cd*>(E), pr.k0, pref, pr.rule7,
                                                            static_cast<cd*>(pr.pot));
    k_assemble<double><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                        pr.inv_perm, static_cast<cd*>(pr.pot), static_cast<cd*>(u));
  }
  s = cuda_check(cudaGetLastError(), "farfield adjoint launch");
  cudaFreeAsync(d_rhat, st);
  return s;
}

}  // namespace pie

namespace pie {

// ---------------------------------------------------------------- Eq. (3) and near-zone fields

// out = src[off:off+n] * scale
__global__ void k_slice_scale(int64_t n, const cd* __restrict__ src, double scale, cd* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = mk<double>(scale * src[i].x, scale * src[i].y);
}

// Single layer of Eq. (3): y_t = <p_t, g, q> for pulse coefficients q
// (mesh order).  It is the pulse-pulse block of the PIE operator divided by
// w^2 eps0, applied to [0 ; q] through the same near and far stages.
pie_status single_layer_one(Problem& pr, const void* q, void* y, cudaStream_t st) {
  const int64_t E = pr.E, T = pr.T;
  cd* v = static_cast<cd*>(pr.vec);
  cd* v2 = static_cast<cd*>(pr.vec2);
  pie_status s = cuda_check(cudaMemsetAsync(v, 0, sizeof(cd) * E, st), "memset");
  if (s == PIE_OK) s = cuda_check(cudaMemcpyAsync(v + E, q, sizeof(cd) * T, cudaMemcpyDeviceToDevice, st), "copy");
  if (s == PIE_OK) s = apply_one(pr, v, v2, st);
  if (s != PIE_OK) return s;
  k_slice_scale<<<nblk(T, 256), 256, 0, st>>>(T, v2 + E, 1.0 / (pr.w * pr.w * eps0()), static_cast<cd*>(y));
  return cuda_check(cudaGetLastError(), "single layer launch");
}

// b_t = <p_t, Phi^inc> = int_t Phi^inc for the plane-wave potential
// Phi^inc = -E0 (pol.r) exp(i k khat.r); 7-point rule; b in mesh order.
__global__ void k_phi_inc(int64_t T, const double* __restrict__ vert, const double* __restrict__ area,
                          const int64_t* __restrict__ perm, double k0, double kx, double ky, double kz, double ex,
                          double ey, double ez, double E0, const double* __restrict__ rule, cd* __restrict__ b) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
  const double* v = vert + 9 * t;
  double pr_ = 0, pi_ = 0;
  for (int q = 0; q < 7; ++q) {
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = rule[4 * q] * v[d] + rule[4 * q + 1] * v[3 + d] + rule[4 * q + 2] * v[6 + d];
    const double wq = rule[4 * q + 3] * area[t];
    double s, c;
    sincos(k0 * (kx * r[0] + ky * r[1] + kz * r[2]), &s, &c);
    const double er = ex * r[0] + ey * r[1] + ez * r[2];
    pr_ += -wq * E0 * er * c;
    pi_ += -wq * E0 * er * s;
  }
  b[perm[t]] = mk<double>(pr_, pi_);
}

pie_status rhs_potential(Problem& pr, const double* khat, const double* pol, double E0, void* b, cudaStream_t st) {
  k_phi_inc<<<nblk(pr.T, 128), 128, 0, st>>>(pr.T, pr.vert, pr.area, pr.perm, pr.k0, khat[0], khat[1], khat[2],
                                             pol[0], pol[1], pol[2], E0, pr.rule7, static_cast<cd*>(b));
  return cuda_check(cudaGetLastError(), "rhs potential launch");
}

// Scattered field at observation points off the surface (Section 2:
// near-zone E from J and the charge density rho):
//   E_s(r) = i w mu0 sum_t int_t J g  -  (1/eps0) sum_t rho_t int_t grad_r g,
// grad_r g = (r - r') (i k - 1/R) g / R; 7-point rule on every triangle (the
// rule is accurate for points farther than about a triangle size).  One block
// per point; coef holds the local coefficients of J (tree order), rho the
// pulse coefficients of the charge density (mesh order).
template <typename Rio>
__global__ void k_nearzone(int64_t T, const double* __restrict__ vert, const double* __restrict__ cent,
                           const double* __restrict__ area, const int64_t* __restrict__ perm,
                           const C2<Rio>* __restrict__ coef, const cd* __restrict__ rho, const double* __restrict__ pts,
                           double k0, double wmu, double inv_eps, const double* __restrict__ rule, cd* __restrict__ E) {
  __shared__ double red[6][32];
  const int ip = blockIdx.x;
  const double px = pts[3 * ip], py = pts[3 * ip + 1], pz = pts[3 * ip + 2];
  double Er[3] = {0, 0, 0}, Ei[3] = {0, 0, 0};
  for (int64_t t = threadIdx.x; t < T; t += blockDim.x) {
    const double* v = vert + 9 * t;
    const C2<Rio>* c = coef + 6 * t;
    const double ar = double(c[0].x), ai = double(c[0].y);
    const cd rh = rho[perm[t]];
    for (int q = 0; q < 7; ++q) {
      double r[3];
      for (int d = 0; d < 3; ++d) r[d] = rule[4 * q] * v[d] + rule[4 * q + 1] * v[3 + d] + rule[4 * q + 2] * v[6 + d];
      const double wq = rule[4 * q + 3] * area[t];
      const double dx = px - r[0], dy = py - r[1], dz = pz - r[2];
      const double R = sqrt(dx * dx + dy * dy + dz * dz);
      double s, cs;
      sincos(k0 * R, &s, &cs);
      const double gr = wq * cs / (4.0 * kPi * R), gi = wq * s / (4.0 * kPi * R);
      // grad g factor: (ik - 1/R)/R * g
      const double fr = (-gr / R - k0 * gi) / R, fi = (-gi / R + k0 * gr) / R;
      const double dd[3] = {dx, dy, dz};
      for (int d = 0; d < 3; ++d) {
        const double u = r[d] - cent[3 * t + d];
        const double jr = ar * u + double(c[1 + d].x), ji = ai * u + double(c[1 + d].y);
        // i w mu0 J g
        const double agr = jr * gr - ji * gi, agi = jr * gi + ji * gr;
        Er[d] += -wmu * agi;
        Ei[d] += wmu * agr;
        // -(1/eps0) rho grad g
        const double gdr = fr * dd[d], gdi = fi * dd[d];
        Er[d] -= inv_eps * (rh.x * gdr - rh.y * gdi);
        Ei[d] -= inv_eps * (rh.x * gdi + rh.y * gdr);
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
    Er[d] = warp_sum(Er[d]);
    Ei[d] = warp_sum(Ei[d]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int d = 0; d < 3; ++d) {
      red[d][wid] = Er[d];
      red[3 + d][wid] = Ei[d];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < int(blockDim.x >> 5); ++w)
      for (int i = 0; i < 6; ++i) S[i] += red[i][w];
    for (int d = 0; d < 3; ++d) E[3 * ip + d] = mk<double>(S[d], S[3 + d]);
  }
}

pie_status nearzone(Problem& pr, const void* x, const void* rho, const double* pts, int64_t npts, void* E,
                    cudaStream_t st) {
  double* d_pts = nullptr;
  pie_status s = cuda_check(cudaMallocAsync((void**)&d_pts, sizeof(double) * 3 * npts, st), "nearfield alloc");
  if (s != PIE_OK) return s;
  s = cuda_check(cudaMemcpyAsync(d_pts, pts, sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, st), "copy");
  if (s != PIE_OK) return s;
  const double w2e = pr.w * pr.w * eps0();
  k_coef<double><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const cd*>(x), pr.perm, pr.tri_edge,
                                                  pr.tri_c, pr.tri_dcp, w2e, static_cast<cd*>(pr.coef), nullptr);
  k_nearzone<double><<<unsigned(npts), 256, 0, st>>>(pr.T, pr.vert, pr.cent, pr.area, pr.perm,
                                                     static_cast<const cd*>(pr.coef), static_cast<const cd*>(rho),
                                                     d_pts, pr.k0, pr.w * kMu0, 1.0 / eps0(), pr.rule7,
                                                     static_cast<cd*>(E));
  s = cuda_check(cudaGetLastError(), "nearfield launch");
  cudaFreeAsync(d_pts, st);
  return s;
}

}  // namespace pie
