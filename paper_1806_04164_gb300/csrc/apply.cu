// One MLFMA matrix-vector product y = Z x for the PIEs (Section 3):
// local coefficients, near pair products, leaf aggregation, interpolation,
// translation (Eq. (5) operators), anterpolation, leaf disaggregation and
// Galerkin assembly (Section 2).
#include <cstdio>

#include "device.cuh"

namespace pie {

// a0: affine restriction of J to every triangle (tree order),
// J|_t = a (r - c_t) + beta, and the pulse densities sigma, d = 2a + w^2 eps0 sigma.
template <typename Rio>
__global__ void k_coef(int64_t T, int64_t E, const C2<Rio>* __restrict__ x, const int64_t* __restrict__ perm,
                       const int32_t* __restrict__ tri_edge, const double* __restrict__ tri_c,
                       const double* __restrict__ tri_dcp, double w2e, C2<Rio>* __restrict__ coef) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= T) return;
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
  C2<Rio>* o = coef + 6 * t;
  o[0] = mk<Rio>(Rio(ar), Rio(ai));
  for (int d = 0; d < 3; ++d) o[1 + d] = mk<Rio>(Rio(br[d]), Rio(bi[d]));
  o[4] = s;
  o[5] = mk<Rio>(Rio(2.0 * ar + w2e * sr), Rio(2.0 * ai + w2e * si));
}

// a1: near part.  One warp per test triangle t; lanes run over the source
// triangles of the neighbouring leaf boxes (contiguous in tree order), whose
// eight pair moments are stored plane by plane ([8][nnz]), so a warp reads
// 32 consecutive entries of each plane.  Writes pot[t] (initialises it).
template <typename Rm, typename Rio>
__global__ void __launch_bounds__(256) k_near(int64_t T, int64_t nnz, const int32_t* __restrict__ leaf_of,
                                              const int32_t* __restrict__ leaf_start,
                                              const int32_t* __restrict__ near_ptr,
                                              const int32_t* __restrict__ near_idx,
                                              const int64_t* __restrict__ row_ptr, const C2<Rm>* __restrict__ mom,
                                              const C2<Rio>* __restrict__ coef, Rm mu0, C2<Rio>* __restrict__ pot) {
  int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (t >= T) return;
  int b = leaf_of[t];
  int64_t e = row_ptr[t];
  C2<Rm> U = mk<Rm>(0, 0), V0 = U, V1 = U, V2 = U, T1 = U, T2 = U;
  for (int qi = near_ptr[b]; qi < near_ptr[b + 1]; ++qi) {
    int q = near_idx[qi];
    int s0 = leaf_start[q];
    int ns = leaf_start[q + 1] - s0;
    for (int j = lane; j < ns; j += 32) {
      int64_t ee = e + j;
      const C2<Rio>* c = coef + 6 * (int64_t)(s0 + j);
      C2<Rm> a = cvt<Rm>(c[0]), b0 = cvt<Rm>(c[1]), b1 = cvt<Rm>(c[2]), b2 = cvt<Rm>(c[3]);
      C2<Rm> sg = cvt<Rm>(c[4]), dd = cvt<Rm>(c[5]);
      C2<Rm> m0 = mom[ee];
      C2<Rm> mt0 = mom[nnz + ee], mt1 = mom[2 * nnz + ee], mt2 = mom[3 * nnz + ee];
      C2<Rm> ms0 = mom[4 * nnz + ee], ms1 = mom[5 * nnz + ee], ms2 = mom[6 * nnz + ee];
      C2<Rm> mts = mom[7 * nnz + ee];
      cfma(U, a, mts);
      cfma(U, b0, mt0);
      cfma(U, b1, mt1);
      cfma(U, b2, mt2);
      cfma(V0, a, ms0);
      cfma(V0, b0, m0);
      cfma(V1, a, ms1);
      cfma(V1, b1, m0);
      cfma(V2, a, ms2);
      cfma(V2, b2, m0);
      cfma(T1, sg, m0);
      cfma(T2, dd, m0);
    }
    e += ns;
  }
  C2<Rm> acc[6] = {U, V0, V1, V2, T1, T2};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    acc[i].x = warp_sum(acc[i].x);
    acc[i].y = warp_sum(acc[i].y);
  }
  if (lane == 0) {
    C2<Rio>* o = pot + 6 * t;
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = mk<Rio>(Rio(mu0 * acc[i].x), Rio(mu0 * acc[i].y));
    o[4] = cvt<Rio>(acc[4]);
    o[5] = cvt<Rio>(acc[5]);
  }
}

// a2: leaf aggregation.  One block per leaf box, one thread per angular
// sample p: S[b][c][p] = sum_t rho_c radiation patterns (Pi, M tables).
template <typename Rf, typename Rio>
__global__ void k_agg(int P, const int32_t* __restrict__ leaf_start, const C2<Rf>* __restrict__ Pi,
                      const C2<Rf>* __restrict__ M, const C2<Rio>* __restrict__ coef, Rf mu0,
                      C2<Rf>* __restrict__ S) {
  int b = blockIdx.x;
  int t0 = leaf_start[b], t1 = leaf_start[b + 1];
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    C2<Rf> s0 = mk<Rf>(0, 0), s1 = s0, s2 = s0, s3 = s0, s4 = s0;
    for (int t = t0; t < t1; ++t) {
      const C2<Rio>* c = coef + 6 * (int64_t)t;
      C2<Rf> a = cvt<Rf>(c[0]);
      C2<Rf> pi = Pi[(int64_t)t * P + p];
      C2<Rf> m0 = M[((int64_t)t * 3 + 0) * P + p];
      C2<Rf> m1 = M[((int64_t)t * 3 + 1) * P + p];
      C2<Rf> m2 = M[((int64_t)t * 3 + 2) * P + p];
      cfma(s0, a, m0);
      cfma(s0, cvt<Rf>(c[1]), pi);
      cfma(s1, a, m1);
      cfma(s1, cvt<Rf>(c[2]), pi);
      cfma(s2, a, m2);
      cfma(s2, cvt<Rf>(c[3]), pi);
      cfma(s3, cvt<Rf>(c[4]), pi);
      cfma(s4, cvt<Rf>(c[5]), pi);
    }
    C2<Rf>* o = S + (int64_t)b * kComp * P + p;
    o[0] = mk<Rf>(mu0 * s0.x, mu0 * s0.y);
    o[P] = mk<Rf>(mu0 * s1.x, mu0 * s1.y);
    o[2 * P] = mk<Rf>(mu0 * s2.x, mu0 * s2.y);
    o[3 * P] = s3;
    o[4 * P] = s4;
  }
}

// a3: interpolation from level l+1 to its parents at level l:
// S_l[b] = sum_children phase_o (F S_child); one block per parent, one thread
// per sample; the child pattern is staged in shared memory.
template <typename Rf>
__global__ void k_interp(int P, const int32_t* __restrict__ child_start, const int8_t* __restrict__ oct_child,
                         const C2<Rf>* __restrict__ Sc, const Rf* __restrict__ Ft, const C2<Rf>* __restrict__ phase,
                         C2<Rf>* __restrict__ Sp) {
  extern __shared__ unsigned char smem_raw[];
  C2<Rf>* sm = reinterpret_cast<C2<Rf>*>(smem_raw);
  int b = blockIdx.x;
  int p = threadIdx.x;
  C2<Rf> acc[kComp];
#pragma unroll
  for (int c = 0; c < kComp; ++c) acc[c] = mk<Rf>(0, 0);
  for (int ch = child_start[b]; ch < child_start[b + 1]; ++ch) {
    __syncthreads();
    for (int i = threadIdx.x; i < kComp * P; i += blockDim.x) sm[i] = Sc[(int64_t)ch * kComp * P + i];
    __syncthreads();
    if (p < P) {
      C2<Rf> sum[kComp];
#pragma unroll
      for (int c = 0; c < kComp; ++c) sum[c] = mk<Rf>(0, 0);
      for (int q = 0; q < P; ++q) {
        Rf f = Ft[(int64_t)q * P + p];
#pragma unroll
        for (int c = 0; c < kComp; ++c) rfma(sum[c], f, sm[c * P + q]);
      }
      C2<Rf> ph = phase[oct_child[ch] * P + p];
#pragma unroll
      for (int c = 0; c < kComp; ++c) cfma(acc[c], ph, sum[c]);
    }
  }
  if (p < P) {
#pragma unroll
    for (int c = 0; c < kComp; ++c) Sp[((int64_t)b * kComp + c) * P + p] = acc[c];
  }
}

// a4: translation at one level: G[d] = sum_{s in IL(d)} T[off] * S[s];
// one block per destination box, one thread per sample, five components.
template <typename Rf>
__global__ void k_trans(int P, const int32_t* __restrict__ il_ptr, const int32_t* __restrict__ il_idx,
                        const int32_t* __restrict__ il_off, const C2<Rf>* __restrict__ Tt,
                        const C2<Rf>* __restrict__ S, C2<Rf>* __restrict__ G) {
  int d = blockIdx.x;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    C2<Rf> acc[kComp];
#pragma unroll
    for (int c = 0; c < kComp; ++c) acc[c] = mk<Rf>(0, 0);
    for (int j = il_ptr[d]; j < il_ptr[d + 1]; ++j) {
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

// a5: anterpolation from level l to level l+1:
// G_child += F^T (conj(phase_o) G_parent); one block per child box.
template <typename Rf>
__global__ void k_anterp(int P, const int32_t* __restrict__ parent, const int8_t* __restrict__ oct_child,
                         const C2<Rf>* __restrict__ Gp, const Rf* __restrict__ F, const C2<Rf>* __restrict__ phase,
                         C2<Rf>* __restrict__ Gc) {
  extern __shared__ unsigned char smem_raw[];
  C2<Rf>* sm = reinterpret_cast<C2<Rf>*>(smem_raw);
  int ch = blockIdx.x;
  int par = parent[ch];
  int o = oct_child[ch];
  for (int i = threadIdx.x; i < kComp * P; i += blockDim.x) {
    int q = i % P;
    C2<Rf> g = Gp[(int64_t)par * kComp * P + i];
    C2<Rf> ph = phase[o * P + q];
    C2<Rf> h;
    h.x = ph.x * g.x + ph.y * g.y;   // conj(ph) * g
    h.y = ph.x * g.y - ph.y * g.x;
    sm[i] = h;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    C2<Rf> sum[kComp];
#pragma unroll
    for (int c = 0; c < kComp; ++c) sum[c] = mk<Rf>(0, 0);
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

// a6: leaf disaggregation with the receiving (conjugate) patterns; one warp
// per triangle, lanes over samples; adds to pot[t].
template <typename Rf, typename Rio>
__global__ void __launch_bounds__(256) k_disagg(int64_t T, int P, const int32_t* __restrict__ leaf_of,
                                                const C2<Rf>* __restrict__ Pi, const C2<Rf>* __restrict__ M,
                                                const C2<Rf>* __restrict__ G, C2<Rio>* __restrict__ pot) {
  int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (t >= T) return;
  const C2<Rf>* g = G + (int64_t)leaf_of[t] * kComp * P;
  C2<Rf> U = mk<Rf>(0, 0), V0 = U, V1 = U, V2 = U, T1 = U, T2 = U;
  for (int p = lane; p < P; p += 32) {
    C2<Rf> pi = Pi[t * P + p];
    C2<Rf> m0 = M[(t * 3 + 0) * P + p], m1 = M[(t * 3 + 1) * P + p], m2 = M[(t * 3 + 2) * P + p];
    C2<Rf> g0 = g[p], g1 = g[P + p], g2 = g[2 * P + p], g3 = g[3 * P + p], g4 = g[4 * P + p];
    cfma_conj(U, m0, g0);
    cfma_conj(U, m1, g1);
    cfma_conj(U, m2, g2);
    cfma_conj(V0, pi, g0);
    cfma_conj(V1, pi, g1);
    cfma_conj(V2, pi, g2);
    cfma_conj(T1, pi, g3);
    cfma_conj(T2, pi, g4);
  }
  C2<Rf> acc[6] = {U, V0, V1, V2, T1, T2};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    acc[i].x = warp_sum(acc[i].x);
    acc[i].y = warp_sum(acc[i].y);
  }
  if (lane == 0) {
    C2<Rio>* o = pot + 6 * t;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      o[i].x = Rio(double(o[i].x) + double(acc[i].x));
      o[i].y = Rio(double(o[i].y) + double(acc[i].y));
    }
  }
}

// a7: Galerkin testing of the per-triangle potentials (Section 2):
// RWG m: sum over its two triangles of c [U + (c_t - p).V] + 2c T1; pulse t: T2.
template <typename Rio>
__global__ void k_assemble(int64_t N, int64_t E, const int32_t* __restrict__ edge_tt,
                           const int8_t* __restrict__ edge_k, const double* __restrict__ tri_c,
                           const double* __restrict__ tri_dcp, const int64_t* __restrict__ inv_perm,
                           const C2<Rio>* __restrict__ pot, C2<Rio>* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (i < E) {
    double yr = 0, yi = 0;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int64_t t = edge_tt[2 * i + side];
      int k = edge_k[2 * i + side];
      double c = tri_c[3 * t + k];
      const double* dcp = tri_dcp + 9 * t + 3 * k;
      const C2<Rio>* p = pot + 6 * t;
      double ur = double(p[0].x) + dcp[0] * double(p[1].x) + dcp[1] * double(p[2].x) + dcp[2] * double(p[3].x);
      double ui = double(p[0].y) + dcp[0] * double(p[1].y) + dcp[1] * double(p[2].y) + dcp[2] * double(p[3].y);
      yr += c * (ur + 2.0 * double(p[4].x));
      yi += c * (ui + 2.0 * double(p[4].y));
    }
    y[i] = mk<Rio>(Rio(yr), Rio(yi));
  } else {
    int64_t t = inv_perm[i - E];
    y[i] = pot[6 * t + 5];
  }
}

// ---------------------------------------------------------------- orchestration

static inline unsigned nblk(int64_t n, int b) { return unsigned((n + b - 1) / b); }

void prof_mark(Problem& pr, int stage, bool end, cudaStream_t st) {
  if (pr.prof_n >= pr.prof_cap) return;
  cudaEventRecord(pr.prof_ev[(size_t(pr.prof_n) * kStages + stage) * 2 + (end ? 1 : 0)], st);
}

template <typename Rm, typename Rf, typename Rio>
static pie_status apply_t(Problem& pr, const void* xv, void* yv, cudaStream_t st) {
  const int P = pr.P;
  const int L = pr.tree.L;
  const C2<Rio>* x = static_cast<const C2<Rio>*>(xv);
  C2<Rio>* y = static_cast<C2<Rio>*>(yv);
  C2<Rio>* coef = static_cast<C2<Rio>*>(pr.coef);
  C2<Rio>* pot = static_cast<C2<Rio>*>(pr.pot);
  const double w2e = pr.w * pr.w * eps0();
  prof_mark(pr, 0, false, st);
  k_coef<Rio><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, x, pr.perm, pr.tri_edge, pr.tri_c, pr.tri_dcp, w2e,
                                               coef);
  prof_mark(pr, 0, true, st);
  prof_mark(pr, 1, false, st);
  k_near<Rm, Rio><<<nblk(pr.T * 32, 256), 256, 0, st>>>(pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr,
                                                        pr.near_idx, pr.row_ptr,
                                                        static_cast<const C2<Rm>*>(pr.mom), coef, Rm(kMu0), pot);
  prof_mark(pr, 1, true, st);
  const int tpb = P < 1024 ? ((P + 31) / 32) * 32 : 1024;
  const C2<Rf>* Pi = static_cast<const C2<Rf>*>(pr.Pi);
  const C2<Rf>* M = static_cast<const C2<Rf>*>(pr.M);
  prof_mark(pr, 2, false, st);
  k_agg<Rf, Rio><<<unsigned(pr.lev[L].nb), tpb, 0, st>>>(P, pr.leaf_start, Pi, M, coef, Rf(kMu0),
                                                        static_cast<C2<Rf>*>(pr.lev[L].S));
  prof_mark(pr, 2, true, st);
  const size_t sm = sizeof(C2<Rf>) * kComp * P;
  prof_mark(pr, 3, false, st);
  for (int l = L - 1; l >= 3; --l) {
    k_interp<Rf><<<unsigned(pr.lev[l].nb), tpb, sm, st>>>(
        P, pr.lev[l].child_start, pr.lev[l + 1].octant, static_cast<const C2<Rf>*>(pr.lev[l + 1].S),
        static_cast<const Rf*>(pr.Ft), static_cast<const C2<Rf>*>(pr.lev[l].phase), static_cast<C2<Rf>*>(pr.lev[l].S));
  }
  prof_mark(pr, 3, true, st);
  prof_mark(pr, 4, false, st);
  for (int l = 3; l <= L; ++l) {
    k_trans<Rf><<<unsigned(pr.lev[l].nb), tpb, 0, st>>>(P, pr.lev[l].il_ptr, pr.lev[l].il_idx, pr.lev[l].il_off,
                                                        static_cast<const C2<Rf>*>(pr.lev[l].trans),
                                                        static_cast<const C2<Rf>*>(pr.lev[l].S),
                                                        static_cast<C2<Rf>*>(pr.lev[l].G));
  }
  prof_mark(pr, 4, true, st);
  prof_mark(pr, 5, false, st);
  for (int l = 3; l < L; ++l) {
    k_anterp<Rf><<<unsigned(pr.lev[l + 1].nb), tpb, sm, st>>>(
        P, pr.lev[l + 1].parent, pr.lev[l + 1].octant, static_cast<const C2<Rf>*>(pr.lev[l].G),
        static_cast<const Rf*>(pr.F), static_cast<const C2<Rf>*>(pr.lev[l].phase), static_cast<C2<Rf>*>(pr.lev[l + 1].G));
  }
  prof_mark(pr, 5, true, st);
  prof_mark(pr, 6, false, st);
  k_disagg<Rf, Rio><<<nblk(pr.T * 32, 256), 256, 0, st>>>(pr.T, P, pr.leaf_of, Pi, M,
                                                         static_cast<const C2<Rf>*>(pr.lev[L].G), pot);
  prof_mark(pr, 6, true, st);
  prof_mark(pr, 7, false, st);
  k_assemble<Rio><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                   pr.inv_perm, pot, y);
  prof_mark(pr, 7, true, st);
  if (pr.prof_n < pr.prof_cap) ++pr.prof_n;
  return cuda_check(cudaGetLastError(), "apply launch");
}

// Near part alone: y = Z_near x (pairs of triangles in neighbouring leaf boxes).
template <typename Rm, typename Rio>
static pie_status apply_near_t(Problem& pr, const void* xv, void* yv, cudaStream_t st) {
  C2<Rio>* coef = static_cast<C2<Rio>*>(pr.coef);
  C2<Rio>* pot = static_cast<C2<Rio>*>(pr.pot);
  k_coef<Rio><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const C2<Rio>*>(xv), pr.perm, pr.tri_edge,
                                               pr.tri_c, pr.tri_dcp, pr.w * pr.w * eps0(), coef);
  k_near<Rm, Rio><<<nblk(pr.T * 32, 256), 256, 0, st>>>(pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr,
                                                        pr.near_idx, pr.row_ptr,
                                                        static_cast<const C2<Rm>*>(pr.mom), coef, Rm(kMu0), pot);
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
    default:
      return apply_near_t<float, double>(pr, x, y, st);
  }
}

pie_status apply_one(Problem& pr, const void* x, void* y, cudaStream_t st) {
  switch (pr.par.precision) {
    case PIE_FP64:
      return apply_t<double, double, double>(pr, x, y, st);
    case PIE_FP32:
      return apply_t<float, float, float>(pr, x, y, st);
    case PIE_MIXED:
      return apply_t<float, double, double>(pr, x, y, st);
  }
  set_error("unknown precision");
  return PIE_ERR_PARAM;
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
                                                   pr.tri_c, pr.tri_dcp, w2e, static_cast<cf*>(pr.coef));
    k_farfield<float><<<unsigned(ndir), 256, 0, st>>>(pr.T, pr.vert, pr.cent, pr.area, static_cast<cf*>(pr.coef),
                                                      d_rhat, pr.k0, pref, rule, static_cast<cd*>(E));
  } else {
    k_coef<double><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const cd*>(x), pr.perm, pr.tri_edge,
                                                    pr.tri_c, pr.tri_dcp, w2e, static_cast<cd*>(pr.coef));
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
                                                   pr.tri_c, pr.tri_dcp, w2e, static_cast<cf*>(coef));
    k_near<float, float><<<nblk(pr.T * 32, 256), 256, 0, st>>>(pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr,
                                                               pr.near_idx, pr.row_ptr, static_cast<const cf*>(pr.mom),
                                                               static_cast<const cf*>(coef), float(kMu0),
                                                               static_cast<cf*>(pot));
    k_assemble<float><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                       pr.inv_perm, static_cast<const cf*>(pot), static_cast<cf*>(y));
  } else {
    k_coef<double><<<nblk(pr.T, 256), 256, 0, st>>>(pr.T, pr.E, static_cast<const cd*>(x), pr.perm, pr.tri_edge,
                                                    pr.tri_c, pr.tri_dcp, w2e, static_cast<cd*>(coef));
    if (pr.near_f32())
      k_near<float, double><<<nblk(pr.T * 32, 256), 256, 0, st>>>(
          pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.row_ptr,
          static_cast<const cf*>(pr.mom), static_cast<const cd*>(coef), float(kMu0), static_cast<cd*>(pot));
    else
      k_near<double, double><<<nblk(pr.T * 32, 256), 256, 0, st>>>(
          pr.T, pr.nnz, pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.row_ptr,
          static_cast<const cd*>(pr.mom), static_cast<const cd*>(coef), kMu0, static_cast<cd*>(pot));
    k_assemble<double><<<nblk(pr.N, 256), 256, 0, st>>>(pr.N, pr.E, pr.edge_tt, pr.edge_k, pr.tri_c, pr.tri_dcp,
                                                        pr.inv_perm, static_cast<const cd*>(pot), static_cast<cd*>(y));
  }
  return cuda_check(cudaGetLastError(), "apply_near_noalloc launch");
}

}  // namespace pie
