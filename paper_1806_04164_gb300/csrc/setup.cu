// Operator set-up on the device, all in FP64 (Sections 2-3):
//  - near pair moments of g over triangle pairs in neighbouring leaf boxes,
//    with closed-form static inner integrals for near-singular pairs (rule
//    averaged over both orders of the pair);
//  - leaf radiation tables (Pi, M) at the leaf wavenumber kappa_L;
//  - translation operators of Eq. (5) per level and offset;
//  - interpolation filter (degree rescale) and phases.
#include <cstring>
#include <cmath>

#include "device.cuh"

namespace pie {

constexpr double kFourPi = 4.0 * kPi;
constexpr int kMaxTau = 30;

// ------------------------------------------------------------ closed forms
// int_T 1/|r-r'| dS' and int_T (r'-r)/|r-r'| dS' over the flat triangle
// (v0, v1, v2) (Wilton et al. 1984; Graglia 1993).  With unit normal n, height
// d = n.(r - v0), per edge a->b: tangent s, outward normal m = s x n,
// l+ = (b-r).s, l- = (a-r).s, P0 = (a-r).m, R0^2 = P0^2 + d^2,
// f = ln((R+ + l+)/(R- + l-)):
//   I1 = sum [P0 f - |d|(atan(P0 l+/(R0^2+|d|R+)) - atan(P0 l-/(R0^2+|d|R-)))]
//   Ir = 1/2 sum m [R0^2 f + l+R+ - l-R-] - d n I1.
__device__ void static_potentials(const double* r, const double* v, double& I1, double* Ir) {
  double e1[3], e2[3], n[3];
  for (int i = 0; i < 3; ++i) {
    e1[i] = v[3 + i] - v[i];
    e2[i] = v[6 + i] - v[i];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int i = 0; i < 3; ++i) n[i] /= nn;
  double d = n[0] * (r[0] - v[0]) + n[1] * (r[1] - v[1]) + n[2] * (r[2] - v[2]);
  double ad = fabs(d);
  I1 = 0;
  double Ip[3] = {0, 0, 0};
  for (int k = 0; k < 3; ++k) {
    const double* a = v + 3 * k;
    const double* b = v + 3 * ((k + 1) % 3);
    double s[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double el = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int i = 0; i < 3; ++i) s[i] /= el;
    double m[3] = {s[1] * n[2] - s[2] * n[1], s[2] * n[0] - s[0] * n[2], s[0] * n[1] - s[1] * n[0]};
    double lp = 0, lm = 0, P0 = 0, Rp2 = 0, Rm2 = 0;
    for (int i = 0; i < 3; ++i) {
      lp += (b[i] - r[i]) * s[i];
      lm += (a[i] - r[i]) * s[i];
      P0 += (a[i] - r[i]) * m[i];
      Rp2 += (r[i] - b[i]) * (r[i] - b[i]);
      Rm2 += (r[i] - a[i]) * (r[i] - a[i]);
    }
    double Rp = sqrt(Rp2), Rm = sqrt(Rm2);
    double R02 = P0 * P0 + d * d;
    double f = 0;
    if (R02 > 1e-24 * el * el) {
      if (lm >= 0)
        f = log((Rp + lp) / (Rm + lm));
      else if (lp <= 0)
        f = log((Rm - lm) / (Rp - lp));
      else
        f = log((Rp + lp) * (Rm - lm) / R02);
    }
    double dp = R02 + ad * Rp, dm = R02 + ad * Rm;
    double at = (dp > 0 ? atan(P0 * lp / dp) : 0.0) - (dm > 0 ? atan(P0 * lm / dm) : 0.0);
    I1 += P0 * f - ad * at;
    double c = 0.5 * (R02 * f + lp * Rp - lm * Rm);
    for (int i = 0; i < 3; ++i) Ip[i] += c * m[i];
  }
  for (int i = 0; i < 3; ++i) Ir[i] = Ip[i] - d * I1 * n[i];
}

// (exp(ikR) - 1)/(4 pi R) without cancellation; ik/(4 pi) at R = 0.
__device__ __forceinline__ void green_rem(double k, double R, double& gr, double& gi) {
  if (R > 0) {
    double sh = sin(0.5 * k * R);
    gr = -2.0 * sh * sh / (kFourPi * R);
    gi = sin(k * R) / (kFourPi * R);
  } else {
    gr = 0;
    gi = k / kFourPi;
  }
}

struct Moments {
  double m0r, m0i, mtr[3], mti[3], msr[3], msi[3], mtsr, mtsi;
};

__device__ void moments_regular(const double* vt, const double* ct, double At, const double* vs, const double* cs,
                                double As, double k, const double* rule7, Moments& o) {
  double rs[7][3], ws[7];
  for (int j = 0; j < 7; ++j) {
    for (int d = 0; d < 3; ++d)
      rs[j][d] = rule7[4 * j] * vs[d] + rule7[4 * j + 1] * vs[3 + d] + rule7[4 * j + 2] * vs[6 + d];
    ws[j] = rule7[4 * j + 3] * As;
  }
  o = Moments{};
  for (int i = 0; i < 7; ++i) {
    double ri[3];
    for (int d = 0; d < 3; ++d)
      ri[d] = rule7[4 * i] * vt[d] + rule7[4 * i + 1] * vt[3 + d] + rule7[4 * i + 2] * vt[6 + d];
    double wi = rule7[4 * i + 3] * At;
    double Kr = 0, Ki = 0, K1r[3] = {0, 0, 0}, K1i[3] = {0, 0, 0};
    for (int j = 0; j < 7; ++j) {
      double dx = ri[0] - rs[j][0], dy = ri[1] - rs[j][1], dz = ri[2] - rs[j][2];
      double R = sqrt(dx * dx + dy * dy + dz * dz);
      double sn, cs_;
      sincos(k * R, &sn, &cs_);
      double g = ws[j] / (kFourPi * R);
      double gr = g * cs_, gi = g * sn;
      Kr += gr;
      Ki += gi;
      for (int d = 0; d < 3; ++d) {
        double u = rs[j][d] - cs[d];
        K1r[d] += gr * u;
        K1i[d] += gi * u;
      }
    }
    o.m0r += wi * Kr;
    o.m0i += wi * Ki;
    for (int d = 0; d < 3; ++d) {
      double u = ri[d] - ct[d];
      o.mtr[d] += wi * u * Kr;
      o.mti[d] += wi * u * Ki;
      o.msr[d] += wi * K1r[d];
      o.msi[d] += wi * K1i[d];
      o.mtsr += wi * u * K1r[d];
      o.mtsi += wi * u * K1i[d];
    }
  }
}

__device__ void moments_singular(const double* vt, const double* ct, double At, const double* vs, const double* cs,
                                 double As, double k, const double* rule7, const double* rule64, Moments& o) {
  o = Moments{};
  for (int i = 0; i < 64; ++i) {
    double ri[3];
    for (int d = 0; d < 3; ++d)
      ri[d] = rule64[4 * i] * vt[d] + rule64[4 * i + 1] * vt[3 + d] + rule64[4 * i + 2] * vt[6 + d];
    double wi = rule64[4 * i + 3] * At;
    double I1, Ir[3];
    static_potentials(ri, vs, I1, Ir);
    double Kr = I1 / kFourPi, Ki = 0;
    double K1r[3], K1i[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) K1r[d] = (Ir[d] + (ri[d] - cs[d]) * I1) / kFourPi;
    for (int j = 0; j < 7; ++j) {
      double rj[3];
      for (int d = 0; d < 3; ++d)
        rj[d] = rule7[4 * j] * vs[d] + rule7[4 * j + 1] * vs[3 + d] + rule7[4 * j + 2] * vs[6 + d];
      double wj = rule7[4 * j + 3] * As;
      double dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
      double gr, gi;
      green_rem(k, sqrt(dx * dx + dy * dy + dz * dz), gr, gi);
      gr *= wj;
      gi *= wj;
      Kr += gr;
      Ki += gi;
      for (int d = 0; d < 3; ++d) {
        double u = rj[d] - cs[d];
        K1r[d] += gr * u;
        K1i[d] += gi * u;
      }
    }
    o.m0r += wi * Kr;
    o.m0i += wi * Ki;
    for (int d = 0; d < 3; ++d) {
      double u = ri[d] - ct[d];
      o.mtr[d] += wi * u * Kr;
      o.mti[d] += wi * u * Ki;
      o.msr[d] += wi * K1r[d];
      o.msi[d] += wi * K1i[d];
      o.mtsr += wi * u * K1r[d];
      o.mtsi += wi * u * K1i[d];
    }
  }
}

// Near-singular test: ((dx*dx + dy*dy) + dz*dz) < 2.25 max(h_t^2, h_s^2), in
// round-to-nearest double with no contraction.
__device__ __forceinline__ bool near_singular(const double* ct, const double* cs, double h2t, double h2s) {
  double dx = __dsub_rn(ct[0], cs[0]), dy = __dsub_rn(ct[1], cs[1]), dz = __dsub_rn(ct[2], cs[2]);
  double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return d2 < __dmul_rn(2.25, fmax(h2t, h2s));
}

// Near-part set-up in three passes, so that the few expensive near-singular
// pairs do not stall the warps computing the regular ones:
//  1. k_count_singular: count the near-singular pairs with t <= s;
//  2. k_near_regular: regular pairs by the 7 x 7 rule; near-singular pairs
//     with t <= s are appended to a list;
//  3. k_near_singular: one thread per listed pair computes the rule in both
//     orders, averages, and writes the (t,s) and (s,t) entries (mt and ms
//     swapped), which keeps Z^T = Z.
// Lanes walk a test row flat, as the product kernel does.
struct NearGeom {
  const int32_t* leaf_of;
  const int32_t* leaf_start;
  const int32_t* near_ptr;
  const int32_t* near_idx;
  const int32_t* near_off;
  const int64_t* row_ptr;
  const double* vert;
  const double* cent;
  const double* area;
  const double* h2;
};

__global__ void __launch_bounds__(256) k_count_singular(int64_t T, NearGeom g, unsigned long long* count) {
  int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (t >= T) return;
  const int b = g.leaf_of[t];
  const int q0 = g.near_ptr[b], q1 = g.near_ptr[b + 1];
  const int len = int(g.row_ptr[t + 1] - g.row_ptr[t]);
  int qi = q0;
  unsigned n = 0;
  for (int j = lane; j < len; j += 32) {
    while (qi + 1 < q1 && g.near_off[qi + 1] <= j) ++qi;
    const int64_t s = g.leaf_start[g.near_idx[qi]] + (j - g.near_off[qi]);
    if (t <= s && near_singular(g.cent + 3 * t, g.cent + 3 * s, g.h2[t], g.h2[s])) ++n;
  }
  n = __reduce_add_sync(0xffffffffu, n);
  if (lane == 0 && n) atomicAdd(count, (unsigned long long)n);
}

struct SingPair {
  int32_t t, s;
  int64_t e;
};

template <typename Rm>
__device__ __forceinline__ void store_moments(C2<Rm>* mom, int64_t nnz, int64_t e, const Moments& m, bool swap) {
  mom[e] = mk<Rm>(Rm(m.m0r), Rm(m.m0i));
  for (int d = 0; d < 3; ++d) {
    const double tr = swap ? m.msr[d] : m.mtr[d], ti = swap ? m.msi[d] : m.mti[d];
    const double sr = swap ? m.mtr[d] : m.msr[d], si = swap ? m.mti[d] : m.msi[d];
    mom[(1 + d) * nnz + e] = mk<Rm>(Rm(tr), Rm(ti));
    mom[(4 + d) * nnz + e] = mk<Rm>(Rm(sr), Rm(si));
  }
  mom[7 * nnz + e] = mk<Rm>(Rm(m.mtsr), Rm(m.mtsi));
}

template <typename Rm>
__global__ void __launch_bounds__(128) k_near_regular(int64_t T, int64_t nnz, NearGeom g, double k,
                                                      const double* __restrict__ rule7, C2<Rm>* __restrict__ mom,
                                                      SingPair* __restrict__ list, unsigned long long* __restrict__ nlist,
                                                      unsigned long long cap) {
  int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (t >= T) return;
  const int b = g.leaf_of[t];
  const int q0 = g.near_ptr[b], q1 = g.near_ptr[b + 1];
  const int64_t e0 = g.row_ptr[t];
  const int len = int(g.row_ptr[t + 1] - e0);
  const double* vt = g.vert + 9 * t;
  const double* ct = g.cent + 3 * t;
  int qi = q0;
  for (int j = lane; j < len; j += 32) {
    while (qi + 1 < q1 && g.near_off[qi + 1] <= j) ++qi;
    const int64_t s = g.leaf_start[g.near_idx[qi]] + (j - g.near_off[qi]);
    const int64_t e = e0 + j;
    if (near_singular(ct, g.cent + 3 * s, g.h2[t], g.h2[s])) {
      if (t <= s) {
        unsigned long long slot = atomicAdd(nlist, 1ull);
        if (slot < cap) list[slot] = SingPair{int32_t(t), int32_t(s), e};
      }
      continue;
    }
    Moments m;
    moments_regular(vt, ct, g.area[t], g.vert + 9 * s, g.cent + 3 * s, g.area[s], k, rule7, m);
    store_moments(mom, nnz, e, m, false);
  }
}

template <typename Rm>
__global__ void __launch_bounds__(128) k_near_singular(int64_t npairs, int64_t nnz, NearGeom g, double k,
                                                       const double* __restrict__ rule7,
                                                       const double* __restrict__ rule64,
                                                       const SingPair* __restrict__ list, C2<Rm>* __restrict__ mom) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const SingPair pq = list[i];
  const int64_t t = pq.t, s = pq.s;
  Moments m, m2;
  moments_singular(g.vert + 9 * t, g.cent + 3 * t, g.area[t], g.vert + 9 * s, g.cent + 3 * s, g.area[s], k, rule7,
                   rule64, m);
  moments_singular(g.vert + 9 * s, g.cent + 3 * s, g.area[s], g.vert + 9 * t, g.cent + 3 * t, g.area[t], k, rule7,
                   rule64, m2);
  // two-sided average, as seen from t (test) and s (source)
  m.m0r = 0.5 * (m.m0r + m2.m0r);
  m.m0i = 0.5 * (m.m0i + m2.m0i);
  m.mtsr = 0.5 * (m.mtsr + m2.mtsr);
  m.mtsi = 0.5 * (m.mtsi + m2.mtsi);
  for (int d = 0; d < 3; ++d) {
    const double tr = 0.5 * (m.mtr[d] + m2.msr[d]), ti = 0.5 * (m.mti[d] + m2.msi[d]);
    const double sr = 0.5 * (m.msr[d] + m2.mtr[d]), si = 0.5 * (m.msi[d] + m2.mti[d]);
    m.mtr[d] = tr;
    m.mti[d] = ti;
    m.msr[d] = sr;
    m.msi[d] = si;
  }
  store_moments(mom, nnz, pq.e, m, false);
  if (s != t) {
    // entry (s, t): row s, at the position of t inside the near box of t
    const int bs = g.leaf_of[s], bt = g.leaf_of[t];
    int64_t e2 = -1;
    for (int qi = g.near_ptr[bs]; qi < g.near_ptr[bs + 1]; ++qi)
      if (g.near_idx[qi] == bt) e2 = g.row_ptr[s] + g.near_off[qi] + (t - g.leaf_start[bt]);
    if (e2 >= 0) store_moments(mom, nnz, e2, m, true);
  }
}

// Leaf radiation tables at kappa_L: Pi_t(p) = int_t exp(-i kappa khat_p.(r - C_b)),
// M_t(p) = int_t (r - c_t) exp(-i kappa khat_p.(r - C_b)); 7-point rule.
// Called with P = the half grid (theta rows 0..ntheta/2-1): the other half
// is the complex conjugate.
template <typename Rf>
__global__ void k_rad(int64_t T, int P, const double* __restrict__ vert, const double* __restrict__ cent,
                      const double* __restrict__ area, const int32_t* __restrict__ leaf_of,
                      const double* __restrict__ leaf_center, const double* __restrict__ khat, double kappa,
                      const double* __restrict__ rule7, C2<Rf>* __restrict__ Pi, C2<Rf>* __restrict__ M,
                      C2<Rf>* __restrict__ PiR, C2<Rf>* __restrict__ MR) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= T * P) return;
  int64_t t = i / P;
  int p = int(i % P);
  const double* v = vert + 9 * t;
  const double* C = leaf_center + 3 * leaf_of[t];
  double kx = khat[3 * p], ky = khat[3 * p + 1], kz = khat[3 * p + 2];
  double pr = 0, pi = 0, mr[3] = {0, 0, 0}, mi[3] = {0, 0, 0};
  for (int q = 0; q < 7; ++q) {
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = rule7[4 * q] * v[d] + rule7[4 * q + 1] * v[3 + d] + rule7[4 * q + 2] * v[6 + d];
    double w = rule7[4 * q + 3] * area[t];
    double ph = -kappa * (kx * (r[0] - C[0]) + ky * (r[1] - C[1]) + kz * (r[2] - C[2]));
    double s, c;
    sincos(ph, &s, &c);
    pr += w * c;
    pi += w * s;
    for (int d = 0; d < 3; ++d) {
      double u = r[d] - cent[3 * t + d];
      mr[d] += w * u * c;
      mi[d] += w * u * s;
    }
  }
  Pi[t * P + p] = mk<Rf>(Rf(pr), Rf(pi));
  for (int d = 0; d < 3; ++d) M[(t * 3 + d) * P + p] = mk<Rf>(Rf(mr[d]), Rf(mi[d]));
  PiR[(int64_t)p * T + t] = mk<Rf>(Rf(pr), Rf(pi));
  for (int d = 0; d < 3; ++d) MR[((int64_t)d * P + p) * T + t] = mk<Rf>(Rf(mr[d]), Rf(mi[d]));
}

// Translation operator of Eq. (5) with the quadrature weight and the
// i k / (16 pi^2) prefactor of Eq. (4) folded in:
//   T[off][p] = (i k/(16 pi^2)) w_p sum_{t<=tau} i^t (2t+1) s^t h_t(k|w|) P_t(khat_p . what),
// w = offset * a.  s^t y_t by the scaled upward recurrence
// Y_{t+1} = (2t+1)(s/z) Y_t - s^2 Y_{t-1}; s^t j_t by its power series (z <= 4).
template <typename Rf>
__global__ void k_trans_table(int P, int tau, double k, double s, double a, const double* __restrict__ khat,
                              const double* __restrict__ wgt, C2<Rf>* __restrict__ Tt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNoffs * P) return;
  int off = i / P, p = i % P;
  // offset code -> (dx, dy, dz), lexicographic over {-3..3}^3 without {-1..1}^3
  int code = 0, dx = 0, dy = 0, dz = 0;
  for (int x = -3; x <= 3; ++x)
    for (int y = -3; y <= 3; ++y)
      for (int z = -3; z <= 3; ++z) {
        int mx = max(abs(x), max(abs(y), abs(z)));
        if (mx <= 1) continue;
        if (code == off) {
          dx = x;
          dy = y;
          dz = z;
        }
        ++code;
      }
  double wv[3] = {dx * a, dy * a, dz * a};
  double wn = sqrt(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
  double z = k * wn;
  double cosang = (khat[3 * p] * wv[0] + khat[3 * p + 1] * wv[1] + khat[3 * p + 2] * wv[2]) / wn;
  double sz, cz;
  sincos(z, &sz, &cz);
  double Yv[kMaxTau + 2], Pv[kMaxTau + 2];
  Yv[0] = -cz / z;
  Yv[1] = s * (-cz / (z * z) - sz / z);
  for (int t = 1; t < tau; ++t) Yv[t + 1] = (2.0 * t + 1.0) * (s / z) * Yv[t] - s * s * Yv[t - 1];
  Pv[0] = 1.0;
  Pv[1] = cosang;
  for (int t = 1; t < tau; ++t) Pv[t + 1] = ((2.0 * t + 1.0) * cosang * Pv[t] - t * Pv[t - 1]) / (t + 1.0);
  double ar = 0, ai = 0;
  double sz_pow = 1.0;  // (s z)^t
  double dfact = 1.0;   // (2t+1)!!
  for (int t = 0; t <= tau; ++t) {
    if (t >= 1) {
      sz_pow *= s * z;
      dfact *= (2.0 * t + 1.0);
    }
    // s^t j_t(z) = (s z)^t / (2t+1)!! * sum_n (-z^2/2)^n / (n! prod_{i=1..n} (2t+2i+1))
    double term = 1.0, ser = 1.0;
    for (int n = 1; n < 60; ++n) {
      term *= -0.5 * z * z / (n * (2.0 * t + 2.0 * n + 1.0));
      ser += term;
      if (fabs(term) < 1e-18 * fabs(ser)) break;
    }
    double Jt = sz_pow / dfact * ser;
    // i^t (2t+1) (J + i Y) P_t
    double hr = (2.0 * t + 1.0) * Jt * Pv[t], hi = (2.0 * t + 1.0) * Yv[t] * Pv[t];
    switch (t & 3) {
      case 0: ar += hr; ai += hi; break;
      case 1: ar -= hi; ai += hr; break;
      case 2: ar -= hr; ai -= hi; break;
      default: ar += hi; ai -= hr; break;
    }
  }
  // times i k w_p / (16 pi^2)
  double f = k * wgt[p] / (16.0 * kPi * kPi);
  Tt[(int64_t)off * P + p] = mk<Rf>(Rf(-f * ai), Rf(f * ar));
}

// Degree-rescale filter from level l+1 to level l with ratio
// r = kappa_l / kappa_{l+1} (1/2 while both levels are scaled, 1 once s = 1):
// F[p][q] = sum_{n<ntheta} r^n (2n+1)/(4 pi) P_n(khat_p.khat_q) w_q.
template <typename Rf>
__global__ void k_filter(int P, int ntheta, double ratio, const double* __restrict__ khat,
                         const double* __restrict__ wgt, Rf* __restrict__ F, Rf* __restrict__ Ft) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * P) return;
  int p = i / P, q = i % P;
  double x = khat[3 * p] * khat[3 * q] + khat[3 * p + 1] * khat[3 * q + 1] + khat[3 * p + 2] * khat[3 * q + 2];
  x = fmin(1.0, fmax(-1.0, x));
  double Pm = 1.0, Pc = x, sum = 1.0 / kFourPi, r = 1.0;
  for (int l = 1; l < ntheta; ++l) {
    r *= ratio;
    double Pl = (l == 1) ? x : Pc;
    if (l >= 2) {
      Pl = ((2.0 * l - 1.0) * x * Pc - (l - 1.0) * Pm) / l;
      Pm = Pc;
      Pc = Pl;
    }
    sum += r * (2.0 * l + 1.0) / kFourPi * Pl;
  }
  double v = sum * wgt[q];
  F[(int64_t)p * P + q] = Rf(v);
  Ft[(int64_t)q * P + p] = Rf(v);
}

// Azimuthal blocks of the block-circulant filter:
// K_m[i][k] = (1/NPHI) sum_d F[(i, d)][(k, 0)] cos(2 pi m d / NPHI)
// (F[(i,d)][(k,0)] is even in d, so the sine part vanishes).
template <typename Rf>
__global__ void k_filter_fourier(int ntheta, const Rf* __restrict__ F, Rf* __restrict__ Kf) {
  const int nphi = 2 * ntheta, P = ntheta * nphi;
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nphi * ntheta * ntheta) return;
  int m = id / (ntheta * ntheta), i = (id / ntheta) % ntheta, k = id % ntheta;
  double acc = 0;
  for (int d = 0; d < nphi; ++d) {
    double c = cospi(2.0 * double(m * d % nphi) / nphi);
    acc += double(F[(int64_t)(i * nphi + d) * P + k * nphi]) * c;
  }
  Kf[id] = Rf(acc / nphi);
}

// Interpolation phases for the children of level-l boxes:
// exp(-i kappa_l khat_p . (C_child - C_parent)), C_child - C_parent = (a_{l+1}/2)(+-1,+-1,+-1).
template <typename Rf>
__global__ void k_phase(int P, double kappa, double half, const double* __restrict__ khat, C2<Rf>* __restrict__ ph) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * P) return;
  int o = i / P, p = i % P;
  double d[3] = {half * (2 * ((o >> 2) & 1) - 1), half * (2 * ((o >> 1) & 1) - 1), half * (2 * (o & 1) - 1)};
  double arg = -kappa * (khat[3 * p] * d[0] + khat[3 * p + 1] * d[1] + khat[3 * p + 2] * d[2]);
  double s, c;
  sincos(arg, &s, &c);
  ph[i] = mk<Rf>(Rf(c), Rf(s));
}

// ------------------------------------------------------------ host side

pie_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PIE_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PIE_ERR_OOM : PIE_ERR_CUDA;
}

void* dalloc(Problem& pr, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  pr.allocs.push_back(p);
  pr.bytes += bytes;
  return p;
}

template <typename T>
static T* upload(Problem& pr, const std::vector<T>& h, cudaStream_t st, pie_status& s) {
  if (s != PIE_OK) return nullptr;
  T* d = static_cast<T*>(dalloc(pr, sizeof(T) * h.size()));
  if (!d) {
    set_error("device allocation failed");
    s = PIE_ERR_OOM;
    return nullptr;
  }
  if (!h.empty()) s = cuda_check(cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st), "upload");
  return d;
}

static void* zalloc(Problem& pr, size_t bytes, pie_status& s) {
  if (s != PIE_OK) return nullptr;
  void* d = dalloc(pr, bytes);
  if (!d) {
    set_error("device allocation failed");
    s = PIE_ERR_OOM;
  }
  return d;
}

template <typename Rm, typename Rf>
static pie_status setup_t(Problem& pr, cudaStream_t st) {
  const Mesh& m = pr.mesh;
  const Tree& tr = pr.tree;
  const int64_t T = pr.T, E = pr.E;
  const int L = tr.L;
  const int P = pr.P;
  pie_status s = PIE_OK;

  // tree-ordered triangle tables
  std::vector<int32_t> tri_edge(T * 3), leaf_of(T);
  std::vector<double> tri_c(T * 3, 0.0), tri_dcp(T * 9, 0.0), vert(T * 9), cent(T * 3), h2(T), area(T);
  for (int64_t i = 0; i < T; ++i) {
    int64_t tm = tr.perm[i];
    for (int k = 0; k < 3; ++k) {
      int32_t v = m.tri[3 * tm + k];
      for (int d = 0; d < 3; ++d) vert[9 * i + 3 * k + d] = m.xyz[3 * v + d];
    }
    for (int d = 0; d < 3; ++d) cent[3 * i + d] = m.centroid[3 * tm + d];
    h2[i] = m.h2[tm];
    area[i] = m.area[tm];
    for (int k = 0; k < 3; ++k) {
      int32_t n = m.tri_edge[3 * tm + k];
      tri_edge[3 * i + k] = n;
      if (n < 0) continue;
      int sg = m.tri_sign[3 * tm + k];
      const double* a = &m.xyz[3 * m.edges[2 * n]];
      const double* b = &m.xyz[3 * m.edges[2 * n + 1]];
      double len = std::sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) + (b[2] - a[2]) * (b[2] - a[2]));
      tri_c[3 * i + k] = sg * len / (2.0 * m.area[tm]);
      int32_t fv = m.edge_free[2 * n + (sg > 0 ? 0 : 1)];
      for (int d = 0; d < 3; ++d) tri_dcp[9 * i + 3 * k + d] = m.centroid[3 * tm + d] - m.xyz[3 * fv + d];
    }
  }
  std::vector<int32_t> edge_tt(E * 2);
  std::vector<int8_t> edge_k(E * 2);
  for (int64_t n = 0; n < E; ++n)
    for (int side = 0; side < 2; ++side) {
      int32_t tm = m.edge_tri[2 * n + side];
      edge_tt[2 * n + side] = int32_t(tr.inv_perm[tm]);
      int kk = 0;
      for (int k = 0; k < 3; ++k)
        if (m.tri_edge[3 * tm + k] == n) kk = k;
      edge_k[2 * n + side] = int8_t(kk);
    }
  const int64_t nleaf = int64_t(tr.keys[L].size());
  pr.nleaf = nleaf;
  std::vector<int32_t> leaf_start(nleaf + 1), near_ptr(nleaf + 1), near_idx(tr.near_idx.size());
  std::vector<double> leaf_center(nleaf * 3);
  const double aL = tr.box_size(L);
  for (int64_t b = 0; b <= nleaf; ++b) leaf_start[b] = int32_t(tr.leaf_start[b]);
  for (int64_t b = 0; b < nleaf; ++b) {
    for (int64_t i = tr.leaf_start[b]; i < tr.leaf_start[b + 1]; ++i) leaf_of[i] = int32_t(b);
    int64_t key = tr.keys[L][b], ii[3] = {0, 0, 0};
    for (int bit = 0; bit < L - 1; ++bit) {
      ii[0] |= ((key >> (3 * bit + 2)) & 1) << bit;
      ii[1] |= ((key >> (3 * bit + 1)) & 1) << bit;
      ii[2] |= ((key >> (3 * bit)) & 1) << bit;
    }
    for (int d = 0; d < 3; ++d) leaf_center[3 * b + d] = tr.x0[d] + (double(ii[d]) + 0.5) * aL;
  }
  for (size_t i = 0; i < near_ptr.size(); ++i) near_ptr[i] = int32_t(tr.near_ptr[i]);
  for (size_t i = 0; i < near_idx.size(); ++i) near_idx[i] = int32_t(tr.near_idx[i]);
  std::vector<int32_t> near_off(near_idx.size());
  for (int64_t b = 0; b < nleaf; ++b) {
    int32_t acc = 0;
    for (int64_t qi = tr.near_ptr[b]; qi < tr.near_ptr[b + 1]; ++qi) {
      near_off[qi] = acc;
      acc += int32_t(tr.leaf_start[tr.near_idx[qi] + 1] - tr.leaf_start[tr.near_idx[qi]]);
    }
  }
  std::vector<int64_t> row_ptr(T + 1, 0);
  for (int64_t i = 0; i < T; ++i) {
    int64_t b = leaf_of[i], cnt = 0;
    for (int64_t q = tr.near_ptr[b]; q < tr.near_ptr[b + 1]; ++q) {
      int64_t nb = tr.near_idx[q];
      cnt += tr.leaf_start[nb + 1] - tr.leaf_start[nb];
    }
    row_ptr[i + 1] = row_ptr[i] + cnt;
  }
  pr.nnz = row_ptr[T];

  // angular grid: ntheta Gauss-Legendre nodes in cos(theta) x 2 ntheta azimuths
  const int nt = pr.par.ntheta;
  std::vector<double> gx, gw;
  gauss_legendre(nt, gx, gw);
  // The lower theta rows are computed; the upper rows are their exact
  // negatives (antipodes), so that -khat is on the grid bit for bit.
  std::vector<double> khat(3 * P), wgt(P);
  for (int i = 0; i < nt / 2; ++i)
    for (int j = 0; j < 2 * nt; ++j) {
      int p = i * 2 * nt + j;
      int pa = (nt - 1 - i) * 2 * nt + (j + nt) % (2 * nt);
      double ct = gx[i], stt = std::sqrt(1.0 - ct * ct), ph = kPi * j / nt;
      khat[3 * p] = stt * std::cos(ph);
      khat[3 * p + 1] = stt * std::sin(ph);
      khat[3 * p + 2] = ct;
      for (int d = 0; d < 3; ++d) khat[3 * pa + d] = -khat[3 * p + d];
      wgt[p] = gw[i] * kPi / nt;
      wgt[pa] = gw[nt - 1 - i] * kPi / nt;
    }
  // 7-point degree-5 rule (Radon), closed form; and the 8 x 8 collapsed Gauss rule
  std::vector<double> r7, r64;
  {
    const double s15 = std::sqrt(15.0);
    r7 = {1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40};
    const double as[2] = {(6.0 - s15) / 21.0, (6.0 + s15) / 21.0};
    const double ws[2] = {(155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0};
    for (int o = 0; o < 2; ++o) {
      double a = as[o], b = 1.0 - 2.0 * a;
      double pts[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
      for (auto& q : pts) r7.insert(r7.end(), {q[0], q[1], q[2], ws[o]});
    }
    std::vector<double> ux, uw;
    gauss_legendre(8, ux, uw);
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) {
        double u = 0.5 * (ux[i] + 1.0), v = 0.5 * (ux[j] + 1.0);
        double x = u, y = (1.0 - u) * v;
        r64.insert(r64.end(), {1.0 - x - y, x, y, 2.0 * (0.5 * uw[i]) * (0.5 * uw[j]) * (1.0 - u)});
      }
  }

  pr.tri_edge = upload(pr, tri_edge, st, s);
  pr.tri_c = upload(pr, tri_c, st, s);
  pr.tri_dcp = upload(pr, tri_dcp, st, s);
  pr.perm = upload(pr, tr.perm, st, s);
  pr.inv_perm = upload(pr, tr.inv_perm, st, s);
  pr.edge_tt = upload(pr, edge_tt, st, s);
  pr.edge_k = upload(pr, edge_k, st, s);
  pr.vert = upload(pr, vert, st, s);
  pr.rule7_host = r7;
  pr.cent = upload(pr, cent, st, s);
  pr.h2 = upload(pr, h2, st, s);
  pr.area = upload(pr, area, st, s);
  pr.leaf_of = upload(pr, leaf_of, st, s);
  pr.leaf_start = upload(pr, leaf_start, st, s);
  pr.leaf_center = upload(pr, leaf_center, st, s);
  pr.near_ptr = upload(pr, near_ptr, st, s);
  pr.near_idx = upload(pr, near_idx, st, s);
  pr.near_off = upload(pr, near_off, st, s);
  pr.row_ptr = upload(pr, row_ptr, st, s);
  pr.khat = upload(pr, khat, st, s);
  pr.wgt = upload(pr, wgt, st, s);
  pr.rule7 = upload(pr, r7, st, s);
  pr.rule64 = upload(pr, r64, st, s);
  if (s != PIE_OK) return s;

  // near pair moments (three passes, see k_near_regular)
  pr.mom = zalloc(pr, sizeof(C2<Rm>) * kMom * size_t(pr.nnz), s);
  unsigned long long* dcount = static_cast<unsigned long long*>(zalloc(pr, 2 * sizeof(unsigned long long), s));
  if (s != PIE_OK) return s;
  NearGeom ng{pr.leaf_of, pr.leaf_start, pr.near_ptr, pr.near_idx, pr.near_off, pr.row_ptr,
              pr.vert, pr.cent, pr.area, pr.h2};
  cudaMemsetAsync(dcount, 0, 2 * sizeof(unsigned long long), st);
  k_count_singular<<<unsigned((T * 32 + 255) / 256), 256, 0, st>>>(T, ng, dcount);
  unsigned long long nsing = 0;
  if ((s = cuda_check(cudaMemcpyAsync(&nsing, dcount, sizeof(nsing), cudaMemcpyDeviceToHost, st), "count")) != PIE_OK)
    return s;
  if ((s = cuda_check(cudaStreamSynchronize(st), "count sync")) != PIE_OK) return s;
  SingPair* list = static_cast<SingPair*>(zalloc(pr, sizeof(SingPair) * std::max<unsigned long long>(nsing, 1), s));
  if (s != PIE_OK) return s;
  k_near_regular<Rm><<<unsigned((T * 32 + 127) / 128), 128, 0, st>>>(
      T, pr.nnz, ng, pr.k0, pr.rule7, static_cast<C2<Rm>*>(pr.mom), list, dcount + 1, nsing);
  k_near_singular<Rm><<<unsigned((nsing + 127) / 128), 128, 0, st>>>(int64_t(nsing), pr.nnz, ng, pr.k0, pr.rule7,
                                                                     pr.rule64, list, static_cast<C2<Rm>*>(pr.mom));
  if ((s = cuda_check(cudaGetLastError(), "near build")) != PIE_OK) return s;

  // leaf radiation tables
  const double x = pr.par.kappa_a;
  // kappa_l = k0 / s_l with s_l = min(k0 a_l / x, 1): boxes small in
  // wavelengths use the scaled plane waves of Eq. (4), larger ones the
  // standard diagonalization (s = 1)
  auto kappa_of = [&](int l) { return std::max(x / tr.box_size(l), pr.k0); };
  pr.Pi = zalloc(pr, sizeof(C2<Rf>) * size_t(T) * (P / 2), s);
  pr.M = zalloc(pr, sizeof(C2<Rf>) * size_t(T) * 3 * (P / 2), s);
  pr.PiR = zalloc(pr, sizeof(C2<Rf>) * size_t(T) * (P / 2), s);
  pr.MR = zalloc(pr, sizeof(C2<Rf>) * size_t(T) * 3 * (P / 2), s);
  if (s != PIE_OK) return s;
  k_rad<Rf><<<unsigned((T * (P / 2) + 255) / 256), 256, 0, st>>>(T, P / 2, pr.vert, pr.cent, pr.area, pr.leaf_of,
                                                           pr.leaf_center, pr.khat, kappa_of(L), pr.rule7,
                                                           static_cast<C2<Rf>*>(pr.Pi), static_cast<C2<Rf>*>(pr.M),
                                                           static_cast<C2<Rf>*>(pr.PiR), static_cast<C2<Rf>*>(pr.MR));
  if ((s = cuda_check(cudaGetLastError(), "radiation tables")) != PIE_OK) return s;

  // levels
  pr.lev.assign(L + 1, LevelDev{});
  for (int l = 1; l <= L; ++l) {
    LevelDev& lv = pr.lev[l];
    lv.nb = int64_t(tr.keys[l].size());
    if (l >= 4) {
      std::vector<int32_t> par(lv.nb);
      std::vector<int8_t> oct(lv.nb);
      for (int64_t b = 0; b < lv.nb; ++b) {
        par[b] = int32_t(tr.parent[l][b]);
        oct[b] = int8_t(tr.keys[l][b] & 7);
      }
      lv.parent = upload(pr, par, st, s);
      lv.octant = upload(pr, oct, st, s);
    }
    if (l >= 3 && l < L) {
      std::vector<int32_t> cs(tr.child_start[l].begin(), tr.child_start[l].end());
      lv.child_start = upload(pr, cs, st, s);
    }
    if (l >= 3) {
      std::vector<int32_t> ptr(tr.il_ptr[l].begin(), tr.il_ptr[l].end());
      std::vector<int32_t> idx(tr.il_idx[l].begin(), tr.il_idx[l].end());
      lv.il_ptr = upload(pr, ptr, st, s);
      lv.il_idx = upload(pr, idx, st, s);
      lv.il_off = upload(pr, tr.il_off[l], st, s);
      lv.S = zalloc(pr, sizeof(C2<Rf>) * size_t(pr.par.max_nrhs) * size_t(lv.nb) * kComp * P, s);
      lv.G = zalloc(pr, sizeof(C2<Rf>) * size_t(pr.par.max_nrhs) * size_t(lv.nb) * kComp * P, s);
      lv.trans = zalloc(pr, sizeof(C2<Rf>) * kNoffs * P, s);
      if (s != PIE_OK) return s;
      const double al = tr.box_size(l);
      lv.kappa = kappa_of(l);
      k_trans_table<Rf><<<unsigned((kNoffs * P + 127) / 128), 128, 0, st>>>(
          P, pr.par.tau, pr.k0, pr.k0 / lv.kappa, al, pr.khat, pr.wgt, static_cast<C2<Rf>*>(lv.trans));
      if (l < L) {
        lv.phase = zalloc(pr, sizeof(C2<Rf>) * 8 * P, s);
        if (s != PIE_OK) return s;
        k_phase<Rf><<<unsigned((8 * P + 127) / 128), 128, 0, st>>>(P, lv.kappa, 0.5 * tr.box_size(l + 1), pr.khat,
                                                                   static_cast<C2<Rf>*>(lv.phase));
        lv.F = zalloc(pr, sizeof(Rf) * P * P, s);
        lv.Ft = zalloc(pr, sizeof(Rf) * P * P, s);
        lv.Kf = zalloc(pr, sizeof(Rf) * 2 * nt * nt * nt, s);
        if (s != PIE_OK) return s;
        k_filter<Rf><<<unsigned((P * P + 127) / 128), 128, 0, st>>>(P, nt, lv.kappa / kappa_of(l + 1), pr.khat, pr.wgt,
                                                                    static_cast<Rf*>(lv.F), static_cast<Rf*>(lv.Ft));
        k_filter_fourier<Rf><<<unsigned((2 * nt * nt * nt + 127) / 128), 128, 0, st>>>(
            nt, static_cast<const Rf*>(lv.F), static_cast<Rf*>(lv.Kf));
      }
    }
    if (s != PIE_OK) return s;
  }
  const size_t cio = pr.io_f32() ? sizeof(cf) : sizeof(cd);
  const size_t nr = size_t(pr.par.max_nrhs);
  pr.gsgd = zalloc(pr, sizeof(C2<Rf>) * 2 * nr * size_t(pr.lev[L].nb) * kComp * (P / 2), s);
  pr.coef = zalloc(pr, cio * 6 * size_t(T) * nr, s);
  pr.pot = zalloc(pr, cio * 6 * size_t(T) * nr, s);
  pr.pot2 = zalloc(pr, cio * 6 * size_t(T) * nr, s);
  if (pr.par.precision == PIE_MIXED) pr.coef32 = zalloc(pr, sizeof(cf) * 6 * size_t(T) * nr, s);
  pr.vec = zalloc(pr, cio * size_t(pr.N), s);
  pr.vec2 = zalloc(pr, cio * size_t(pr.N), s);
  if (s != PIE_OK) return s;
  if ((s = cuda_check(cudaGetLastError(), "setup launch")) != PIE_OK) return s;
  int dev = 0;
  if ((s = cuda_check(cudaGetDevice(&dev), "device")) != PIE_OK) return s;
  if ((s = cuda_check(cudaDeviceGetAttribute(&pr.nsm, cudaDevAttrMultiProcessorCount, dev), "SM count")) != PIE_OK)
    return s;
  if ((s = cuda_check(cudaStreamCreateWithFlags(&pr.side, cudaStreamNonBlocking), "side stream")) != PIE_OK) return s;
  int prio_low = 0, prio_high = 0;
  if ((s = cuda_check(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high), "stream priorities")) != PIE_OK)
    return s;
  if ((s = cuda_check(cudaStreamCreateWithPriority(&pr.far, cudaStreamNonBlocking, prio_high), "far stream")) !=
      PIE_OK)
    return s;
  if ((s = cuda_check(cudaEventCreateWithFlags(&pr.ev_fork, cudaEventDisableTiming), "event")) != PIE_OK) return s;
  if ((s = cuda_check(cudaEventCreateWithFlags(&pr.ev_join, cudaEventDisableTiming), "event")) != PIE_OK) return s;
  if ((s = cuda_check(cudaEventCreateWithFlags(&pr.ev_far, cudaEventDisableTiming), "event")) != PIE_OK) return s;
  pr.tune = pie_tuning{1, 2, pr.par.max_nrhs, 0, 0, 0};
  return cuda_check(cudaStreamSynchronize(st), "setup");
}

// Largest |re| and |im| of each of the eight moment planes (blockIdx.y):
// non-negative floats order like their bit patterns, so atomicMax on those.
__global__ void k_plane_absmax(int64_t nnz, const cf* __restrict__ mom, unsigned* __restrict__ mx) {
  const int q = blockIdx.y;
  float m = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
    const cf v = mom[q * nnz + e];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx + q, __float_as_uint(m));
}

// out = round-to-nearest half of (value * 2^e[plane]), plane by plane.
// One thread per pair: the eight planes' entries e become the pair's record
// of eight half pairs (32 bytes, entry-major [nnz][8]).
__global__ void k_to_half(int64_t nnz, const cf* __restrict__ mom, MomScale mul, __half2* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
    uint32_t w[kMom];
#pragma unroll
    for (int q = 0; q < kMom; ++q) {
      const cf v = mom[q * nnz + e];
      const __half2 h = __floats2half2_rn(v.x * mul.s[q], v.y * mul.s[q]);
      memcpy(&w[q], &h, sizeof(h));
    }
    uint4* o = reinterpret_cast<uint4*>(out + kMom * e);
    o[0] = make_uint4(w[0], w[1], w[2], w[3]);
    o[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

// PIE_FP32H: the float moments built by setup_t become half pairs, each
// plane scaled by the power of two that puts its largest magnitude in
// [2^14, 2^15) (half's largest finite value is 65504); the scale's inverse is
// kept in pr.mom_scale.  The half moments are stored pair by pair ([nnz][8],
// one 32-byte record per pair, read with two 16-byte loads), unlike the
// plane-major float and double moments.  The float planes are freed.
static pie_status moments_to_half(Problem& pr, cudaStream_t st) {
  pie_status s = PIE_OK;
  const int64_t nnz = pr.nnz;
  unsigned* mx = static_cast<unsigned*>(zalloc(pr, sizeof(unsigned) * kMom, s));
  __half2* h = static_cast<__half2*>(zalloc(pr, sizeof(__half2) * kMom * size_t(nnz), s));
  if (s != PIE_OK) return s;
  const unsigned grid = unsigned(std::min<int64_t>((nnz + 255) / 256, 4096));
  cudaMemsetAsync(mx, 0, sizeof(unsigned) * kMom, st);
  const cf* mom = static_cast<const cf*>(pr.mom);
  k_plane_absmax<<<dim3(std::max(grid, 1u), kMom), 256, 0, st>>>(nnz, mom, mx);
  unsigned hm[kMom];
  if ((s = cuda_check(cudaMemcpyAsync(hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, st), "moment range")) != PIE_OK)
    return s;
  if ((s = cuda_check(cudaStreamSynchronize(st), "moment range")) != PIE_OK) return s;
  MomScale mul;
  for (int q = 0; q < kMom; ++q) {
    float m;
    std::memcpy(&m, &hm[q], sizeof(m));
    int e = 0;
    if (m > 0.f && std::isfinite(m)) std::frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
    const int sh = (m > 0.f && std::isfinite(m)) ? 15 - e : 0;
    mul.s[q] = std::ldexp(1.0f, sh);
    pr.mom_scale[q] = std::ldexp(1.0f, -sh);
  }
  k_to_half<<<std::max(grid, 1u), 256, 0, st>>>(nnz, mom, mul, h);
  if ((s = cuda_check(cudaStreamSynchronize(st), "moments to half")) != PIE_OK) return s;
  // release the float planes and the range buffer
  auto release = [&](void* ptr, size_t bytes) {
    for (size_t i = 0; i < pr.allocs.size(); ++i)
      if (pr.allocs[i] == ptr) {
        cudaFree(ptr);
        pr.allocs.erase(pr.allocs.begin() + i);
        pr.bytes -= bytes;
        return;
      }
  };
  release(pr.mom, sizeof(cf) * kMom * size_t(nnz));
  release(mx, sizeof(unsigned) * kMom);
  pr.mom = h;
  return PIE_OK;
}

pie_status setup_device(Problem& pr, cudaStream_t st) {
  switch (pr.par.precision) {
    case PIE_FP64:
      return setup_t<double, double>(pr, st);
    case PIE_FP32:
      return setup_t<float, float>(pr, st);
    case PIE_FP32H: {
      pie_status s = setup_t<float, float>(pr, st);
      return s == PIE_OK ? moments_to_half(pr, st) : s;
    }
    case PIE_MIXED:
      return setup_t<float, double>(pr, st);
  }
  set_error("unknown precision");
  return PIE_ERR_PARAM;
}

}  // namespace pie
