// Mesh topology (RWG / pulse discretisation of Section 2) and oct-tree with
// one-box-buffer lists (Section 3).  Host C++, compiled with
// -ffp-contract=off so that centroids, squared lengths and leaf indices are
// the IEEE double values of the formulas as written.
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "internal.h"

namespace pie {

static inline double sq3(double x, double y, double z) { return (x * x + y * y) + z * z; }

pie_status build_mesh(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, Mesh& m) {
  if (!xyz || !tri || nv < 3 || nt < 1) {
    set_error("pie_mesh_create: empty mesh or NULL array");
    return PIE_ERR_PARAM;
  }
  m.nv = nv;
  m.nt = nt;
  m.xyz.assign(xyz, xyz + nv * 3);
  m.tri.assign(tri, tri + nt * 3);
  m.centroid.resize(nt * 3);
  m.area.resize(nt);
  m.h2.resize(nt);
  for (int64_t t = 0; t < nt; ++t) {
    int32_t v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
    for (int k = 0; k < 3; ++k)
      if (v[k] < 0 || v[k] >= nv) {
        set_error("pie_mesh_create: vertex index out of range");
        return PIE_ERR_PARAM;
      }
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) {
      set_error("pie_mesh_create: repeated vertex in a triangle");
      return PIE_ERR_DEGENERATE;
    }
    const double* a = xyz + 3 * v[0];
    const double* b = xyz + 3 * v[1];
    const double* c = xyz + 3 * v[2];
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = b[d] - a[d];
      e2[d] = c[d] - a[d];
      m.centroid[3 * t + d] = ((a[d] + b[d]) + c[d]) / 3.0;
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1];
    double cy = e1[2] * e2[0] - e1[0] * e2[2];
    double cz = e1[0] * e2[1] - e1[1] * e2[0];
    double ar = 0.5 * std::sqrt(sq3(cx, cy, cz));
    if (!(ar > 0.0)) {
      set_error("pie_mesh_create: zero-area triangle");
      return PIE_ERR_DEGENERATE;
    }
    m.area[t] = ar;
    double l01 = sq3(b[0] - a[0], b[1] - a[1], b[2] - a[2]);
    double l12 = sq3(c[0] - b[0], c[1] - b[1], c[2] - b[2]);
    double l20 = sq3(a[0] - c[0], a[1] - c[1], a[2] - c[2]);
    m.h2[t] = std::max(std::max(l01, l12), l20);
  }
  // occurrences of every undirected edge: (vmin, vmax, triangle, local edge)
  struct Occ {
    int32_t a, b;
    int32_t t;
    int8_t k;
    bool operator<(const Occ& o) const { return std::tie(a, b, t) < std::tie(o.a, o.b, o.t); }
  };
  std::vector<Occ> occ(nt * 3);
  for (int64_t t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      int32_t u = tri[3 * t + k], w = tri[3 * t + (k + 1) % 3];
      occ[3 * t + k] = {std::min(u, w), std::max(u, w), int32_t(t), int8_t(k)};
    }
  std::sort(occ.begin(), occ.end());
  m.tri_edge.assign(nt * 3, -1);
  m.tri_sign.assign(nt * 3, 0);
  m.edges.clear();
  m.edge_tri.clear();
  m.edge_free.clear();
  size_t i = 0;
  while (i < occ.size()) {
    size_t j = i;
    while (j < occ.size() && occ[j].a == occ[i].a && occ[j].b == occ[i].b) ++j;
    size_t cnt = j - i;
    if (cnt > 2) {
      set_error("pie_mesh_create: edge shared by more than two triangles");
      return PIE_ERR_NONMANIFOLD;
    }
    if (cnt == 2) {
      int32_t n = int32_t(m.edges.size() / 2);
      int side_of[2];
      for (int q = 0; q < 2; ++q) {
        const Occ& o = occ[i + q];
        int32_t from = tri[3 * o.t + o.k];
        side_of[q] = (from == o.a) ? 0 : 1;  // 0: runs vmin -> vmax => "+" triangle
      }
      if (side_of[0] == side_of[1]) {
        set_error("pie_mesh_create: inconsistent triangle orientation");
        return PIE_ERR_ORIENTATION;
      }
      int32_t tp = 0, tm = 0, fp = 0, fm = 0;
      for (int q = 0; q < 2; ++q) {
        const Occ& o = occ[i + q];
        int32_t free = tri[3 * o.t + (o.k + 2) % 3];
        m.tri_edge[3 * o.t + o.k] = n;
        m.tri_sign[3 * o.t + o.k] = side_of[q] == 0 ? 1 : -1;
        if (side_of[q] == 0) {
          tp = o.t;
          fp = free;
        } else {
          tm = o.t;
          fm = free;
        }
      }
      m.edges.push_back(occ[i].a);
      m.edges.push_back(occ[i].b);
      m.edge_tri.push_back(tp);
      m.edge_tri.push_back(tm);
      m.edge_free.push_back(fp);
      m.edge_free.push_back(fm);
    }
    i = j;
  }
  m.ne = int64_t(m.edges.size() / 2);
  return PIE_OK;
}

static int64_t morton(int64_t ix, int64_t iy, int64_t iz, int bits) {
  int64_t key = 0;
  for (int b = 0; b < bits; ++b) {
    key |= ((ix >> b) & 1) << (3 * b + 2);
    key |= ((iy >> b) & 1) << (3 * b + 1);
    key |= ((iz >> b) & 1) << (3 * b);
  }
  return key;
}

static void demorton(int64_t key, int bits, int64_t& ix, int64_t& iy, int64_t& iz) {
  ix = iy = iz = 0;
  for (int b = 0; b < bits; ++b) {
    ix |= ((key >> (3 * b + 2)) & 1) << b;
    iy |= ((key >> (3 * b + 1)) & 1) << b;
    iz |= ((key >> (3 * b)) & 1) << b;
  }
}

int offset_code(int dx, int dy, int dz) {
  if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) <= 1) return -1;
  int code = 0;
  for (int x = -3; x <= 3; ++x)
    for (int y = -3; y <= 3; ++y)
      for (int z = -3; z <= 3; ++z) {
        if (std::max(std::abs(x), std::max(std::abs(y), std::abs(z))) <= 1) continue;
        if (x == dx && y == dy && z == dz) return code;
        ++code;
      }
  return -1;
}

pie_status build_tree(const Mesh& m, int L, double root_side, Tree& tr) {
  if (L < 3 || L > 21) {
    set_error("levels must be in [3, 21]");
    return PIE_ERR_PARAM;
  }
  tr.L = L;
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = hi[d] = m.xyz[d];
  }
  for (int64_t v = 0; v < m.nv; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], m.xyz[3 * v + d]);
      hi[d] = std::max(hi[d], m.xyz[3 * v + d]);
    }
  double side = root_side;
  if (!(side > 0)) side = std::max(std::max(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
  if (!(side > 0)) {
    set_error("degenerate bounding box");
    return PIE_ERR_PARAM;
  }
  tr.side = side;
  for (int d = 0; d < 3; ++d) tr.x0[d] = (lo[d] + hi[d]) * 0.5 - side * 0.5;
  const int64_t nleaf = int64_t(1) << (L - 1);
  const double scale = double(nleaf) / side;
  const int64_t T = m.nt;
  std::vector<int64_t> key(T);
  for (int64_t t = 0; t < T; ++t) {
    int64_t ii[3];
    for (int d = 0; d < 3; ++d) {
      double q = (m.centroid[3 * t + d] - tr.x0[d]) * scale;
      int64_t v = int64_t(std::floor(q));
      ii[d] = std::min(std::max(v, int64_t(0)), nleaf - 1);
    }
    key[t] = morton(ii[0], ii[1], ii[2], L - 1);
  }
  tr.perm.resize(T);
  for (int64_t t = 0; t < T; ++t) tr.perm[t] = t;
  std::stable_sort(tr.perm.begin(), tr.perm.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  tr.inv_perm.resize(T);
  for (int64_t i = 0; i < T; ++i) tr.inv_perm[tr.perm[i]] = i;
  std::vector<int64_t> leafkey(T);
  for (int64_t i = 0; i < T; ++i) leafkey[i] = key[tr.perm[i]];

  tr.keys.assign(L + 1, {});
  tr.parent.assign(L + 1, {});
  tr.child_start.assign(L + 1, {});
  for (int l = 1; l <= L; ++l) {
    auto& k = tr.keys[l];
    int sh = 3 * (L - l);
    for (int64_t i = 0; i < T; ++i) {
      int64_t v = leafkey[i] >> sh;
      if (k.empty() || k.back() != v) k.push_back(v);
    }
  }
  for (int l = 2; l <= L; ++l) {
    auto& p = tr.parent[l];
    const auto& kp = tr.keys[l - 1];
    p.resize(tr.keys[l].size());
    for (size_t b = 0; b < tr.keys[l].size(); ++b)
      p[b] = std::lower_bound(kp.begin(), kp.end(), tr.keys[l][b] >> 3) - kp.begin();
  }
  for (int l = 1; l < L; ++l) {
    auto& cs = tr.child_start[l];
    cs.assign(tr.keys[l].size() + 1, 0);
    const auto& pc = tr.parent[l + 1];
    for (size_t c = 0; c < pc.size(); ++c) cs[pc[c] + 1]++;
    for (size_t b = 0; b < tr.keys[l].size(); ++b) cs[b + 1] += cs[b];
  }
  const auto& lk = tr.keys[L];
  tr.leaf_start.resize(lk.size() + 1);
  for (size_t b = 0; b < lk.size(); ++b)
    tr.leaf_start[b] = std::lower_bound(leafkey.begin(), leafkey.end(), lk[b]) - leafkey.begin();
  tr.leaf_start[lk.size()] = T;

  auto find_box = [&](int l, int64_t ix, int64_t iy, int64_t iz) -> int64_t {
    int64_t n = int64_t(1) << (l - 1);
    if (ix < 0 || iy < 0 || iz < 0 || ix >= n || iy >= n || iz >= n) return -1;
    int64_t k = morton(ix, iy, iz, l - 1);
    const auto& ks = tr.keys[l];
    auto it = std::lower_bound(ks.begin(), ks.end(), k);
    if (it == ks.end() || *it != k) return -1;
    return it - ks.begin();
  };
  // near lists at the leaves
  tr.near_ptr.assign(1, 0);
  tr.near_idx.clear();
  for (size_t b = 0; b < lk.size(); ++b) {
    int64_t ix, iy, iz;
    demorton(lk[b], L - 1, ix, iy, iz);
    std::vector<int64_t> nb;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int64_t q = find_box(L, ix + dx, iy + dy, iz + dz);
          if (q >= 0) nb.push_back(q);
        }
    std::sort(nb.begin(), nb.end());
    tr.near_idx.insert(tr.near_idx.end(), nb.begin(), nb.end());
    tr.near_ptr.push_back(int64_t(tr.near_idx.size()));
  }
  // interaction lists at levels 3..L
  tr.il_ptr.assign(L + 1, {});
  tr.il_idx.assign(L + 1, {});
  tr.il_off.assign(L + 1, {});
  for (int l = 3; l <= L; ++l) {
    auto& ptr = tr.il_ptr[l];
    auto& idx = tr.il_idx[l];
    auto& off = tr.il_off[l];
    ptr.assign(1, 0);
    for (size_t b = 0; b < tr.keys[l].size(); ++b) {
      int64_t ix, iy, iz;
      demorton(tr.keys[l][b], l - 1, ix, iy, iz);
      std::vector<std::pair<int64_t, int32_t>> cand;
      int64_t px = ix >> 1, py = iy >> 1, pz = iz >> 1;
      for (int64_t qx = 2 * (px - 1); qx <= 2 * (px + 1) + 1; ++qx)
        for (int64_t qy = 2 * (py - 1); qy <= 2 * (py + 1) + 1; ++qy)
          for (int64_t qz = 2 * (pz - 1); qz <= 2 * (pz + 1) + 1; ++qz) {
            int64_t dx = ix - qx, dy = iy - qy, dz = iz - qz;
            if (std::max(std::llabs(dx), std::max(std::llabs(dy), std::llabs(dz))) <= 1) continue;
            int64_t q = find_box(l, qx, qy, qz);
            if (q >= 0) cand.push_back({q, int32_t(offset_code(int(dx), int(dy), int(dz)))});
          }
      std::sort(cand.begin(), cand.end());
      for (auto& c : cand) {
        idx.push_back(c.first);
        off.push_back(c.second);
      }
      ptr.push_back(int64_t(idx.size()));
    }
  }
  return PIE_OK;
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton iteration
// on the three-term recurrence of the Legendre polynomials.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) {
        p1 = z;
        p0 = 1.0;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace pie
