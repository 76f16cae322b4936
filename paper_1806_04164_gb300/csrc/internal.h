// Internal declarations of the PIE MLFMA library (host side).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pie.h"

namespace pie {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;
constexpr double kC0 = 299792458.0;
inline double eps0() { return 1.0 / (kMu0 * kC0 * kC0); }

void set_error(const std::string& msg);

struct Mesh {
  int64_t nv = 0, nt = 0, ne = 0;
  std::vector<double> xyz;            // [nv*3]
  std::vector<int32_t> tri;           // [nt*3]
  std::vector<int32_t> edges;         // [ne*2] (vmin, vmax)
  std::vector<int32_t> edge_tri;      // [ne*2] (T+, T-)
  std::vector<int32_t> edge_free;     // [ne*2]
  std::vector<int32_t> tri_edge;      // [nt*3] RWG of local edge k (k: v_k -> v_k+1), -1 if boundary
  std::vector<int8_t> tri_sign;       // [nt*3] +1 / -1 / 0
  std::vector<double> centroid;       // [nt*3] ((v0 + v1) + v2) / 3
  std::vector<double> area;           // [nt]
  std::vector<double> h2;             // [nt] longest squared edge, ((x*x + y*y) + z*z)
};

// Oct-tree of Section 3 (one-box buffer).  Level index 1..L.
struct Tree {
  int L = 0;
  double x0[3] = {0, 0, 0};
  double side = 0;
  std::vector<int64_t> perm;                  // tree position -> mesh triangle
  std::vector<int64_t> inv_perm;              // mesh triangle -> tree position
  std::vector<std::vector<int64_t>> keys;     // [L+1][nb]
  std::vector<std::vector<int64_t>> parent;   // [L+1][nb] box number at l-1
  std::vector<std::vector<int64_t>> child_start;  // [L+1][nb+1] children at l+1
  std::vector<int64_t> leaf_start;            // [nleaf+1]
  std::vector<int64_t> near_ptr, near_idx;    // leaf near lists
  std::vector<std::vector<int64_t>> il_ptr, il_idx;  // [L+1]
  std::vector<std::vector<int32_t>> il_off;           // [L+1]
  double box_size(int l) const { return side / double(int64_t(1) << (l - 1)); }
};

pie_status build_mesh(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, Mesh& m);
pie_status build_tree(const Mesh& m, int L, double root_side, Tree& t);
int offset_code(int dx, int dy, int dz);
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

}  // namespace pie
