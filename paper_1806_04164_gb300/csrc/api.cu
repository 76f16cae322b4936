// extern "C" entry points of include/pie.h.
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include <cuda_fp16.h>

#include "handles.h"

namespace pie {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

pie_status check_device(const Problem& pr, const char* who) {
  int dev = -1;
  pie_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (s == PIE_OK && dev != pr.device) {
    set_error(std::string(who) + ": the current device (" + std::to_string(dev) +
              ") is not the one the problem was built on (" + std::to_string(pr.device) + ")");
    s = PIE_ERR_PARAM;
  }
  return s;
}
}  // namespace pie

using namespace pie;

extern "C" {

const char* pie_last_error(void) { return g_err.c_str(); }

void pie_params_default(pie_params* p) {
  if (!p) return;
  p->levels = 3;
  p->root_side = 0.0;
  p->tau = 7;
  p->kappa_a = 0.08;
  p->ntheta = 8;
  p->precision = PIE_FP64;
  p->max_nrhs = 1;
}

pie_status pie_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, pie_mesh** out) {
  if (!out) {
    set_error("pie_mesh_create: out is NULL");
    return PIE_ERR_PARAM;
  }
  *out = nullptr;
  pie_mesh* m = new (std::nothrow) pie_mesh;
  if (!m) return PIE_ERR_OOM;
  pie_status s = build_mesh(xyz, nv, tri, nt, m->m);
  if (s != PIE_OK) {
    delete m;
    return s;
  }
  *out = m;
  return PIE_OK;
}

void pie_mesh_destroy(pie_mesh* m) { delete m; }

pie_status pie_mesh_info(const pie_mesh* m, int64_t* nv, int64_t* nt, int64_t* ne) {
  if (!m) {
    set_error("NULL mesh");
    return PIE_ERR_PARAM;
  }
  if (nv) *nv = m->m.nv;
  if (nt) *nt = m->m.nt;
  if (ne) *ne = m->m.ne;
  return PIE_OK;
}

pie_status pie_mesh_edges(const pie_mesh* m, int32_t* edges, int32_t* edge_tri, int32_t* edge_free) {
  if (!m) {
    set_error("NULL mesh");
    return PIE_ERR_PARAM;
  }
  size_t n = m->m.edges.size();
  if (edges) std::memcpy(edges, m->m.edges.data(), n * sizeof(int32_t));
  if (edge_tri) std::memcpy(edge_tri, m->m.edge_tri.data(), n * sizeof(int32_t));
  if (edge_free) std::memcpy(edge_free, m->m.edge_free.data(), n * sizeof(int32_t));
  return PIE_OK;
}

static void free_profile(Problem& pr) {
  for (cudaEvent_t e : pr.prof_ev) cudaEventDestroy(e);
  pr.prof_ev.clear();
  pr.prof_cap = pr.prof_n = 0;
}

static void free_problem(Problem& pr) {
  free_profile(pr);
  if (pr.side) cudaStreamSynchronize(pr.side), cudaStreamDestroy(pr.side);
  if (pr.far) cudaStreamSynchronize(pr.far), cudaStreamDestroy(pr.far);
  if (pr.ev_fork) cudaEventDestroy(pr.ev_fork);
  if (pr.ev_join) cudaEventDestroy(pr.ev_join);
  if (pr.ev_far) cudaEventDestroy(pr.ev_far);
  pr.side = pr.far = nullptr;
  pr.ev_fork = pr.ev_join = pr.ev_far = nullptr;
  for (void* p : pr.allocs) cudaFree(p);
  pr.allocs.clear();
}

pie_status pie_problem_create(const pie_mesh* m, double k0, const pie_params* par, void* stream, pie_problem** out) {
  if (!m || !par || !out) {
    set_error("pie_problem_create: NULL argument");
    return PIE_ERR_PARAM;
  }
  *out = nullptr;
  if (!(k0 > 0) || par->levels < 3 || par->levels > 21 || par->tau < 0 || par->tau > 30 || par->ntheta < 1 ||
      2 * par->ntheta * par->ntheta > 1024 || (par->ntheta & 1) || !(par->kappa_a > 0) || par->precision < 0 ||
      par->precision > 3 || par->max_nrhs < 1 || par->max_nrhs > 1024) {
    set_error("pie_problem_create: parameter out of range");
    return PIE_ERR_PARAM;
  }
  if (m->m.ne == 0) {
    set_error("pie_problem_create: mesh has no interior edge");
    return PIE_ERR_PARAM;
  }
  pie_problem* h = new (std::nothrow) pie_problem;
  if (!h) return PIE_ERR_OOM;
  Problem& pr = h->p;
  pr.mesh = m->m;
  pr.k0 = k0;
  pr.w = k0 * kC0;
  pr.par = *par;
  pr.P = 2 * par->ntheta * par->ntheta;
  pr.T = m->m.nt;
  pr.E = m->m.ne;
  pr.N = pr.T + pr.E;
  pie_status s = build_tree(pr.mesh, par->levels, par->root_side, pr.tree);
  if (s == PIE_OK) {
    double aL = pr.tree.box_size(par->levels);
    double h2max = 0;
    for (double v : pr.mesh.h2) h2max = std::max(h2max, v);
    if (aL * aL < 2.25 * h2max) {
      set_error("leaf box smaller than 1.5 x the longest triangle edge");
      s = PIE_ERR_LEAF;
    }
    // the power series used for s^t j_t(k w) is accurate for k w <= 4
    if (s == PIE_OK && k0 * 3.0 * std::sqrt(3.0) * pr.tree.box_size(3) > 4.0) {
      set_error("k0 too large for the low-frequency translation build (k0 |w| > 4 at level 3)");
      s = PIE_ERR_PARAM;
    }
  }
  if (s == PIE_OK) s = cuda_check(cudaGetDevice(&pr.device), "cudaGetDevice");
  if (s == PIE_OK) s = setup_device(pr, static_cast<cudaStream_t>(stream));
  if (s == PIE_OK) s = noalloc_bind(pr);
  if (s != PIE_OK) {
    free_problem(pr);
    delete h;
    return s;
  }
  *out = h;
  return PIE_OK;
}

void pie_problem_destroy(pie_problem* h) {
  if (!h) return;
  free_problem(h->p);
  delete h;
}

pie_status pie_problem_info(const pie_problem* h, pie_info* info) {
  if (!h || !info) {
    set_error("NULL argument");
    return PIE_ERR_PARAM;
  }
  const Problem& pr = h->p;
  std::memset(info, 0, sizeof(*info));
  info->N = pr.N;
  info->E = pr.E;
  info->T = pr.T;
  info->L = pr.tree.L;
  info->P = pr.P;
  for (int l = 1; l <= pr.tree.L && l < 24; ++l) info->boxes[l] = int64_t(pr.tree.keys[l].size());
  info->near_pairs = pr.nnz;
  info->device_bytes = int64_t(pr.bytes);
  info->leaf_size = pr.tree.box_size(pr.tree.L);
  return PIE_OK;
}

pie_status pie_problem_perm(const pie_problem* h, int64_t* perm) {
  if (!h || !perm) {
    set_error("NULL argument");
    return PIE_ERR_PARAM;
  }
  std::memcpy(perm, h->p.tree.perm.data(), sizeof(int64_t) * h->p.T);
  return PIE_OK;
}

pie_status pie_problem_level(const pie_problem* h, int level, int64_t* nb, int64_t* nlist, int64_t* keys,
                             int64_t* ptr, int64_t* idx, int32_t* off) {
  if (!h) {
    set_error("NULL problem");
    return PIE_ERR_PARAM;
  }
  const Tree& tr = h->p.tree;
  if (level < 1 || level > tr.L) {
    set_error("level out of range");
    return PIE_ERR_PARAM;
  }
  int64_t n = int64_t(tr.keys[level].size());
  int64_t nl = level >= 3 ? int64_t(tr.il_idx[level].size()) : 0;
  if (nb) *nb = n;
  if (nlist) *nlist = nl;
  if (keys) std::memcpy(keys, tr.keys[level].data(), sizeof(int64_t) * n);
  if (level >= 3) {
    if (ptr) std::memcpy(ptr, tr.il_ptr[level].data(), sizeof(int64_t) * (n + 1));
    if (idx) std::memcpy(idx, tr.il_idx[level].data(), sizeof(int64_t) * nl);
    if (off) std::memcpy(off, tr.il_off[level].data(), sizeof(int32_t) * nl);
  }
  return PIE_OK;
}

pie_status pie_problem_near(const pie_problem* h, int64_t* nlist, int64_t* ptr, int64_t* idx) {
  if (!h) {
    set_error("NULL problem");
    return PIE_ERR_PARAM;
  }
  const Tree& tr = h->p.tree;
  if (nlist) *nlist = int64_t(tr.near_idx.size());
  if (ptr) std::memcpy(ptr, tr.near_ptr.data(), sizeof(int64_t) * tr.near_ptr.size());
  if (idx) std::memcpy(idx, tr.near_idx.data(), sizeof(int64_t) * tr.near_idx.size());
  return PIE_OK;
}

static pie_status apply_api(pie_problem* h, const void* x, void* y, int nrhs, int dtype, void* stream, bool near) {
  if (!h || (!x && nrhs > 0) || (!y && nrhs > 0) || nrhs < 0) {
    set_error("pie_apply: invalid argument");
    return PIE_ERR_PARAM;
  }
  Problem& pr = h->p;
  int want = pr.io_f32() ? PIE_C64 : PIE_C128;
  if (dtype != want) {
    set_error("pie_apply: dtype does not match the problem precision");
    return PIE_ERR_PARAM;
  }
  if (pie_status sd = check_device(pr, "pie_apply")) return sd;
  size_t es = pr.io_f32() ? sizeof(cf) : sizeof(cd);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (near) {
    for (int j = 0; j < nrhs; ++j) {
      pie_status s = apply_near_one(pr, static_cast<const char*>(x) + es * size_t(pr.N) * j,
                                    static_cast<char*>(y) + es * size_t(pr.N) * j, st);
      if (s != PIE_OK) return s;
    }
    return PIE_OK;
  }
  // batches of up to tune.rhs_chunk (<= max_nrhs) right-hand sides share
  // each pass over the operator
  return pie::apply_cols(pr, x, y, nrhs, st);
}

pie_status pie_apply(pie_problem* h, const void* x, void* y, int nrhs, int dtype, void* stream) {
  return apply_api(h, x, y, nrhs, dtype, stream, false);
}

pie_status pie_apply_levels(pie_problem* h, const void* x, void* y, uint32_t level_mask, int near, int dtype,
                            void* stream) {
  if (!h || !x || !y || (near != 0 && near != 1)) {
    set_error("pie_apply_levels: invalid argument");
    return PIE_ERR_PARAM;
  }
  Problem& pr = h->p;
  if (dtype != (pr.io_f32() ? PIE_C64 : PIE_C128)) {
    set_error("pie_apply_levels: dtype does not match the problem precision");
    return PIE_ERR_PARAM;
  }
  if (pie_status sd = check_device(pr, "pie_apply_levels")) return sd;
  pr.far_mask = level_mask;
  pr.with_near = near == 1;
  pie_status s = apply_batch(pr, x, y, 1, static_cast<cudaStream_t>(stream));
  pr.far_mask = 0xffffffffu;
  pr.with_near = true;
  return s;
}

pie_status pie_apply_near(pie_problem* h, const void* x, void* y, int nrhs, int dtype, void* stream) {
  return apply_api(h, x, y, nrhs, dtype, stream, true);
}

pie_status pie_apply_t(pie_problem* h, const void* x, void* y, int nrhs, int dtype, int conj, void* stream) {
  if (!h || (!x && nrhs > 0) || (!y && nrhs > 0) || nrhs < 0 || (conj != 0 && conj != 1)) {
    set_error("pie_apply_t: invalid argument");
    return PIE_ERR_PARAM;
  }
  Problem& pr = h->p;
  if (dtype != (pr.io_f32() ? PIE_C64 : PIE_C128)) {
    set_error("pie_apply_t: dtype does not match the problem precision");
    return PIE_ERR_PARAM;
  }
  if (pie_status sd = check_device(pr, "pie_apply_t")) return sd;
  size_t es = pr.io_f32() ? sizeof(cf) : sizeof(cd);
  for (int j = 0; j < nrhs; ++j) {
    pie_status s = apply_t_one(pr, static_cast<const char*>(x) + es * size_t(pr.N) * j,
                               static_cast<char*>(y) + es * size_t(pr.N) * j, conj == 1,
                               static_cast<cudaStream_t>(stream));
    if (s != PIE_OK) return s;
  }
  return PIE_OK;
}

pie_status pie_farfield_adjoint(pie_problem* h, const double* rhat, int64_t ndir, const void* E, void* u,
                                void* stream) {
  if (!h || !rhat || !E || !u || ndir < 1) {
    set_error("pie_farfield_adjoint: invalid argument");
    return PIE_ERR_PARAM;
  }
  return farfield_adjoint(h->p, rhat, ndir, E, u, static_cast<cudaStream_t>(stream));
}

pie_status pie_profile_begin(pie_problem* h, int max_applies) {
  if (!h || max_applies < 1) {
    set_error("pie_profile_begin: invalid argument");
    return PIE_ERR_PARAM;
  }
  Problem& pr = h->p;
  free_profile(pr);
  pr.prof_ev.resize(size_t(max_applies) * kStages * 2);
  for (auto& e : pr.prof_ev) {
    pie_status s = cuda_check(cudaEventCreate(&e), "event create");
    if (s != PIE_OK) {
      e = nullptr;
      free_profile(pr);
      return s;
    }
  }
  pr.prof_cap = max_applies;
  pr.prof_n = 0;
  return PIE_OK;
}

pie_status pie_profile_end(pie_problem* h, double* stage_ms, int32_t* applies) {
  if (!h) {
    set_error("NULL problem");
    return PIE_ERR_PARAM;
  }
  Problem& pr = h->p;
  double acc[kStages] = {0};
  pie_status s = PIE_OK;
  for (int a = 0; a < pr.prof_n && s == PIE_OK; ++a)
    for (int k = 0; k < kStages && s == PIE_OK; ++k) {
      cudaEvent_t e0 = pr.prof_ev[(size_t(a) * kStages + k) * 2], e1 = pr.prof_ev[(size_t(a) * kStages + k) * 2 + 1];
      s = cuda_check(cudaEventSynchronize(e1), "profile sync");
      float ms = 0;
      if (s == PIE_OK) s = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "profile elapsed");
      acc[k] += ms;
    }
  if (stage_ms)
    for (int k = 0; k < kStages; ++k) stage_ms[k] = acc[k];
  if (applies) *applies = pr.prof_n;
  free_profile(pr);
  return s;
}

pie_status pie_problem_stage(pie_problem* h, int which, int level, double* out, void* stream) {
  if (!h || !out) {
    set_error("NULL argument");
    return PIE_ERR_PARAM;
  }
  Problem& pr = h->p;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pie_status s = cuda_check(cudaStreamSynchronize(st), "stage sync");
  if (s != PIE_OK) return s;
  const void* src = nullptr;
  size_t n = 0;
  bool f32 = false;
  if (which == 0 || which == 1) {
    if (level < 3 || level > pr.tree.L) {
      set_error("level out of range");
      return PIE_ERR_PARAM;
    }
    src = which == 0 ? pr.lev[level].S : pr.lev[level].G;
    n = size_t(pr.lev[level].nb) * kComp * pr.P;
    f32 = pr.far_f32();
  } else if (which == 2 || which == 3) {
    src = which == 2 ? pr.coef : pr.pot;
    n = size_t(pr.T) * 6;
    f32 = pr.io_f32();
  } else if (which == 4) {
    src = pr.mom;
    n = size_t(pr.nnz) * kMom;
    f32 = pr.near_f32();
    if (pr.near_h16()) {  // half pairs times the plane scales
      std::vector<__half2> tmp(n);
      s = cuda_check(cudaMemcpy(tmp.data(), src, n * sizeof(__half2), cudaMemcpyDeviceToHost), "stage copy");
      if (s != PIE_OK) return s;
      // stored pair by pair ([nnz][8]); exported plane by plane like the others
      const size_t nnz = size_t(pr.nnz);
      for (size_t i = 0; i < n; ++i) {
        const size_t q = i / nnz, e = i % nnz;
        const __half2 h = tmp[e * kMom + q];
        out[2 * i] = double(__low2float(h)) * pr.mom_scale[q];
        out[2 * i + 1] = double(__high2float(h)) * pr.mom_scale[q];
      }
      return PIE_OK;
    }
  } else if (which == 5 || which == 6) {
    src = which == 5 ? pr.Pi : pr.M;
    n = size_t(pr.T) * (pr.P / 2) * (which == 5 ? 1 : 3);
    f32 = pr.far_f32();
  } else {
    set_error("unknown stage");
    return PIE_ERR_PARAM;
  }
  std::vector<double> buf(2 * n);
  if (!f32) {
    s = cuda_check(cudaMemcpy(buf.data(), src, n * sizeof(cd), cudaMemcpyDeviceToHost), "stage copy");
  } else {
    std::vector<float> tmp(2 * n);
    s = cuda_check(cudaMemcpy(tmp.data(), src, n * sizeof(cf), cudaMemcpyDeviceToHost), "stage copy");
    for (size_t i = 0; i < 2 * n; ++i) buf[i] = tmp[i];
  }
  if (s != PIE_OK) return s;
  std::memcpy(out, buf.data(), sizeof(double) * 2 * n);
  return s;
}

pie_status pie_rhs_planewave(pie_problem* h, const double khat[3], const double pol[3], double E0, void* b,
                             int dtype, void* stream) {
  if (!h || !khat || !pol || !b) {
    set_error("NULL argument");
    return PIE_ERR_PARAM;
  }
  int want = h->p.io_f32() ? PIE_C64 : PIE_C128;
  if (dtype != want) {
    set_error("pie_rhs_planewave: dtype does not match the problem precision");
    return PIE_ERR_PARAM;
  }
  return rhs_planewave(h->p, khat, pol, E0, b, static_cast<cudaStream_t>(stream));
}

pie_status pie_farfield(pie_problem* h, const void* x, const double* rhat, int64_t ndir, void* E, int nrhs,
                        void* stream) {
  if (!h || !x || !rhat || !E || ndir < 0 || nrhs < 1) {
    set_error("pie_farfield: invalid argument");
    return PIE_ERR_PARAM;
  }
  if (ndir == 0) return PIE_OK;
  Problem& pr = h->p;
  const size_t col = (pr.io_f32() ? sizeof(cf) : sizeof(cd)) * size_t(pr.N);
  for (int j = 0; j < nrhs; ++j) {
    pie_status s = farfield(pr, static_cast<const char*>(x) + col * j, rhat, ndir,
                            static_cast<cd*>(E) + size_t(ndir) * 3 * j, static_cast<cudaStream_t>(stream));
    if (s != PIE_OK) return s;
  }
  return PIE_OK;
}

static pie_status solve_cols(pie_problem* h, const void* b, void* x, int nrhs, double tol, int maxit, int restart,
                             pie_solve_stats* stats, void* stream, bool guess) {
  if (!h || !b || !x || nrhs < 1 || !(tol > 0) || maxit < 1 || restart < 1) {
    set_error("pie_solve: invalid argument");
    return PIE_ERR_PARAM;
  }
  // one GMRES per column; a column that does not converge does not stop the
  // others, a failure of the device or the arithmetic does
  Problem& pr = h->p;
  if (pie_status sd = check_device(pr, "pie_solve")) return sd;
  const size_t col = sizeof(cd) * size_t(pr.N);
  pie_status worst = PIE_OK;
  std::string msg;
  for (int j = 0; j < nrhs; ++j) {
    pie_status s = solve(pr, static_cast<const char*>(b) + col * j, static_cast<char*>(x) + col * j, tol, maxit,
                         restart, stats ? stats + j : nullptr, static_cast<cudaStream_t>(stream), guess);
    if (s == PIE_ERR_NOCONV || s == PIE_ERR_BREAKDOWN) {
      if (worst == PIE_OK) {
        worst = s;
        msg = g_err;
      }
      continue;
    }
    if (s != PIE_OK) return s;
  }
  if (worst != PIE_OK) set_error(msg);
  return worst;
}

pie_status pie_solve(pie_problem* h, const void* b, void* x, int nrhs, double tol, int maxit, int restart,
                     pie_solve_stats* stats, void* stream) {
  return solve_cols(h, b, x, nrhs, tol, maxit, restart, stats, stream, false);
}

pie_status pie_solve_guess(pie_problem* h, const void* b, void* x, int nrhs, double tol, int maxit, int restart,
                           pie_solve_stats* stats, void* stream) {
  return solve_cols(h, b, x, nrhs, tol, maxit, restart, stats, stream, true);
}

pie_status pie_solve_nested(pie_problem* ho, pie_problem* hi, const void* b, void* x, int nrhs,
                            const pie_nested_params* np, pie_nested_stats* stats, void* stream) {
  if (!ho || !hi || !b || !x || !np || nrhs < 1 || !(np->tol > 0) || np->maxit < 1 || np->inner_restart < 1 ||
      np->inner_restart > 1000 || !(np->inner_tol > 0) || !(np->inner_tol < 1) || np->outer_restart < 0 ||
      np->outer_restart > 200 || np->max_outer < 1) {
    set_error("pie_solve_nested: invalid argument");
    return PIE_ERR_PARAM;
  }
  Problem& po = ho->p;
  Problem& pi = hi->p;
  if (po.io_f32()) {
    set_error("pie_solve_nested: the outer problem must be PIE_FP64 or PIE_MIXED (complex double vectors)");
    return PIE_ERR_PARAM;
  }
  if (pi.N != po.N || pi.T != po.T || pi.E != po.E || pi.k0 != po.k0 || pi.mesh.tri != po.mesh.tri ||
      pi.mesh.xyz != po.mesh.xyz) {
    set_error("pie_solve_nested: inner and outer problems differ in mesh or k0");
    return PIE_ERR_PARAM;
  }
  if (pi.device != po.device) {
    set_error("pie_solve_nested: inner and outer problems are on different devices");
    return PIE_ERR_PARAM;
  }
  if (pie_status sd = check_device(po, "pie_solve_nested")) return sd;
  const size_t col = sizeof(cd) * size_t(po.N);
  pie_status worst = PIE_OK;
  std::string msg;
  for (int j = 0; j < nrhs; ++j) {
    pie_status s = solve_nested(po, pi, static_cast<const char*>(b) + col * j, static_cast<char*>(x) + col * j, *np,
                                stats ? stats + j : nullptr, static_cast<cudaStream_t>(stream));
    if (s == PIE_ERR_NOCONV) {
      if (worst == PIE_OK) {
        worst = s;
        msg = g_err;
      }
      continue;
    }
    if (s != PIE_OK) return s;
  }
  if (worst != PIE_OK) set_error(msg);
  return worst;
}

pie_status pie_problem_quadrature(const pie_problem* h, double* pts, double* wts) {
  if (!h) {
    set_error("pie_problem_quadrature: NULL problem");
    return PIE_ERR_PARAM;
  }
  const Problem& pr = h->p;
  const Mesh& m = pr.mesh;
  const std::vector<double>& r = pr.rule7_host;
  for (int64_t t = 0; t < m.nt; ++t) {
    const double* v0 = &m.xyz[3 * size_t(m.tri[3 * t])];
    const double* v1 = &m.xyz[3 * size_t(m.tri[3 * t + 1])];
    const double* v2 = &m.xyz[3 * size_t(m.tri[3 * t + 2])];
    for (int q = 0; q < 7; ++q) {
      if (pts)
        for (int d = 0; d < 3; ++d)
          pts[(t * 7 + q) * 3 + d] = r[4 * q] * v0[d] + r[4 * q + 1] * v1[d] + r[4 * q + 2] * v2[d];
      if (wts) wts[t * 7 + q] = r[4 * q + 3] * m.area[t];
    }
  }
  return PIE_OK;
}

pie_status pie_rhs_potentials(pie_problem* h, const void* A_q, const void* Phi_q, void* b, int dtype, void* stream) {
  if (!h || !A_q || !Phi_q || !b) {
    set_error("pie_rhs_potentials: NULL argument");
    return PIE_ERR_PARAM;
  }
  if (dtype != (h->p.io_f32() ? PIE_C64 : PIE_C128)) {
    set_error("pie_rhs_potentials: dtype does not match the problem precision");
    return PIE_ERR_PARAM;
  }
  return rhs_potentials(h->p, A_q, Phi_q, b, static_cast<cudaStream_t>(stream));
}

static bool c128_problem(pie_problem* h, const char* who) {
  if (h->p.io_f32()) {
    set_error(std::string(who) + ": needs a PIE_FP64 or PIE_MIXED problem (complex double vectors)");
    return false;
  }
  return true;
}

pie_status pie_apply_single_layer(pie_problem* h, const void* q, void* y, void* stream) {
  if (!h || !q || !y) {
    set_error("pie_apply_single_layer: NULL argument");
    return PIE_ERR_PARAM;
  }
  if (!c128_problem(h, "pie_apply_single_layer")) return PIE_ERR_PARAM;
  return single_layer_one(h->p, q, y, static_cast<cudaStream_t>(stream));
}

pie_status pie_solve_single_layer(pie_problem* h, const void* b, void* x, double tol, int maxit, int restart,
                                  pie_solve_stats* stats, void* stream) {
  if (!h || !b || !x || !(tol > 0) || maxit < 1 || restart < 1) {
    set_error("pie_solve_single_layer: invalid argument");
    return PIE_ERR_PARAM;
  }
  return solve_single_layer(h->p, b, x, tol, maxit, restart, stats, static_cast<cudaStream_t>(stream));
}

pie_status pie_rhs_potential(pie_problem* h, const double khat[3], const double pol[3], double E0, void* b,
                             void* stream) {
  if (!h || !khat || !pol || !b) {
    set_error("pie_rhs_potential: NULL argument");
    return PIE_ERR_PARAM;
  }
  return rhs_potential(h->p, khat, pol, E0, b, static_cast<cudaStream_t>(stream));
}

pie_status pie_nearfield(pie_problem* h, const void* x, const void* rho, const double* pts, int64_t npts, void* E,
                         void* stream) {
  if (!h || !x || !rho || !pts || !E || npts < 0) {
    set_error("pie_nearfield: invalid argument");
    return PIE_ERR_PARAM;
  }
  if (!c128_problem(h, "pie_nearfield")) return PIE_ERR_PARAM;
  if (npts == 0) return PIE_OK;
  return nearzone(h->p, x, rho, pts, npts, E, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
