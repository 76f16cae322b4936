// Launch tuning of the product, its autotuner (launch settings and level
// count per mesh) and multi-mesh groups applied in one CUDA-graph launch.
// None of this changes the arithmetic of the product: every setting gives
// the same result to the last bit.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "handles.h"

using namespace pie;

namespace {

bool tuning_valid(const Problem& pr, const pie_tuning& t) {
  return (t.overlap == 0 || t.overlap == 1) && t.near_ctas_per_sm >= 0 && t.near_ctas_per_sm <= 32 &&
         t.rhs_chunk >= 1 && t.rhs_chunk <= pr.par.max_nrhs &&
         (t.near_rhs_block == 0 || t.near_rhs_block == 1 || t.near_rhs_block == 2 || t.near_rhs_block == 4 ||
          t.near_rhs_block == 8) &&
         (t.far_rows == 0 || t.far_rows == 1 || t.far_rows == 2 || t.far_rows == 4 || t.far_rows == 8 ||
          t.far_rows == 16 || t.far_rows == 32) &&
         t.near_kernel >= 0 && t.near_kernel <= 2;
}

bool profiling(const Problem& pr) { return pr.prof_n < pr.prof_cap; }

// Median milliseconds per right-hand side of products of nrhs columns under
// the problem's current tuning (one untimed product first).
pie_status time_products(Problem& pr, const void* x, void* y, int nrhs, int reps, cudaStream_t st, cudaEvent_t e0,
                         cudaEvent_t e1, double* ms) {
  pie_status s = apply_cols(pr, x, y, nrhs, st);
  if (s != PIE_OK) return s;
  std::vector<float> t(reps);
  for (int r = 0; r < reps; ++r) {
    if ((s = cuda_check(cudaEventRecord(e0, st), "event")) != PIE_OK) return s;
    if ((s = apply_cols(pr, x, y, nrhs, st)) != PIE_OK) return s;
    if ((s = cuda_check(cudaEventRecord(e1, st), "event")) != PIE_OK) return s;
    if ((s = cuda_check(cudaEventSynchronize(e1), "autotune product")) != PIE_OK) return s;
    if ((s = cuda_check(cudaEventElapsedTime(&t[r], e0, e1), "event")) != PIE_OK) return s;
  }
  std::sort(t.begin(), t.end());
  *ms = double(t[reps / 2]) / nrhs;
  return PIE_OK;
}

struct Scratch {
  void* x = nullptr;
  void* y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Scratch() {
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

pie_status autotune(Problem& pr, int nrhs, int reps, cudaStream_t st, pie_tuning* best, double* best_ms) {
  Scratch sc;
  const size_t bytes = (pr.io_f32() ? sizeof(cf) : sizeof(cd)) * size_t(pr.N) * nrhs;
  if (cudaMalloc(&sc.x, bytes) != cudaSuccess || cudaMalloc(&sc.y, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("pie_problem_autotune: out of device memory for the scratch vectors");
    return PIE_ERR_OOM;
  }
  pie_status s = cuda_check(cudaEventCreate(&sc.e0), "event");
  if (s == PIE_OK) s = cuda_check(cudaEventCreate(&sc.e1), "event");
  // finite nonzero input (bytes 0x3f: 2.4e-4 as double, 0.75 as float)
  if (s == PIE_OK) s = cuda_check(cudaMemsetAsync(sc.x, 0x3f, bytes, st), "memset");
  if (s != PIE_OK) return s;
  const pie_tuning saved = pr.tune;
  const int cmax = std::min(nrhs, pr.par.max_nrhs);
  pie_tuning win{0, 0, cmax, 0, 0, 0};
  double win_ms = 1e300;
  auto trial = [&](pie_tuning t) -> pie_status {
    pr.tune = t;
    double ms = 0;
    pie_status r = time_products(pr, sc.x, sc.y, nrhs, reps, st, sc.e0, sc.e1, &ms);
    if (r == PIE_OK && ms < win_ms) {
      win_ms = ms;
      win = t;
    }
    return r;
  };
  // overlap and the near kernel's grid, at the widest chunk
  s = trial(pie_tuning{0, 0, cmax, 0, 0, 0});
  const int ctas[] = {1, 2, 3, 4, 6, 8, 0};
  for (int c : ctas)
    if (s == PIE_OK) s = trial(pie_tuning{1, c, cmax, 0, 0, 0});
  // then the chunk of right-hand sides per pass
  const pie_tuning lead = win;
  for (int c = 1; c < cmax && s == PIE_OK; c *= 2)
    s = trial(pie_tuning{lead.overlap, lead.near_ctas_per_sm, c, 0, 0, 0});
  // then the right-hand sides per near-kernel thread (the automatic choice
  // is the one already timed)
  const pie_tuning lead2 = win;
  for (int rb = 1; rb <= 8 && rb <= lead2.rhs_chunk && lead2.rhs_chunk > 1 && s == PIE_OK; rb *= 2)
    s = trial(pie_tuning{lead2.overlap, lead2.near_ctas_per_sm, lead2.rhs_chunk, rb, 0, 0});
  // then the tile of the per-box far kernels (N_theta = 8 uses the
  // factorised filter kernels, whose tile is fixed)
  if (pr.par.ntheta != 8)
    for (int rows = 1; rows <= 16 && s == PIE_OK; rows *= 2) {
      pie_tuning t = win;
      t.far_rows = rows;
      s = trial(t);
    }
  // then the near kernel, where both apply
  if (pr.near_f32() && s == PIE_OK) {
    const pie_tuning lead3 = win;
    for (int nk = 1; nk <= 2 && s == PIE_OK; ++nk) {
      pie_tuning t = lead3;
      t.near_kernel = nk;
      if (nk == 2 && t.near_rhs_block == 8) continue;  // the box kernel carries at most 4
      s = trial(t);
    }
  }
  if (s != PIE_OK) {
    pr.tune = saved;
    return s;
  }
  pr.tune = win;
  *best = win;
  if (best_ms) *best_ms = win_ms;
  return PIE_OK;
}

}  // namespace

// A group's captured graph for one set of buffers and member tunings.
struct GroupGraph {
  std::vector<const void*> x;
  std::vector<void*> y;
  std::vector<pie_tuning> tune;
  int nrhs = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t used = 0;
};

struct pie_group {
  std::vector<Problem*> mem;
  std::vector<cudaStream_t> branch;  // one capture branch per member
  std::vector<cudaEvent_t> done;
  cudaStream_t cap = nullptr;        // the stream the capture starts on
  cudaEvent_t start = nullptr;
  std::vector<GroupGraph> graphs;    // at most kKeep, least recently used replaced
  uint64_t tick = 0;
  int64_t captured = 0, launches = 0;
  static constexpr size_t kKeep = 4;
  ~pie_group() {
    for (GroupGraph& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaStream_t s : branch)
      if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : done)
      if (e) cudaEventDestroy(e);
    if (cap) cudaStreamDestroy(cap);
    if (start) cudaEventDestroy(start);
  }
};

namespace {

// Records the products of all members, each on its own branch forked from
// and joined back into the capture stream, as one graph.
pie_status capture(pie_group& g, const void* const* x, void* const* y, int nrhs, cudaGraphExec_t* exec) {
  pie_status s = cuda_check(cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (s != PIE_OK) return s;
  s = cuda_check(cudaEventRecord(g.start, g.cap), "capture fork");
  for (size_t i = 0; i < g.mem.size() && s == PIE_OK; ++i) {
    s = cuda_check(cudaStreamWaitEvent(g.branch[i], g.start, 0), "capture fork");
    if (s == PIE_OK) s = apply_cols(*g.mem[i], x[i], y[i], nrhs, g.branch[i]);
    if (s == PIE_OK) s = cuda_check(cudaEventRecord(g.done[i], g.branch[i]), "capture join");
    if (s == PIE_OK) s = cuda_check(cudaStreamWaitEvent(g.cap, g.done[i], 0), "capture join");
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g.cap, &graph);
  if (s == PIE_OK) s = cuda_check(e, "end capture");
  if (s == PIE_OK) s = cuda_check(cudaGraphInstantiate(exec, graph, 0), "graph instantiate");
  if (graph) cudaGraphDestroy(graph);
  if (s != PIE_OK) cudaGetLastError();
  return s;
}

}  // namespace

extern "C" {

pie_status pie_problem_get_tuning(const pie_problem* h, pie_tuning* t) {
  if (!h || !t) {
    set_error("pie_problem_get_tuning: NULL argument");
    return PIE_ERR_PARAM;
  }
  *t = h->p.tune;
  return PIE_OK;
}

pie_status pie_problem_set_tuning(pie_problem* h, const pie_tuning* t) {
  if (!h || !t || !tuning_valid(h->p, *t)) {
    set_error("pie_problem_set_tuning: NULL argument or field out of range");
    return PIE_ERR_PARAM;
  }
  h->p.tune = *t;
  return PIE_OK;
}

pie_status pie_problem_autotune(pie_problem* h, int nrhs, int reps, pie_tuning* best, double* best_ms,
                                void* stream) {
  if (!h || !best || nrhs < 1 || nrhs > 1024 || reps < 1 || reps > 100) {
    set_error("pie_problem_autotune: invalid argument");
    return PIE_ERR_PARAM;
  }
  if (profiling(h->p)) {
    set_error("pie_problem_autotune: per-stage profiling is active");
    return PIE_ERR_PARAM;
  }
  return autotune(h->p, nrhs, reps, static_cast<cudaStream_t>(stream), best, best_ms);
}

pie_status pie_tune_levels(const pie_mesh* m, double k0, const pie_params* base, int lmin, int lmax, int nrhs,
                           void* stream, int* best_levels, double* ms_per_level) {
  if (!m || !base || !best_levels || lmin < 3 || lmax > 21 || lmin > lmax || nrhs < 1 || nrhs > 1024) {
    set_error("pie_tune_levels: invalid argument");
    return PIE_ERR_PARAM;
  }
  int best = -1;
  double best_ms = 1e300;
  for (int L = lmin; L <= lmax; ++L) {
    if (ms_per_level) ms_per_level[L - lmin] = 0;
    pie_params p = *base;
    p.levels = L;
    pie_problem* h = nullptr;
    pie_status s = pie_problem_create(m, k0, &p, stream, &h);
    if (s == PIE_ERR_LEAF) continue;  // leaf box too small for the mesh
    if (s != PIE_OK) return s;
    pie_tuning t{};
    double ms = 0;
    s = pie_problem_autotune(h, nrhs, 3, &t, &ms, stream);
    pie_problem_destroy(h);
    if (s != PIE_OK) return s;
    if (ms_per_level) ms_per_level[L - lmin] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = L;
    }
  }
  if (best < 0) {
    set_error("pie_tune_levels: no level count in range admits the mesh");
    return PIE_ERR_LEAF;
  }
  *best_levels = best;
  return PIE_OK;
}

pie_status pie_group_create(pie_problem* const* members, int n, pie_group** out) {
  if (!members || n < 1 || n > 1024 || !out) {
    set_error("pie_group_create: invalid argument");
    return PIE_ERR_PARAM;
  }
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!members[i]) {
      set_error("pie_group_create: NULL member");
      return PIE_ERR_PARAM;
    }
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) {
        set_error("pie_group_create: a problem appears twice");
        return PIE_ERR_PARAM;
      }
  }
  pie_group* g = new (std::nothrow) pie_group;
  if (!g) return PIE_ERR_OOM;
  pie_status s = PIE_OK;
  for (int i = 0; i < n && s == PIE_OK; ++i) {
    g->mem.push_back(&members[i]->p);
    g->branch.push_back(nullptr);
    g->done.push_back(nullptr);
    s = cuda_check(cudaStreamCreateWithFlags(&g->branch.back(), cudaStreamNonBlocking), "group stream");
    if (s == PIE_OK) s = cuda_check(cudaEventCreateWithFlags(&g->done.back(), cudaEventDisableTiming), "event");
    if (s == PIE_OK) s = prepare_apply(members[i]->p);
  }
  if (s == PIE_OK) s = cuda_check(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking), "group stream");
  if (s == PIE_OK) s = cuda_check(cudaEventCreateWithFlags(&g->start, cudaEventDisableTiming), "event");
  if (s != PIE_OK) {
    delete g;
    return s;
  }
  *out = g;
  return PIE_OK;
}

pie_status pie_group_apply(pie_group* g, const void* const* x, void* const* y, int nrhs, void* stream) {
  if (!g || !x || !y || nrhs < 1 || nrhs > 1 << 20) {
    set_error("pie_group_apply: invalid argument");
    return PIE_ERR_PARAM;
  }
  const size_t n = g->mem.size();
  for (size_t i = 0; i < n; ++i) {
    if (!x[i] || !y[i]) {
      set_error("pie_group_apply: NULL buffer");
      return PIE_ERR_PARAM;
    }
    if (profiling(*g->mem[i])) {
      set_error("pie_group_apply: per-stage profiling is active on a member");
      return PIE_ERR_PARAM;
    }
  }
  GroupGraph* hit = nullptr;
  for (GroupGraph& gg : g->graphs) {
    if (gg.nrhs != nrhs) continue;
    bool same = true;
    for (size_t i = 0; i < n && same; ++i)
      same = gg.x[i] == x[i] && gg.y[i] == y[i] && std::memcmp(&gg.tune[i], &g->mem[i]->tune, sizeof(pie_tuning)) == 0;
    if (same) {
      hit = &gg;
      break;
    }
  }
  if (!hit) {
    GroupGraph gg;
    gg.x.assign(x, x + n);
    gg.y.assign(y, y + n);
    for (Problem* p : g->mem) gg.tune.push_back(p->tune);
    gg.nrhs = nrhs;
    pie_status s = capture(*g, x, y, nrhs, &gg.exec);
    if (s != PIE_OK) return s;
    ++g->captured;
    if (g->graphs.size() >= pie_group::kKeep) {
      auto lru = std::min_element(g->graphs.begin(), g->graphs.end(),
                                  [](const GroupGraph& a, const GroupGraph& b) { return a.used < b.used; });
      cudaGraphExecDestroy(lru->exec);
      *lru = gg;
      hit = &*lru;
    } else {
      g->graphs.push_back(gg);
      hit = &g->graphs.back();
    }
  }
  hit->used = ++g->tick;
  pie_status s = cuda_check(cudaGraphLaunch(hit->exec, static_cast<cudaStream_t>(stream)), "graph launch");
  if (s == PIE_OK) ++g->launches;
  return s;
}

pie_status pie_group_info(const pie_group* g, int64_t* graphs, int64_t* launches) {
  if (!g) {
    set_error("pie_group_info: NULL group");
    return PIE_ERR_PARAM;
  }
  if (graphs) *graphs = g->captured;
  if (launches) *launches = g->launches;
  return PIE_OK;
}

void pie_group_destroy(pie_group* g) { delete g; }

}  // extern "C"
