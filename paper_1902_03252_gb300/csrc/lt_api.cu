// C ABI of the library (include/lt.h): model lifetime, workspaces, the batch
// plan (samples grouped into chunks whose node workspace fits a budget, each
// chunk a flat list of equal-size work items for the persistent kernels), and
// the stream-ordered sequence of kernels behind every entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lt_internal.cuh"

using namespace lt;

namespace {

constexpr int64_t kDefaultCap = 4096;
constexpr int kDefl64Nodes = 128;    // nodes per FP64 deflection item
constexpr int kSearch64Cells = 128;  // cells per FP64 search item

struct Chunk {
  int b0, b1;            // samples [b0, b1)
  int64_t defl_items;    // work items of the deflection kernel
  int64_t search_items;  // work items of the search kernel
  size_t defl_off;       // offset (elements) of this chunk's item table in d_plan_items
  size_t search_off;
};

struct Plan {
  std::vector<lt_grid> grids;
  int precision = -1, shape = -1;
  std::vector<Chunk> chunks;
  size_t max_chunk_nodes = 0;
};

}  // namespace

struct lt_model {
  int n_pot = 0, batch = 0;
  int64_t hit_cap = kDefaultCap, work_cap = kDefaultCap;
  int device = 0, sm_count = 1;
  int shape = 0;  // FP32 deflection launch shape (autotuned)
  size_t ws_budget = (size_t)4 << 30;
  double* d_params = nullptr;
  Pot64* d_pot64 = nullptr;
  Pot32* d_pot32 = nullptr;
  Seg32* d_seg = nullptr;
  uint32_t* d_status = nullptr;
  long long* d_counters = nullptr;
  // node workspace (float4 per node in mixed precision, double2 in FP64)
  void* d_nodes = nullptr;
  size_t nodes_bytes = 0;
  // hits and FP64 work lists, [batch][cap]
  Hit* d_hits = nullptr;
  Work64* d_work = nullptr;
  unsigned long long* d_hit_count = nullptr;
  unsigned long long* d_work_count = nullptr;
  int64_t hits_cap_alloc = 0, work_cap_alloc = 0;
  // plan on the device: SampleGrid [batch] and per-chunk item tables
  SampleGrid* d_plan_grids = nullptr;
  int64_t* d_plan_items = nullptr;
  size_t plan_items_alloc = 0;
  float* d_plan_coords = nullptr;  // FP32 node coordinates of every grid (SampleGrid::coord_off)
  size_t plan_coords_alloc = 0;
  // the coordinate table of the last single-grid deflection (lt_deflect_grid),
  // uploaded again only when the grid changes
  lt_grid dg_grid{};
  float* d_dg_coords = nullptr;
  size_t dg_coords_alloc = 0;
  // dynamic item counters: [0] single-grid calls, then (deflect, search) per chunk
  unsigned long long* d_sched = nullptr;
  size_t sched_alloc = 0;
  // side stream for the barycentres, overlapping the FP32 deflection
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  Plan plan;
  // chi^2 intermediates
  double* d_beta_obs = nullptr;
  double* d_bary = nullptr;
  int64_t* d_match_tri = nullptr;
  int32_t* d_match_hit = nullptr;
  double* d_match_xy = nullptr;
  double* d_chi2_terms = nullptr;  // chi^2 term of each observed image [batch][n_obs]
  // FP64 resolution scratch (node table, vertex slots, distinct-node list)
  ResolveScratch rs{nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                    nullptr, nullptr, nullptr, nullptr};
  size_t rs_vslot_alloc = 0;
  double2* d_adj_lam = nullptr;   // adjoint: lambda per matched observed image
  AdjPt* d_adj_pts = nullptr;   // adjoint points (x, y, coefficient) [batch][4 n_obs]
  int obs_alloc = 0, sys_alloc = 0;
  int last_nobs = -1, last_nsys = -1;
  // source-plane chi^2 scratch: beta and mu [batch][n_obs], barycentres [batch][n_sys]
  double2* d_src_beta = nullptr;
  double* d_src_mu = nullptr;
  double2* d_src_bary = nullptr;
  int src_obs_alloc = 0, src_sys_alloc = 0;
  // CUDA graph cache of lt_chi2_graph
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::vector<lt_grid> graph_grids;
  lt_obs graph_obs{};
  int graph_prec = -1;
  double* graph_out = nullptr;
  uint64_t graph_epoch = 0;
  uint64_t ws_epoch = 1;  // bumped whenever a workspace captured by a graph moves
  // optional per-kernel event timing
  unsigned prof_mask = 0;  // stages bracketed by events (bit k = stage k)
  struct ProfRec {
    int kind;
    cudaEvent_t e0, e1;
    double node_pot;
    int fp64;
    int kernels;  // kernel launches inside the timed scope
  };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  lt_profile prof_acc{};
  std::string err;
};

namespace {

#define LT_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      m->err = std::string(#call) + ": " + cudaGetErrorString(e_);                       \
      return e_ == cudaErrorMemoryAllocation ? LT_ERR_NOMEM : LT_ERR_CUDA;               \
    }                                                                                    \
  } while (0)

#define LT_CHECK_ARG(cond, msg)   \
  do {                            \
    if (!(cond)) {                \
      m->err = (msg);             \
      return LT_ERR_INVALID_ARG;  \
    }                             \
  } while (0)

inline cudaStream_t S(uintptr_t s) { return reinterpret_cast<cudaStream_t>(s); }

// Event bracket around one launch when profiling is enabled (never inside a
// stream capture).
struct ProfScope {
  lt_model* m;
  cudaStream_t st;
  int kind;
  double node_pot;
  int fp64;
  int kernels;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProfScope(lt_model* m_, cudaStream_t st_, int kind_, double np = 0.0, int fp64_ = 0,
            int kernels_ = 1)
      : m(m_), st(st_), kind(kind_), node_pot(np), fp64(fp64_), kernels(kernels_) {
    if (!(m->prof_mask & (1u << kind))) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    e0 = take();
    e1 = take();
    if (e0 && e1) cudaEventRecord(e0, st);
  }
  cudaEvent_t take() {
    cudaEvent_t e = nullptr;
    if (!m->prof_pool.empty()) {
      e = m->prof_pool.back();
      m->prof_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
    }
    return e;
  }
  ~ProfScope() {
    if (!e0 || !e1) return;
    cudaEventRecord(e1, st);
    m->prof_pending.push_back({kind, e0, e1, node_pot, fp64, kernels});
  }
};

template <class T>
lt_status grow(lt_model* m, T** p, size_t* have, size_t need_elems) {
  if (*have >= need_elems && *p) return LT_OK;
  ++m->ws_epoch;
  if (*p) LT_CUDA(cudaFree(*p));
  *p = nullptr;
  *have = 0;
  LT_CUDA(cudaMalloc((void**)p, std::max<size_t>(need_elems, 1) * sizeof(T)));
  *have = need_elems;
  return LT_OK;
}

bool grid_ok(const lt_grid& g) {
  return g.nx >= 1 && g.ny >= 1 && std::isfinite(g.x0) && std::isfinite(g.y0) &&
         std::isfinite(g.dx) && std::isfinite(g.dy) && g.dx > 0 && g.dy > 0 &&
         (int64_t)g.nx * g.ny < ((int64_t)1 << 40);
}

bool same_grids(const std::vector<lt_grid>& a, const lt_grid* b, int n) {
  if ((int)a.size() != n) return false;
  return std::memcmp(a.data(), b, sizeof(lt_grid) * n) == 0;
}

// Device description of one sample's grid whose nodes start at node_off.
SampleGrid sample_grid(const lt_grid& g, int64_t node_off, int64_t coord_off) {
  SampleGrid s;
  s.x0 = g.x0; s.y0 = g.y0; s.dx = g.dx; s.dy = g.dy; s.nx = g.nx; s.ny = g.ny;
  s.node_off = node_off;
  const double tm = std::max(std::max(std::fabs(g.x0), std::fabs(g.x0 + (g.nx - 1) * g.dx)),
                             std::max(std::fabs(g.y0), std::fabs(g.y0 + (g.ny - 1) * g.dy)));
  s.theta_max = (float)(tm * (1.0 + 1e-6));
  s.pad = 0.f;
  s.x0f = (float)g.x0; s.y0f = (float)g.y0; s.dxf = (float)g.dx; s.dyf = (float)g.dy;
  s.coord_off = coord_off;
  return s;
}

// Append a grid's FP32 node coordinates, nx values x0 + i dx then ny values
// y0 + j dy: each evaluated in FP64 as written (this file is compiled without
// floating-point contraction, so the product and the sum round separately, as
// in an FP64 reference that states the grid the same way) and rounded once
// to FP32.
void grid_coords(const lt_grid& g, std::vector<float>& out) {
  for (int i = 0; i < g.nx; ++i) out.push_back((float)(g.x0 + (double)i * g.dx));
  for (int j = 0; j < g.ny; ++j) out.push_back((float)(g.y0 + (double)j * g.dy));
}

// Deflection work items of one grid: node ranges of kDefl64Nodes in FP64,
// column bands of the launch shape in FP32 (defl32_items).
int64_t defl_items(const lt_grid& g, int precision, int shape) {
  if (precision == LT_PREC_FP64) return ((int64_t)g.nx * g.ny + kDefl64Nodes - 1) / kDefl64Nodes;
  const DeflectShape sh = deflect_shape(shape);
  return defl32_items(g.nx, g.ny, sh.threads, sh.npt);
}

// Group samples into chunks whose node workspace fits the budget, build each
// chunk's item tables and upload the SampleGrid array and the tables.
lt_status make_plan(lt_model* m, const lt_grid* grids, int n, int precision, cudaStream_t st) {
  const int shape = m->shape;
  if (same_grids(m->plan.grids, grids, n) && m->plan.precision == precision &&
      m->plan.shape == shape)
    return LT_OK;
  for (int b = 0; b < n; ++b)
    LT_CHECK_ARG(grid_ok(grids[b]), "invalid grid (need nx, ny >= 1, dx, dy > 0, finite)");
  const size_t node_bytes = precision == LT_PREC_FP64 ? sizeof(double2) : sizeof(float4);
  const size_t budget_nodes = std::max<size_t>(m->ws_budget / node_bytes, 1);
  Plan p;
  p.grids.assign(grids, grids + n);
  p.precision = precision;
  p.shape = shape;
  std::vector<SampleGrid> sg(n);
  std::vector<int64_t> items;
  std::vector<float> coords;
  int b = 0;
  while (b < n) {
    Chunk c;
    c.b0 = b;
    size_t nodes = 0;
    while (b < n) {
      size_t nb = (size_t)grids[b].nx * grids[b].ny;
      if (b > c.b0 && nodes + nb > budget_nodes) break;
      const lt_grid& g = grids[b];
      sg[b] = sample_grid(g, (int64_t)nodes, (int64_t)coords.size());
      grid_coords(g, coords);
      nodes += nb;
      ++b;
    }
    c.b1 = b;
    p.max_chunk_nodes = std::max(p.max_chunk_nodes, nodes);
    c.defl_off = items.size();
    int64_t acc = 0;
    for (int k = c.b0; k < c.b1; ++k) {
      items.push_back(acc);
      acc += defl_items(grids[k], precision, shape);
    }
    items.push_back(acc);
    c.defl_items = acc;
    c.search_off = items.size();
    acc = 0;
    for (int k = c.b0; k < c.b1; ++k) {
      items.push_back(acc);
      acc += precision == LT_PREC_FP64
                 ? ((int64_t)(grids[k].nx - 1) * (grids[k].ny - 1) + kSearch64Cells - 1) /
                       kSearch64Cells
                 : search32_items(grids[k].nx, grids[k].ny);
    }
    items.push_back(acc);
    c.search_items = acc;
    p.chunks.push_back(c);
  }
  lt_status s = grow(m, &m->d_plan_items, &m->plan_items_alloc, items.size());
  if (s != LT_OK) return s;
  s = grow(m, &m->d_sched, &m->sched_alloc, 1 + 2 * p.chunks.size());
  if (s != LT_OK) return s;
  s = grow(m, &m->d_plan_coords, &m->plan_coords_alloc, coords.size());
  if (s != LT_OK) return s;
  LT_CUDA(cudaMemcpyAsync(m->d_plan_coords, coords.data(), sizeof(float) * coords.size(),
                          cudaMemcpyHostToDevice, st));
  LT_CUDA(cudaMemcpyAsync(m->d_plan_grids, sg.data(), sizeof(SampleGrid) * n,
                          cudaMemcpyHostToDevice, st));
  LT_CUDA(cudaMemcpyAsync(m->d_plan_items, items.data(), sizeof(int64_t) * items.size(),
                          cudaMemcpyHostToDevice, st));
  m->plan = std::move(p);
  return LT_OK;
}

lt_status ensure_nodes(lt_model* m, size_t bytes) {
  if (m->nodes_bytes >= bytes && m->d_nodes) return LT_OK;
  ++m->ws_epoch;
  if (m->d_nodes) LT_CUDA(cudaFree(m->d_nodes));
  m->d_nodes = nullptr;
  m->nodes_bytes = 0;
  LT_CUDA(cudaMalloc(&m->d_nodes, std::max<size_t>(bytes, 16)));
  m->nodes_bytes = bytes;
  return LT_OK;
}

lt_status ensure_lists(lt_model* m, int64_t hit_cap, int64_t work_cap) {
  if (m->hits_cap_alloc < hit_cap || !m->d_hits) {
    ++m->ws_epoch;
    if (m->d_hits) LT_CUDA(cudaFree(m->d_hits));
    m->d_hits = nullptr;
    LT_CUDA(cudaMalloc(&m->d_hits, sizeof(Hit) * (size_t)m->batch * hit_cap));
    m->hits_cap_alloc = hit_cap;
  }
  if (m->work_cap_alloc < work_cap || !m->d_work) {
    ++m->ws_epoch;
    if (m->d_work) LT_CUDA(cudaFree(m->d_work));
    m->d_work = nullptr;
    LT_CUDA(cudaMalloc(&m->d_work, sizeof(Work64) * (size_t)m->batch * work_cap));
    m->work_cap_alloc = work_cap;
  }
  return LT_OK;
}

lt_status ensure_obs(lt_model* m, int n_obs, int n_sys) {
  if (n_obs > m->obs_alloc) {
    ++m->ws_epoch;
    if (m->d_beta_obs) LT_CUDA(cudaFree(m->d_beta_obs));
    if (m->d_match_tri) LT_CUDA(cudaFree(m->d_match_tri));
    if (m->d_match_hit) LT_CUDA(cudaFree(m->d_match_hit));
    if (m->d_match_xy) LT_CUDA(cudaFree(m->d_match_xy));
    if (m->d_adj_lam) LT_CUDA(cudaFree(m->d_adj_lam));
    if (m->d_adj_pts) LT_CUDA(cudaFree(m->d_adj_pts));
    if (m->d_chi2_terms) LT_CUDA(cudaFree(m->d_chi2_terms));
    m->d_beta_obs = nullptr; m->d_match_tri = nullptr; m->d_match_hit = nullptr;
    m->d_match_xy = nullptr; m->d_adj_lam = nullptr; m->d_adj_pts = nullptr;
    m->d_chi2_terms = nullptr;
    LT_CUDA(cudaMalloc(&m->d_beta_obs, sizeof(double) * 2 * (size_t)m->batch * n_obs));
    LT_CUDA(cudaMalloc(&m->d_match_tri, sizeof(int64_t) * (size_t)m->batch * n_obs));
    LT_CUDA(cudaMalloc(&m->d_match_hit, sizeof(int32_t) * (size_t)m->batch * n_obs));
    LT_CUDA(cudaMalloc(&m->d_match_xy, sizeof(double) * 2 * (size_t)m->batch * n_obs));
    LT_CUDA(cudaMalloc(&m->d_adj_lam, sizeof(double2) * (size_t)m->batch * n_obs));
    LT_CUDA(cudaMalloc(&m->d_adj_pts, sizeof(AdjPt) * 4 * (size_t)m->batch * n_obs));
    LT_CUDA(cudaMalloc(&m->d_chi2_terms, sizeof(double) * (size_t)m->batch * n_obs));
    m->obs_alloc = n_obs;
  }
  if (n_sys > m->sys_alloc) {
    ++m->ws_epoch;
    if (m->d_bary) LT_CUDA(cudaFree(m->d_bary));
    m->d_bary = nullptr;
    LT_CUDA(cudaMalloc(&m->d_bary, sizeof(double) * 2 * (size_t)m->batch * n_sys));
    m->sys_alloc = n_sys;
  }
  return LT_OK;
}

// Scratch of the FP64 resolution for the largest chunk of the current plan.
lt_status ensure_resolve(lt_model* m) {
  int max_nb = 1;
  for (const Chunk& c : m->plan.chunks) max_nb = std::max(max_nb, c.b1 - c.b0);
  unsigned long long cap = 1024;
  while (cap < 6ull * (unsigned long long)max_nb * (unsigned long long)m->work_cap) cap <<= 1;
  LT_CHECK_ARG(cap <= (1ull << 31), "FP64 work capacity too large for one chunk");
  const size_t vslots = (size_t)max_nb * m->work_cap * 3;
  if (cap > m->rs.cap) {
    ++m->ws_epoch;
    void* old[] = {m->rs.keys, m->rs.hval, m->rs.ulist, m->rs.tval, m->rs.flag64, m->rs.ulist64};
    for (void* q : old)
      if (q) LT_CUDA(cudaFree(q));
    m->rs.keys = nullptr; m->rs.hval = nullptr; m->rs.ulist = nullptr; m->rs.cap = 0;
    m->rs.tval = nullptr; m->rs.flag64 = nullptr; m->rs.ulist64 = nullptr;
    LT_CUDA(cudaMalloc(&m->rs.keys, sizeof(unsigned long long) * cap));
    LT_CUDA(cudaMalloc(&m->rs.hval, sizeof(double2) * cap));
    LT_CUDA(cudaMalloc(&m->rs.ulist, sizeof(int32_t) * cap));
    LT_CUDA(cudaMalloc(&m->rs.tval, sizeof(TightVal) * cap));
    LT_CUDA(cudaMalloc(&m->rs.flag64, sizeof(uint32_t) * cap));
    LT_CUDA(cudaMalloc(&m->rs.ulist64, sizeof(int32_t) * cap));
    // empty once here; every resolution leaves them empty again (k_res_tri)
    LT_CUDA(cudaMemset(m->rs.keys, 0xff, sizeof(unsigned long long) * cap));
    LT_CUDA(cudaMemset(m->rs.flag64, 0, sizeof(uint32_t) * cap));
    m->rs.cap = cap;
  }
  if (!m->rs.n_unique) {
    LT_CUDA(cudaMalloc(&m->rs.n_unique, sizeof(unsigned int)));
    LT_CUDA(cudaMemset(m->rs.n_unique, 0, sizeof(unsigned int)));
  }
  if (!m->rs.n64) {
    LT_CUDA(cudaMalloc(&m->rs.n64, sizeof(unsigned int)));
    LT_CUDA(cudaMemset(m->rs.n64, 0, sizeof(unsigned int)));
  }
  if (vslots > m->rs_vslot_alloc) {
    ++m->ws_epoch;
    if (m->rs.vslot) LT_CUDA(cudaFree(m->rs.vslot));
    m->rs.vslot = nullptr;
    LT_CUDA(cudaMalloc(&m->rs.vslot, sizeof(int32_t) * vslots));
    m->rs_vslot_alloc = vslots;
  }
  return LT_OK;
}

// Prepare everything an enqueue needs (plan, workspaces) -- may allocate and
// upload; must run outside stream capture.
lt_status prepare(lt_model* m, const lt_grid* grids, int precision, int64_t hit_cap,
                  cudaStream_t st) {
  lt_status s = make_plan(m, grids, m->batch, precision, st);
  if (s != LT_OK) return s;
  const size_t node_bytes = precision == LT_PREC_FP64 ? sizeof(double2) : sizeof(float4);
  s = ensure_nodes(m, m->plan.max_chunk_nodes * node_bytes);
  if (s != LT_OK) return s;
  s = ensure_lists(m, std::max(hit_cap, m->hit_cap), m->work_cap);
  if (s != LT_OK || precision == LT_PREC_FP64) return s;
  return ensure_resolve(m);
}

// Deflection + search (+ FP64 resolution) of one chunk into the hit lists.
lt_status enqueue_search(lt_model* m, size_t ci, int precision, Sources src, int64_t hit_cap,
                         cudaStream_t st, cudaEvent_t wait_before_search) {
  const Chunk& c = m->plan.chunks[ci];
  unsigned long long* next_defl = m->d_sched + 1 + 2 * ci;
  unsigned long long* next_search = next_defl + 1;
  const int nb = c.b1 - c.b0;
  const SampleGrid* g = m->d_plan_grids + c.b0;
  const int64_t* di = m->d_plan_items + c.defl_off;
  const int64_t* si = m->d_plan_items + c.search_off;
  Hit* hits = m->d_hits + (size_t)c.b0 * hit_cap;
  Work64* work = m->d_work + (size_t)c.b0 * m->work_cap;
  unsigned long long* hc = m->d_hit_count + c.b0;
  unsigned long long* wc = m->d_work_count + c.b0;
  src.sample_base = c.b0;
  double np = 0.0;
  for (int b = c.b0; b < c.b1; ++b)
    np += (double)m->plan.grids[b].nx * m->plan.grids[b].ny * m->n_pot;
  if (precision == LT_PREC_FP64) {
    double2* nodes = (double2*)m->d_nodes;
    {
      ProfScope ps(m, st, 0, np, 1);
      LT_CUDA(launch_deflect64(m->d_pot64 + (size_t)c.b0 * m->n_pot, m->n_pot, g, di, nb,
                               c.defl_items, nodes, m->sm_count, st));
    }
    if (wait_before_search) LT_CUDA(cudaStreamWaitEvent(st, wait_before_search, 0));
    ProfScope ps(m, st, 1);
    LT_CUDA(launch_search64(nodes, g, si, nb, c.search_items, src, hits, hit_cap, hc,
                            m->d_counters, m->d_status, m->sm_count, st));
  } else {
    float4* nodes = (float4*)m->d_nodes;
    {
      ProfScope ps(m, st, 0, np, 0);
      // the coarse bound: the resolution re-evaluates undecided nodes tightly
      LT_CUDA(launch_deflect32(m->d_pot32 + (size_t)c.b0 * m->n_pot, m->d_seg + c.b0, m->n_pot,
                               g, m->d_plan_coords, di, nb, c.defl_items, m->shape, false, nodes,
                               next_defl, m->sm_count, st));
    }
    if (wait_before_search) LT_CUDA(cudaStreamWaitEvent(st, wait_before_search, 0));
    {
      ProfScope ps(m, st, 1);
      LT_CUDA(launch_search32(nodes, g, si, nb, c.search_items, src, hits, hit_cap, work,
                              m->work_cap, hc, wc, m->d_counters, m->d_status, next_search,
                              m->sm_count, st));
    }
    // k_res_insert, k_res_tight32, k_res_tri32, k_res_nodes, k_res_tri
    ProfScope ps(m, st, 2, 0.0, 0, 5);
    const cudaError_t re =
        launch_resolve64(m->d_pot64, m->d_pot32 + (size_t)c.b0 * m->n_pot, m->d_seg + c.b0,
                         m->n_pot, g, src, work, wc, nb, m->work_cap, hits, hit_cap, hc,
                         m->d_counters, m->d_status, m->rs, m->sm_count, st);
    // a failed launch may leave the table partly filled: reallocate (and so
    // clear) it on the next call
    if (re != cudaSuccess) {
      m->rs.cap = 0;
      if (m->rs.n_unique) cudaMemsetAsync(m->rs.n_unique, 0, sizeof(unsigned int), st);
      if (m->rs.n64) cudaMemsetAsync(m->rs.n64, 0, sizeof(unsigned int), st);
    }
    LT_CUDA(re);
  }
  return LT_OK;
}

lt_status reset_counts(lt_model* m, cudaStream_t st) {
  LT_CUDA(launch_zero64((unsigned long long*)m->d_counters, CNT_N, m->d_sched,
                        (int64_t)m->sched_alloc, m->d_hit_count, m->batch, m->d_work_count,
                        m->batch, st));
  return LT_OK;
}

lt_status check_obs(lt_model* m, const lt_obs* obs) {
  LT_CHECK_ARG(obs != nullptr, "obs is NULL");
  LT_CHECK_ARG(obs->n_obs >= 1 && obs->n_sys >= 1, "obs: need n_obs >= 1 and n_sys >= 1");
  LT_CHECK_ARG(obs->x && obs->y && obs->sigma && obs->sys && obs->dls_ds,
               "obs: a device pointer is NULL");
  return LT_OK;
}

// The whole chi^2 sequence (no allocation, no host synchronisation: safe to
// capture in a CUDA graph once prepare() has run).
lt_status enqueue_chi2(lt_model* m, const lt_obs& obs, int precision, double* chi2_out,
                       cudaStream_t st) {
  lt_status s = reset_counts(m, st);
  if (s != LT_OK) return s;
  // the barycentres need only the parameters: run them on the side stream,
  // overlapping the first chunk's deflection; the search waits for them
  LT_CUDA(cudaEventRecord(m->ev_fork, st));
  LT_CUDA(cudaStreamWaitEvent(m->side, m->ev_fork, 0));
  {
    ProfScope ps(m, m->side, 4, 0.0, 0, 2);  // k_bary_obs, k_bary_sys
    LT_CUDA(launch_barycentres(m->d_pot64, m->n_pot, m->batch, obs, m->d_beta_obs, m->d_bary,
                               m->side));
  }
  LT_CUDA(cudaEventRecord(m->ev_join, m->side));
  Sources src{m->d_bary, obs.dls_ds, obs.n_sys, 0, 0};
  const int64_t hc = m->hits_cap_alloc;
  for (size_t ci = 0; ci < m->plan.chunks.size(); ++ci) {
    const Chunk& c = m->plan.chunks[ci];
    s = enqueue_search(m, ci, precision, src, hc, st, ci == 0 ? m->ev_join : nullptr);
    if (s != LT_OK) return s;
    ProfScope ps(m, st, 3, 0.0, 0, 2);  // k_chi2_match, k_chi2_sum
    LT_CUDA(launch_chi2(m->d_hits + (size_t)c.b0 * hc, m->d_hit_count + c.b0, c.b1 - c.b0, hc,
                        c.b0, m->d_plan_grids + c.b0, obs, chi2_out, m->d_chi2_terms,
                        m->d_match_tri, m->d_match_hit, m->d_match_xy, st));
  }
  m->last_nobs = obs.n_obs;
  m->last_nsys = obs.n_sys;
  return LT_OK;
}

}  // namespace

extern "C" {

const char* lt_version(void) { return "lenstool-gb300 0.1 (sm_103a)"; }

const char* lt_status_string(lt_status s) {
  switch (s) {
    case LT_OK: return "ok";
    case LT_ERR_INVALID_ARG: return "invalid argument";
    case LT_ERR_CUDA: return "CUDA error";
    case LT_ERR_NOMEM: return "out of device memory";
    case LT_ERR_OVERFLOW: return "capacity overflow";
    case LT_ERR_TIMEOUT: return "timeout";
    case LT_ERR_NONFINITE: return "non-finite or invalid lens parameter";
  }
  return "unknown status";
}

const char* lt_last_error(const lt_model* m) { return m ? m->err.c_str() : "model is NULL"; }

lt_status lt_model_create(const lt_model_desc* desc, lt_model** out) {
  if (!out) return LT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || desc->n_pot < 1 || desc->batch < 1 || desc->hit_capacity < 0)
    return LT_ERR_INVALID_ARG;
  lt_model* m = new lt_model();
  m->n_pot = desc->n_pot;
  m->batch = desc->batch;
  m->hit_cap = desc->hit_capacity > 0 ? desc->hit_capacity : kDefaultCap;
  m->work_cap = m->hit_cap;
  if (const char* e = std::getenv("LT_WORKSPACE_MB")) {
    long long mb = std::atoll(e);
    if (mb > 0) m->ws_budget = (size_t)mb << 20;
  }
  auto fail = [&](cudaError_t e) {
    lt_status st = e == cudaErrorMemoryAllocation ? LT_ERR_NOMEM : LT_ERR_CUDA;
    lt_model_destroy(m);
    return st;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&m->device)) != cudaSuccess) return fail(e);
  if ((e = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device)) !=
      cudaSuccess)
    return fail(e);
  const size_t np = (size_t)m->n_pot * m->batch;
  if ((e = cudaMalloc(&m->d_params, sizeof(double) * LT_N_ROWS * np)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->d_pot64, sizeof(Pot64) * np)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->d_pot32, sizeof(Pot32) * np)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->d_seg, sizeof(Seg32) * m->batch)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->d_status, sizeof(uint32_t))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->d_counters, sizeof(long long) * CNT_N)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->d_hit_count, sizeof(unsigned long long) * m->batch)) != cudaSuccess)
    return fail(e);
  if ((e = cudaMalloc(&m->d_work_count, sizeof(unsigned long long) * m->batch)) != cudaSuccess)
    return fail(e);
  if ((e = cudaMalloc(&m->d_plan_grids, sizeof(SampleGrid) * m->batch)) != cudaSuccess)
    return fail(e);
  if ((e = cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
    return fail(e);
  if ((e = cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming)) != cudaSuccess)
    return fail(e);
  if ((e = cudaMemset(m->d_status, 0, sizeof(uint32_t))) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(m->d_counters, 0, sizeof(long long) * CNT_N)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(m->d_hit_count, 0, sizeof(unsigned long long) * m->batch)) != cudaSuccess)
    return fail(e);
  if ((e = cudaMemset(m->d_work_count, 0, sizeof(unsigned long long) * m->batch)) != cudaSuccess)
    return fail(e);
  // zero parameters: a valid, massless model until lt_model_set_params
  if ((e = cudaMemset(m->d_params, 0, sizeof(double) * LT_N_ROWS * np)) != cudaSuccess)
    return fail(e);
  if ((e = launch_prep(m->d_params, m->batch, m->n_pot, m->d_pot64, m->d_pot32, m->d_seg,
                       m->d_status, 0)) != cudaSuccess)
    return fail(e);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  *out = m;
  return LT_OK;
}

void lt_model_destroy(lt_model* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  void* ptrs[] = {m->d_params, m->d_pot64, m->d_pot32, m->d_seg, m->d_status, m->d_counters,
                  m->d_nodes, m->d_hits, m->d_work, m->d_hit_count, m->d_work_count,
                  m->d_plan_grids, m->d_plan_items, m->d_plan_coords, m->d_dg_coords,
                  m->d_beta_obs, m->d_bary, m->d_match_tri,
                  m->d_match_hit, m->d_match_xy, m->d_adj_lam, m->d_adj_pts, m->d_sched,
                  m->d_src_beta, m->d_src_mu, m->d_src_bary, m->d_chi2_terms, m->rs.keys,
                  m->rs.hval,
                  m->rs.vslot, m->rs.ulist, m->rs.n_unique, m->rs.tval, m->rs.flag64,
                  m->rs.ulist64, m->rs.n64};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
  if (m->side) cudaStreamDestroy(m->side);
  if (m->ev_fork) cudaEventDestroy(m->ev_fork);
  if (m->ev_join) cudaEventDestroy(m->ev_join);
  for (auto& r : m->prof_pending) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (cudaEvent_t e : m->prof_pool) cudaEventDestroy(e);
  delete m;
}

lt_status lt_model_set_params(lt_model* m, const double* params, int on_device,
                              uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(params != nullptr, "params is NULL");
  const size_t bytes = sizeof(double) * LT_N_ROWS * (size_t)m->n_pot * m->batch;
  // device parameters are read in place by the preparation kernel (stream
  // ordered, like a copy would be); host parameters are uploaded first
  const double* src = params;
  if (!on_device) {
    LT_CUDA(cudaMemcpyAsync(m->d_params, params, bytes, cudaMemcpyHostToDevice, S(stream)));
    src = m->d_params;
  }
  LT_CUDA(launch_prep(src, m->batch, m->n_pot, m->d_pot64, m->d_pot32, m->d_seg, m->d_status,
                      S(stream)));
  return LT_OK;
}

lt_status lt_deflect_grid(lt_model* m, int32_t sample, const lt_grid* grid,
                          lt_precision precision, void* alpha_out, float* err_out,
                          uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(sample >= 0 && sample < m->batch, "sample out of range");
  LT_CHECK_ARG(grid && grid_ok(*grid), "invalid grid");
  LT_CHECK_ARG(alpha_out != nullptr, "alpha_out is NULL");
  LT_CHECK_ARG(precision == LT_PREC_FP64 || precision == LT_PREC_MIXED ||
                   precision == LT_PREC_PAPER,
               "invalid precision");
  LT_CHECK_ARG(precision != LT_PREC_FP64 || err_out == nullptr,
               "err_out is not produced in FP64 precision");
  cudaStream_t st = S(stream);
  // a one-sample plan over the caller's grid (does not disturb the batch plan)
  const lt_grid& g = *grid;
  const SampleGrid sg = sample_grid(g, 0, 0);
  const int64_t nodes = (int64_t)g.nx * g.ny;
  LT_CHECK_ARG(precision != LT_PREC_PAPER || nodes < ((int64_t)1 << 31),
               "LT_PREC_PAPER grids are limited to 2^31 nodes");
  int64_t items[2] = {
      0, defl_items(g, precision == LT_PREC_FP64 ? LT_PREC_FP64 : LT_PREC_MIXED, m->shape)};
  static_assert(sizeof(SampleGrid) % 8 == 0, "alignment");
  struct OneSample {
    SampleGrid g;
    int64_t items[2];
    unsigned long long count;
  } host{sg, {items[0], items[1]}, 0ull};
  // node workspace layout: [float4 nodes][flags][int32 list][OneSample]; the
  // sample's plan lives after its nodes, so the batch plan's tables stay intact
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const bool fp32 = precision != LT_PREC_FP64;
  const size_t node_bytes = fp32 ? up(sizeof(float4) * (size_t)nodes) : 0;
  const size_t flag_bytes = precision == LT_PREC_PAPER ? up((size_t)nodes) : 0;
  const size_t list_bytes = precision == LT_PREC_PAPER ? up(sizeof(int32_t) * (size_t)nodes) : 0;
  if (fp32 && (!m->d_dg_coords || std::memcmp(&m->dg_grid, &g, sizeof(lt_grid)) != 0)) {
    std::vector<float> coords;
    grid_coords(g, coords);
    if (m->dg_coords_alloc < coords.size()) {
      if (m->d_dg_coords) LT_CUDA(cudaFree(m->d_dg_coords));
      m->d_dg_coords = nullptr;
      m->dg_coords_alloc = 0;
      LT_CUDA(cudaMalloc(&m->d_dg_coords, sizeof(float) * coords.size()));
      m->dg_coords_alloc = coords.size();
    }
    LT_CUDA(cudaMemcpyAsync(m->d_dg_coords, coords.data(), sizeof(float) * coords.size(),
                            cudaMemcpyHostToDevice, st));
    m->dg_grid = g;
  }
  const size_t need = node_bytes + flag_bytes + list_bytes + up(sizeof(OneSample));
  lt_status s = ensure_nodes(m, need);
  if (s != LT_OK) return s;
  char* base = (char*)m->d_nodes;
  unsigned char* flags = (unsigned char*)(base + node_bytes);
  int32_t* list = (int32_t*)(base + node_bytes + flag_bytes);
  OneSample* dev = (OneSample*)(base + node_bytes + flag_bytes + list_bytes);
  LT_CUDA(cudaMemcpyAsync(dev, &host, sizeof(OneSample), cudaMemcpyHostToDevice, st));
  if (precision == LT_PREC_FP64) {
    LT_CUDA(launch_deflect64(m->d_pot64 + (size_t)sample * m->n_pot, m->n_pot, &dev->g,
                             dev->items, 1, items[1], (double2*)alpha_out, m->sm_count, st));
    return LT_OK;
  }
  float4* nodes4 = (float4*)base;
  if (!m->d_sched) {
    lt_status s2 = grow(m, &m->d_sched, &m->sched_alloc, 1);
    if (s2 != LT_OK) return s2;
  }
  LT_CUDA(cudaMemsetAsync(m->d_sched, 0, sizeof(unsigned long long), st));
  // the tight bound where the caller asks for it, the cheaper coarse kernel
  // otherwise (its bound is not output; the deflection is the same)
  const bool tight = err_out != nullptr && precision == LT_PREC_MIXED;
  LT_CUDA(launch_deflect32(m->d_pot32 + (size_t)sample * m->n_pot, m->d_seg + sample, m->n_pot,
                           &dev->g, m->d_dg_coords, dev->items, 1, items[1], m->shape, tight,
                           nodes4, m->d_sched, m->sm_count, st));
  if (precision == LT_PREC_MIXED) {
    LT_CUDA(launch_unpack32(nodes4, nodes, (float2*)alpha_out, err_out, st));
    return LT_OK;
  }
  // the paper's rule: FP32 widened, FP64 in halo patches and where the
  // distortion criteria fire
  const Pot64* p64 = m->d_pot64 + (size_t)sample * m->n_pot;
  LT_CUDA(launch_paper_flags(nodes4, p64, m->n_pot, g, (double2*)alpha_out, flags, list,
                             &dev->count, err_out, m->sm_count, st));
  LT_CUDA(launch_paper_fp64(p64, m->n_pot, g, list, &dev->count, (double2*)alpha_out,
                            m->sm_count, st));
  LT_CUDA(cudaMemcpyAsync(&m->d_counters[CNT_FP64_NODES], &dev->count, sizeof(long long),
                          cudaMemcpyDeviceToDevice, st));
  return LT_OK;
}

lt_status lt_find_images(lt_model* m, const lt_grid* grids, int32_t n_src, const double* src_xy,
                         const double* dls_ds, lt_precision precision, int64_t capacity,
                         lt_image* out, int64_t* n_out, uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(grids != nullptr, "grids is NULL");
  LT_CHECK_ARG(n_src >= 0, "n_src < 0");
  LT_CHECK_ARG(n_src == 0 || (src_xy && dls_ds), "src_xy / dls_ds is NULL");
  LT_CHECK_ARG(capacity >= 0 && (capacity == 0 || out), "out is NULL");
  LT_CHECK_ARG(n_out != nullptr, "n_out is NULL");
  LT_CHECK_ARG(precision == LT_PREC_FP64 || precision == LT_PREC_MIXED, "invalid precision");
  cudaStream_t st = S(stream);
  const int64_t hc = std::max<int64_t>(capacity, m->hit_cap);
  lt_status s = prepare(m, grids, precision, hc, st);
  if (s != LT_OK) return s;
  s = reset_counts(m, st);
  if (s != LT_OK) return s;
  Sources src{src_xy, dls_ds, n_src, 1, 0};
  const int64_t hca = m->hits_cap_alloc;
  for (size_t ci = 0; ci < m->plan.chunks.size(); ++ci) {
    const Chunk& c = m->plan.chunks[ci];
    if (n_src > 0) {
      s = enqueue_search(m, ci, precision, src, hca, st, nullptr);
      if (s != LT_OK) return s;
    }
    LT_CUDA(launch_sort_hits(m->d_hits + (size_t)c.b0 * hca, m->d_hit_count + c.b0, c.b1 - c.b0,
                             hca, c.b0, out, capacity, n_out, m->d_status, st));
  }
  return LT_OK;
}

lt_status lt_chi2(lt_model* m, const lt_grid* grids, const lt_obs* obs, lt_precision precision,
                  double* chi2_out, uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(grids != nullptr, "grids is NULL");
  LT_CHECK_ARG(chi2_out != nullptr, "chi2_out is NULL");
  LT_CHECK_ARG(precision == LT_PREC_FP64 || precision == LT_PREC_MIXED, "invalid precision");
  lt_status s = check_obs(m, obs);
  if (s != LT_OK) return s;
  cudaStream_t st = S(stream);
  s = prepare(m, grids, precision, m->hit_cap, st);
  if (s != LT_OK) return s;
  s = ensure_obs(m, obs->n_obs, obs->n_sys);
  if (s != LT_OK) return s;
  return enqueue_chi2(m, *obs, precision, chi2_out, st);
}

lt_status lt_chi2_graph(lt_model* m, const lt_grid* grids, const lt_obs* obs,
                        lt_precision precision, double* chi2_out, uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(grids != nullptr, "grids is NULL");
  LT_CHECK_ARG(chi2_out != nullptr, "chi2_out is NULL");
  LT_CHECK_ARG(precision == LT_PREC_FP64 || precision == LT_PREC_MIXED, "invalid precision");
  lt_status s = check_obs(m, obs);
  if (s != LT_OK) return s;
  cudaStream_t st = S(stream);
  const bool same = m->graph_exec && m->graph_prec == precision && m->graph_out == chi2_out &&
                    same_grids(m->graph_grids, grids, m->batch) &&
                    std::memcmp(&m->graph_obs, obs, sizeof(lt_obs)) == 0 &&
                    same_grids(m->plan.grids, grids, m->batch) &&
                    m->plan.precision == precision && m->plan.shape == m->shape &&
                    m->graph_epoch == m->ws_epoch;
  if (!same) {
    s = prepare(m, grids, precision, m->hit_cap, st);
    if (s != LT_OK) return s;
    s = ensure_obs(m, obs->n_obs, obs->n_sys);
    if (s != LT_OK) return s;
    LT_CUDA(cudaStreamSynchronize(st));  // uploads done before capture
    m->graph_epoch = m->ws_epoch;
    if (!m->capture_stream)
      LT_CUDA(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
    if (m->graph_exec) {
      cudaGraphExecDestroy(m->graph_exec);
      m->graph_exec = nullptr;
    }
    LT_CUDA(cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal));
    s = enqueue_chi2(m, *obs, precision, chi2_out, m->capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(m->capture_stream, &graph);
    if (s != LT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    LT_CUDA(ce);
    cudaError_t ie = cudaGraphInstantiate(&m->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    LT_CUDA(ie);
    m->graph_grids.assign(grids, grids + m->batch);
    m->graph_obs = *obs;
    m->graph_prec = precision;
    m->graph_out = chi2_out;
  }
  LT_CUDA(cudaGraphLaunch(m->graph_exec, st));
  m->last_nobs = obs->n_obs;
  m->last_nsys = obs->n_sys;
  return LT_OK;
}

lt_status lt_chi2_grad(lt_model* m, const lt_grid* grids, const lt_obs* obs,
                       lt_precision precision, double* chi2_out, double* grad_out,
                       uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(grad_out != nullptr, "grad_out is NULL");
  lt_status s = lt_chi2(m, grids, obs, precision, chi2_out, stream);
  if (s != LT_OK) return s;
  cudaStream_t st = S(stream);
  LT_CUDA(launch_adjoint(m->d_pot64, m->n_pot, m->batch, m->d_plan_grids, m->d_hits,
                         m->hits_cap_alloc, *obs, m->d_match_hit, m->d_adj_lam, m->d_adj_pts,
                         grad_out, m->sm_count, st));
  return LT_OK;
}

lt_status lt_chi2_source(lt_model* m, const lt_obs* obs, double* chi2_out, double* mu_out,
                         uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(chi2_out != nullptr, "chi2_out is NULL");
  lt_status s = check_obs(m, obs);
  if (s != LT_OK) return s;
  cudaStream_t st = S(stream);
  if (obs->n_obs > m->src_obs_alloc) {
    if (m->d_src_beta) LT_CUDA(cudaFree(m->d_src_beta));
    if (m->d_src_mu) LT_CUDA(cudaFree(m->d_src_mu));
    m->d_src_beta = nullptr;
    m->d_src_mu = nullptr;
    LT_CUDA(cudaMalloc(&m->d_src_beta, sizeof(double2) * (size_t)m->batch * obs->n_obs));
    LT_CUDA(cudaMalloc(&m->d_src_mu, sizeof(double) * (size_t)m->batch * obs->n_obs));
    m->src_obs_alloc = obs->n_obs;
  }
  if (obs->n_sys > m->src_sys_alloc) {
    if (m->d_src_bary) LT_CUDA(cudaFree(m->d_src_bary));
    m->d_src_bary = nullptr;
    LT_CUDA(cudaMalloc(&m->d_src_bary, sizeof(double2) * (size_t)m->batch * obs->n_sys));
    m->src_sys_alloc = obs->n_sys;
  }
  double* mu = mu_out ? mu_out : m->d_src_mu;
  LT_CUDA(launch_chi2_source(m->d_pot64, m->n_pot, m->batch, *obs, m->d_src_beta, mu,
                             m->d_src_bary, chi2_out, m->sm_count, st));
  return LT_OK;
}

lt_status lt_last_magnifications(lt_model* m, const lt_obs* obs, double* mu_out,
                                 uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(mu_out != nullptr, "mu_out is NULL");
  LT_CHECK_ARG(m->last_nobs > 0, "no chi^2 evaluation has run");
  lt_status s = check_obs(m, obs);
  if (s != LT_OK) return s;
  LT_CHECK_ARG(obs->n_obs == m->last_nobs && obs->n_sys == m->last_nsys,
               "obs differ from the last chi^2 evaluation's");
  LT_CUDA(launch_mag_pred(m->d_pot64, m->n_pot, m->batch, m->d_plan_grids, m->d_hits,
                          m->hits_cap_alloc, *obs, m->d_match_hit, mu_out, m->sm_count,
                          S(stream)));
  return LT_OK;
}

lt_status lt_last_matches(lt_model* m, int64_t* match_tri, double* match_xy, double* bary,
                          uintptr_t stream) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(m->last_nobs > 0, "no chi^2 evaluation has run");
  cudaStream_t st = S(stream);
  const size_t no = (size_t)m->batch * m->last_nobs, ns = (size_t)m->batch * m->last_nsys;
  if (match_tri)
    LT_CUDA(cudaMemcpyAsync(match_tri, m->d_match_tri, sizeof(int64_t) * no,
                            cudaMemcpyDeviceToDevice, st));
  if (match_xy)
    LT_CUDA(cudaMemcpyAsync(match_xy, m->d_match_xy, sizeof(double) * 2 * no,
                            cudaMemcpyDeviceToDevice, st));
  if (bary)
    LT_CUDA(cudaMemcpyAsync(bary, m->d_bary, sizeof(double) * 2 * ns, cudaMemcpyDeviceToDevice,
                            st));
  return LT_OK;
}

lt_status lt_model_sync(lt_model* m, uintptr_t stream, lt_stats* stats) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CUDA(cudaStreamSynchronize(S(stream)));
  uint32_t status = 0;
  long long cnt[CNT_N] = {0};
  LT_CUDA(cudaMemcpy(&status, m->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  LT_CUDA(cudaMemcpy(cnt, m->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  LT_CUDA(cudaMemset(m->d_status, 0, sizeof(uint32_t)));
  if (stats) {
    stats->hits = cnt[CNT_HITS];
    stats->ambiguous = cnt[CNT_AMBIG];
    stats->refined = cnt[CNT_REFINE];
    stats->fp64_nodes = cnt[CNT_FP64_NODES];
    stats->work_overflow = cnt[CNT_DROPPED];
    stats->tight_nodes = cnt[CNT_TIGHT_NODES];
    stats->fp64_items = cnt[CNT_FP64_ITEMS];
  }
  if (status & ST_NONFINITE) {
    m->err = "non-finite or out-of-domain lens parameter";
    return LT_ERR_NONFINITE;
  }
  if (status & (ST_OVERFLOW_HITS | ST_OVERFLOW_WORK)) {
    m->err = (status & ST_OVERFLOW_HITS) ? "hit capacity exceeded" : "FP64 work capacity exceeded";
    return LT_ERR_OVERFLOW;
  }
  return LT_OK;
}

lt_status lt_profile_enable(lt_model* m, int on) {
  if (!m) return LT_ERR_INVALID_ARG;
  m->prof_mask = on ? 0x1fu : 0u;
  return LT_OK;
}

lt_status lt_profile_stages(lt_model* m, uint32_t mask) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(mask <= 0x1fu, "stage mask has bits beyond the five stages");
  m->prof_mask = mask;
  return LT_OK;
}

lt_status lt_profile_read(lt_model* m, lt_profile* out, int reset) {
  if (!m) return LT_ERR_INVALID_ARG;
  for (auto& r : m->prof_pending) {
    LT_CUDA(cudaEventSynchronize(r.e1));
    float ms = 0.f;
    LT_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
    m->prof_acc.launches[r.kind] += r.kernels;
    m->prof_acc.ms[r.kind] += ms;
    if (r.kind == 0) m->prof_acc.node_pot[r.fp64] += r.node_pot;
    m->prof_pool.push_back(r.e0);
    m->prof_pool.push_back(r.e1);
  }
  m->prof_pending.clear();
  if (out) *out = m->prof_acc;
  if (reset) m->prof_acc = lt_profile{};
  return LT_OK;
}

lt_status lt_model_set_shape(lt_model* m, int32_t shape) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(shape >= 0 && shape < kNumShapes, "shape out of range");
  if (m->shape != shape) {
    m->shape = shape;
    m->plan.grids.clear();  // item sizes depend on the shape
  }
  return LT_OK;
}

int32_t lt_num_shapes(void) { return kNumShapes; }

lt_status lt_autotune(lt_model* m, const lt_grid* grid, uintptr_t stream, int32_t* choice) {
  if (!m) return LT_ERR_INVALID_ARG;
  LT_CHECK_ARG(grid && grid_ok(*grid), "invalid grid");
  cudaStream_t st = S(stream);
  const lt_grid& g = *grid;
  const int64_t nodes = (int64_t)g.nx * g.ny;
  // the grid's plan for every shape (the work-item count depends on it),
  // uploaded once; then only the deflection kernel of sample 0 is timed, by
  // CUDA events around each launch
  struct OneShape {
    SampleGrid g;
    int64_t items[2];
  };
  static_assert(sizeof(OneShape) % 8 == 0, "alignment");
  std::vector<OneShape> hs(kNumShapes);
  for (int v = 0; v < kNumShapes; ++v) {
    hs[v] = OneShape{sample_grid(g, 0, 0), {0, defl_items(g, LT_PREC_MIXED, v)}};
  }
  std::vector<float> coords;
  grid_coords(g, coords);
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t node_bytes = up(sizeof(float4) * (size_t)nodes);
  const size_t plan_bytes = up(sizeof(OneShape) * hs.size());
  lt_status s = ensure_nodes(m, node_bytes + plan_bytes + up(sizeof(float) * coords.size()));
  if (s != LT_OK) return s;
  if (!m->d_sched) {
    s = grow(m, &m->d_sched, &m->sched_alloc, 1);
    if (s != LT_OK) return s;
  }
  char* base = (char*)m->d_nodes;
  OneShape* dplan = (OneShape*)(base + node_bytes);
  float* dcoords = (float*)(base + node_bytes + plan_bytes);
  LT_CUDA(cudaMemcpyAsync(dplan, hs.data(), sizeof(OneShape) * hs.size(), cudaMemcpyHostToDevice,
                          st));
  LT_CUDA(cudaMemcpyAsync(dcoords, coords.data(), sizeof(float) * coords.size(),
                          cudaMemcpyHostToDevice, st));
  cudaEvent_t e0, e1;
  LT_CUDA(cudaEventCreate(&e0));
  LT_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 1e30f;
  constexpr int kReps = 5;
  for (int v = 0; v < kNumShapes; ++v) {
    float vmin = 1e30f;
    for (int r = 0; r <= kReps; ++r) {  // r = 0 warms up
      LT_CUDA(cudaMemsetAsync(m->d_sched, 0, sizeof(unsigned long long), st));
      LT_CUDA(cudaEventRecord(e0, st));
      LT_CUDA(launch_deflect32(m->d_pot32, m->d_seg, m->n_pot, &dplan[v].g, dcoords,
                               dplan[v].items, 1, hs[v].items[1], v, false, (float4*)base,
                               m->d_sched, m->sm_count, st));
      LT_CUDA(cudaEventRecord(e1, st));
      LT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      LT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0) vmin = std::min(vmin, ms);
    }
    // a later shape must be clearly faster to replace an earlier one
    if (vmin < best_ms * 0.995f) {
      best_ms = vmin;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->shape = best;
  m->plan.grids.clear();
  if (choice) *choice = best;
  return LT_OK;
}

}  // extern "C"
