// C ABI of the library (declared in include/como3r.h): graph handles, workspaces,
// per-iteration launch sequence and its CUDA-graph replay.
//
// One iteration is six launches on the handle's stream:
//   K0 edge_prep -> K1 residual_reduce -> K2 edge_reduce -> assemble -> K3 factor_solve -> K4 retract
// como3r_solve captures them once into a CUDA graph (on a private capture stream) and
// replays it; a device counter indexes the per-iteration cost trace.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/como3r.h"
#include "como3r_internal.h"
#include "plan.h"

using namespace como3r;

namespace {
thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return set_error(COMO3R_ERR_OOM, std::string(where) + ": out of device memory");
  return set_error(COMO3R_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

// Error reporting for the entry points defined in other files (como3r_last_error).
int como3r::report_error(int code, const char* msg) { return set_error(code, msg); }
int como3r::report_cuda_error(cudaError_t e, const char* where) { return cuda_error(e, where); }

namespace {
#define CK(expr, where)                      \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return cuda_error(e_, where); \
  } while (0)

constexpr int kDefaultChunk = 2048;
constexpr int kChunks[] = {1024, 2048, 4096};  // K1 pixels per warp work item (autotuned)
}  // namespace

struct como3r_graph {
  HostPlan plan;
  int device = 0, sms = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  RobustParams rp{};
  double lambda = 0.0, eps0 = 1e-6;
  int max_attempts = 6;
  int k1_cfg = 0, k1_chunk = kDefaultChunk, k1_grid = 0, num_items = 0, max_items = 0;
  float k1_tuned_ms = 0.f;
  bool idx_rows_aligned = false;
  std::vector<void*> allocs;
  const void* points = nullptr;
  const int32_t* midx = nullptr;
  void* own_points = nullptr;
  int32_t* own_midx = nullptr;
  size_t points_bytes = 0, idx_bytes = 0;
  EdgeStatic* d_es = nullptr;
  Item* d_items = nullptr;
  int32_t* d_item_off = nullptr;
  // balanced K1 schedule (rebuilt on the device when the match indices change)
  int32_t *d_counts = nullptr, *d_wstart = nullptr, *d_wseg = nullptr, *d_seg_off = nullptr;
  uint32_t* d_compact = nullptr;  // valid-match lists per 1024-pixel item (kCompactSlot entries per item)
  bool k1_compact = false;        // d_compact is allocated (index rows aligned, P <= 2^22)
  long long* d_cum = nullptr;
  int max_warps = 0, k1_wv = 0, k1_wp = 1;
  double *d_T64 = nullptr, *d_Ad = nullptr, *d_partials = nullptr;
  float* d_T32 = nullptr;
  double *d_edge_M = nullptr, *d_edge_b = nullptr, *d_edge_cost = nullptr, *d_edge_skip = nullptr;
  long long* d_edge_valid = nullptr;
  int32_t *d_slot_kf_r = nullptr, *d_slot_kf_c = nullptr, *d_slot_contrib_off = nullptr, *d_slot_contrib = nullptr;
  int32_t *d_kf_contrib_off = nullptr, *d_kf_contrib = nullptr, *d_edge_offset = nullptr;
  double *d_A = nullptr, *d_L = nullptr, *d_colscratch = nullptr, *d_gvec = nullptr, *d_tau = nullptr;
  uint8_t* d_frozen = nullptr;
  GraphInfoDev* d_ginfo = nullptr;
  long long* d_start_ns = nullptr;  // device clock at the start of the last gn_step / solve
  DepthState* depth = nullptr;      // segment-level structure refinement (como3r_depth_setup)
  int *d_iter = nullptr, *d_warn = nullptr;
  double* d_cost_hist = nullptr;
  int64_t cost_hist_cap = 0;
  double* d_poses = nullptr;
  GraphInfoDev* h_ginfo = nullptr;
  int* h_warn = nullptr;
  unsigned long long* d_bad = nullptr;
  bool smem_solve = false;
  size_t solve_smem = 0;
  SolverPlan sp{};
  // multi-SM solve (one cluster of cluster_ctas CTAs per graph), when chosen at create
  int cluster_ctas = 0;
  // grid-wide solve of a single large graph (grid_ctas co-resident CTAs), when chosen
  int grid_ctas = 0;
  // batches with large graphs: one launch of CTA groups (group_ctas CTAs, group_big graphs
  // solved by a whole cluster), when chosen
  int group_ctas = 0, group_big = 0;
  int4* d_gtask = nullptr;
  int32_t* d_glist = nullptr;
  int* d_gfail = nullptr;
  GridSync* d_gsync = nullptr;
  unsigned grid_extra = 0;  // COMO3R_GRID_BARRIER_EXTRA: test of the barrier's wait limit
  double* d_diag_shift = nullptr;  // COMO3R_TEST_DIAG_SHIFT: per-graph diagonal shift (tests only)
  size_t cluster_smem = 0;
  ClusterPlan cp{};
  cudaGraphExec_t iter_exec = nullptr, eval_exec = nullptr;
  int64_t last_launches = 0;
  std::vector<long long> edge_valid;
  // adjoint workspaces (allocated by the first como3r_vjp call, grown with iters)
  int vjp_iters_cap = -1;
  double *d_ckpt = nullptr, *d_tau_hist = nullptr;
  GraphInfoDev *d_ginfo_hist = nullptr, *d_ginfo_final = nullptr;
  double *d_adj_a = nullptr, *d_adj_a2 = nullptr, *d_adj_rhs = nullptr, *d_adj_u = nullptr;
  double *d_evec = nullptr, *d_adj_rec = nullptr, *d_edge_adj = nullptr, *d_gacc = nullptr;
  // the factor of every forward iteration (blocks, column scratch), solved again backwards
  double *d_keep_L = nullptr, *d_keep_S = nullptr, *d_sub_z = nullptr;
  size_t sub_smem = 0;  // shared memory of the kept-factor substitution (0: d_sub_z)
  bool sub_fsmem = false;  // ... the kept factor staged into it as well
};

namespace {

template <typename T>
int dalloc(como3r_graph* g, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc");
  g->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return COMO3R_OK;
}

template <typename T>
int upload(como3r_graph* g, T** p, const std::vector<T>& v) {
  int rc = dalloc(g, p, v.size());
  if (rc) return rc;
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, g->stream), "upload");
  return COMO3R_OK;
}

void free_all(como3r_graph* g) {
  depth_free(g->depth);
  g->depth = nullptr;
  if (g->iter_exec) cudaGraphExecDestroy(g->iter_exec);
  if (g->eval_exec) cudaGraphExecDestroy(g->eval_exec);
  for (void* p : g->allocs) cudaFree(p);
  g->allocs.clear();
  if (g->h_ginfo) cudaFreeHost(g->h_ginfo);
  if (g->h_warn) cudaFreeHost(g->h_warn);
  if (g->cap) cudaStreamDestroy(g->cap);
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

WarpSched sched(const como3r_graph* g) { return WarpSched{g->d_wstart, g->d_wseg, g->d_counts, g->d_compact}; }

// Balanced K1 schedule for the current items and a grid of `grid` CTAs.
int rebuild_schedule(como3r_graph* g, int cfg, int grid, int wv, int wp, cudaStream_t s) {
  const int W = grid * residual_reduce_workers_per_cta(cfg);
  if (W > g->max_warps) return set_error(COMO3R_ERR_UNSUPPORTED, "K1 grid larger than the schedule buffers");
  CK(launch_schedule(g->midx, g->d_es, g->d_items, g->num_items, g->d_item_off, g->plan.E, W, wv, wp, g->d_counts,
                     g->d_cum, g->d_wstart, g->d_wseg, g->d_seg_off, g->k1_compact ? g->d_compact : nullptr, s),
     "schedule");
  return COMO3R_OK;
}

// Cost-weight candidates (valid match, pixel) of a launch configuration's schedule; the
// environment variable COMO3R_K1_WEIGHTS=<wv>,<wp> replaces them (studies).
std::vector<std::pair<int, int>> weight_candidates(int cfg) {
  if (const char* w = getenv("COMO3R_K1_WEIGHTS")) {
    int a = 0, b = 0;
    if (sscanf(w, "%d,%d", &a, &b) == 2 && a >= 0 && b >= 0 && a + b > 0) return {{a, b}};
  }
  int wv = 0, wp = 1;
  residual_reduce_cost_weights(cfg, wv, wp);
  std::vector<std::pair<int, int>> c{{wv, wp}};
  for (int a : {0, 1, 2, 3, 5, 8})
    if (a != wv || wp != 1) c.push_back({a, 1});
  c.push_back({1, 0});  // valid matches only (the precompacted lists skip the index rows)
  return c;
}

int enqueue_linearize(como3r_graph* g, cudaStream_t s, double* cost_hist, const int* iter, double* edge_rec) {
  const HostPlan& p = g->plan;
  CK(launch_edge_prep(g->d_poses, g->d_es, p.E, g->d_T64, g->d_T32, g->d_Ad, s), "edge_prep");
  CK(launch_residual_reduce(p.mode, p.dtype, g->k1_cfg, g->k1_grid, g->points, g->midx, g->d_items, g->num_items,
                            g->d_es, g->d_T64, g->d_T32, g->rp, g->d_partials, sched(g), s),
     "residual_reduce");
  CK(launch_edge_reduce(p.mode, g->d_partials, g->d_seg_off, p.E, g->d_Ad, g->d_edge_M, g->d_edge_b, g->d_edge_cost,
                        g->d_edge_skip, edge_rec, g->d_edge_valid, s),
     "edge_reduce");
  const int nslots = p.slot_begin.back();
  CK(launch_assemble(nslots, g->d_slot_contrib_off, g->d_slot_contrib, g->d_edge_M, g->d_A, p.N, g->d_kf_contrib_off,
                     g->d_kf_contrib, g->d_edge_b, g->d_gvec, p.G, g->d_edge_offset, g->d_edge_cost, g->d_edge_skip,
                     g->d_ginfo, cost_hist, iter, g->d_warn, s),
     "assemble");
  if (g->d_diag_shift) CK(launch_diag_shift(p.G, g->sp, g->d_A, g->d_diag_shift, s), "diag_shift");
  return COMO3R_OK;
}

// The damped factorisation and solve of every graph: the grid-wide or the multi-SM
// variant when one was chosen at create, else one CTA per graph.
// `keep` (the vjp's forward iterations): where a successful factorisation also leaves L.
cudaError_t launch_solver(como3r_graph* g, const double* gvec, double* tau, GraphInfoDev* ginfo, int* warn,
                          cudaStream_t s, FactorKeep keep = {}) {
  if (g->group_ctas > 0)
    return launch_factor_solve_group(g->group_ctas, g->sp, g->d_gtask, g->d_glist, g->d_A, g->d_L, g->d_colscratch,
                                     gvec, tau, g->lambda, g->eps0, g->max_attempts, ginfo, warn, g->d_gfail, s, keep);
  if (g->grid_ctas > 0)
    return launch_factor_solve_grid(g->grid_ctas, g->sp, g->d_A, g->d_L, g->d_colscratch, gvec, tau, g->lambda,
                                    g->eps0, g->max_attempts, ginfo, warn, g->d_gsync, s, keep, g->grid_extra);
  if (g->cluster_ctas > 0)
    return launch_factor_solve_cluster(g->plan.G, g->sp, g->cp, g->cluster_smem, g->d_A, gvec, tau, g->lambda,
                                       g->eps0, g->max_attempts, ginfo, warn, s, keep);
  return launch_factor_solve(g->plan.G, g->sp, g->smem_solve, g->solve_smem, g->d_A, g->d_L, g->d_colscratch, gvec,
                             tau, g->lambda, g->eps0, g->max_attempts, ginfo, warn, s, keep);
}

int enqueue_solve(como3r_graph* g, cudaStream_t s, int* iter, FactorKeep keep = {}) {
  const HostPlan& p = g->plan;
  CK(launch_solver(g, g->d_gvec, g->d_tau, g->d_ginfo, g->d_warn, s, keep), "factor_solve");
  CK(launch_retract(g->d_tau, g->d_poses, g->d_frozen, p.N, iter, s), "retract");
  return COMO3R_OK;
}

int finish_info(como3r_graph* g, como3r_graph_info* info) {
  const HostPlan& p = g->plan;
  if (info) {
    for (int k = 0; k < p.G; ++k) {
      info[k].cost = g->h_ginfo[k].cost;
      info[k].attempts = g->h_ginfo[k].attempts;
      info[k].solved = g->h_ginfo[k].solved;
      info[k].skipped_matches = g->h_ginfo[k].skipped;
      int64_t v = 0;
      for (int e = p.edge_offset[k]; e < p.edge_offset[k + 1]; ++e) v += g->edge_valid[e];
      info[k].valid_matches = v;
    }
  }
  return *g->h_warn;
}

int capture(como3r_graph* g, bool with_solve, cudaGraphExec_t* exec) {
  CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal), "capture begin");
  int rc = enqueue_linearize(g, g->cap, g->d_cost_hist, g->d_iter, nullptr);
  if (!rc && with_solve) rc = enqueue_solve(g, g->cap, g->d_iter);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "capture end");
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_error(e, "graph instantiate");
  return COMO3R_OK;
}

int autotune_k1(como3r_graph* g);

int create_impl(como3r_graph* g, const como3r_graph_desc* d) {
  HostPlan& p = g->plan;
  int rc = build_plan(d, p);
  if (rc) return set_error(rc, p.error);
  CK(cudaGetDevice(&g->device), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device), "attribute");
  // a batch too large for one cluster per graph: CTA groups when they beat one CTA per graph
  // (COMO3R_SOLVE_GROUPS=<k> puts the k slowest graphs on clusters, 0 disables them); a graph
  // solved by a cluster may take the other ordering, and the plan is built again with it
  GroupPlan gp;
  {
    int force = -1;
    bool want = p.G > 1 && kGroupCTAs * p.G > g->sms;
    if (const char* e = getenv("COMO3R_SOLVE_GROUPS")) {
      force = std::max(0, atoi(e));
      want = force > 0 && p.G > 1;
    }
    if (want) build_group_plan(p, g->sms, force, gp);
    if (gp.ctas > 0) {
      bool changed = false;
      for (int k = 0; k < p.G; ++k) changed = changed || (gp.order[k] >= 0 && gp.order[k] != p.order_kind[k]);
      if (changed) {
        HostPlan p2;
        if ((rc = build_plan(d, p2, &gp.order))) return set_error(rc, p2.error);
        p = std::move(p2);
      }
    }
  }
  CK(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking), "stream create");
  g->rp = make_robust_params(d->sigma_ray, d->sigma_dist, d->huber_k);
  g->lambda = d->lambda;
  g->eps0 = d->eps0;
  g->max_attempts = d->max_attempts;
  const size_t bpp = d->dtype == COMO3R_F16 ? 8 : (d->dtype == COMO3R_F32 ? 16 : 32);
  g->points_bytes = (size_t)p.total_px * bpp;
  g->idx_bytes = (size_t)p.total_idx * sizeof(int32_t);
  if (d->copy_inputs) {
    if ((rc = dalloc(g, (char**)&g->own_points, g->points_bytes))) return rc;
    if ((rc = dalloc(g, &g->own_midx, p.total_idx))) return rc;
    CK(cudaMemcpyAsync(g->own_points, d->points_conf, g->points_bytes, cudaMemcpyDefault, g->stream), "copy points");
    if (p.total_idx)
      CK(cudaMemcpyAsync(g->own_midx, d->match_idx, g->idx_bytes, cudaMemcpyDefault, g->stream), "copy matches");
    g->points = g->own_points;
    g->midx = g->own_midx;
  } else {
    if (!is_device_pointer(d->points_conf) || (p.total_idx && !is_device_pointer(d->match_idx)))
      return set_error(COMO3R_ERR_INVALID_ARG, "points_conf / match_idx must be device memory unless copy_inputs = 1");
    if (reinterpret_cast<uintptr_t>(d->points_conf) % 16 || reinterpret_cast<uintptr_t>(d->match_idx) % 4)
      return set_error(COMO3R_ERR_INVALID_ARG, "points_conf must be 16-byte and match_idx 4-byte aligned");
    g->points = d->points_conf;
    g->midx = d->match_idx;
  }
  // K1 work items: allocated for the smallest candidate chunk, chosen by autotune_k1()
  std::vector<Item> items;
  std::vector<int32_t> item_off;
  build_items(p, kChunks[0], items, item_off);
  g->max_items = (int)items.size();
  g->max_warps = g->sms * (2048 / 32);  // the most warps a persistent grid can hold
  // the shared-memory-staged residual kernel copies match indices in 16-byte pieces
  g->idx_rows_aligned = reinterpret_cast<uintptr_t>(g->midx) % 16 == 0 && reinterpret_cast<uintptr_t>(g->points) % 16 == 0;
  for (int k = 0; k < p.N; ++k)
    g->idx_rows_aligned = g->idx_rows_aligned && (p.npix[k] % 4 == 0) && p.npix[k] <= (1 << 22);
  g->k1_compact = g->idx_rows_aligned;
  const int E = p.E, N = p.N, G = p.G;
  const int nslots = p.slot_begin.back(), ncols = p.col_begin.back();
  if ((rc = upload(g, &g->d_es, p.es)) || (rc = upload(g, &g->d_items, items)) ||
      (rc = upload(g, &g->d_item_off, item_off)) || (rc = dalloc(g, &g->d_T64, (size_t)E * 12)) ||
      (rc = dalloc(g, &g->d_T32, (size_t)E * 16)) || (rc = dalloc(g, &g->d_Ad, (size_t)E * 49)) ||
      (rc = dalloc(g, &g->d_partials, (size_t)std::max(g->max_items, g->max_warps + E) * kPartial)) ||
      (g->idx_rows_aligned && (rc = dalloc(g, &g->d_compact, (size_t)g->max_items * kCompactSlot))) ||
      (rc = dalloc(g, &g->d_counts, (size_t)g->max_items)) || (rc = dalloc(g, &g->d_cum, (size_t)g->max_items + 1)) ||
      (rc = dalloc(g, &g->d_wstart, (size_t)g->max_warps + 1)) || (rc = dalloc(g, &g->d_wseg, (size_t)g->max_warps)) ||
      (rc = dalloc(g, &g->d_seg_off, (size_t)E + 1)) ||
      (rc = dalloc(g, &g->d_edge_M, (size_t)E * 49)) || (rc = dalloc(g, &g->d_edge_b, (size_t)E * 7)) ||
      (rc = dalloc(g, &g->d_edge_cost, E)) || (rc = dalloc(g, &g->d_edge_skip, E)) ||
      (rc = dalloc(g, &g->d_edge_valid, E)) || (rc = upload(g, &g->d_slot_kf_r, p.slot_kf_r)) ||
      (rc = upload(g, &g->d_slot_kf_c, p.slot_kf_c)) || (rc = upload(g, &g->d_slot_contrib_off, p.slot_contrib_off)) ||
      (rc = upload(g, &g->d_slot_contrib, p.slot_contrib)) ||
      (rc = upload(g, &g->d_kf_contrib_off, p.kf_contrib_off)) || (rc = upload(g, &g->d_kf_contrib, p.kf_contrib)) ||
      (rc = upload(g, &g->d_edge_offset, p.edge_offset)) || (rc = dalloc(g, &g->d_A, (size_t)nslots * 49)) ||
      (rc = dalloc(g, &g->d_L, (size_t)nslots * 49)) ||
      (rc = dalloc(g, &g->d_colscratch, (size_t)ncols * kColScratch)) ||
 (rc = dalloc(g, &g->d_gvec, (size_t)N * 7)) ||
      (rc = dalloc(g, &g->d_tau, (size_t)N * 7)) || (rc = upload(g, &g->d_frozen, p.frozen)) ||
      (rc = dalloc(g, &g->d_ginfo, G)) || (rc = dalloc(g, &g->d_start_ns, 1)) || (rc = dalloc(g, &g->d_iter, 1)) || (rc = dalloc(g, &g->d_warn, 1)) ||
      (rc = dalloc(g, &g->d_poses, (size_t)N * 8)) || (rc = dalloc(g, &g->d_bad, 1)))
    return rc;
  // solver plan
  int32_t *meta, *col_kf, *lcol_slot, *lslot_row, *lsched, *llvl, *lrow_off;
  int4 *ltri, *lutask;
  int2 *lttask, *lrow_ent;
  if ((rc = upload(g, &meta, p.meta)) || (rc = upload(g, &col_kf, p.col_kf)) ||
      (rc = upload(g, &lcol_slot, p.lcol_slot)) || (rc = upload(g, &lslot_row, p.lslot_row)) ||
      (rc = upload(g, &lsched, p.lsched)) || (rc = upload(g, &ltri, p.ltri)) || (rc = upload(g, &lutask, p.lutask)) ||
      (rc = upload(g, &lttask, p.lttask)) || (rc = upload(g, &llvl, p.llvl)) ||
      (rc = upload(g, &lrow_off, p.lrow_off)) || (rc = upload(g, &lrow_ent, p.lrow_ent)))
    return rc;
  g->sp = SolverPlan{meta, col_kf, lcol_slot, lslot_row, lsched, ltri, lutask, lttask, llvl, lrow_off, lrow_ent};
  // test setting COMO3R_TEST_DIAG_SHIFT=<s0>,<s1>,...: graph g's assembled diagonal is
  // lowered by s_g before every solve (missing entries 0), which makes the first epsilon
  // attempts fail by construction; off unless the variable is set
  if (const char* e = getenv("COMO3R_TEST_DIAG_SHIFT")) {
    std::vector<double> sh(p.G, 0.0);
    const char* c = e;
    for (int k = 0; k < p.G && *c; ++k) {
      char* end = nullptr;
      sh[k] = strtod(c, &end);
      if (end == c) return set_error(COMO3R_ERR_INVALID_ARG, "COMO3R_TEST_DIAG_SHIFT: expected numbers separated by commas");
      c = *end == ',' ? end + 1 : end;
    }
    if ((rc = upload(g, &g->d_diag_shift, sh))) return rc;
  }
  CK(cudaMallocHost(&g->h_ginfo, sizeof(GraphInfoDev) * G), "cudaMallocHost");
  CK(cudaMallocHost(&g->h_warn, sizeof(int)), "cudaMallocHost");
  CK(cudaMemsetAsync(g->d_tau, 0, sizeof(double) * 7 * (size_t)N, g->stream), "memset");
  CK(cudaMemsetAsync(g->d_ginfo, 0, sizeof(GraphInfoDev) * G, g->stream), "memset");
  CK(residual_reduce_prepare(), "residual kernel smem attribute");
  // shared-memory factor when every graph fits
  const size_t smax = factor_solve_max_smem();
  g->smem_solve = p.max_graph_smem <= smax;
  if (gp.ctas > 0) {
    if ((rc = upload(g, &g->d_gtask, gp.gtask)) || (rc = upload(g, &g->d_glist, gp.glist)) ||
        (rc = dalloc(g, &g->d_gfail, (size_t)2 * p.G)))
      return rc;
    CK(cudaMemsetAsync(g->d_gfail, 0, sizeof(int) * 2 * (size_t)p.G, g->stream), "memset");
    g->group_ctas = gp.ctas;
    g->group_big = gp.big;
  }
  // multi-SM solve for a few large graphs (it needs the graphs' clusters to fit on the GPU):
  // eight CTAs per graph, or sixteen (a non-portable cluster size) when a factor does not fit
  // eight CTAs' shared memory and the GPU can schedule such a cluster;
  // COMO3R_SOLVE_CLUSTER=<C> forces C CTAs per graph, 0 disables it
  if (g->group_ctas == 0) {
    int C = 0, max_col = 0;
    for (int k = 0; k < p.G; ++k) max_col = std::max(max_col, p.col_begin[k + 1] - p.col_begin[k]);
    if (max_col >= 32 && 8 * p.G <= g->sms) C = 8;
    const char* force_c = getenv("COMO3R_SOLVE_CLUSTER");
    if (force_c) C = std::max(0, std::min(16, atoi(force_c)));
    if (C > 1) {
      HostClusterPlan hc;
      build_cluster_plan(p, C, hc);
      if (!force_c && hc.max_cta_smem > smax && 16 * p.G <= g->sms) {
        HostClusterPlan h16;
        build_cluster_plan(p, 16, h16);
        if (h16.max_cta_smem <= smax && factor_solve_cluster_max_active(h16.max_cta_smem, 16) > 0) {
          hc = std::move(h16);
          C = 16;
        }
      }
      if (hc.max_cta_smem <= smax) {
        int32_t *cmeta, *csched, *clvl, *own, *shome, *chome;
        int4 *cut, *ctri;
        int2* ctt;
        if ((rc = upload(g, &cmeta, hc.cmeta)) || (rc = upload(g, &csched, hc.csched)) ||
            (rc = upload(g, &clvl, hc.clvl)) || (rc = upload(g, &own, hc.own_slot)) ||
            (rc = upload(g, &shome, hc.slot_home)) || (rc = upload(g, &chome, hc.col_home)) ||
            (rc = upload(g, &cut, hc.cutask)) || (rc = upload(g, &ctt, hc.cttask)) || (rc = upload(g, &ctri, hc.ctri)))
          return rc;
        g->cp = ClusterPlan{C, cmeta, csched, cut, ctt, clvl, own, shome, chome, ctri};
        g->cluster_smem = hc.max_cta_smem;
        CK(factor_solve_cluster_prepare(g->cluster_smem, C), "cluster solver attributes");
        g->cluster_ctas = C;
      }
    }
  }
  // grid-wide solve for one graph whose factor fits neither one SM nor a cluster
  // (COMO3R_SOLVE_GRID=0 disables it, =1 forces it for any one-graph plan)
  if (p.G == 1 && g->cluster_ctas == 0) {
    const int ncol = p.col_begin[1] - p.col_begin[0];
    bool want = !g->smem_solve && ncol >= 64;
    if (const char* e = getenv("COMO3R_SOLVE_GRID")) want = atoi(e) != 0;
    const int ctas = want ? factor_solve_grid_ctas() : 0;
    if (ctas > 0) {
      if ((rc = dalloc(g, &g->d_gsync, 1))) return rc;
      CK(cudaMemsetAsync(g->d_gsync, 0, sizeof(GridSync), g->stream), "memset");
      g->grid_ctas = ctas;
      // test setting: arrivals that never come, so every barrier wait runs out its limit
      if (const char* e = getenv("COMO3R_GRID_BARRIER_EXTRA")) g->grid_extra = (unsigned)std::max(0, atoi(e));
    }
  }
  if (g->smem_solve) {
    g->solve_smem = p.max_graph_smem;
    CK(factor_solve_prepare(g->solve_smem), "solver smem attribute");
  }
  {  // the kept-factor substitution of the vjp: its vector, plan and (if they fit) the kept
     // factor in shared memory
    size_t z = 16, zf = 16;
    for (int k = 0; k < G; ++k) {
      const int32_t* m = p.meta.data() + kMetaCount * k;
      const size_t b = substitute_smem_bytes(m[kMetaNSlot], m[kMetaNCol], m[kMetaNLvl]);
      z = std::max(z, b);
      zf = std::max(zf, b + substitute_factor_bytes(m[kMetaNSlot], m[kMetaNCol]));
    }
    // test setting: 0 forces global memory, 1 keeps the factor out of shared memory
    const char* e = getenv("COMO3R_SUBSTITUTE_SMEM");
    const int want = e ? atoi(e) : 2;
    const size_t smax = factor_solve_max_smem();
    if (want >= 2 && zf <= smax) {
      g->sub_smem = zf;
      g->sub_fsmem = true;
    } else if (want >= 1 && z <= smax) {
      g->sub_smem = z;
    }
    if (g->sub_smem) CK(factor_substitute_prepare(g->sub_smem, g->sub_fsmem), "substitute smem attribute");
  }
  // match index check and valid counts
  CK(cudaMemsetAsync(g->d_bad, 0, sizeof(unsigned long long), g->stream), "memset");
  CK(cudaMemsetAsync(g->d_edge_valid, 0, sizeof(long long) * std::max(E, 1), g->stream), "memset");
  CK(launch_check_matches(g->midx, g->d_es, E, g->d_bad, g->d_edge_valid, g->stream), "check_matches");
  unsigned long long bad = 0;
  g->edge_valid.assign(E, 0);
  CK(cudaMemcpyAsync(&bad, g->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, g->stream), "readback");
  if (E) CK(cudaMemcpyAsync(g->edge_valid.data(), g->d_edge_valid, sizeof(long long) * E, cudaMemcpyDeviceToHost, g->stream), "readback");
  CK(cudaStreamSynchronize(g->stream), "create sync");
  if (bad) return set_error(COMO3R_ERR_INVALID_ARG, std::to_string(bad) + " match indices outside [-1, P_j)");
  return autotune_k1(g);
}

// Chooses K1's (chunk, CTA residency) by timing every candidate on this graph's data
// with CUDA events (identity poses: the arithmetic per match does not depend on them).
int autotune_k1(como3r_graph* g) {
  const HostPlan& p = g->plan;
  std::vector<double> ident((size_t)p.N * 8, 0.0);
  for (int k = 0; k < p.N; ++k) ident[8 * k + 6] = ident[8 * k + 7] = 1.0;
  CK(cudaMemcpyAsync(g->d_poses, ident.data(), sizeof(double) * ident.size(), cudaMemcpyHostToDevice, g->stream),
     "tune poses");
  CK(launch_edge_prep(g->d_poses, g->d_es, p.E, g->d_T64, g->d_T32, g->d_Ad, g->stream), "tune edge_prep");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  int best_chunk = kChunks[0], best_cfg = 0;
  // COMO3R_K1_CFG=<n> restricts the search to one launch configuration (tests, studies)
  const char* force = getenv("COMO3R_K1_CFG");
  const int forced = force ? atoi(force) : -1;
  // COMO3R_K1_CHUNK=<n> restricts it to work items of n pixels (with COMO3R_K1_CFG and
  // COMO3R_K1_WEIGHTS the residual kernel's schedule, and so its rounding, is then fixed)
  const char* force_chunk = getenv("COMO3R_K1_CHUNK");
  const int forced_chunk = force_chunk ? atoi(force_chunk) : 0;
  // FP64 launches are long (the FP64 pipe bounds them): try two chunk sizes only
  const int nchunks = p.mode == COMO3R_MIXED ? (int)(sizeof(kChunks) / sizeof(kChunks[0])) : 2;
  std::vector<Item> items;
  std::vector<int32_t> item_off;
  int rc = COMO3R_OK;
  for (int ci = 0; ci < nchunks && !rc; ++ci) {
    const int chunk = kChunks[ci];
    if (forced_chunk > 0 && chunk != forced_chunk) continue;
    build_items(p, chunk, items, item_off);
    CK(cudaMemcpyAsync(g->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, g->stream),
       "tune items");
    CK(cudaMemcpyAsync(g->d_item_off, item_off.data(), sizeof(int32_t) * item_off.size(), cudaMemcpyHostToDevice,
                       g->stream),
       "tune items");
    g->num_items = (int)items.size();
    for (int cfg = 0; cfg < residual_reduce_num_cfgs(p.mode); ++cfg) {
      const int need = residual_reduce_cfg_chunk(cfg);
      if (need && (chunk != need || !g->idx_rows_aligned)) continue;
      if (forced >= 0 && cfg != forced) continue;
      if (p.mode == COMO3R_PLAIN_FP64 && forced < 0 && cfg != 1 && cfg != 4) continue;
      const int occ = residual_reduce_max_blocks_per_sm(p.mode, p.dtype, cfg);
      if (occ <= 0) continue;
      const int warps_per_cta = residual_reduce_block() / 32;
      const int grid = std::max(1, std::min(g->sms * std::max(occ, 1), ((int)items.size() + warps_per_cta - 1) / warps_per_cta));
      for (const auto& wt : weight_candidates(cfg)) {
        if ((rc = rebuild_schedule(g, cfg, grid, wt.first, wt.second, g->stream))) break;
        float tot = 0.f;
        for (int r = 0; r < 4; ++r) {
          cudaError_t err = cudaEventRecord(e0, g->stream);
          if (!err) err = launch_residual_reduce(p.mode, p.dtype, cfg, grid, g->points, g->midx, g->d_items,
                                                 (int)items.size(), g->d_es, g->d_T64, g->d_T32, g->rp, g->d_partials,
                                                 sched(g), g->stream);
          if (!err) err = cudaEventRecord(e1, g->stream);
          if (!err) err = cudaEventSynchronize(e1);
          if (err) {
            rc = cuda_error(err, "autotune");
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (r > 0) tot += ms;  // first run warms caches and clocks
        }
        if (rc) break;
        if (tot / 3 < best) {
          best = tot / 3;
          best_chunk = chunk;
          best_cfg = cfg;
          g->k1_wv = wt.first;
          g->k1_wp = wt.second;
        }
      }
      if (rc) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  build_items(p, best_chunk, items, item_off);
  CK(cudaMemcpyAsync(g->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, g->stream),
     "items");
  CK(cudaMemcpyAsync(g->d_item_off, item_off.data(), sizeof(int32_t) * item_off.size(), cudaMemcpyHostToDevice,
                     g->stream),
     "items");
  g->num_items = (int)items.size();
  g->k1_chunk = best_chunk;
  g->k1_cfg = best_cfg;
  g->k1_tuned_ms = best;
  const int occ = residual_reduce_max_blocks_per_sm(p.mode, p.dtype, best_cfg);
  const int warps_per_cta = residual_reduce_block() / 32;
  g->k1_grid = std::max(1, std::min(g->sms * std::max(occ, 1), (g->num_items + warps_per_cta - 1) / warps_per_cta));
  if ((rc = rebuild_schedule(g, g->k1_cfg, g->k1_grid, g->k1_wv, g->k1_wp, g->stream))) return rc;
  CK(cudaStreamSynchronize(g->stream), "tune sync");
  return COMO3R_OK;
}

int begin_call(como3r_graph* g, const double* poses) {
  if (!g) return set_error(COMO3R_ERR_INVALID_ARG, "graph handle is NULL");
  if (!poses) return set_error(COMO3R_ERR_INVALID_ARG, "poses is NULL");
  CK(cudaMemcpyAsync(g->d_poses, poses, sizeof(double) * 8 * (size_t)g->plan.N, cudaMemcpyDefault, g->stream),
     "poses in");
  CK(cudaMemsetAsync(g->d_warn, 0, sizeof(int), g->stream), "memset");
  return COMO3R_OK;
}

int end_call(como3r_graph* g, double* poses_out) {
  if (poses_out)
    CK(cudaMemcpyAsync(poses_out, g->d_poses, sizeof(double) * 8 * (size_t)g->plan.N, cudaMemcpyDefault, g->stream),
       "poses out");
  CK(cudaMemcpyAsync(g->h_ginfo, g->d_ginfo, sizeof(GraphInfoDev) * g->plan.G, cudaMemcpyDeviceToHost, g->stream),
     "info");
  CK(cudaMemcpyAsync(g->h_warn, g->d_warn, sizeof(int), cudaMemcpyDeviceToHost, g->stream), "info");
  CK(cudaStreamSynchronize(g->stream), "sync");
  return COMO3R_OK;
}

}  // namespace

extern "C" {

int como3r_graph_create(const como3r_graph_desc* desc, void* cuda_stream, como3r_graph_t* out) {
  if (!out) return set_error(COMO3R_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  como3r_graph* g = new (std::nothrow) como3r_graph();
  if (!g) return set_error(COMO3R_ERR_OOM, "host allocation failed");
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  const int rc = create_impl(g, desc);
  if (rc) {
    cudaStreamSynchronize(g->stream);
    free_all(g);
    delete g;
    return rc;
  }
  *out = g;
  return COMO3R_OK;
}

void como3r_graph_destroy(como3r_graph_t g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  free_all(g);
  delete g;
}

int como3r_gn_step(como3r_graph_t g, double* poses, double* H_out, double* g_out, como3r_graph_info* info) {
  int rc = begin_call(g, poses);
  if (rc) return rc;
  const HostPlan& p = g->plan;
  CK(launch_stamp(g->d_start_ns, g->stream), "stamp");
  if ((rc = enqueue_linearize(g, g->stream, nullptr, nullptr, nullptr))) return rc;
  int64_t launches = 5;
  if (H_out || g_out) {
    if (H_out)
      CK(cudaMemsetAsync(H_out, 0, sizeof(double) * 49 * (size_t)p.N * p.N, g->stream), "memset H_out");
    CK(launch_export_dense(p.slot_begin.back(), g->d_slot_kf_r, g->d_slot_kf_c, g->d_A, p.N, g->d_gvec, H_out, g_out,
                           g->stream),
       "export");
    ++launches;
  }
  if ((rc = enqueue_solve(g, g->stream, nullptr))) return rc;
  g->last_launches = launches + 2;
  if ((rc = end_call(g, poses))) return rc;
  return finish_info(g, info);
}

int como3r_solve(como3r_graph_t g, double* poses, int32_t iters, double* cost_trace, como3r_graph_info* info) {
  if (g && iters < 0) return set_error(COMO3R_ERR_INVALID_ARG, "iters must be >= 0");
  int rc = begin_call(g, poses);
  if (rc) return rc;
  const int64_t need = (int64_t)(iters + 1) * g->plan.G;
  if (need > g->cost_hist_cap) {
    // graphs hold the trace pointer: rebuild them around a larger buffer
    cudaStreamSynchronize(g->stream);
    if (g->iter_exec) cudaGraphExecDestroy(g->iter_exec);
    if (g->eval_exec) cudaGraphExecDestroy(g->eval_exec);
    g->iter_exec = g->eval_exec = nullptr;
    const int64_t cap = std::max<int64_t>(need, 64 * (int64_t)g->plan.G);
    if ((rc = dalloc(g, &g->d_cost_hist, (size_t)cap))) return rc;
    g->cost_hist_cap = cap;
  }
  if (!g->iter_exec && (rc = capture(g, true, &g->iter_exec))) return rc;
  if (!g->eval_exec && (rc = capture(g, false, &g->eval_exec))) return rc;
  CK(cudaMemsetAsync(g->d_iter, 0, sizeof(int), g->stream), "memset");
  CK(launch_stamp(g->d_start_ns, g->stream), "stamp");
  for (int k = 0; k < iters; ++k) CK(cudaGraphLaunch(g->iter_exec, g->stream), "graph launch");
  CK(cudaGraphLaunch(g->eval_exec, g->stream), "graph launch");
  g->last_launches = 6 * (int64_t)iters + 5;
  if (cost_trace)
    CK(cudaMemcpyAsync(cost_trace, g->d_cost_hist, sizeof(double) * need, cudaMemcpyDeviceToHost, g->stream),
       "trace");
  if ((rc = end_call(g, poses))) return rc;
  return finish_info(g, info);
}

int como3r_last_step(como3r_graph_t g, double* tau_out) {
  if (!g) return set_error(COMO3R_ERR_INVALID_ARG, "graph handle is NULL");
  if (!tau_out) return set_error(COMO3R_ERR_INVALID_ARG, "tau_out is NULL");
  CK(cudaMemcpyAsync(tau_out, g->d_tau, sizeof(double) * 7 * (size_t)g->plan.N, cudaMemcpyDefault, g->stream),
     "step out");
  CK(cudaStreamSynchronize(g->stream), "sync");
  return COMO3R_OK;
}

int como3r_solve_timestamps(como3r_graph_t g, int64_t* start_ns, int64_t* done_ns) {
  if (!g) return set_error(COMO3R_ERR_INVALID_ARG, "graph handle is NULL");
  const int G = g->plan.G;
  long long t0 = 0;
  CK(cudaMemcpyAsync(&t0, g->d_start_ns, sizeof(t0), cudaMemcpyDeviceToHost, g->stream), "readback");
  CK(cudaMemcpyAsync(g->h_ginfo, g->d_ginfo, sizeof(GraphInfoDev) * G, cudaMemcpyDeviceToHost, g->stream),
     "readback");
  CK(cudaStreamSynchronize(g->stream), "sync");
  if (start_ns) *start_ns = t0;
  if (done_ns)
    for (int k = 0; k < G; ++k) done_ns[k] = g->h_ginfo[k].done_ns;
  return COMO3R_OK;
}

int como3r_depth_setup(como3r_graph_t g, const como3r_depth_desc* d, int64_t* num_segments) {
  if (!g || !d || !d->labels) return set_error(COMO3R_ERR_INVALID_ARG, "graph, desc and desc->labels must be non-NULL");
  if (!(d->sigma_point > 0) || !(d->lambda_smooth >= 0) || !(d->lambda_prior >= 0) || !(d->lambda_lm >= 0) ||
      !(d->eta_max > 0) || d->min_pixels < 1 || !(d->c_min == d->c_min))
    return set_error(COMO3R_ERR_INVALID_ARG, "depth parameters out of range");
  depth_free(g->depth);
  g->depth = nullptr;
  return depth_setup(g->plan, g->points, g->plan.dtype, g->plan.mode, d->labels, d, g->stream, &g->depth,
                     num_segments);
}

int como3r_depth_refine(como3r_graph_t g, const double* poses, double* eta, int32_t iters, double* cost_trace,
                        void* points_out, float* match_ms) {
  if (!g) return set_error(COMO3R_ERR_INVALID_ARG, "graph handle is NULL");
  if (!g->depth) return set_error(COMO3R_ERR_INVALID_ARG, "como3r_depth_setup was not called");
  if (iters < 0 || !eta) return set_error(COMO3R_ERR_INVALID_ARG, "iters must be >= 0 and eta non-NULL");
  int rc = begin_call(g, poses);
  if (rc) return rc;
  const HostPlan& p = g->plan;
  CK(launch_edge_prep(g->d_poses, g->d_es, p.E, g->d_T64, g->d_T32, g->d_Ad, g->stream), "edge_prep");
  g->last_launches = 1 + 2 * ((int64_t)iters + 1) + (points_out ? 1 : 0);
  const bool lists = g->k1_compact && g->k1_chunk <= kCompactSlot;
  return depth_run(g->depth, p, g->d_items, g->num_items, g->d_es, g->midx, lists ? g->d_counts : nullptr,
                   lists ? g->d_compact : nullptr, g->d_T64, g->d_T32, g->rp.kappa, g->sms, eta, iters, cost_trace,
                   points_out, g->points, match_ms, g->stream);
}

int como3r_linearize(como3r_graph_t g, const double* poses, double* edge_out, double* cost_out) {
  int rc = begin_call(g, poses);
  if (rc) return rc;
  if ((rc = enqueue_linearize(g, g->stream, nullptr, nullptr, edge_out))) return rc;
  g->last_launches = 4;
  if ((rc = end_call(g, nullptr))) return rc;
  if (cost_out)
    for (int k = 0; k < g->plan.G; ++k) cost_out[k] = g->h_ginfo[k].cost;
  return *g->h_warn & COMO3R_WARN_SKIPPED;
}

}  // extern "C"

namespace {
// CUDA events of one timed adjoint call: ev[0] start, ev[1] after the forward pass,
// ev[2] after the envelope pass, ev[3] end; ev[4 + 2k], ev[5 + 2k] around the per-match
// adjoint kernel of backward step k.
struct VjpEvents {
  std::vector<cudaEvent_t> ev;
};

int vjp_impl(como3r_graph_t g, const double* poses_init, int32_t iters, int32_t mode, double upstream,
             float* grad_logdepth, float* grad_conf, double* poses_out, double* loss_out, VjpEvents* tm) {
  auto mark = [&](int k) -> cudaError_t { return tm ? cudaEventRecord(tm->ev[k], g->stream) : cudaSuccess; };
  if (!g) return set_error(COMO3R_ERR_INVALID_ARG, "graph handle is NULL");
  if (iters < 0) return set_error(COMO3R_ERR_INVALID_ARG, "iters must be >= 0");
  if (mode != COMO3R_VJP_UNROLLED && mode != COMO3R_VJP_ENVELOPE)
    return set_error(COMO3R_ERR_INVALID_ARG, "mode must be COMO3R_VJP_UNROLLED or COMO3R_VJP_ENVELOPE");
  if (!grad_logdepth || !grad_conf) return set_error(COMO3R_ERR_INVALID_ARG, "gradient outputs are NULL");
  if (!is_device_pointer(grad_logdepth) || !is_device_pointer(grad_conf))
    return set_error(COMO3R_ERR_INVALID_ARG, "gradient outputs must be device memory");
  if (mode == COMO3R_VJP_UNROLLED && g->lambda != 0.0)
    return set_error(COMO3R_ERR_UNSUPPORTED, "the unrolled adjoint requires lambda = 0");
  const HostPlan& p = g->plan;
  const int N = p.N, E = p.E, G = p.G;
  const int64_t P = p.total_px;
  int rc;
  const size_t keep_L = (size_t)p.slot_begin.back() * 49, keep_S = (size_t)p.col_begin.back() * kColScratch;
  if (iters > g->vjp_iters_cap) {
    const int cap = std::max<int>(iters, 8);
    CK(cudaStreamSynchronize(g->stream), "sync");
    if ((rc = dalloc(g, &g->d_ckpt, (size_t)(cap + 1) * 8 * N)) || (rc = dalloc(g, &g->d_tau_hist, (size_t)cap * 7 * N)) ||
        (rc = dalloc(g, &g->d_ginfo_hist, (size_t)cap * G)) || (rc = dalloc(g, &g->d_keep_L, (size_t)cap * keep_L)) ||
        (rc = dalloc(g, &g->d_keep_S, (size_t)cap * keep_S)))
      return rc;
    if (g->vjp_iters_cap < 0 &&
        ((rc = dalloc(g, &g->d_ginfo_final, G)) ||
         (g->sub_smem == 0 && (rc = dalloc(g, &g->d_sub_z, (size_t)7 * p.col_begin.back()))) ||
         (rc = dalloc(g, &g->d_adj_a, (size_t)7 * N)) ||
         (rc = dalloc(g, &g->d_adj_a2, (size_t)7 * N)) || (rc = dalloc(g, &g->d_adj_rhs, (size_t)7 * N)) ||
         (rc = dalloc(g, &g->d_adj_u, (size_t)7 * N)) || (rc = dalloc(g, &g->d_evec, (size_t)16 * E)) ||
         (rc = dalloc(g, &g->d_adj_rec, (size_t)kAdjointRecord * std::max(g->max_items, 1))) ||
         (rc = dalloc(g, &g->d_edge_adj, (size_t)14 * E)) ||
         (p.mode == COMO3R_PLAIN_FP64 && (rc = dalloc(g, &g->d_gacc, (size_t)2 * P)))))
      return rc;
    g->vjp_iters_cap = cap;
  }
  if ((rc = begin_call(g, poses_init))) return rc;
  cudaStream_t s = g->stream;
  int64_t launches = 0;
  CK(mark(0), "event");
  // forward with checkpoints: T^k, tau_k, the solve outcome and the factor of every iteration
  auto keep_of = [&](int k) { return FactorKeep{g->d_keep_L + (size_t)k * keep_L, g->d_keep_S + (size_t)k * keep_S}; };
  for (int k = 0; k < iters; ++k) {
    CK(cudaMemcpyAsync(g->d_ckpt + (size_t)k * 8 * N, g->d_poses, sizeof(double) * 8 * N, cudaMemcpyDeviceToDevice, s),
       "checkpoint");
    if ((rc = enqueue_linearize(g, s, nullptr, nullptr, nullptr)) || (rc = enqueue_solve(g, s, nullptr, keep_of(k))))
      return rc;
    CK(cudaMemcpyAsync(g->d_tau_hist + (size_t)k * 7 * N, g->d_tau, sizeof(double) * 7 * N, cudaMemcpyDeviceToDevice,
                       s),
       "checkpoint");
    CK(cudaMemcpyAsync(g->d_ginfo_hist + (size_t)k * G, g->d_ginfo, sizeof(GraphInfoDev) * G, cudaMemcpyDeviceToDevice,
                       s),
       "checkpoint");
    launches += 6;
  }
  CK(cudaMemcpyAsync(g->d_ckpt + (size_t)iters * 8 * N, g->d_poses, sizeof(double) * 8 * N, cudaMemcpyDeviceToDevice, s),
     "checkpoint");
  CK(mark(1), "event");
  // the refined cost at T^K, its pose gradient g(T^K) and the envelope pixel term
  if ((rc = enqueue_linearize(g, s, nullptr, nullptr, nullptr))) return rc;
  CK(cudaMemcpyAsync(g->d_ginfo_final, g->d_ginfo, sizeof(GraphInfoDev) * G, cudaMemcpyDeviceToDevice, s), "info");
  launches += 4;
  const bool plain = p.mode == COMO3R_PLAIN_FP64;
  void* gl = plain ? (void*)g->d_gacc : (void*)grad_logdepth;
  void* gc = plain ? (void*)(g->d_gacc + P) : (void*)grad_conf;
  CK(cudaMemsetAsync(gl, 0, (plain ? sizeof(double) : sizeof(float)) * (size_t)P, s), "memset");
  CK(cudaMemsetAsync(gc, 0, (plain ? sizeof(double) : sizeof(float)) * (size_t)P, s), "memset");
  // K1's valid-match lists, when its items are small enough to have them
  const bool lists = g->k1_compact && g->k1_chunk <= kCompactSlot;
  const int32_t* lcounts = lists ? g->d_counts : nullptr;
  const uint32_t* lcompact = lists ? g->d_compact : nullptr;
  CK(launch_adjoint_match(p.mode, p.dtype, false, g->points, g->midx, g->d_items, g->num_items, g->d_es, g->d_T64,
                          g->d_T32, nullptr, g->rp, upstream, gl, gc, nullptr, lcounts, lcompact, s),
     "adjoint envelope");
  ++launches;
  CK(mark(2), "event");
  if (mode == COMO3R_VJP_UNROLLED && iters > 0) {
    CK(launch_adjoint_gather(nullptr, nullptr, nullptr, nullptr, g->d_frozen, N, g->d_gvec, upstream, g->d_adj_a, s),
       "adjoint start");
    ++launches;
    for (int k = iters - 1; k >= 0; --k) {
      const double* tau_k = g->d_tau_hist + (size_t)k * 7 * N;
      CK(launch_adjoint_keyframe(g->d_adj_a, tau_k, g->d_frozen, N, g->d_adj_a2, g->d_adj_rhs, s), "adjoint keyframe");
      CK(cudaMemcpyAsync(g->d_poses, g->d_ckpt + (size_t)k * 8 * N, sizeof(double) * 8 * N, cudaMemcpyDeviceToDevice,
                         s),
         "restore");
      // the edge transforms at T^k; H(T^k) is not formed again: its factor was kept
      CK(launch_edge_prep(g->d_poses, g->d_es, p.E, g->d_T64, g->d_T32, g->d_Ad, s), "edge_prep");
      CK(cudaMemsetAsync(g->d_adj_u, 0, sizeof(double) * 7 * N, s), "memset");
      CK(launch_factor_substitute(G, g->sp, keep_of(k), g->d_ginfo_hist + (size_t)k * G, g->d_adj_rhs, g->d_adj_u,
                                  g->sub_smem, g->d_sub_z, s, g->sub_fsmem),
         "adjoint solve");
      CK(launch_adjoint_edge_prep(p.mode, g->d_es, E, g->d_Ad, g->d_adj_u, tau_k, g->d_evec, s), "adjoint edge prep");
      CK(mark(4 + 2 * k), "event");
      CK(launch_adjoint_match(p.mode, p.dtype, true, g->points, g->midx, g->d_items, g->num_items, g->d_es, g->d_T64,
                              g->d_T32, g->d_evec, g->rp, -1.0, gl, gc, g->d_adj_rec, lcounts, lcompact, s),
         "adjoint match");
      CK(mark(5 + 2 * k), "event");
      CK(launch_adjoint_edge(g->d_adj_rec, g->d_item_off, E, g->d_es, g->d_Ad, g->d_adj_u, tau_k, g->d_edge_adj, s),
         "adjoint edge");
      CK(launch_adjoint_gather(g->d_adj_a2, g->d_edge_adj, g->d_kf_contrib_off, g->d_kf_contrib, g->d_frozen, N,
                               nullptr, 1.0, g->d_adj_a, s),
         "adjoint gather");
      launches += 7;
    }
    CK(cudaMemcpyAsync(g->d_poses, g->d_ckpt + (size_t)iters * 8 * N, sizeof(double) * 8 * N,
                       cudaMemcpyDeviceToDevice, s),
       "restore");
  }
  CK(mark(3), "event");
  if (plain) {
    CK(launch_to_float(g->d_gacc, grad_logdepth, P, s), "to float");
    CK(launch_to_float(g->d_gacc + P, grad_conf, P, s), "to float");
    launches += 2;
  }
  g->last_launches = launches;
  // the per-graph cost and status of the evaluation at T^K (not of the backward re-solves)
  CK(cudaMemcpyAsync(g->d_ginfo, g->d_ginfo_final, sizeof(GraphInfoDev) * G, cudaMemcpyDeviceToDevice, s), "info");
  if ((rc = end_call(g, poses_out))) return rc;
  if (loss_out)
    for (int k = 0; k < G; ++k) loss_out[k] = g->h_ginfo[k].cost;
  return *g->h_warn;
}

}  // namespace

extern "C" {

int como3r_vjp(como3r_graph_t g, const double* poses_init, int32_t iters, int32_t mode, double upstream,
               float* grad_logdepth, float* grad_conf, double* poses_out, double* loss_out) {
  return vjp_impl(g, poses_init, iters, mode, upstream, grad_logdepth, grad_conf, poses_out, loss_out, nullptr);
}

int como3r_time_vjp(como3r_graph_t g, const double* poses_init, int32_t iters, int32_t reps, float* ms) {
  if (!g || !ms || reps < 1 || iters < 0) return set_error(COMO3R_ERR_INVALID_ARG, "bad time_vjp arguments");
  const int64_t P = g->plan.total_px;
  float* grads = nullptr;
  CK(cudaMalloc(&grads, sizeof(float) * 2 * (size_t)std::max<int64_t>(P, 1)), "cudaMalloc");
  VjpEvents tm;
  tm.ev.resize(4 + 2 * (size_t)iters);
  int rc = COMO3R_OK;
  for (auto& e : tm.ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = set_error(COMO3R_ERR_CUDA, "event create");
  double acc[4] = {0, 0, 0, 0};
  for (int r = 0; r <= reps && rc >= 0; ++r) {  // the first call warms up
    rc = vjp_impl(g, poses_init, iters, COMO3R_VJP_UNROLLED, 1.0, grads, grads + P, nullptr, nullptr, &tm);
    if (rc < 0 || r == 0) continue;
    float a = 0.f, b = 0.f, c = 0.f;
    cudaEventElapsedTime(&a, tm.ev[0], tm.ev[1]);
    cudaEventElapsedTime(&b, tm.ev[1], tm.ev[2]);
    cudaEventElapsedTime(&c, tm.ev[2], tm.ev[3]);
    acc[0] += a;
    acc[1] += b;
    acc[2] += c;
    for (int k = 0; k < iters; ++k) {
      float d = 0.f;
      cudaEventElapsedTime(&d, tm.ev[4 + 2 * k], tm.ev[5 + 2 * k]);
      acc[3] += d;
    }
  }
  for (auto& e : tm.ev)
    if (e) cudaEventDestroy(e);
  cudaFree(grads);
  if (rc < 0) return rc;
  for (int k = 0; k < 4; ++k) ms[k] = (float)(acc[k] / reps);
  return COMO3R_OK;
}

int como3r_points_from_logdepth(const float* rays, const float* logdepth, const float* conf, int64_t n,
                                int32_t dtype, void* points_out, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!rays || !logdepth || !conf || !points_out)))
    return set_error(COMO3R_ERR_INVALID_ARG, "bad points_from_logdepth arguments");
  if (dtype < COMO3R_F16 || dtype > COMO3R_F64) return set_error(COMO3R_ERR_INVALID_ARG, "bad dtype");
  CK(launch_points_from_logdepth(dtype, rays, logdepth, conf, n, points_out, static_cast<cudaStream_t>(cuda_stream)),
     "points_from_logdepth");
  return COMO3R_OK;
}

int como3r_rays_from_points(const void* points, int64_t n, int32_t dtype, float* rays, float* logdepth, float* conf,
                            void* cuda_stream) {
  if (n < 0 || (n > 0 && (!points || !rays || !logdepth || !conf)))
    return set_error(COMO3R_ERR_INVALID_ARG, "bad rays_from_points arguments");
  if (dtype < COMO3R_F16 || dtype > COMO3R_F64) return set_error(COMO3R_ERR_INVALID_ARG, "bad dtype");
  CK(launch_rays_from_points(dtype, points, n, rays, logdepth, conf, static_cast<cudaStream_t>(cuda_stream)),
     "rays_from_points");
  return COMO3R_OK;
}

int como3r_sim3_retract(const double* tau, double* poses, int32_t n, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!tau || !poses))) return set_error(COMO3R_ERR_INVALID_ARG, "bad retract arguments");
  CK(launch_retract(tau, poses, nullptr, n, nullptr, static_cast<cudaStream_t>(cuda_stream)), "retract");
  return COMO3R_OK;
}

int como3r_update_inputs(como3r_graph_t g, const void* points_conf, const int32_t* match_idx) {
  if (!g) return set_error(COMO3R_ERR_INVALID_ARG, "graph handle is NULL");
  if (!g->own_points) return set_error(COMO3R_ERR_INVALID_ARG, "graph was created with copy_inputs = 0");
  if (points_conf)
    CK(cudaMemcpyAsync(g->own_points, points_conf, g->points_bytes, cudaMemcpyDefault, g->stream), "copy points");
  if (match_idx && g->idx_bytes) {
    CK(cudaMemcpyAsync(g->own_midx, match_idx, g->idx_bytes, cudaMemcpyDefault, g->stream), "copy matches");
    // new valid counts: rebalance K1 (device only, no synchronisation)
    const int rc = rebuild_schedule(g, g->k1_cfg, g->k1_grid, g->k1_wv, g->k1_wp, g->stream);
    if (rc) return rc;
  }
  return COMO3R_OK;
}

int como3r_time_stages(como3r_graph_t g, const double* poses, int32_t reps, float* ms) {
  if (!g || !ms || reps < 1) return set_error(COMO3R_ERR_INVALID_ARG, "bad time_stages arguments");
  int rc = begin_call(g, poses);
  if (rc) return rc;
  const HostPlan& p = g->plan;
  cudaEvent_t ev[7];
  for (auto& e : ev) CK(cudaEventCreate(&e), "event create");
  double acc[COMO3R_STAGES] = {0};
  cudaStream_t s = g->stream;
  const int nslots = p.slot_begin.back();
  for (int r = 0; r < reps && !rc; ++r) {
    cudaError_t err = cudaEventRecord(ev[0], s);
    if (!err) err = launch_edge_prep(g->d_poses, g->d_es, p.E, g->d_T64, g->d_T32, g->d_Ad, s);
    if (!err) err = cudaEventRecord(ev[1], s);
    if (!err) err = launch_residual_reduce(p.mode, p.dtype, g->k1_cfg, g->k1_grid, g->points, g->midx, g->d_items,
                                           g->num_items, g->d_es, g->d_T64, g->d_T32, g->rp, g->d_partials, sched(g),
                                           s);
    if (!err) err = cudaEventRecord(ev[2], s);
    if (!err) err = launch_edge_reduce(p.mode, g->d_partials, g->d_seg_off, p.E, g->d_Ad, g->d_edge_M, g->d_edge_b,
                                       g->d_edge_cost, g->d_edge_skip, nullptr, g->d_edge_valid, s);
    if (!err) err = cudaEventRecord(ev[3], s);
    if (!err) err = launch_assemble(nslots, g->d_slot_contrib_off, g->d_slot_contrib, g->d_edge_M, g->d_A, p.N,
                                    g->d_kf_contrib_off, g->d_kf_contrib, g->d_edge_b, g->d_gvec, p.G,
                                    g->d_edge_offset, g->d_edge_cost, g->d_edge_skip, g->d_ginfo, nullptr, nullptr,
                                    g->d_warn, s);
    if (!err) err = cudaEventRecord(ev[4], s);
    if (!err) err = launch_solver(g, g->d_gvec, g->d_tau, g->d_ginfo, g->d_warn, s);
    if (!err) err = cudaEventRecord(ev[5], s);
    if (!err) err = launch_retract(g->d_tau, g->d_poses, g->d_frozen, p.N, nullptr, s);
    if (!err) err = cudaEventRecord(ev[6], s);
    if (!err) err = cudaEventSynchronize(ev[6]);
    if (err) {
      rc = cuda_error(err, "time_stages");
      break;
    }
    for (int k = 0; k < 6; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
    float tot = 0.f;
    cudaEventElapsedTime(&tot, ev[0], ev[6]);
    acc[6] += tot;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  for (int k = 0; k < COMO3R_STAGES; ++k) ms[k] = (float)(acc[k] / reps);
  g->last_launches = 6 * (int64_t)reps;
  return COMO3R_OK;
}

int64_t como3r_last_launch_count(como3r_graph_t g) { return g ? g->last_launches : 0; }

int como3r_graph_stats(como3r_graph_t g, int64_t* stats) {
  if (!g || !stats) return set_error(COMO3R_ERR_INVALID_ARG, "NULL argument");
  plan_stats(g->plan, stats);
  stats[COMO3R_STAT_ITEMS] = g->num_items;
  int64_t v = 0;
  for (long long x : g->edge_valid) v += x;
  stats[COMO3R_STAT_VALID] = v;
  stats[COMO3R_STAT_CHUNK] = g->k1_chunk;
  stats[COMO3R_STAT_BLOCK] = residual_reduce_block() * 100 + g->k1_cfg;
  stats[COMO3R_STAT_GRID] = g->k1_grid;
  stats[COMO3R_STAT_SMEM_SOLVE] = g->smem_solve ? 1 : 0;
  stats[COMO3R_STAT_SOLVE_CTAS] = g->grid_ctas > 0 ? g->grid_ctas
                                 : g->cluster_ctas > 0 ? g->cluster_ctas
                                 : g->group_ctas > 0 ? kGroupCTAs : 1;
  stats[COMO3R_STAT_SOLVE_GROUPS] = g->group_big;
  stats[COMO3R_STAT_K1_STALLS] = residual_reduce_stalls();
  return COMO3R_OK;
}

int como3r_plan_stats(const como3r_graph_desc* desc, int64_t* stats) {
  if (!stats) return set_error(COMO3R_ERR_INVALID_ARG, "stats is NULL");
  HostPlan p;
  const int rc = build_plan(desc, p);
  if (rc) return set_error(rc, p.error);
  plan_stats(p, stats);
  std::vector<Item> items;
  std::vector<int32_t> item_off;
  build_items(p, kDefaultChunk, items, item_off);
  stats[COMO3R_STAT_ITEMS] = (int64_t)items.size();
  stats[COMO3R_STAT_CHUNK] = kDefaultChunk;
  return COMO3R_OK;
}

const char* como3r_status_str(int code) {
  switch (code) {
    case COMO3R_OK: return "ok";
    case COMO3R_WARN_SOLVE_FAILED: return "warning: every factorisation attempt failed in >= 1 graph (zero update)";
    case COMO3R_WARN_SKIPPED: return "warning: degenerate or non-finite matches were skipped";
    case COMO3R_WARN_SOLVE_FAILED | COMO3R_WARN_SKIPPED: return "warning: solve failed and matches skipped";
    case COMO3R_ERR_INVALID_ARG: return "error: invalid argument";
    case COMO3R_ERR_CUDA: return "error: CUDA runtime error";
    case COMO3R_ERR_OOM: return "error: out of device memory";
    case COMO3R_ERR_UNSUPPORTED: return "error: unsupported";
    default: return "unknown status";
  }
}

const char* como3r_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
