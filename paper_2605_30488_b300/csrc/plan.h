// Host-side planning of a batch of pose graphs: validation, fill-reducing ordering,
// symbolic block factorisation, level schedule, assembly lists and K1 work items.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/como3r.h"
#include "como3r_internal.h"

namespace como3r {

struct HostPlan {
  int G = 0, N = 0, E = 0;
  int mode = 1, dtype = 1;
  int64_t total_px = 0, total_idx = 0, valid_hint = 0;
  std::vector<int32_t> kf_offset, edge_offset, anchor;
  std::vector<int32_t> width;     // [G] pointmap width of each graph
  std::vector<int64_t> pix_off;   // [N+1]
  std::vector<int32_t> npix;      // [N]
  std::vector<EdgeStatic> es;     // [E]
  std::vector<uint8_t> frozen;    // [N] anchors
  // solver plan (see SolverPlan)
  // global numbering (assembly, export): columns and slots of graph g start at
  // col_begin[g] / slot_begin[g]; col_slot (global) gives each column's diagonal slot
  std::vector<int32_t> col_begin, slot_begin, col_kf, col_slot;
  // solver plan in per-graph local indices (see SolverPlan)
  std::vector<int32_t> meta, lcol_slot, lslot_row, lsched, llvl;
  std::vector<int4> ltri, lutask;
  std::vector<int2> lttask;
  // blocks of L by block row: per graph ncol + 1 offsets (at col_begin[g] + g) into
  // (local slot, column) entries (graph g's at slot_begin[g] - col_begin[g])
  std::vector<int32_t> lrow_off;
  std::vector<int2> lrow_ent;
  std::vector<int8_t> order_kind;  // per graph: 0 minimum degree, 1 nested dissection
  // per graph, both candidate orderings: elimination-tree levels and block updates
  // (minimum degree, nested dissection), for the CTA-group assignment of batched solves
  std::vector<int32_t> nlev_md, nlev_nd;
  std::vector<int64_t> upd_md, upd_nd;
  std::vector<int32_t> slot_kf_r, slot_kf_c;
  // assembly (entries edge * 2 + negate, in edge order)
  std::vector<int32_t> slot_contrib_off, slot_contrib, kf_contrib_off, kf_contrib;
  int max_levels = 0;
  int64_t fill_blocks = 0;
  size_t max_graph_smem = 0;      // bytes of the largest graph's factor + vectors
  std::string error;
};

// Host side of ClusterPlan (concatenated arrays; see como3r_internal.h).
struct HostClusterPlan {
  int C = 0;
  std::vector<int32_t> cmeta, csched, clvl, own_slot, slot_home, col_home;
  std::vector<int4> cutask, ctri;
  std::vector<int2> cttask;
  size_t max_cta_smem = 0;  // shared memory of the largest (graph, rank) CTA
};

// Splits every graph's columns over C CTAs (see ClusterPlan).
void build_cluster_plan(const HostPlan& p, int C, HostClusterPlan& cp);

// Validates `d` and fills `p`; returns COMO3R_OK or COMO3R_ERR_INVALID_ARG (message in p.error).
// order (optional, per graph): 0 minimum degree, 1 nested dissection, -1 the cheaper one for
// one SM (the default).
int build_plan(const como3r_graph_desc* d, HostPlan& p, const std::vector<int8_t>* order = nullptr);

// CTA groups of a batched solve (factor_solve_group_kernel): per graph the estimated time
// (microseconds) of one CTA with its one-SM ordering, and of a cluster of kGroupCTAs with the
// better ordering for it; the assignment minimising the estimated makespan on `sms` SMs.
struct GroupPlan {
  int ctas = 0;                    // multiple of kGroupCTAs; 0: no group solve
  int big = 0;                     // graphs solved by a whole cluster
  double makespan_us = 0.0, single_us = 0.0;  // estimates: grouped, and one CTA per graph
  std::vector<int4> gtask;         // per CTA (list offset, count, rank, group size)
  std::vector<int32_t> glist;
  std::vector<int8_t> order;       // per graph, for build_plan
};
void build_group_plan(const HostPlan& p, int sms, int force_big, GroupPlan& gp);

// Splits every edge's streamed pixels into items of at most `chunk` pixels.
void build_items(const HostPlan& p, int chunk, std::vector<Item>& items, std::vector<int32_t>& item_off);

// Fills the COMO3R_STAT_* entries that depend on the plan only.
void plan_stats(const HostPlan& p, int64_t* stats);

// Segment-level structure refinement state (k_depth.cu): built by depth_setup from the
// graph's current pointmaps, run by depth_run, released by depth_free.
struct DepthState;
int depth_setup(const HostPlan& p, const void* points, int dtype, int mode, const int32_t* labels,
                const como3r_depth_desc* d, cudaStream_t s, DepthState** out, int64_t* num_segments);
// counts / compact: the residual kernel's valid-match lists of the items (both NULL: none)
int depth_run(DepthState* st, const HostPlan& p, const Item* items, int num_items, const EdgeStatic* es,
              const int32_t* midx, const int32_t* counts, const uint32_t* compact, const double* T64,
              const float* T32, double kappa, int sms, double* eta, int iters, double* cost_trace,
              void* points_out, const void* points_src, float* match_ms, cudaStream_t s);
void depth_free(DepthState* st);

}  // namespace como3r
