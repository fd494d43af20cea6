// Internal declarations shared by the host planner, the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace como3r {

// 8-byte slots per K1 work-item record: [0..24] H_rel unique entries, [25..31] g_rel,
// [32] cost, [33] skipped matches, [34..35] zero.  MIXED: float2 (sum, compensation)
// per slot; PLAIN: double.
constexpr int kPartial = 36;
// Unique nonzero H_rel entries kept by K1 (the (omega, zeta) block is identically zero):
// vv (00 01 02 11 12 22), v-omega (3x3 row-major), omega-omega (00 01 02 11 12 22),
// v-zeta (3), zeta-zeta (1).
constexpr int kHUnique = 25;
constexpr int kEdgeRec = 64;   // exported edge record (doubles)

struct Item {                  // one K1 work item: pixels [begin, end) of edge `edge`
  int32_t edge, begin, end, pad;
};

struct EdgeStatic {            // per edge, fixed at create
  int64_t pix_i;               // first pixel of keyframe i in the packed points
  int64_t pix_j;               // first pixel of keyframe j
  int64_t idx_off;             // first entry of the edge in match_idx
  int32_t i, j;                // global keyframe ids
  int32_t npix_i, npix_j;      // pixel counts of i and j
};

// K1 schedule (k_schedule.cu): warp w of the persistent grid processes items
// [start[w], start[w+1]) and writes its records at seg[w], seg[w] + 1, ... (one per run of
// items of one edge).  With start == nullptr the items are split evenly by count and every
// item gets its own record (zeros unless it ends a run).
struct WarpSched {
  const int32_t* start;
  const int32_t* seg;
  // valid-match lists (or nullptr): item it's counts[it] valid matches, packed
  // (n << 10) | (pixel offset in the item), at compact + it * kCompactSlot
  const int32_t* counts = nullptr;
  const uint32_t* compact = nullptr;
};
constexpr int kCompactSlot = 1024;  // entries per item slot of the valid-match lists

struct RobustParams {          // whitening and Huber constants (Sec. III-A)
  double inv_sigma_ray, inv_sigma_dist;      // 1/sigma_r, 1/sigma_d
  double inv_var_ray, inv_var_dist;          // 1/sigma_r^2, 1/sigma_d^2
  double kappa;
  // FP32 copies for the mixed form, rounded once on the host: a kernel that converted the
  // FP64 values itself could have the conversion rematerialised inside its hot loop, where
  // every FP64-pipe instruction holds the pipe for a whole warp's time
  float f_inv_sigma_ray, f_inv_sigma_dist, f_inv_var_ray, f_inv_var_dist, f_kappa;
  float f_kappa_inv_var_ray, f_kappa_inv_var_dist;  // kappa / sigma_r^2, kappa / sigma_d^2
};

inline RobustParams make_robust_params(double sigma_ray, double sigma_dist, double kappa) {
  RobustParams rp{};
  rp.inv_sigma_ray = 1.0 / sigma_ray;
  rp.inv_sigma_dist = 1.0 / sigma_dist;
  rp.inv_var_ray = 1.0 / (sigma_ray * sigma_ray);
  rp.inv_var_dist = 1.0 / (sigma_dist * sigma_dist);
  rp.kappa = kappa;
  rp.f_inv_sigma_ray = (float)rp.inv_sigma_ray;
  rp.f_inv_sigma_dist = (float)rp.inv_sigma_dist;
  rp.f_inv_var_ray = (float)rp.inv_var_ray;
  rp.f_inv_var_dist = (float)rp.inv_var_dist;
  rp.f_kappa = (float)kappa;
  rp.f_kappa_inv_var_ray = (float)(kappa * rp.inv_var_ray);
  rp.f_kappa_inv_var_dist = (float)(kappa * rp.inv_var_dist);
  return rp;
}

struct GraphInfoDev {          // per graph, written on the device
  double cost;
  int32_t attempts;
  int32_t solved;
  long long skipped;
  long long done_ns;           // %globaltimer when this graph's last factorisation ended
};

#ifdef __CUDACC__
// FP32 -> FP64 on the integer ALU (exact for normal numbers and zero; FP32 denormals flush
// to signed zero; inf / NaN keep their class).  On this GPU a warp's FP64-pipe
// instruction -- a conversion included -- takes the pipe for a whole warp's time however
// few lanes are active, so widening in a hot FP32 loop goes through the ALU instead.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  const unsigned ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  unsigned long long bits;
  if (ex == 0u) bits = sgn;
  else if (ex == 0xffu) bits = sgn | (0x7ffull << 52) | ((unsigned long long)man << 29);
  else bits = sgn | ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)man << 29);
  return __longlong_as_double((long long)bits);
}

// Device clock (ns): %globaltimer, the same time base on every SM.
__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#endif

// Solver plan of all graphs (device arrays).  Every index inside a graph's plan is local
// to that graph (slots 0..nslot-1, columns 0..ncol-1 in elimination order, triplets and
// tasks from 0), so a CTA can stage its graph's plan in shared memory as is; meta[g]
// locates the graph's part of each concatenated array.  Slot s is one stored 7x7 block
// (row-major) of the factor.  Each elimination-tree level has three task lists, executed
// in this order with a CTA barrier after each:
//   D: the level's columns (diagonal factorisation + forward substitution);
//   T: (slot, col): the off-diagonal blocks of the level's columns, solved against L_cc;
//   U: right-looking updates from the level's columns to all their ancestors, one task
//      per destination block, (dst, t0, t1, col): L[dst] -= sum_{t0 <= t < t1}
//      L[tri[t].x] L[tri[t].y]^T; col >= 0 marks a diagonal destination, whose task also
//      updates the forward right-hand side of column col with L[tri[t].x] y_{tri[t].w}.
//      The tasks into the next level's columns ("near") come first; the others ("far")
//      run together with the next level's D list.
enum GraphMeta {
  kMetaColBase, kMetaNCol, kMetaSlotBase, kMetaNSlot, kMetaTriBase, kMetaNTri,
  kMetaUBase, kMetaNU, kMetaTBase, kMetaNT, kMetaLvlBase, kMetaNLvl, kMetaCount
};
struct SolverPlan {
  const int32_t* meta;      // [G][kMetaCount]
  const int32_t* col_kf;    // [C] keyframe (global id) of each column, at col_base
  const int32_t* col_slot;  // per graph ncol+1 local slot offsets (diagonal first), at col_base + g
  const int32_t* slot_row;  // local block-row column of each slot, at slot_base
  const int32_t* sched;     // local columns in level order, at col_base
  const int4* tri;          // (src_r, src_k, dst, j) local slots / column, at tri_base
  const int4* utask;        // (dst, t0, t1, col or -1), at u_base
  const int2* ttask;        // (slot, col), at t_base
  const int32_t* lvl;       // per graph (nlev+1) x 4: level offsets in sched, utask (near), utask (far), ttask;
                            // at 4 * lvl_base
  const int32_t* row_off;   // per graph ncol+1 offsets of each block row's entries, at col_base + g
  const int2* row_ent;      // (slot of L_rj, j) by block row r, j ascending, at slot_base - col_base
};

// Multi-SM solve: one thread-block cluster of `C` CTAs per graph.  Every column has an
// owner CTA (round robin within its elimination level) that keeps the column's blocks and
// scratch in its shared memory and runs its diagonal factorisation, off-diagonal solves,
// backward step, and every update whose destination lies in one of its columns (sources
// are read from the owners' shared memory through the cluster window).  Per (graph, rank):
// the owned columns, update tasks and off-diagonal tasks in level order, with offsets
// (nlev + 1) x 4 like SolverPlan::lvl.  Homes are encoded rank << 24 | local index.
// Every CTA of a graph lays out its shared memory identically up to the blocks (column
// scratch for kCNColMax columns first, then the blocks), so a remote column or block is
// found at the same offset as a local one.
// kCTopLocal: the lowest level from which on every level's columns are all owned by rank 0
// (the narrow top of the elimination tree): the back substitution of those levels needs no
// cluster barrier between them (only rank 0 works, and only rank 0 reads their solutions).
// kCTri / kCNTri: the CTA's own triplet list (the triplets of the update tasks it runs, in
// task order; its tasks' triplet ranges index into it), so that a CTA stages only what it
// reads, not the whole graph's list.
enum ClusterMeta {
  kCSched, kCNSched, kCU, kCNU, kCT, kCNT, kCLvl, kCNSlot, kCNCol, kCOwn, kCNColMax, kCTopLocal, kCTri, kCNTri,
  kCMetaCount
};
struct ClusterPlan {
  int C;                    // CTAs per graph
  const int32_t* cmeta;     // [G * C][kCMetaCount]
  const int32_t* csched;    // owned columns (graph-local), level order
  const int4* cutask;       // owned update tasks (graph-local slots), per level near then far
  const int2* cttask;       // owned off-diagonal tasks
  const int32_t* clvl;      // [(nlev + 1) * 4] per (graph, rank)
  const int32_t* own_slot;  // graph-local slot of each local slot, per (graph, rank)
  const int32_t* slot_home; // per slot (at slot_base)
  const int32_t* col_home;  // per column (at col_base)
  const int4* ctri;         // triplets of each (graph, rank)'s update tasks
};

// Bytes of shared memory one graph's factor, per-column scratch and plan occupy.
inline size_t solver_smem_bytes(int nslot, int ncol, int ntri, int nu, int nt, int nlev) {
  auto r16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  size_t b = r16(sizeof(double) * ((size_t)nslot * 49 + (size_t)ncol * 63));
  b += r16(16 * (size_t)ntri) + r16(16 * (size_t)nu) + r16(8 * (size_t)nt);
  b += r16(4 * (size_t)(ncol + 1)) + r16(4 * (size_t)nslot) + r16(4 * (size_t)ncol) + r16(16 * (size_t)(nlev + 1));
  return b;
}

// Bytes of shared memory of the kept-factor substitution of one graph: its working vector,
// block-row entries and offsets, column-slot offsets, slot rows, schedule and levels.
inline size_t substitute_smem_bytes(int nslot, int ncol, int nlev) {
  auto r16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  return r16(8 * 7 * (size_t)ncol) + r16(8 * (size_t)(nslot - ncol)) + 2 * r16(4 * (size_t)(ncol + 1)) +
         r16(4 * (size_t)nslot) + r16(4 * (size_t)ncol) + r16(16 * (size_t)(nlev + 1));
}

// ... and of its kept blocks and L_cc^{-1} when those are staged as well.
inline size_t substitute_factor_bytes(int nslot, int ncol) {
  auto r16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  return r16(8 * 49 * (size_t)nslot) + r16(8 * 49 * (size_t)ncol);
}

// Bytes of shared memory of one CTA of the multi-SM solve: its blocks and column scratch,
// the triplets of its update tasks, its task lists and the graph's home / column-slot / row
// maps.
inline size_t cluster_smem_bytes(int nslot_loc, int ncol_loc, int ncol_max, int ntri, int nu, int nt, int nlev,
                                 int nslot, int ncol) {
  auto r16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  size_t b = r16(sizeof(double) * (size_t)ncol_max * 63) + r16(sizeof(double) * (size_t)nslot_loc * 49);
  b += r16(16 * (size_t)ntri) + r16(16 * (size_t)nu) + r16(8 * (size_t)nt);
  b += r16(4 * (size_t)ncol_loc) + r16(16 * (size_t)(nlev + 1)) + r16(4 * (size_t)nslot_loc);
  b += r16(4 * (size_t)nslot) + r16(4 * (size_t)ncol) + r16(4 * (size_t)(ncol + 1)) + r16(4 * (size_t)nslot);
  return b;
}

// ---- kernel launchers (defined in the .cu files) ----
cudaError_t launch_edge_prep(const double* poses, const EdgeStatic* es, int E, double* T64, float* T32,
                             double* Ad, cudaStream_t s);
cudaError_t launch_residual_reduce(int mode, int dtype, int cfg, int grid, const void* points,
                                   const int32_t* midx, const Item* items, int num_items,
                                   const EdgeStatic* es, const double* T64, const float* T32,
                                   RobustParams rp, void* partials, WarpSched ws, cudaStream_t s);
int residual_reduce_max_blocks_per_sm(int mode, int dtype, int cfg);
int residual_reduce_num_cfgs(int mode);
int residual_reduce_cfg_chunk(int cfg);      // required pixels per item, 0 = any
cudaError_t residual_reduce_prepare();       // once, before any capture
int residual_reduce_block();
// Balanced schedule for W workers (warps or CTAs) with item cost wv x valid + wp x pixels:
// per-item valid counts, cost prefix `cum` [num_items + 1], worker starts [W + 1], segment
// bases [W], first segment per edge [E + 1].
cudaError_t launch_schedule(const int32_t* midx, const EdgeStatic* es, const Item* items, int num_items,
                            const int32_t* item_off, int E, int W, int wv, int wp, int32_t* counts, long long* cum,
                            int32_t* start, int32_t* seg, int32_t* seg_off, uint32_t* compact, cudaStream_t s);
// Schedule workers of a launch configuration per CTA (1) or per warp (block / 32), and
// the cost weights of its loop.
int residual_reduce_workers_per_cta(int cfg);
void residual_reduce_cost_weights(int cfg, int& wv, int& wp);
unsigned int residual_reduce_stalls();  // bounded waits of the TMA variant that gave up
cudaError_t launch_edge_reduce(int mode, const void* partials, const int32_t* item_off, int E, const double* Ad,
                               double* edge_M, double* edge_b, double* edge_cost, double* edge_skip,
                               double* edge_rec, const long long* edge_valid, cudaStream_t s);
cudaError_t launch_assemble(int num_slots, const int32_t* slot_contrib_off, const int32_t* slot_contrib,
                            const double* edge_M, double* A, int N, const int32_t* kf_contrib_off,
                            const int32_t* kf_contrib, const double* edge_b, double* gvec, int G,
                            const int32_t* edge_offset, const double* edge_cost, const double* edge_skip,
                            GraphInfoDev* ginfo, double* cost_hist, const int* iter_counter, int* warn,
                            cudaStream_t s);
cudaError_t launch_export_dense(int num_slots, const int32_t* slot_kf_r, const int32_t* slot_kf_c,
                                const double* A, int N, const double* gvec, double* H_out, double* g_out,
                                cudaStream_t s);
// Workspace doubles per column (outside the slots): 7 Dinv + 7 rhs/solution + 49 L_cc^{-1}.
constexpr int kColScratch = 63;
// A factorisation kept for later solves: the graph's blocks of L at L + 49 (slot_base + s)
// and its column scratch at S + kColScratch (col_base + c), written by a solve that
// succeeded when L is not NULL.
struct FactorKeep {
  double* L;
  double* S;
};
// Panel levels of the factorisation: at most this many columns, each with at most this
// many off-diagonal blocks (7 diagonal rows + the right-hand side + 7 rows per block fit a
// warp's 32 lanes).
constexpr int kPanelCols = 4;
constexpr int kPanelBlocks = 3;
// A level (or a CTA's part of a level in the multi-SM solve) with a single column is a
// panel when that column has at most this many off-diagonal blocks: four warps eliminate
// its first 32 rows and then solve the rest of its 8 + 7 nb rows against L_cc, one row per
// thread of the four warps (8 + 7 x 20 - 32 = 116 <= 128).
constexpr int kPanel4Blocks = 20;
// A CTA of the multi-SM solve (8 warps) factors up to this many of its columns of a level
// as whole panels, one warp each (a fifth column would otherwise turn the CTA's level into
// diagonal factorisations followed by off-diagonal solves, about twice the dependent chain).
constexpr int kClusterPanelCols = 8;
// The multi-SM solve (same arguments; `cp` adds the cluster plan; smem_bytes per CTA).
cudaError_t launch_factor_solve_cluster(int G, const SolverPlan& plan, const ClusterPlan& cp, size_t smem_bytes,
                                        const double* A, const double* gvec, double* tau, double lambda, double eps0,
                                        int max_attempts, GraphInfoDev* ginfo, int* warn, cudaStream_t s,
                                        FactorKeep keep = {});
cudaError_t factor_solve_cluster_prepare(size_t smem_bytes, int C);
cudaError_t launch_factor_solve(int G, const SolverPlan& plan, bool smem, size_t smem_bytes, const double* A,
                                double* L, double* colscratch, const double* gvec, double* tau, double lambda,
                                double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn, cudaStream_t s,
                                FactorKeep keep = {});
size_t factor_solve_max_smem();
// Clusters of C CTAs (with smem_bytes each) of the multi-SM solver that the GPU can hold at
// once (0: none, e.g. a cluster size it cannot schedule); sets the kernel's attributes.
int factor_solve_cluster_max_active(size_t smem_bytes, int C);
// out = -(L L^T)^{-1} rhs with the factor a successful solve kept (the adjoint systems of
// the unrolled vjp), per graph; zero on the columns of a graph whose recorded solve
// (rec[g].solved) failed.  rhs / out are [N][7] by keyframe; anchors are not written.
// One CTA per graph; the working vector and the plan arrays live in shared memory
// (smem = the largest graph's substitute_smem_bytes, set up by factor_substitute_prepare)
// or, with smem == 0, in global memory (zwork: [total columns][7] doubles).
// factor_in_smem: the kept blocks and L_cc^{-1} are staged into shared memory too (smem then
// includes substitute_factor_bytes of the largest graph).
cudaError_t factor_substitute_prepare(size_t smem_bytes, bool factor_in_smem);
cudaError_t launch_factor_substitute(int G, const SolverPlan& plan, FactorKeep keep, const GraphInfoDev* rec,
                                     const double* rhs, double* out, size_t smem_bytes, double* zwork, cudaStream_t s,
                                     bool factor_in_smem);
// Test setting only (COMO3R_TEST_DIAG_SHIFT): A_gg -= shift[g] I on every graph's
// assembled diagonal, launched after the assembly when the setting is given at create.
cudaError_t launch_diag_shift(int G, const SolverPlan& plan, double* A, const double* shift, cudaStream_t s);

cudaError_t factor_solve_prepare(size_t smem_bytes);  // once, before any capture
// Grid-wide solve of graph 0 of a one-graph plan with the factor in global memory: the
// per-level task lists over every warp of `ctas` co-resident CTAs (a cooperative launch),
// phases separated by a grid barrier on `sync` (zeroed once; it resets itself).  A barrier
// wait has an iteration limit; when it runs out the kernel sets sync->err, every CTA
// leaves, and the graph gets the zero update of a failed factorisation (extra_arrivals > 0,
// a test setting only, makes every wait run out that way).
struct GridSync {
  unsigned count;  // arrivals at the current barrier
  unsigned gen;    // barrier generation
  int fail[2];     // pivot failure flags of the factorisation levels, by level parity
  int err;         // a barrier wait ran out
  int pad[3];
};
int factor_solve_grid_ctas();  // CTAs of the grid solve on this GPU (one per SM), 0 if unavailable
cudaError_t launch_factor_solve_grid(int ctas, const SolverPlan& plan, const double* A, double* L, double* colscratch,
                                     const double* gvec, double* tau, double lambda, double eps0, int max_attempts,
                                     GraphInfoDev* ginfo, int* warn, GridSync* sync, cudaStream_t s,
                                     FactorKeep keep = {}, unsigned extra_arrivals = 0);
// Batches with large graphs: one launch of clusters of kGroupCTAs CTAs (factor in global
// memory, L/colscratch as for the one-CTA kernel).  gtask[b] = (offset in glist, count,
// rank, group size) for CTA b: a cluster whose CTAs all name one graph with group size
// kGroupCTAs solves it together (cluster barriers); a CTA with group size 1 solves its
// graphs in turn.  Every CTA of the launch has an entry (count 0: idle).  gfail: 2 ints per
// graph.  ctas is a multiple of kGroupCTAs.
constexpr int kGroupCTAs = 8;
cudaError_t launch_factor_solve_group(int ctas, const SolverPlan& plan, const int4* gtask, const int32_t* glist,
                                      const double* A, double* L, double* colscratch, const double* gvec, double* tau,
                                      double lambda, double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn,
                                      int* gfail, cudaStream_t s, FactorKeep keep = {});
cudaError_t launch_retract(const double* tau, double* poses, const uint8_t* frozen, int N, int* iter_counter,
                           cudaStream_t s);
// ---- adjoint of the refined cost (k_adjoint.cu)
constexpr int kAdjointRecord = 21;  // doubles per K1 work item
cudaError_t launch_adjoint_match(int mode, int dtype, bool phi, const void* points, const int32_t* midx,
                                 const Item* items, int num_items, const EdgeStatic* es, const double* T64,
                                 const float* T32, const void* evec, RobustParams rp, double out_scale, void* gl,
                                 void* gc, double* rec, const int32_t* counts, const uint32_t* compact, cudaStream_t s);
cudaError_t launch_adjoint_edge_prep(int mode, const EdgeStatic* es, int E, const double* Ad, const double* u,
                                     const double* tau, void* evec, cudaStream_t s);
cudaError_t launch_adjoint_edge(const double* rec, const int32_t* item_off, int E, const EdgeStatic* es,
                                const double* Ad, const double* u, const double* tau, double* out, cudaStream_t s);
cudaError_t launch_adjoint_keyframe(const double* a, const double* tau, const uint8_t* frozen, int N, double* a_out,
                                    double* rhs, cudaStream_t s);
cudaError_t launch_adjoint_gather(const double* a_prime, const double* edge_out, const int32_t* kf_contrib_off,
                                  const int32_t* kf_contrib, const uint8_t* frozen, int N, const double* gvec,
                                  double scale, double* a, cudaStream_t s);
cudaError_t launch_to_float(const double* src, float* dst, int64_t n, cudaStream_t s);
cudaError_t launch_points_from_logdepth(int dtype, const float* rays, const float* logdepth, const float* conf,
                                        int64_t n, void* out, cudaStream_t s);
cudaError_t launch_rays_from_points(int dtype, const void* points, int64_t n, float* rays, float* logdepth,
                                    float* conf, cudaStream_t s);
cudaError_t launch_stamp(long long* out, cudaStream_t s);
// Sets the calling thread's como3r_last_error message and returns `code` (defined in api.cu).
int report_error(int code, const char* msg);
int report_cuda_error(cudaError_t e, const char* where);
cudaError_t launch_check_matches(const int32_t* midx, const EdgeStatic* es, int E, unsigned long long* bad,
                                 long long* edge_valid, cudaStream_t s);

}  // namespace como3r
