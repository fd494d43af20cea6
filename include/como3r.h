/*
 * como3r.h -- C ABI of the B300 (sm_103a) unified multi-agent Sim(3) graph refinement.
 *
 * The library evaluates and minimises, by Gauss-Newton, the global cost of CoMo3R-SLAM
 * (arXiv 2605.30488), Sec. III-D, Eq. (global):
 *
 *   E = sum_{(i,j) in E} sum_{(m,n) in M_ij} sum_{c=1..4} rho([Sigma_mn^{-1/2} e_mn(T_ij)]_c)
 *
 * with the ray-plus-range residual of Eq. (residual), e = [psi(T_ij X_j,n) - psi(X_i,m);
 * ||T_ij X_j,n|| - ||X_i,m||], psi(X) = X/||X||, T_ij = T_i^{-1} T_j, Sigma_mn = Sigma/q_mn,
 * Sigma = diag(sigma_r^2 I_3, sigma_d^2), q_mn = sqrt(c_i,m c_j,n) and a component-wise
 * Huber kernel rho of breakpoint kappa with IRLS weights min(1, kappa/|r|) (Sec. III-A).
 * Every iteration linearises all edges with the analytic Jacobians of Eq. (jacobian)
 * chained to both endpoints by -/+ Ad_{T_i^{-1}}, assembles the block-sparse normal
 * matrix (two diagonal and one off-diagonal 7x7 block per edge), solves Eq. (normal)
 * (H + lambda diag(H) + eps_r I) tau = -g with eps_r = eps0 * 100^r escalated on
 * factorisation failure (zero update after max_attempts failures), and retracts
 * T_i <- Exp(tau_i) T_i with tau = (v, omega, zeta) (Sec. III-D).  The first keyframe
 * of agent 0 (or the keyframe given as anchor) is held fixed.
 *
 * Conventions shared by every call:
 *   Poses:   double [N][8] = (tx, ty, tz, qx, qy, qz, qw, s): T = [s R(q) t; 0 1] maps
 *            camera coordinates to world coordinates (Sec. III-A).  Pose arguments may be
 *            host or device pointers; the library detects which.
 *   Points:  per keyframe k a row-major H_g x W_g pointmap in k's own camera frame, each
 *            pixel packed as (x, y, z, confidence) in the storage type of the graph
 *            (FP16: 8 B, FP32: 16 B, FP64: 32 B per pixel); keyframes concatenated in
 *            global keyframe order.  Pixels of keyframe k start at sum_{k'<k} P_k'.
 *   Matches: for edge e = (i, j), int32 [P_i]: the pixel n of keyframe j matched to pixel
 *            m of keyframe i, or -1 (masked / invalid).  Edges concatenated in edge order.
 *   Ownership: device input buffers passed at create are borrowed (zero copy) and must
 *            stay alive and unchanged until como3r_graph_destroy, unless
 *            desc.copy_inputs = 1, in which case the library copies them into buffers it
 *            owns (source may then be host or device memory).  The library owns all
 *            workspaces, the ordering / symbolic factorisation and the captured CUDA
 *            graphs.
 *   Streams: all work is enqueued on the stream given at create (0 = legacy default).
 *            Calls return after the results they write to host memory are available;
 *            device outputs are complete when the stream reaches the call's end.
 *   Errors:  0 = OK; > 0 = warning bit set (COMO3R_WARN_*), results valid;
 *            < 0 = error (COMO3R_ERR_*), outputs untouched unless stated.  No call aborts
 *            the process or traps on the device.  Handles are not thread-safe: one
 *            host thread at a time per handle.
 */
#ifndef COMO3R_H
#define COMO3R_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct como3r_graph* como3r_graph_t;

/* Storage type of the packed (x, y, z, confidence) pixels. */
typedef enum { COMO3R_F16 = 0, COMO3R_F32 = 1, COMO3R_F64 = 2 } como3r_dtype;

/* Arithmetic of the per-match residual / Jacobian / reduction.
 * PLAIN_FP64: every step in FP64.
 * MIXED: residuals, Jacobians and per-thread Hessian-block accumulation in FP32 with
 *        compensated warp merges and FP64 beyond the warp; edge preparation, assembly,
 *        Cholesky factorisation, solve and Sim(3) retraction stay FP64. */
typedef enum { COMO3R_PLAIN_FP64 = 0, COMO3R_MIXED = 1 } como3r_mode;

#define COMO3R_OK 0
#define COMO3R_WARN_SOLVE_FAILED 1   /* all eps attempts failed in >= 1 graph: zero update there */
#define COMO3R_WARN_SKIPPED 2        /* >= 1 degenerate / non-finite match was skipped */
#define COMO3R_ERR_INVALID_ARG (-1)
#define COMO3R_ERR_CUDA (-2)
#define COMO3R_ERR_OOM (-3)
#define COMO3R_ERR_UNSUPPORTED (-4)

/* Size of one exported edge record (doubles), see como3r_linearize. */
#define COMO3R_EDGE_RECORD 64

/* One batch of independent graphs in a flat keyframe index space (Sec. III-D: all
 * keyframes of all agents in one global index with a side map a(i)). */
typedef struct {
  int32_t num_graphs;            /* G >= 1 */
  const int32_t* kf_offset;      /* host [G+1]: keyframes of graph g are [kf_offset[g], kf_offset[g+1]) */
  const int32_t* height;         /* host [G]: pointmap rows of graph g (> 0) */
  const int32_t* width;          /* host [G]: pointmap columns of graph g (> 0) */
  const int32_t* agent_of;       /* host [N] or NULL: originating agent a(i) of each keyframe */
  const void* points_conf;       /* [sum_k P_k][4] packed pixels, see Points above */
  int32_t dtype;                 /* como3r_dtype of points_conf */
  const int32_t* edge_offset;    /* host [G+1]: edges of graph g are [edge_offset[g], edge_offset[g+1]) */
  const int32_t* edge_i;         /* host [E]: streamed keyframe (global id) */
  const int32_t* edge_j;         /* host [E]: gathered keyframe (global id), same graph, != edge_i */
  const int32_t* match_idx;      /* [sum_e P_{edge_i[e]}] pixel of j or -1, see Matches above */
  const int32_t* anchor;         /* host [G] or NULL: fixed keyframe of each graph (default:
                                    the first keyframe of the graph's lowest agent) */
  double sigma_ray;              /* sigma_r > 0, paper: 0.003 */
  double sigma_dist;             /* sigma_d > 0, paper: 10 */
  double huber_k;                /* kappa > 0, paper: 1.345 */
  double lambda;                 /* lambda >= 0 of Eq. (normal); back-end default 0 */
  double eps0;                   /* eps_0 > 0, paper: 1e-6 */
  int32_t max_attempts;          /* 1..16, paper: 6 */
  int32_t mode;                  /* como3r_mode */
  int32_t copy_inputs;           /* 0: borrow device buffers; 1: copy points/matches (host or device) */
} como3r_graph_desc;

/* Per-graph result of one linearisation / iteration. */
typedef struct {
  double cost;                   /* E at the linearisation point (Eq. global) */
  int32_t attempts;              /* factorisation attempts made (1..max_attempts) */
  int32_t solved;                /* 1: a factorisation succeeded; 0: zero update applied */
  int64_t valid_matches;         /* matches with match_idx >= 0 */
  int64_t skipped_matches;       /* of those, skipped as degenerate / non-finite */
} como3r_graph_info;

/* Validate the description, plan the solve (fill-reducing ordering, symbolic block
 * factorisation, work lists; for a few large graphs a multi-SM solve with one cluster of 8
 * CTAs per graph (16 when a factor does not fit eight CTAs' shared memory and the device
 * can schedule a 16-CTA cluster), COMO3R_SOLVE_CLUSTER=<C> forcing C CTAs or 0 none; for
 * one graph whose factor fits neither one SM nor a cluster, a grid-wide solve over one CTA
 * per SM (a
 * cooperative launch), COMO3R_SOLVE_GRID=1 forcing it for any one-graph plan, 0 disabling
 * it; for a batch too large for one cluster per graph, one launch of CTA groups when the
 * planner's estimates favour it: the slowest graphs each solved by a cluster of 8 CTAs, the
 * others packed onto single CTAs, factors in global memory, COMO3R_SOLVE_GROUPS=<k> forcing k
 * cluster-solved graphs or 0 none), allocate workspaces, check every match index on the
 * device (-1 <= n < P_j) and autotune the residual kernel's work-item size and launch
 * configuration on this graph's data (a few milliseconds of timed trial launches; the
 * environment variables COMO3R_K1_CFG=<n>, COMO3R_K1_CHUNK=<pixels> and
 * COMO3R_K1_WEIGHTS=<wv>,<wp> restrict the search, and together fix the residual kernel's
 * schedule, so that two graphs of the same problem round alike).
 * Synchronises the stream.  On error *out is NULL.
 * Errors: INVALID_ARG (bad sizes / ids / indices / parameters), OOM, CUDA. */
int como3r_graph_create(const como3r_graph_desc* desc, void* cuda_stream, como3r_graph_t* out);

/* Release every resource of the handle (NULL is allowed). */
void como3r_graph_destroy(como3r_graph_t graph);

/* One Gauss-Newton iteration for every graph: linearise all edges at `poses`, assemble,
 * solve Eq. (normal) with eps escalation, retract `poses` in place (Sec. III-D).
 *   poses  [N][8] in/out (host or device).
 *   H_out  device [7N][7N] row-major or NULL: the assembled H before damping, on the
 *          flat keyframe index; rows/columns of anchors and every pair without a block
 *          are zero.  g_out device [7N] or NULL: the assembled gradient (anchors zero).
 *   info   host [G] or NULL.
 * Returns OK or a warning bitmask, or an error. */
int como3r_gn_step(como3r_graph_t graph, double* poses, double* H_out, double* g_out,
                   como3r_graph_info* info);

/* `iters` Gauss-Newton iterations (>= 0), replayed from a captured CUDA graph.
 *   poses       [N][8] in/out (host or device).
 *   cost_trace  host [(iters+1) * G] or NULL: cost of graph g before iteration k at
 *               [k*G + g], and after the last retraction at [iters*G + g].
 *   info        host [G] or NULL: result of the last iteration.
 * Returns OK or the OR of the warnings of all iterations, or an error. */
int como3r_solve(como3r_graph_t graph, double* poses, int32_t iters, double* cost_trace,
                 como3r_graph_info* info);

/* The step tau of the last Gauss-Newton iteration of como3r_gn_step or como3r_solve, the
 * solution of Eq. (normal), (H + lambda diag(H) + eps_r I) tau = -g (Sec. III-D), before
 * its retraction T_i <- Exp(tau_i) T_i.
 *   tau_out  [N][7] (host or device), tau = (v, omega, zeta) per keyframe on the flat
 *            keyframe index; rows of fixed keyframes, and every row of a graph whose six
 *            attempts all failed, are zero.  Undefined before the first iteration.
 * Synchronises the graph's stream.  Errors: INVALID_ARG (NULL argument), CUDA. */
int como3r_last_step(como3r_graph_t graph, double* tau_out);

/* Device-clock stamps (ns, the GPU's %globaltimer) of the last como3r_gn_step or
 * como3r_solve: the moment its first kernel ran (after the pose upload), and for every
 * graph the moment its last damped factorisation and solve (Eq. 7) finished.  In a batch
 * all graphs share each residual launch and each graph's solve ends on its own CTA(s),
 * so done_ns[g] - start_ns is graph g's latency within the call.
 *   start_ns host [1] or NULL;  done_ns host [G] or NULL.
 * Synchronises the graph's stream.  Errors: INVALID_ARG (NULL graph), CUDA. */
int como3r_solve_timestamps(como3r_graph_t graph, int64_t* start_ns, int64_t* done_ns);

/* Linearise every edge at `poses` without solving.
 *   edge_out device [E][COMO3R_EDGE_RECORD] or NULL: per edge e = (i, j) the blocks with
 *            respect to a left perturbation of T_ij: [0..48] H_rel = sum J^T W J row-major,
 *            [49..55] g_rel = sum J^T W e, [56] cost, [57] valid matches, [58] skipped.
 *            (The endpoint blocks follow as H_jj = H_ii = -H_ij = Ad^T H_rel Ad,
 *            g_j = -g_i = Ad^T g_rel with Ad = Ad_{T_i^{-1}}.)
 *   cost_out host [G] or NULL. */
int como3r_linearize(como3r_graph_t graph, const double* poses, double* edge_out, double* cost_out);

/* Gradient of the refined cost with respect to the dense structure (pose-depth
 * alternation, Sec. III-E).  Each pixel p is parameterised by its log-range l_p, with
 * X_p = exp(l_p) psi(X_p) (the point slides along its viewing ray, so this is also the
 * derivative with respect to log-depth), and by its confidence c_p.  The refined cost is
 *   L = sum over graphs of E_global(T^K, theta)                              (Eq. global)
 * where T^K are the poses after `iters` Gauss-Newton iterations (Sec. III-D) from
 * `poses_init`.
 *   mode      COMO3R_VJP_UNROLLED: the total derivative through the K iterations (their
 *             IRLS weights, damped factorisations and retractions); requires lambda = 0
 *             (else UNSUPPORTED).  COMO3R_VJP_ENVELOPE: the partial derivative at fixed
 *             T^K (equal to the total one at a stationary point).
 *   upstream  factor applied to every output gradient (dLoss/dL of the caller).
 *   grad_logdepth, grad_conf  device float [sum_k P_k], pixels in the packed order of
 *             points_conf: upstream * dL/dl_p and upstream * dL/dc_p (overwritten).
 *   poses_out [N][8] (host or device) or NULL: T^K.   loss_out host [G] or NULL: E_g(T^K).
 * The forward iterations are recomputed inside the call and keep, per iteration, the poses,
 * the step, the solve outcome and the damped factor (7N + 8N doubles and 49 per factor
 * block + 63 per unknown keyframe); each backward step solves its adjoint system with the
 * kept factor of its iteration (the system is not linearised or factorised again).  The
 * kept-factor solve holds its working vector, plan and the kept factor in shared memory when
 * the largest graph's fit (about 500 bytes per keyframe and 400 per factor block), else the
 * vector and plan alone (about 100 and 12), else global memory (COMO3R_SUBSTITUTE_SMEM=1 / 0
 * at create force the second / the third, test settings).  Pixel gradients are accumulated with atomics (FP32
 * in the MIXED form, so bitwise results can vary between runs; FP64 then rounded once in
 * the PLAIN form).  A match with c_i c_j = 0 contributes no confidence gradient.
 * Synchronises the stream.
 * Returns OK or the warning bitmask of the forward iterations, or an error. */
typedef enum { COMO3R_VJP_UNROLLED = 0, COMO3R_VJP_ENVELOPE = 1 } como3r_vjp_mode;
int como3r_vjp(como3r_graph_t graph, const double* poses_init, int32_t iters, int32_t mode, double upstream,
               float* grad_logdepth, float* grad_conf, double* poses_out, double* loss_out);

/* Timing of `reps` unrolled como3r_vjp calls of `iters` iterations from poses_init (one
 * more untimed call first), CUDA events on the graph's stream; ms[k] receives the mean
 * duration of: 0 the forward pass with checkpoints, 1 the evaluation at T^K with the
 * envelope pixel term, 2 the backward iterations, 3 the per-match adjoint kernels of the
 * backward iterations (part of 2).  Allocates and frees its own gradient buffers. */
int como3r_time_vjp(como3r_graph_t graph, const double* poses_init, int32_t iters, int32_t reps,
                    float* ms /* [4] */);

/* Packs pointmaps from the structure parameters: X_p = exp(logdepth_p) rays_p and c_p.
 *   rays device float [n][3] (unit), logdepth / conf device float [n];
 *   points_out device [n][4] in the storage type `dtype` (como3r_dtype); async on stream. */
int como3r_points_from_logdepth(const float* rays, const float* logdepth, const float* conf, int64_t n,
                                int32_t dtype, void* points_out, void* cuda_stream);

/* The inverse split of packed points: unit ray, log-range (log ||X_p||) and confidence
 * per point (device arrays; a point with zero or non-finite range gets ray 0 and log-range
 * -inf); async on stream. */
int como3r_rays_from_points(const void* points, int64_t n, int32_t dtype, float* rays, float* logdepth, float* conf,
                            void* cuda_stream);

/* Left retraction T_k <- Exp(tau_k) T_k (Sec. III-D) of n poses, tau_k = (v, omega, zeta).
 *   tau   device [n][7]; poses device [n][8] in/out; stream as at create (may be NULL).
 * Independent of any graph handle. */
int como3r_sim3_retract(const double* tau, double* poses, int32_t n, void* cuda_stream);

/* Replace the pointmaps and matches of a graph created with copy_inputs = 1 (same sizes);
 * sources may be host or device memory.  Either pointer may be NULL (kept).  The copy is
 * enqueued on the graph's stream; host sources must stay valid until the stream passes it
 * (pinned host memory makes the copy asynchronous). */
int como3r_update_inputs(como3r_graph_t graph, const void* points_conf, const int32_t* match_idx);

/* Per-stage timing of `reps` full iterations from `poses` (host or device; not modified):
 * the six kernels of an iteration are launched individually on the graph's stream with
 * CUDA events recorded between them, and ms[k] receives the mean duration of stage k:
 * 0 edge prep, 1 residual/Jacobian/reduction (K1), 2 per-edge reduction, 3 assembly,
 * 4 factorisation + solve, 5 retraction; ms[6] = mean time of a whole iteration. */
#define COMO3R_STAGES 7
int como3r_time_stages(como3r_graph_t graph, const double* poses, int32_t reps, float* ms /* [COMO3R_STAGES] */);

/* Number of kernels the last gn_step / solve / linearize / vjp call enqueued (for accounting). */
int64_t como3r_last_launch_count(como3r_graph_t graph);

/* Static description of the planned work (see COMO3R_STAT_* indices). */
#define COMO3R_STAT_GRAPHS 0
#define COMO3R_STAT_KEYFRAMES 1
#define COMO3R_STAT_EDGES 2
#define COMO3R_STAT_ITEMS 3          /* K1 work items */
#define COMO3R_STAT_COLUMNS 4        /* block columns of the factor (all graphs) */
#define COMO3R_STAT_BLOCKS 5         /* stored 7x7 blocks of the factor, incl. diagonal */
#define COMO3R_STAT_FILL 6           /* of those, fill blocks (no edge) */
#define COMO3R_STAT_UPDATES 7        /* 7x7 block updates of one factorisation */
#define COMO3R_STAT_LEVELS 8         /* max elimination-tree levels of one graph */
#define COMO3R_STAT_VALID 9          /* valid matches (all edges) */
#define COMO3R_STAT_CHUNK 10         /* K1 pixels per work item */
#define COMO3R_STAT_BLOCK 11         /* K1 threads per CTA * 100 + chosen register/residency config */
#define COMO3R_STAT_GRID 12          /* K1 CTAs */
#define COMO3R_STAT_SMEM_SOLVE 13    /* 1 if the factor of every graph fits in shared memory */
#define COMO3R_STAT_ND_GRAPHS 14     /* graphs ordered by nested dissection (others: minimum degree) */
#define COMO3R_STAT_K1_STALLS 15     /* bounded waits of the TMA-staged K1 that gave up (process-wide; 0 = healthy) */
#define COMO3R_STAT_SOLVE_CTAS 16    /* CTAs per graph of the factorisation: 1, the cluster of the multi-SM solve, the grid of the grid-wide solve of one large graph, or the cluster of a batch's CTA groups */
#define COMO3R_STAT_SOLVE_FLOPS 17   /* FP64 operations of one factorisation + solve, all graphs (FMA = 2) */
#define COMO3R_STAT_SOLVE_GROUPS 18  /* graphs of a batch solved by a whole cluster (CTA-group solve), 0 if none */
#define COMO3R_STAT_COUNT 19
int como3r_graph_stats(como3r_graph_t graph, int64_t* stats /* [COMO3R_STAT_COUNT] */);

/* Plan a description on the host only (no device memory touched): fills the same stats
 * as como3r_graph_stats (K1 launch fields 0).  For inspecting orderings without a GPU. */
int como3r_plan_stats(const como3r_graph_desc* desc, int64_t* stats /* [COMO3R_STAT_COUNT] */);

/* ---- Allocation-free linearisation ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory when they need a linearisation: real-time loops that must never
 * wait on the allocator, and host frameworks that reserve the whole device memory budget
 * for themselves and forbid side allocations.  It computes what como3r_linearize writes
 * to edge_out, without a graph handle and without allocating anything: every
 * intermediate lives in one fixed device array of COMO3R_NOALLOC_SCRATCH_BYTES that the
 * library declares statically, so every GPU that loads the library holds that memory
 * until the process exits.
 *   desc      as for como3r_graph_create, with copy_inputs = 0: points_conf and
 *             match_idx must be device memory (16- / 4-byte aligned); host arrays as usual.
 *   poses     device [N][8], read only.
 *   edge_out  device [E][COMO3R_EDGE_RECORD], written as by como3r_linearize.
 *   stream    stream to run on (NULL = legacy default stream).
 * Limits: at most COMO3R_NOALLOC_MAX_EDGES edges and COMO3R_NOALLOC_MAX_GRAPHS graphs;
 * larger descriptions are rejected with COMO3R_ERR_INVALID_ARG before any GPU work
 * (the work-item size is raised as needed to stay within COMO3R_NOALLOC_MAX_ITEMS).
 * The first call on a device looks up the array's device address (once per device);
 * make that first call before any stream capture.  All calls share the one array and a
 * call overwrites what the previous call left there, so calls whose GPU work may
 * overlap (different streams or host threads) race and must be serialised by the
 * caller; the entry point is also not reentrant on the host.  The call synchronises the
 * stream once (to check the match indices) and returns with the rest enqueued.
 * Returns OK or an error (como3r_last_error says which).  Unlike como3r_linearize it
 * does not return COMO3R_WARN_SKIPPED: matches skipped as degenerate or non-finite are
 * counted only in each edge record's skip slot (entry 58), which the caller reads. */
#define COMO3R_NOALLOC_MAX_EDGES 2048
#define COMO3R_NOALLOC_MAX_ITEMS 16384
#define COMO3R_NOALLOC_MAX_GRAPHS 256
#define COMO3R_NOALLOC_SCRATCH_BYTES (7u * 1024u * 1024u)
int como3r_linearize_noalloc(const como3r_graph_desc* desc, const double* poses, double* edge_out,
                             void* cuda_stream);

/* ---- Cross-agent candidate verification and gauge synchronisation (Sec. III-B, III-C).
 *
 * Candidate c = (kf_i[c], kf_j[c]) is a pair of keyframes of different agents with the two
 * decoded match directions of the two-view prior.  Keyframe i belongs to the reference
 * component, j to the moving one.  A match of pixel m (of the view whose pixels are listed)
 * to pixel n is valid when its index is >= 0, and high-confidence when moreover both points
 * are finite and c_m c_n >= q_min^2, i.e. q_mn = sqrt(c_m c_n) >= q_min (the exact product of
 * the stored confidences, decided as in FP64 by both arithmetic modes).
 *   nu_i = high-confidence matches of i's pixels into j / P_i, nu_j likewise from j into i;
 *   admitted = min(nu_i, nu_j) >= nu_min (Sec. III-B);
 *   T* (Sec. III-C) maps j's component onto i's and is to be left-multiplied onto every pose
 *   of the moving component: with x = T_i X_i,m and y = T_j X_j,n over the forward
 *   high-confidence matches (N_c = n_i of them), the Umeyama similarity of Eq. (umeyama)
 *   minimising sum |x - (s R y + t)|^2 when N_c >= nc_min; otherwise (and when the
 *   cross-covariance has rank < 2, so R is undetermined) the endpoint transform
 *   T_i T_j^{-1}, which puts j's pose onto i's.
 * The pass over the matches is HBM-bound: match rows and the streamed pixels are read once,
 * the gathered pixels once per valid match.  MIXED accumulates the camera-frame moments in
 * FP32 with Kahan-compensated lane sums and TwoSum warp merges (FP64 above the warp);
 * PLAIN_FP64 in FP64.  The 3x3 SVD and everything after it are FP64. */
typedef struct {
  int32_t num_candidates;       /* C >= 0 */
  int32_t num_kf;               /* keyframes described by pix_off and poses */
  const int64_t* pix_off;       /* host [num_kf + 1]: first pixel of keyframe k in points_conf (non-decreasing) */
  const void* points_conf;      /* device, packed (x, y, z, confidence) pixels of every keyframe (see above) */
  int32_t dtype;                /* como3r_dtype of points_conf */
  const int32_t* kf_i;          /* host [C] reference-side keyframe of each candidate */
  const int32_t* kf_j;          /* host [C] moving-side keyframe (!= kf_i) */
  const int32_t* match_ij;      /* device: per candidate P_{kf_i[c]} entries (pixel of j or -1), candidates concatenated */
  const int32_t* match_ji;      /* device: per candidate P_{kf_j[c]} entries (pixel of i or -1), candidates concatenated */
  const double* poses;          /* [num_kf][8] current poses, host or device */
  double q_min;                 /* high-confidence threshold on q = sqrt(c_m c_n) (>= 0) */
  double nu_min;                /* admission threshold of min(nu_i, nu_j), 0.1 in the paper */
  int32_t nc_min;               /* fewest correspondences for the point-based alignment, 64 in the paper */
  int32_t mode;                 /* COMO3R_MIXED or COMO3R_PLAIN_FP64 */
} como3r_gauge_desc;

typedef struct {
  double T[8];                  /* T* as (tx, ty, tz, qx, qy, qz, qw, s) */
  double nu_i, nu_j;            /* support fractions of the two views */
  int64_t n_i, n_j;             /* high-confidence matches of each direction (n_i = N_c) */
  int64_t valid_i, valid_j;     /* matches with index >= 0 of each direction */
  int32_t admitted;             /* 1 if min(nu_i, nu_j) >= nu_min */
  int32_t fallback;             /* 0 Umeyama; 1 endpoint transform (N_c < nc_min); 2 endpoint transform (rank < 2) */
} como3r_gauge_result;

/* Verifies and aligns C candidates on `cuda_stream` (device temporaries allocated and freed
 * inside the call; synchronises the stream).  out host [C].  kernel_ms (host, nullable)
 * receives the duration of the pass over the matches (CUDA events).
 * Errors: INVALID_ARG (NULL pointers, bad ids or sizes, a match index outside [-1, P)),
 * OOM, CUDA. */
int como3r_gauge_sync(const como3r_gauge_desc* desc, void* cuda_stream, como3r_gauge_result* out,
                      float* kernel_ms);

/* Gauge transport (Sec. III-C): poses[k] <- T[which[k]] * poses[k] (Sim(3) left
 * multiplication) for every keyframe k with 0 <= which[k] < num_candidates; others are
 * left unchanged.  poses device [num_kf][8] in/out, which device [num_kf], T device
 * [num_candidates][8] (e.g. the T fields of como3r_gauge_sync's results, uploaded).
 * Asynchronous on `cuda_stream`.  Errors: INVALID_ARG, CUDA. */
int como3r_gauge_transport(double* poses, int32_t num_kf, const int32_t* which, const double* T,
                           int32_t num_candidates, void* cuda_stream);

/* ---- Terminal segment-level structure refinement (Sec. III-E).
 *
 * One log-scale eta_g per segment: a pixel p of segment g moves along the ray of its
 * snapshot point, X_p(eta_g) = |X_p,init| exp(eta_g) psi(X_p,init) (Eq. depth_parameter);
 * with the poses fixed, E' = E_data + lambda_smooth E_bnd / 2 + lambda_prior E_prior / 2
 * where E_data = sum over the graph's matches and c = 1..3 of
 * rho(sqrt(q_mn) [T_ij X_j,n(eta) - X_i,m(eta)]_c / sigma_point) (Eq. depth_data, Huber of
 * the graph's kappa), E_bnd = sum over 4-adjacent segment pairs of ((eta_g - eta_h) +
 * Delta_gh)^2 and E_prior = sum eta_g^2 (Eq. depth_total; the halves follow from the
 * printed H_prior = lambda_prior I).  Each iteration takes the Jacobi 1x1 damped Newton
 * step delta_g = -g_g / ((1 + lambda_lm) H_gg), |delta_g| <= eta_max, with the full gradient
 * and the diagonal of the normal matrix (cross terms dropped); segments of the graph's
 * fixed keyframes do not move.
 * Segments: a pixel belongs to segment (its keyframe's base + label) when its label is
 * >= 0, its confidence >= c_min, its point finite with range > 1e-12, and the segment has
 * >= min_pixels such pixels; otherwise it keeps its snapshot point.  Keyframe k's base =
 * sum over earlier keyframes of (max label + 1); M = the total.  Delta_gh (g < h) is the
 * mean over the 4-adjacent pixel pairs (p in g, p' in h) of log|X_p| - log|X_p'| of the
 * snapshot. */
typedef struct {
  const int32_t* labels;        /* [sum P_k] host or device: segment of each pixel within its keyframe, or -1 */
  double c_min;                 /* 1.5 */
  int32_t min_pixels;           /* 16 */
  double sigma_point;           /* 0.05 */
  double lambda_smooth;         /* 1 */
  double lambda_prior;          /* 1 */
  double lambda_lm;             /* 0.05 */
  double eta_max;               /* 0.5 */
} como3r_depth_desc;

/* Snapshots the graph's current pointmaps (the pristine reference rays and ranges),
 * builds the segments and boundary pairs on the host and uploads them; replaces an earlier
 * setup.  *num_segments (nullable) receives M.  Synchronises.  Errors: INVALID_ARG, OOM,
 * CUDA. */
int como3r_depth_setup(como3r_graph_t graph, const como3r_depth_desc* desc, int64_t* num_segments);

/* Up to `iters` (>= 0) Jacobi steps at fixed poses.  poses [N][8] host or device;
 * eta [M] host or device, in/out (start and result); cost_trace host [iters + 1] or NULL
 * (E' before each step and at the result); points_out device or NULL: the refined
 * pointmaps in the graph's storage type and layout (pixels without a segment keep the
 * snapshot point; confidences copied) -- e.g. for the next pose pass via
 * como3r_update_inputs.  match_ms host or NULL: mean duration of the per-match pass
 * (CUDA events).  Synchronises.  Errors: INVALID_ARG (no setup), CUDA. */
int como3r_depth_refine(como3r_graph_t graph, const double* poses, double* eta, int32_t iters,
                        double* cost_trace, void* points_out, float* match_ms);

/* ---- Front-end kernels (Sec. III-A).
 *
 * Projective ray matching: for every queried point x (keyframe k's pointmap predicted in
 * frame f's camera, X^k_f), the pixel p* of f minimising |psi([X^f_f]_p) - psi(x)|^2 on f's
 * ray image, by a deterministic descent: from init[q] (or pixel q mod H*W when init is
 * NULL), move to the best of the 8 neighbours (order (-1,-1) (-1,0) (-1,1) (0,-1) (0,1)
 * (1,-1) (1,0) (1,1); strictly smaller distance; the first on ties) while it improves, at
 * most max_steps moves.  Distances are FP32 with every operation correctly rounded in
 * the fixed order n = sqrt((x0 x0 + x1 x1) + x2 x2), psi = x / n,
 * d = ((a0-b0)^2 + (a1-b1)^2) + (a2-b2)^2 (no fused multiply-adds), so the result is
 * reproducible on any IEEE implementation.  match[q] = -1 when x is not finite or has zero
 * norm, or when the final distance exceeds 2 - 2 cos(max_angle) (rounded to FP32).  Pixels
 * of f whose ray is not finite are never entered.  The descriptor-window refinement of the
 * paper needs the prior's descriptors and is not part of this call. */
typedef struct {
  int32_t H, W;                 /* frame f's pointmap size */
  const void* frame_points;     /* device [H*W] packed (x, y, z, c) pixels of X^f_f */
  const void* query_points;     /* device [num_queries] packed (x, y, z, c) points x */
  int32_t num_queries;
  int32_t dtype;                /* como3r_dtype of both point arrays (converted to FP32, round to nearest) */
  const int32_t* init;          /* device [num_queries] start pixels, or NULL */
  int32_t max_steps;            /* >= 0 */
  double max_angle;             /* radians, >= 0 */
} como3r_match_desc;

/* match device int32 [num_queries] (pixel of f or -1); dist device float [num_queries] or
 * NULL (final FP32 distance).  Asynchronous on `cuda_stream` (a scratch ray image is
 * allocated stream-ordered).  Errors: INVALID_ARG, CUDA. */
int como3r_project_match(const como3r_match_desc* desc, int32_t* match, float* dist, void* cuda_stream);

/* Confidence-weighted fusion, Eq. (fusion), per pixel:
 *   X_k <- (C_k X_k + C_f (T_kf X_f)) / (C_k + C_f),  C_k <- C_k + C_f,
 * canon device [num_pixels] packed (X_k, C_k), in/out; pred device [num_pixels] packed
 * (X^k_f in f's frame, C^k_f); T_kf host [8] pose (t, q, s) mapping f's camera to k's.
 * dtype COMO3R_F32 or COMO3R_F64 (a running average is not kept in FP16: UNSUPPORTED).
 * Asynchronous on `cuda_stream`.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
int como3r_fuse(void* canon, const void* pred, int64_t num_pixels, int32_t dtype, const double* T_kf,
                void* cuda_stream);

/* Fusion of many keyframes in one launch (Eq. (fusion) as in como3r_fuse, pixel for pixel
 * the same results): keyframe q owns rows pix_off[q] .. pix_off[q+1]-1 of the packed canon
 * (in/out) and pred device arrays and is fused with its own pose T_kf[8q .. 8q+7].
 * pix_off host int64 [n+1], non-decreasing from 0; T_kf host [n][8]; n >= 0.  The
 * transforms travel as kernel parameters (128 keyframes per launch), so nothing is
 * allocated.  dtype COMO3R_F32 or COMO3R_F64.  Asynchronous on `cuda_stream`.
 * Errors: INVALID_ARG (bad offsets, NULL pointers, a zero quaternion), UNSUPPORTED (FP16),
 * CUDA. */
int como3r_fuse_packed(void* canon, const void* pred, const int64_t* pix_off, const double* T_kf, int32_t n,
                       int32_t dtype, void* cuda_stream);

/* Human-readable text of a status code. */
const char* como3r_status_str(int code);

/* Message of the last error returned to the calling host thread ("" if none). */
const char* como3r_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* COMO3R_H */
