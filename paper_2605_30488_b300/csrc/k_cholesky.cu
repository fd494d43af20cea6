// K3: damped block Cholesky factorisation and solve of the pose system, Eq. (normal),
// with the epsilon escalation of Sec. III-D, all in FP64.
//
// One CTA (16 warps) per graph.  The factor L (lower, 7x7 blocks; pattern, elimination
// order and task lists fixed at create) is computed left-looking one elimination-tree
// level at a time.  Within a level three task lists run, separated by CTA barriers:
//   U  one warp per destination block: L[dst] -= sum L_rj L_cj^T over the descendants j
//      (diagonal destinations also accumulate the forward right-hand side
//      b_c - sum_j L_cj y_j);
//   D  one warp per column: Cholesky of the 7x7 diagonal block in registers (lane r holds
//      row r) with the right-hand side riding along as an eighth row, which yields
//      y_c = L_cc^{-1}(...) for free; a pivot that is not > 0 or not finite fails the attempt;
//   T  one thread per row of every off-diagonal block (B <- B L_cc^{-T}) and per column of
//      L_cc^{-1}, all independent.
// A failed attempt restarts with eps_r = eps0 * 100^r; after max_attempts failures the
// update is zero (Sec. III-D).  Back substitution walks the levels from the root, each
// column x_c = L_cc^{-T}(y_c - sum_r L_rc^T x_r) with the precomputed L_cc^{-1}.
// FP64 on this GPU has a long dependent latency (about 66 cycles per FMA, several
// hundred for rsqrt), so the schedule keeps chains short and spreads independent work.
// The factor lives in shared memory when the graph's blocks fit, else in global memory.
#include <cstdint>

#include "como3r_internal.h"

namespace como3r {
namespace {

constexpr int kSolveThreads = 512;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

struct SolveCtx {
  const SolverPlan* P;
  double* L;   // blocks of this graph: local slot (s - s0) * 49
  double* S;   // per-column scratch: (col - c0) * kColScratch = [Dinv 7 | y 7 | Linv 49]
  int s0, c0;
};

__device__ __forceinline__ double* blk(const SolveCtx& C, int s) { return C.L + (int64_t)(s - C.s0) * 49; }
__device__ __forceinline__ double* dinv_of(const SolveCtx& C, int col) { return C.S + (int64_t)(col - C.c0) * kColScratch; }
__device__ __forceinline__ double* y_of(const SolveCtx& C, int col) { return dinv_of(C, col) + 7; }
__device__ __forceinline__ double* linv_of(const SolveCtx& C, int col) { return dinv_of(C, col) + 14; }

// sum_q a[q] b[q], q < 7, as two interleaved FMA chains (shorter dependent latency)
__device__ __forceinline__ double dot7(const double* a, const double* b, double acc) {
  double p = a[0] * b[0];
  p = fma(a[2], b[2], p);
  p = fma(a[4], b[4], p);
  p = fma(a[6], b[6], p);
  double q = fma(a[1], b[1], acc);
  q = fma(a[3], b[3], q);
  q = fma(a[5], b[5], q);
  return p + q;
}

// U: one destination block (see file header)
__device__ void update_task(const SolveCtx& C, int4 task, int lane) {
  const SolverPlan& P = *C.P;
  const int e0 = lane, e1 = lane + 32;
  const bool has1 = e1 < 49;
  const int r0 = e0 / 7, q0 = e0 % 7, r1 = has1 ? e1 / 7 : 0, q1 = has1 ? e1 % 7 : 0;
  double a0 = 0.0, a1 = 0.0, rh = 0.0;
  const bool rhs = task.w >= 0 && lane < 7;
  for (int t = task.y; t < task.z; ++t) {
    const int4 tr = P.tri[t];
    const double* Lr = blk(C, tr.x);
    const double* Lk = blk(C, tr.y);
    a0 += dot7(Lr + 7 * r0, Lk + 7 * q0, 0.0);
    if (has1) a1 += dot7(Lr + 7 * r1, Lk + 7 * q1, 0.0);
    if (rhs) rh += dot7(Lr + 7 * lane, y_of(C, tr.w), 0.0);
  }
  double* D = blk(C, task.x);
  D[e0] -= a0;
  if (has1) D[e1] -= a1;
  if (rhs) y_of(C, task.w)[lane] -= rh;
}

// D: Cholesky of the diagonal block with the forward right-hand side as row 7
__device__ void diag_factor(const SolveCtx& C, int col, int lane, int* fail) {
  const SolverPlan& P = *C.P;
  double* D = blk(C, P.col_slot[col]);
  double* y = y_of(C, col);
  double a[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) a[c] = lane < 7 ? D[7 * lane + c] : (lane == 7 ? y[c] : 0.0);
  bool bad = false;
  double myinv = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double p = __shfl_sync(kFull, a[k], k);
    const bool okp = (p > 0.0) && (p < __longlong_as_double(0x7ff0000000000000LL));
    bad = bad || !okp;
    const double inv = rsqrt(okp ? p : 1.0);
    const double lk = (lane == k) ? p * inv : a[k] * inv;
    if (lane == k) myinv = inv;
    if (lane >= k) a[k] = lk;
#pragma unroll
    for (int c = k + 1; c < 7; ++c) {
      const double lc = __shfl_sync(kFull, lk, c);
      if (lane >= c) a[c] = fma(-lk, lc, a[c]);
    }
  }
  if (lane < 7) {
#pragma unroll
    for (int c = 0; c < 7; ++c) D[7 * lane + c] = (c <= lane) ? a[c] : 0.0;
    dinv_of(C, col)[lane] = myinv;
  } else if (lane == 7) {
#pragma unroll
    for (int c = 0; c < 7; ++c) y[c] = a[c];
  }
  if (bad && lane == 0) *fail = 1;
}

// T: item x < 7 * nt: row (x % 7) of off-diagonal block ttask[x / 7]; else column (x % 7)
// of L_cc^{-1} for the level column (x - 7 nt) / 7.
__device__ void trsm_or_inverse(const SolveCtx& C, int lv, int x) {
  const SolverPlan& P = *C.P;
  const int nt = P.ttask_off[lv + 1] - P.ttask_off[lv];
  if (x < 7 * nt) {
    const int2 tt = P.ttask[P.ttask_off[lv] + x / 7];
    const int i = x % 7;
    const double* Lc = blk(C, P.col_slot[tt.y]);
    const double* dv = dinv_of(C, tt.y);
    double* B = blk(C, tt.x) + 7 * i;
    double xr[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      double s = B[c];
#pragma unroll
      for (int q = 0; q < c; ++q) s = fma(-Lc[7 * c + q], xr[q], s);
      xr[c] = s * dv[c];
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) B[c] = xr[c];
  } else {
    const int k = (x - 7 * nt) / 7, c = x % 7;
    const int col = P.sched[P.lvl_off[lv] + k];
    const double* Lc = blk(C, P.col_slot[col]);
    const double* dv = dinv_of(C, col);
    double* X = linv_of(C, col);
    double xc[7];
#pragma unroll
    for (int r = 0; r < 7; ++r) {
      if (r < c) {
        xc[r] = 0.0;
      } else if (r == c) {
        xc[r] = dv[r];
      } else {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < r; ++q)
          if (q >= c) s = fma(Lc[7 * r + q], xc[q], s);
        xc[r] = -s * dv[r];
      }
    }
#pragma unroll
    for (int r = 0; r < 7; ++r) X[7 * r + c] = xc[r];
  }
}

// back substitution of one column: x_c = L_cc^{-T} (y_c - sum_r L_rc^T x_r)
__device__ void backward_column(const SolveCtx& C, int col, int lane) {
  const SolverPlan& P = *C.P;
  const int grp = lane / 7, q = lane % 7;
  const int s_begin = P.col_slot[col] + 1, nb = P.col_slot[col + 1] - s_begin;
  double part = 0.0;
  if (grp < 4) {
    for (int b = grp; b < nb; b += 4) {
      const double* B = blk(C, s_begin + b);
      const double* xr = y_of(C, P.slot_row[s_begin + b]);
      double p0 = B[q] * xr[0];
      double p1 = B[7 + q] * xr[1];
      p0 = fma(B[14 + q], xr[2], p0);
      p1 = fma(B[21 + q], xr[3], p1);
      p0 = fma(B[28 + q], xr[4], p0);
      p1 = fma(B[35 + q], xr[5], p1);
      p0 = fma(B[42 + q], xr[6], p0);
      part += p0 + p1;
    }
  }
  const double o1 = __shfl_sync(kFull, part, (q + 7) & 31);
  const double o2 = __shfl_sync(kFull, part, (q + 14) & 31);
  const double o3 = __shfl_sync(kFull, part, (q + 21) & 31);
  double* y = y_of(C, col);
  const double t = (lane < 7) ? y[q] - ((part + o1) + (o2 + o3)) : 0.0;
  const double* X = linv_of(C, col);
  double xq = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const double tr = __shfl_sync(kFull, t, r);
    if (lane < 7 && r >= q) xq = fma(X[7 * r + q], tr, xq);
  }
  __syncwarp();
  if (lane < 7) y[q] = xq;
}

template <bool SMEM>
__global__ void __launch_bounds__(kSolveThreads, 1) factor_solve_kernel(
    SolverPlan P, const double* __restrict__ A, double* Lg, double* Sg, const double* __restrict__ gvec,
    double* __restrict__ tau, double lambda, double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn) {
  extern __shared__ __align__(16) double dyn[];
  __shared__ int s_fail;
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = P.col_begin[g], c1 = P.col_begin[g + 1], ncol = c1 - c0;
  if (ncol == 0) {
    if (tid == 0) {
      ginfo[g].attempts = 1;
      ginfo[g].solved = 1;
    }
    return;
  }
  const int s0 = P.col_slot[c0], nslot = P.col_slot[c1] - s0;
  SolveCtx C;
  C.P = &P;
  C.L = SMEM ? dyn : Lg + (int64_t)s0 * 49;
  C.S = SMEM ? dyn + (int64_t)nslot * 49 : Sg + (int64_t)c0 * kColScratch;
  C.s0 = s0;
  C.c0 = c0;
  const int lv0 = P.lvl_begin[g], lv1 = P.lvl_begin[g + 1];

  bool ok = false;
  int attempt = 0;
  double pow100 = 1.0;  // 100^attempt, exact in FP64
  for (; attempt < max_attempts; ++attempt, pow100 *= 100.0) {
    const double eps = eps0 * pow100;
    for (int64_t x = tid; x < (int64_t)nslot * 49; x += kSolveThreads) C.L[x] = A[(int64_t)s0 * 49 + x];
    __syncthreads();
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) {
      const int col = c0 + x / 7, k = x % 7;
      const int64_t ds = P.col_slot[col];
      blk(C, (int)ds)[8 * k] += lambda * A[ds * 49 + 8 * k] + eps;
      y_of(C, col)[k] = -gvec[7 * P.col_kf[col] + k];
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int lv = lv0; lv < lv1; ++lv) {
      for (int u = P.utask_off[lv] + warp; u < P.utask_off[lv + 1]; u += kSolveWarps) update_task(C, P.utask[u], lane);
      __syncthreads();
      for (int q = P.lvl_off[lv] + warp; q < P.lvl_off[lv + 1]; q += kSolveWarps)
        diag_factor(C, P.sched[q], lane, &s_fail);
      __syncthreads();
      if (s_fail) break;
      const int nx = 7 * (P.ttask_off[lv + 1] - P.ttask_off[lv] + P.lvl_off[lv + 1] - P.lvl_off[lv]);
      for (int x = tid; x < nx; x += kSolveThreads) trsm_or_inverse(C, lv, x);
      __syncthreads();
    }
    ok = (s_fail == 0);
    __syncthreads();
    if (ok) break;
  }
  if (ok) {
    for (int lv = lv1 - 1; lv >= lv0; --lv) {
      for (int q = P.lvl_off[lv] + warp; q < P.lvl_off[lv + 1]; q += kSolveWarps)
        backward_column(C, P.sched[q], lane);
      __syncthreads();
    }
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) tau[7 * P.col_kf[c0 + x / 7] + x % 7] = y_of(C, c0 + x / 7)[x % 7];
  } else {
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) tau[7 * P.col_kf[c0 + x / 7] + x % 7] = 0.0;
  }
  if (tid == 0) {
    ginfo[g].attempts = ok ? attempt + 1 : max_attempts;
    ginfo[g].solved = ok ? 1 : 0;
    if (!ok) atomicOr(warn, 1);
  }
}

}  // namespace

size_t factor_solve_max_smem() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return optin > 64 ? (size_t)optin - 64 : 0;
}

cudaError_t factor_solve_prepare(size_t smem_bytes) {
  return cudaFuncSetAttribute(factor_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t launch_factor_solve(int G, const SolverPlan& plan, bool smem, size_t smem_bytes, const double* A,
                                double* L, double* colscratch, const double* gvec, double* tau, double lambda,
                                double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn, cudaStream_t s) {
  if (G <= 0) return cudaSuccess;
  if (smem) {
    factor_solve_kernel<true><<<G, kSolveThreads, smem_bytes, s>>>(plan, A, L, colscratch, gvec, tau, lambda, eps0,
                                                                   max_attempts, ginfo, warn);
  } else {
    factor_solve_kernel<false><<<G, kSolveThreads, 0, s>>>(plan, A, L, colscratch, gvec, tau, lambda, eps0,
                                                           max_attempts, ginfo, warn);
  }
  return cudaGetLastError();
}

}  // namespace como3r
