// K3: damped block Cholesky factorisation and solve of the pose system, Eq. (normal),
// with the epsilon escalation of Sec. III-D, all in FP64.
//
// One CTA per graph.  The factor L (lower, 7x7 blocks, pattern and elimination order
// fixed at create by a nested-dissection ordering) is computed left-looking, one
// elimination-tree level at a time: the columns of a level are independent, each is
// owned by one warp, which (1) applies the updates L_rc -= L_rj L_cj^T from its
// descendants j, (2) factors its 7x7 diagonal block in registers (lane r holds row r),
// (3) solves the off-diagonal blocks against it.  A pivot that is not > 0 or not finite
// marks the attempt failed; the CTA then restarts with eps_r = eps0 * 100^r, and after
// max_attempts failures writes a zero update (Sec. III-D).  Forward and back
// substitution walk the same levels up and down.  The factor lives in shared memory
// when the graph's blocks fit, otherwise in a global workspace.
#include <cstdint>

#include "como3r_internal.h"

namespace como3r {
namespace {

constexpr int kSolveThreads = 512;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

struct SolveCtx {
  const SolverPlan* P;
  double* L;        // blocks of this graph, local slot index (s - s0) * 49
  double* Dinv;     // 1 / L_kk diagonal entries, local column * 7
  double* y;        // right-hand side / solution, local column * 7
  int s0, c0;
  double* stage;    // this warp's 2 x 49 staging area
  int* fail;
};

__device__ __forceinline__ double* blk(const SolveCtx& c, int s) { return c.L + (int64_t)(s - c.s0) * 49; }

__device__ void factor_column(const SolveCtx& C, int col, int lane) {
  const SolverPlan& P = *C.P;
  const int dslot = P.col_slot[col];
  double* st0 = C.stage;
  double* st1 = C.stage + 49;
  const int e0 = lane, e1 = lane + 32;
  const bool has1 = e1 < 49;
  const int r0 = e0 / 7, q0 = e0 % 7, r1 = e1 / 7, q1 = e1 % 7;

  // (1) left-looking updates, grouped by destination block
  double acc0 = 0.0, acc1 = 0.0;
  int cur = -1;
  for (int t = P.tri_off[col]; t < P.tri_off[col + 1]; ++t) {
    const int4 tr = P.tri[t];
    if (tr.z != cur) {
      if (cur >= 0) {
        double* D = blk(C, cur);
        D[e0] -= acc0;
        if (has1) D[e1] -= acc1;
      }
      cur = tr.z;
      acc0 = 0.0;
      acc1 = 0.0;
    }
    const double* Lr = blk(C, tr.x);
    const double* Lk = blk(C, tr.y);
    __syncwarp();
    st0[e0] = Lr[e0];
    st1[e0] = Lk[e0];
    if (has1) {
      st0[e1] = Lr[e1];
      st1[e1] = Lk[e1];
    }
    __syncwarp();
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int q = 0; q < 7; ++q) sa = fma(st0[7 * r0 + q], st1[7 * q0 + q], sa);
    if (has1) {
#pragma unroll
      for (int q = 0; q < 7; ++q) sb = fma(st0[7 * r1 + q], st1[7 * q1 + q], sb);
    }
    acc0 += sa;
    acc1 += sb;
  }
  if (cur >= 0) {
    double* D = blk(C, cur);
    D[e0] -= acc0;
    if (has1) D[e1] -= acc1;
  }
  __syncwarp();

  // (2) Cholesky of the diagonal block: lane r < 7 holds row r
  double* D = blk(C, dslot);
  double a[7];
  const bool act = lane < 7;
#pragma unroll
  for (int k = 0; k < 7; ++k) a[k] = act ? D[7 * lane + k] : 0.0;
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
  if (act) {
#pragma unroll
    for (int c = 0; c < 7; ++c) D[7 * lane + c] = (c <= lane) ? a[c] : 0.0;
    C.Dinv[7 * (col - C.c0) + lane] = myinv;
  }
  if (bad && lane == 0) *C.fail = 1;
  __syncwarp();

  // (3) off-diagonal blocks: B <- B L_kk^{-T}, one (block, row) per lane
  const int nb = P.col_slot[col + 1] - dslot - 1;
  if (nb > 0) {
    st0[e0] = D[e0];
    if (has1) st0[e1] = D[e1];
    if (act) st1[lane] = myinv;
    __syncwarp();
    for (int task = lane; task < 7 * nb; task += 32) {
      const int b = task / 7, i = task % 7;
      double* B = blk(C, dslot + 1 + b) + 7 * i;
      double x[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        double s = B[c];
#pragma unroll
        for (int q = 0; q < c; ++q) s = fma(-st0[7 * c + q], x[q], s);
        x[c] = s * st1[c];
      }
#pragma unroll
      for (int c = 0; c < 7; ++c) B[c] = x[c];
    }
    __syncwarp();
  }
}

// y_c <- L_cc^{-1} (y_c - sum_j L_cj y_j)
__device__ void forward_column(const SolveCtx& C, int col, int lane) {
  const SolverPlan& P = *C.P;
  const int lc = col - C.c0;
  double acc = 0.0;
  if (lane < 7) {
    acc = C.y[7 * lc + lane];
    for (int q = P.rs_off[col]; q < P.rs_off[col + 1]; ++q) {
      const int2 e = P.rs[q];
      const double* B = blk(C, e.x) + 7 * lane;
      const double* yj = C.y + 7 * (e.y - C.c0);
#pragma unroll
      for (int k = 0; k < 7; ++k) acc = fma(-B[k], yj[k], acc);
    }
  }
  const double* D = blk(C, P.col_slot[col]);
  const double dinv = lane < 7 ? C.Dinv[7 * lc + lane] : 0.0;
  double x = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    if (lane == k) x = acc * dinv;
    const double xk = __shfl_sync(kFull, x, k);
    if (lane > k && lane < 7) acc = fma(-D[7 * lane + k], xk, acc);
  }
  if (lane < 7) C.y[7 * lc + lane] = x;
}

// x_c <- L_cc^{-T} (y_c - sum_{r > c} L_rc^T x_r)
__device__ void backward_column(const SolveCtx& C, int col, int lane) {
  const SolverPlan& P = *C.P;
  const int lc = col - C.c0;
  const int dslot = P.col_slot[col];
  double acc = 0.0;
  if (lane < 7) {
    acc = C.y[7 * lc + lane];
    for (int s = dslot + 1; s < P.col_slot[col + 1]; ++s) {
      const double* B = blk(C, s);
      const double* xr = C.y + 7 * (P.slot_row[s] - C.c0);
#pragma unroll
      for (int i = 0; i < 7; ++i) acc = fma(-B[7 * i + lane], xr[i], acc);
    }
  }
  const double* D = blk(C, dslot);
  const double dinv = lane < 7 ? C.Dinv[7 * lc + lane] : 0.0;
  double x = 0.0;
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    if (lane == k) x = acc * dinv;
    const double xk = __shfl_sync(kFull, x, k);
    if (lane < k) acc = fma(-D[7 * k + lane], xk, acc);
  }
  if (lane < 7) C.y[7 * lc + lane] = x;
}

template <bool SMEM>
__global__ void __launch_bounds__(kSolveThreads) factor_solve_kernel(
    SolverPlan P, const double* __restrict__ A, double* Lg, double* Dg, const double* __restrict__ gvec, double* yg,
    double* __restrict__ tau, double lambda, double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn) {
  extern __shared__ __align__(16) double dyn[];
  __shared__ double stage[kSolveWarps][98];
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
  C.Dinv = SMEM ? dyn + (int64_t)nslot * 49 : Dg + (int64_t)c0 * 7;
  C.y = SMEM ? C.Dinv + (int64_t)ncol * 7 : yg + (int64_t)c0 * 7;
  C.s0 = s0;
  C.c0 = c0;
  C.stage = stage[warp];
  C.fail = &s_fail;
  const int lv0 = P.lvl_begin[g], lv1 = P.lvl_begin[g + 1];

  bool ok = false;
  int attempt = 0;
  double pow100 = 1.0;  // 100^attempt, exact in FP64
  for (; attempt < max_attempts; ++attempt, pow100 *= 100.0) {
    const double eps = eps0 * pow100;
    for (int64_t x = tid; x < (int64_t)nslot * 49; x += kSolveThreads) C.L[x] = A[(int64_t)s0 * 49 + x];
    __syncthreads();
    for (int c = tid; c < ncol; c += kSolveThreads) {
      const int ds = P.col_slot[c0 + c];
      double* D = blk(C, ds);
      const double* AD = A + (int64_t)ds * 49;
#pragma unroll
      for (int k = 0; k < 7; ++k) D[8 * k] += lambda * AD[8 * k] + eps;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int lv = lv0; lv < lv1; ++lv) {
      for (int q = P.lvl_off[lv] + warp; q < P.lvl_off[lv + 1]; q += kSolveWarps) factor_column(C, P.sched[q], lane);
      __syncthreads();
      if (s_fail) break;
    }
    ok = (s_fail == 0);
    __syncthreads();
    if (ok) break;
  }
  if (ok) {
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) C.y[x] = -gvec[7 * P.col_kf[c0 + x / 7] + x % 7];
    __syncthreads();
    for (int lv = lv0; lv < lv1; ++lv) {
      for (int q = P.lvl_off[lv] + warp; q < P.lvl_off[lv + 1]; q += kSolveWarps) forward_column(C, P.sched[q], lane);
      __syncthreads();
    }
    for (int lv = lv1 - 1; lv >= lv0; --lv) {
      for (int q = P.lvl_off[lv] + warp; q < P.lvl_off[lv + 1]; q += kSolveWarps) backward_column(C, P.sched[q], lane);
      __syncthreads();
    }
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) tau[7 * P.col_kf[c0 + x / 7] + x % 7] = C.y[x];
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
  const size_t static_bytes = sizeof(double) * kSolveWarps * 98 + 64;
  return optin > (int)static_bytes ? (size_t)optin - static_bytes : 0;
}

cudaError_t factor_solve_prepare(size_t smem_bytes) {
  return cudaFuncSetAttribute(factor_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t launch_factor_solve(int G, const SolverPlan& plan, bool smem, size_t smem_bytes, const double* A,
                                double* L, double* Dinv, const double* gvec, double* y, double* tau, double lambda,
                                double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn, cudaStream_t s) {
  if (G <= 0) return cudaSuccess;
  if (smem) {
    factor_solve_kernel<true><<<G, kSolveThreads, smem_bytes, s>>>(plan, A, L, Dinv, gvec, y, tau, lambda, eps0,
                                                                   max_attempts, ginfo, warn);
  } else {
    factor_solve_kernel<false><<<G, kSolveThreads, 0, s>>>(plan, A, L, Dinv, gvec, y, tau, lambda, eps0,
                                                           max_attempts, ginfo, warn);
  }
  return cudaGetLastError();
}

}  // namespace como3r
