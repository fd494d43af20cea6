// K3: damped block Cholesky factorisation and solve of the pose system, Eq. (normal),
// with the epsilon escalation of Sec. III-D, all in FP64.
//
// One CTA (16 warps) per graph.  The factor L (lower, 7x7 blocks; pattern, elimination
// order and task lists fixed at create) is computed one elimination-tree level at a
// time.  Within a level three task lists run, separated by CTA barriers:
//   D  four columns per warp (8 lanes each): Cholesky of the 7x7 diagonal block in
//      registers (lane r holds row r) with the right-hand side riding along as an eighth
//      row, which yields y_c = L_cc^{-1}(...) for free; a pivot that is not > 0 or not
//      finite fails the attempt;
//   T  one thread per row of every off-diagonal block (B <- B L_cc^{-T}), all independent
//      (the columns of L_cc^{-1}, needed only by the back substitution, are computed in
//      the U phase by threads the update tasks leave idle);
//   U  right-looking: two warps per destination block in any ancestor column (half the
//      entries each), L[dst] -= sum L_rj L_kj^T over the level's columns j (diagonal
//      destinations also update the forward right-hand side t_c -= L_cj y_j), so every
//      column has received all of its descendants' updates when its own level starts.
// Narrow levels (at most 4 columns of at most 3 off-diagonal blocks: the top of the tree)
// have no T list: one warp per column eliminates the whole column panel, its off-diagonal
// rows riding along with the diagonal block's, bitwise as D then T would.
// The update tasks into the next level's columns run in the U phase; the others run in
// the next level's D phase, alongside its diagonal factorisations (lookahead).
// A failed attempt restarts with eps_r = eps0 * 100^r; after max_attempts failures the
// update is zero (Sec. III-D).  Back substitution walks the levels from the root, each
// column x_c = L_cc^{-T}(y_c - sum_r L_rc^T x_r) with the precomputed L_cc^{-1}.
// FP64 on this GPU issues about one warp instruction per ~80 cycles per SM sub-partition
// (and has a long dependent latency), so the schedule keeps every lane of an FP64
// instruction busy and spreads the work of a level over all warps: a right-looking
// schedule spreads the update work evenly over the levels (a left-looking one piles
// the root's updates into the last, narrowest levels).
// The factor lives in shared memory when the graph's blocks fit, else in global memory.
#include <cooperative_groups.h>

#include <cstdint>
#include <mutex>

#include "como3r_internal.h"

namespace como3r {
namespace {

constexpr int kSolveThreads = 512;
// Pivot hand-over buffer of the four-warp panel (doubles: one 32-row column per pivot).
constexpr int kPanelXchg = 7 * 32;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// Local view of one graph's solver state: blocks, per-column scratch and plan arrays,
// all with graph-local indices (in shared memory, or the graph's part of global memory).
struct SolveCtx {
  double* L;              // slot s at L + 49 s
  double* S;              // column c at S + kColScratch c = [Dinv 7 | y 7 | Linv 49]
  const int* col_slot;    // [ncol + 1]
  const int* slot_row;    // [nslot]
  const int* sched;       // [ncol]
  const int4* tri;        // [ntri]
  const int4* utask;      // [nu]
  const int2* ttask;      // [nt]
  const int* lvl;         // [(nlev + 1) * 4]
  // multi-SM solve only: homes (rank << 24 | local index) of the graph's slots and columns
  const int* slot_home;
  const int* col_home;
  int rank;
  int nranks;             // CTAs of the cluster
};

// A location in the shared memory of CTA `rank` of this cluster (direct when it is ours).
__device__ __forceinline__ double* at_rank(double* p, int rank, int mine) {
  if (rank == mine) return p;
  return cooperative_groups::this_cluster().map_shared_rank(p, (unsigned)rank);
}
template <bool CL>
__device__ __forceinline__ double* blk(const SolveCtx& C, int s) {
  if constexpr (!CL) {
    return C.L + (int64_t)s * 49;
  } else {
    const int h = C.slot_home[s];
    return at_rank(C.L + (int64_t)(h & 0xffffff) * 49, h >> 24, C.rank);
  }
}
template <bool CL>
__device__ __forceinline__ double* dinv_of(const SolveCtx& C, int col) {
  if constexpr (!CL) {
    return C.S + (int64_t)col * kColScratch;
  } else {
    const int h = C.col_home[col];
    return at_rank(C.S + (int64_t)(h & 0xffffff) * kColScratch, h >> 24, C.rank);
  }
}
template <bool CL>
__device__ __forceinline__ double* y_of(const SolveCtx& C, int col) { return dinv_of<CL>(C, col) + 7; }
template <bool CL>
__device__ __forceinline__ double* linv_of(const SolveCtx& C, int col) { return dinv_of<CL>(C, col) + 14; }

// acc + sum_q a[q] b[q], q < 7: seven FP64 instructions (instruction count, not the
// dependent latency, is what limits FP64 work on this GPU)
__device__ __forceinline__ double dot7(const double* a, const double* b, double acc) {
#pragma unroll
  for (int q = 0; q < 7; ++q) acc = fma(a[q], b[q], acc);
  return acc;
}

// U: half h of one destination block (see file header), so that a block's two halves run
// on two warps (two SM sub-partitions: an FP64 warp instruction holds its sub-partition's
// pipe for ~80 cycles however few lanes are active).  Half 0: lane l < 28 owns entry l of
// the 7x7 block, lanes 28..31 rows 0..3 of the forward right-hand side; half 1: lane
// l < 21 owns entry 28 + l, lanes 21..23 rows 4..6 (right-hand side rows: diagonal
// destinations only).  Each entry is one chain of FMAs over the level's triplets.
template <bool CL>
__device__ void update_half(const SolveCtx& C, int4 task, int h, int lane) {
  const int ne = h ? 21 : 28;
  const bool ent = lane < ne;
  if (!ent && (task.w < 0 || lane >= ne + (h ? 3 : 4))) return;
  const int e = (h ? 28 : 0) + lane;
  const int r = ent ? e / 7 : (h ? 4 : 0) + lane - ne, q = e % 7;
  double* dst = ent ? blk<CL>(C, task.x) + e : y_of<CL>(C, task.w) + r;
  // the destination itself seeds the chain: L[dst] - sum = -(sum - L[dst])
  double a = -*dst;
  for (int t = task.y; t < task.z; ++t) {
    const int4 tr = C.tri[t];
    a = dot7(blk<CL>(C, tr.x) + 7 * r, ent ? blk<CL>(C, tr.y) + 7 * q : y_of<CL>(C, tr.w), a);
  }
  *dst = -a;
}

// 1/sqrt(p) of a pivot p > 0: an FP32 seed (exponent and leading mantissa bits moved on
// the ALU, the hardware reciprocal-square-root approximation, widened on the ALU) and one
// Newton step in FP64, y1 = y0 (3/2 - p (y0/2) y0): relative error ~1e-13 (the seed's
// ~2^-22, squared), in about half the dependent latency of the FP64 rsqrt, which sits on
// the factorisation's critical chain seven times per column.  Pivots outside 2^+-100
// take the FP64 rsqrt, out of line (if-converted it would run for every pivot).
__device__ __noinline__ double rsqrt_wide_range(double p) { return rsqrt(p); }
__device__ __forceinline__ double rsqrt_pivot(double p) {
  const long long b = __double_as_longlong(p);
  const int ex = (int)((b >> 52) & 0x7ff) - 1023;
  if (ex < -100 || ex > 100) return rsqrt_wide_range(p);
  const float pf = __uint_as_float(((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff));
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(pf));
  // p (y0 / 2) is bitwise (p / 2) y0: halving is exact on both sides, and it saves an
  // FP64 instruction on the pivot's chain
  const double y0 = widen_f32(yf), hy0 = widen_f32(0.5f * yf);
  const double t = p * hy0;
  return y0 * fma(-t, y0, 1.5);
}

// Right-looking elimination of a column's seven pivots, one row per lane in groups of W
// lanes: lane sl < 7 of a group holds row sl of the diagonal block, lanes sl >= 7 rows
// below it (the forward right-hand side, off-diagonal rows), which end as L_rk = B_rk
// L_cc^{-T} (and y_c = L_cc^{-1} t_c) by the same operations, in the same order, as the
// off-diagonal solve below.  A pivot that is not > 0 or not finite sets `bad`; myinv is
// the pivot's 1 / sqrt for lane sl < 7.
template <int W>
__device__ __forceinline__ void eliminate7(double (&a)[7], int sl, bool& bad, double& myinv) {
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double p = __shfl_sync(kFull, a[k], k, W);
    // p > 0 and finite, tested on the bit pattern (keeps the FP64 pipe free)
    const long long pb = __double_as_longlong(p);
    const bool okp = pb > 0 && pb < 0x7ff0000000000000LL;
    bad = bad || !okp;
    const double inv = rsqrt_pivot(okp ? p : 1.0);
    const double lk = ((sl == k) ? p : a[k]) * inv;
    if (sl == k) myinv = inv;
    if (sl >= k) a[k] = lk;
#pragma unroll
    for (int c = k + 1; c < 7; ++c) {
      const double lc = __shfl_sync(kFull, lk, c, W);
      if (sl >= c) a[c] = fma(-lk, lc, a[c]);
    }
  }
}

template <bool CL>
__device__ __forceinline__ void raise_fail(const SolveCtx& C, int* fail) {
  if constexpr (CL) {  // every CTA's copy of the level's flag: each reads its own after the barrier
    for (int r = 0; r < C.nranks; ++r) *cooperative_groups::this_cluster().map_shared_rank(fail, (unsigned)r) = 1;
  } else {
    *fail = 1;
  }
}

// D: Cholesky of diagonal blocks, four columns per warp (FP64 instructions occupy the
// pipe for the whole warp, so idle lanes would waste it).  Segment s = lane / 8 handles
// column cols[s]; within it lane r < 7 holds row r and lane 7 holds the forward
// right-hand side as an eighth row, so the elimination also yields y_c = L_cc^{-1} t_c.
// Segments without a column factor an identity block and write nothing.
template <bool CL>
__device__ void diag_factor4(const SolveCtx& C, const int* cols, int ncols, int lane, int* fail) {
  const int seg = lane >> 3, sl = lane & 7;
  const bool active = seg < ncols;
  const int col = cols[active ? seg : 0];
  const int dslot = C.col_slot[col];
  double* D = blk<CL>(C, dslot);
  double* y = y_of<CL>(C, col);
  double a[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    if (active) a[c] = sl < 7 ? D[7 * sl + c] : y[c];
    else a[c] = (c == sl) ? 1.0 : 0.0;
  }
  bool bad = false;
  double myinv = 0.0;
  eliminate7<8>(a, sl, bad, myinv);
  if (active) {
    if (sl < 7) {
#pragma unroll
      for (int c = 0; c < 7; ++c) D[7 * sl + c] = (c <= sl) ? a[c] : 0.0;
      dinv_of<CL>(C, col)[sl] = myinv;
    } else {
#pragma unroll
      for (int c = 0; c < 7; ++c) y[c] = a[c];
    }
    if (bad && sl == 0) raise_fail<CL>(C, fail);
  }
}

// D of a panel level (no off-diagonal solve tasks): one column per warp, the whole column
// at once.  Lane r < 7 holds row r of the diagonal block, lane 7 the forward right-hand
// side, lane 8 + 7 b + i row i of the column's off-diagonal block b (at most kPanelBlocks
// blocks), so the elimination also yields the off-diagonal blocks of L, bitwise as the
// separate off-diagonal solve would.  A column with more blocks (never planned) fails the
// attempt rather than leave blocks unsolved.
template <bool CL>
__device__ void panel_factor(const SolveCtx& C, int col, int lane, int* fail) {
  const int dslot = C.col_slot[col], nb = C.col_slot[col + 1] - dslot - 1;
  if (nb > kPanelBlocks) {
    if (lane == 0) raise_fail<CL>(C, fail);
    return;
  }
  double* D = blk<CL>(C, dslot);
  double* y = y_of<CL>(C, col);
  double* row = nullptr;
  if (lane < 7) row = D + 7 * lane;
  else if (lane == 7) row = y;
  else if (lane < 8 + 7 * nb) row = blk<CL>(C, dslot + 1 + (lane - 8) / 7) + 7 * ((lane - 8) % 7);
  double a[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) a[c] = row ? row[c] : 0.0;
  bool bad = false;
  double myinv = 0.0;
  eliminate7<32>(a, lane, bad, myinv);
  if (lane < 7) {
#pragma unroll
    for (int c = 0; c < 7; ++c) row[c] = (c <= lane) ? a[c] : 0.0;
    dinv_of<CL>(C, col)[lane] = myinv;
  } else if (row) {
#pragma unroll
    for (int c = 0; c < 7; ++c) row[c] = a[c];
  }
  if (bad && lane == 0) raise_fail<CL>(C, fail);
}

// The same panel on warps 0..3 of the CTA, for a CTA whose only column of the level it
// is: every FP64 instruction holds its SM sub-partition's FP64 unit for ~80 cycles
// whether or not it depends on the previous one, so one warp's ~50 instructions per
// column are the level's critical path.  Here warp w keeps columns w and w + 4 of every
// row (lane r = row r as in panel_factor) and only the pivot's owner forms 1 / sqrt(p)
// and the scaled column l_.k, which it hands to the others through `xbuf` (slot k per
// pivot, so it is never rewritten within a column) across one named barrier of the four
// warps (barrier 1; all four warps call this together and pass every barrier).  Every
// entry sees the operations of panel_factor in the same order: bitwise the same factor.
// A column with nb >= 4 off-diagonal blocks has 8 + 7 nb > 32 rows: rows 32 and up stay
// out of the elimination (any instruction for them in the pivot loop would lengthen every
// column's chain) and are solved afterwards against the finished L_cc with the operations
// of the off-diagonal solve (bitwise what the elimination would give them): in the narrow
// form (nb <= kPanel4Narrow) rows 32..35 by lanes 0..3 of warp 0, in the wide form row
// 32 + t by thread t of the four warps.
__device__ __forceinline__ void panel_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
constexpr int kPanel4Narrow = 4;

template <bool CL, bool WIDE>
__device__ void panel_factor4_impl(const SolveCtx& C, int col, int warp, int lane, double* xbuf, int* fail) {
  const int dslot = C.col_slot[col], nb = C.col_slot[col + 1] - dslot - 1;
  if (nb > (WIDE ? kPanel4Blocks : kPanel4Narrow)) {  // never planned; the same decision in all four warps
    if (warp == 0 && lane == 0) raise_fail<CL>(C, fail);
    return;
  }
  const int rows = min(8 + 7 * nb, 32);
  const bool has = lane < rows;
  double* D = blk<CL>(C, dslot);
  double* row = nullptr;
  if (has)
    row = lane < 7 ? D + 7 * lane
                   : (lane == 7 ? y_of<CL>(C, col) : blk<CL>(C, dslot + 1 + (lane - 8) / 7) + 7 * ((lane - 8) % 7));
  const int c0 = warp, c1 = warp + 4;
  const bool two = c1 < 7;
  double a0 = has ? row[c0] : 0.0, a1 = (has && two) ? row[c1] : 0.0;
  bool bad = false;
  double myinv = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    if (warp == (k & 3)) {
      const double ak = k < 4 ? a0 : a1;
      const double p = __shfl_sync(kFull, ak, k);
      // p > 0 and finite, tested on the bit pattern (keeps the FP64 pipe free)
      const long long pb = __double_as_longlong(p);
      const bool okp = pb > 0 && pb < 0x7ff0000000000000LL;
      bad = bad || !okp;
      const double inv = rsqrt_pivot(okp ? p : 1.0);
      const double lk = ((lane == k) ? p : ak) * inv;
      if (lane == k) myinv = inv;
      if (lane >= k) {
        if (k < 4) a0 = lk;
        else a1 = lk;
      }
      xbuf[32 * k + lane] = lk;
    }
    panel_barrier();
    const double lr = xbuf[32 * k + lane];
    if (c0 > k) {
      const double lc = xbuf[32 * k + c0];
      if (lane >= c0) a0 = fma(-lr, lc, a0);
    }
    if (two && c1 > k) {
      const double lc = xbuf[32 * k + c1];
      if (lane >= c1) a1 = fma(-lr, lc, a1);
    }
  }
  if (has) {
    if (lane < 7) {
      row[c0] = (c0 <= lane) ? a0 : 0.0;
      if (two) row[c1] = (c1 <= lane) ? a1 : 0.0;
    } else {
      row[c0] = a0;
      if (two) row[c1] = a1;
    }
  }
  if (lane < 7 && (lane & 3) == warp) dinv_of<CL>(C, col)[lane] = myinv;
  if (__any_sync(kFull, bad) && lane == 0) raise_fail<CL>(C, fail);
  const int ntail = 8 + 7 * nb - 32;
  if (ntail > 0) {    // rows 32.. (the same decision in all four warps)
    panel_barrier();  // L_cc and its pivot inverses are in place
    const int t = WIDE ? 32 * warp + lane : (warp == 0 ? lane : 32);
    if (t < ntail) {
      const double* Lc = D;
      const double* dv = dinv_of<CL>(C, col);
      double* B = WIDE ? blk<CL>(C, dslot + 1 + (24 + t) / 7) + 7 * ((24 + t) % 7)
                       : blk<CL>(C, dslot + kPanel4Narrow) + 7 * (3 + lane);
      double sr[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) sr[c] = B[c];
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        sr[q] *= dv[q];
#pragma unroll
        for (int c = q + 1; c < 7; ++c) sr[c] = fma(-Lc[7 * c + q], sr[q], sr[c]);
      }
#pragma unroll
      for (int c = 0; c < 7; ++c) B[c] = sr[c];
    }
  }
}

// Four-warp panel of a single column: the narrow form (at most kPanel4Narrow off-diagonal
// blocks, most single-column levels) and the wide form are separate copies; one copy for
// both made every narrow panel ~0.14 us slower.
template <bool CL>
__device__ __forceinline__ void panel_factor4(const SolveCtx& C, int col, int warp, int lane, double* xbuf,
                                              int* fail) {
  if (C.col_slot[col + 1] - C.col_slot[col] - 1 <= kPanel4Narrow)
    panel_factor4_impl<CL, false>(C, col, warp, lane, xbuf, fail);
  else
    panel_factor4_impl<CL, true>(C, col, warp, lane, xbuf, fail);
}

// T: item x < 7 * nt: row (x % 7) of off-diagonal block ttask[t0 + x / 7]; items from
// tpad = 7 * nt rounded up to a warp on: column (x % 7) of L_cc^{-1} for the level column
// sched[s0 + (x - tpad) / 7].  The two kinds never share a warp (they would diverge).
template <bool CL>
__device__ void trsm_or_inverse(const SolveCtx& C, int t0, int nt, int tpad, int s0, int x) {
  // Both solves are right-looking: once x_q is known its term leaves every later row at
  // once (independent FMAs), so the dependent chain is one multiply and one FMA per
  // unknown (14 deep) instead of a dot product per unknown (28 deep).
  if (x < 7 * nt) {
    const int2 tt = C.ttask[t0 + x / 7];
    const int i = x % 7;
    const double* Lc = blk<CL>(C, C.col_slot[tt.y]);
    const double* dv = dinv_of<CL>(C, tt.y);
    double* B = blk<CL>(C, tt.x) + 7 * i;
    double sr[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) sr[c] = B[c];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      sr[q] *= dv[q];  // x_q
#pragma unroll
      for (int c = q + 1; c < 7; ++c) sr[c] = fma(-Lc[7 * c + q], sr[q], sr[c]);
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) B[c] = sr[c];
  } else if (x >= tpad) {
    const int k = (x - tpad) / 7, c = (x - tpad) % 7;
    const int col = C.sched[s0 + k];
    const double* Lc = blk<CL>(C, C.col_slot[col]);
    const double* dv = dinv_of<CL>(C, col);
    double* X = linv_of<CL>(C, col);
    // column c of L_cc^{-1}: xc[r] = 0 (r < c), dv[c] (r = c), -dv[r] sum_{c<=q<r} L[r][q] xc[q]
    double xc[7], acc[7];
#pragma unroll
    for (int r = 0; r < 7; ++r) acc[r] = 0.0;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      if (q < c) {
        xc[q] = 0.0;
      } else {
        xc[q] = (q == c) ? dv[q] : -acc[q] * dv[q];
#pragma unroll
        for (int r = q + 1; r < 7; ++r) acc[r] = fma(Lc[7 * r + q], xc[q], acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < 7; ++r) X[7 * r + c] = xc[r];
  }
}

// back substitution of one column: x_c = L_cc^{-T} (y_c - sum_r L_rc^T x_r)
template <bool CL>
__device__ void backward_column(const SolveCtx& C, int col, int lane) {
  const int grp = lane / 7, q = lane % 7;
  const int s_begin = C.col_slot[col] + 1, nb = C.col_slot[col + 1] - s_begin;
  double part = 0.0;
  if (grp < 4) {
    for (int b = grp; b < nb; b += 4) {
      const double* B = blk<CL>(C, s_begin + b);
      const double* xr = y_of<CL>(C, C.slot_row[s_begin + b]);
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
  double* y = y_of<CL>(C, col);
  const double t = (lane < 7) ? y[q] - ((part + o1) + (o2 + o3)) : 0.0;
  const double* X = linv_of<CL>(C, col);
  double xq = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const double tr = __shfl_sync(kFull, t, r);
    if (lane < 7 && r >= q) xq = fma(X[7 * r + q], tr, xq);
  }
  __syncwarp();
  if (lane < 7) y[q] = xq;
}

template <typename T>
__device__ __forceinline__ T* carve(unsigned char*& p, size_t count) {
  T* r = reinterpret_cast<T*>(p);
  p += (sizeof(T) * count + 15) & ~size_t(15);
  return r;
}

// Global -> shared copies issued as cp.async (all in flight at once; completed by
// async_wait_all): element sizes 4, 8 and 16 bytes, each source element naturally aligned.
template <typename T>
__device__ __forceinline__ void stage(T* dst, const T* src, int64_t n, int tid, int nthreads = kSolveThreads) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "cp.async element size");
  for (int64_t x = tid; x < n; x += nthreads) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + x);
    if constexpr (sizeof(T) == 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + x) : "memory");
    else if constexpr (sizeof(T) == 8)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src + x) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src + x) : "memory");
  }
}
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <bool SMEM>
__global__ void __launch_bounds__(kSolveThreads, 1) factor_solve_kernel(
    SolverPlan P, const double* __restrict__ A, double* Lg, double* Sg, const double* __restrict__ gvec,
    double* __restrict__ tau, double lambda, double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn,
    FactorKeep keep) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ int s_fail;
  __shared__ double s_xbuf[kPanelXchg];
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int* m = P.meta + kMetaCount * g;
  const int cbase = m[kMetaColBase], ncol = m[kMetaNCol], sbase = m[kMetaSlotBase], nslot = m[kMetaNSlot];
  const int nlev = m[kMetaNLvl];
  if (ncol == 0) {
    if (tid == 0) {
      ginfo[g].attempts = 1;
      ginfo[g].solved = 1;
      ginfo[g].done_ns = globaltimer_ns();
    }
    return;
  }
  const int* gcol_slot = P.col_slot + cbase + g;
  const int* gslot_row = P.slot_row + sbase;
  const int* gsched = P.sched + cbase;
  const int4* gtri = P.tri + m[kMetaTriBase];
  const int4* gutask = P.utask + m[kMetaUBase];
  const int2* gttask = P.ttask + m[kMetaTBase];
  const int* glvl = P.lvl + 4 * m[kMetaLvlBase];
  SolveCtx C;
  if (SMEM) {
    unsigned char* q = dyn;
    C.L = carve<double>(q, (size_t)nslot * 49 + (size_t)ncol * kColScratch);
    C.S = C.L + (size_t)nslot * 49;
    int4* tri = carve<int4>(q, m[kMetaNTri]);
    int4* ut = carve<int4>(q, m[kMetaNU]);
    int2* tt = carve<int2>(q, m[kMetaNT]);
    int* cs = carve<int>(q, ncol + 1);
    int* sr = carve<int>(q, nslot);
    int* sc = carve<int>(q, ncol);
    int* lv = carve<int>(q, 4 * (nlev + 1));
    stage(tri, gtri, m[kMetaNTri], tid);
    stage(ut, gutask, m[kMetaNU], tid);
    stage(tt, gttask, m[kMetaNT], tid);
    stage(cs, gcol_slot, ncol + 1, tid);
    stage(sr, gslot_row, nslot, tid);
    stage(sc, gsched, ncol, tid);
    stage(lv, glvl, 4 * (nlev + 1), tid);
    C.tri = tri; C.utask = ut; C.ttask = tt; C.col_slot = cs; C.slot_row = sr; C.sched = sc; C.lvl = lv;
  } else {
    C.L = Lg + (int64_t)sbase * 49;
    C.S = Sg + (int64_t)cbase * kColScratch;
    C.tri = gtri; C.utask = gutask; C.ttask = gttask; C.col_slot = gcol_slot; C.slot_row = gslot_row;
    C.sched = gsched; C.lvl = glvl;
  }
  const double* Ag = A + (int64_t)sbase * 49;
  const int* col_kf = P.col_kf + cbase;

  int attempt = 0;
  bool ok = false;
  double pow100 = 1.0;  // 100^attempt, exact in FP64
  for (; attempt < max_attempts; ++attempt, pow100 *= 100.0) {
    const double eps = eps0 * pow100;
    if (SMEM) {
      stage(C.L, Ag, (int64_t)nslot * 49, tid);
      async_wait_all();  // also completes the plan staged above
    } else {
      for (int64_t x = tid; x < (int64_t)nslot * 49; x += kSolveThreads) C.L[x] = Ag[x];
    }
    __syncthreads();
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) {
      const int col = x / 7, k = x % 7;
      const int ds = C.col_slot[col];
      blk<false>(C, ds)[8 * k] += lambda * Ag[(int64_t)ds * 49 + 8 * k] + eps;
      y_of<false>(C, col)[k] = -gvec[7 * col_kf[col] + k];
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int lv = 0; lv < nlev; ++lv) {
      // [sched, near updates, far updates, ttask] offsets of this level; the next level's at +4
      const int* L0 = C.lvl + 4 * lv;
      // D(lv) in groups of four columns, with the far updates of level lv - 1 (their
      // destinations lie two or more levels up, so they do not touch this level's blocks):
      // the latency-bound factorisations and the FP64-throughput-bound updates overlap
      // a level without off-diagonal solve tasks is a panel level: one column per warp
      const int ncl = L0[4] - L0[0], nt = L0[7] - L0[3];
      const bool panel = nt == 0;
      const int nd = panel ? ncl : (ncl + 3) / 4;
      const int f0 = lv > 0 ? C.lvl[4 * (lv - 1) + 2] : 0, nf = lv > 0 ? L0[1] - f0 : 0;
      if (panel && ncl == 1) {  // one column: spread over four warps, far updates on the rest
        if (warp < 4) panel_factor4<false>(C, C.sched[L0[0]], warp, lane, s_xbuf, &s_fail);
        else
          for (int i = warp - 4; i < 2 * nf; i += kSolveWarps - 4)
            update_half<false>(C, C.utask[f0 + i / 2], i & 1, lane);
      } else {
        for (int i = warp; i < nd + 2 * nf; i += kSolveWarps) {
          if (i >= nd) update_half<false>(C, C.utask[f0 + (i - nd) / 2], (i - nd) & 1, lane);
          else if (panel) panel_factor<false>(C, C.sched[L0[0] + i], lane, &s_fail);
          else diag_factor4<false>(C, C.sched + L0[0] + 4 * i, min(4, ncl - 4 * i), lane, &s_fail);
        }
      }
      __syncthreads();
      if (s_fail) break;
      if (!panel) {
        for (int x = tid; x < 7 * nt; x += kSolveThreads) trsm_or_inverse<false>(C, L0[3], nt, 7 * nt, L0[0], x);
        __syncthreads();
      }
      for (int x = warp; x < 2 * (L0[2] - L0[1]); x += kSolveWarps)
        update_half<false>(C, C.utask[L0[1] + x / 2], x & 1, lane);
      // the level's L_cc^{-1} (read only by the back substitution), off the critical path:
      // threads of the last warps, which the update tasks leave idle first
      for (int x = kSolveThreads - 1 - tid; x < 7 * ncl; x += kSolveThreads)
        trsm_or_inverse<false>(C, 0, 0, 0, L0[0], x);
      __syncthreads();
    }
    if (s_fail == 0 && nlev > 0) {
      // far updates of the last level (none in an elimination tree: its columns are roots)
      const int* L0 = C.lvl + 4 * (nlev - 1);
      for (int x = warp; x < 2 * (L0[5] - L0[2]); x += kSolveWarps)
        update_half<false>(C, C.utask[L0[2] + x / 2], x & 1, lane);
      __syncthreads();
    }
    ok = (s_fail == 0);
    __syncthreads();
    if (ok) break;
  }
  async_wait_all();  // nothing left in flight when no attempt ran
  if (ok) {
    for (int lv = nlev - 1; lv >= 0; --lv) {
      const int* L0 = C.lvl + 4 * lv;
      for (int q = L0[0] + warp; q < L0[4]; q += kSolveWarps) backward_column<false>(C, C.sched[q], lane);
      __syncthreads();
    }
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) tau[7 * col_kf[x / 7] + x % 7] = y_of<false>(C, x / 7)[x % 7];
    if (keep.L) {
      for (int64_t x = tid; x < (int64_t)nslot * 49; x += kSolveThreads) keep.L[(int64_t)sbase * 49 + x] = C.L[x];
      for (int64_t x = tid; x < (int64_t)ncol * kColScratch; x += kSolveThreads)
        keep.S[(int64_t)cbase * kColScratch + x] = C.S[x];
    }
  } else {
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) tau[7 * col_kf[x / 7] + x % 7] = 0.0;
  }
  __syncthreads();  // every thread's tau is written before the stamp
  if (tid == 0) {
    ginfo[g].attempts = ok ? attempt + 1 : max_attempts;
    ginfo[g].solved = ok ? 1 : 0;
    ginfo[g].done_ns = globaltimer_ns();
    if (!ok) atomicOr(warn, 1);
  }
}

// ---- grid-wide solve of one large graph (factor in global memory) -------------------
// For a graph whose factor fits neither one SM's nor a cluster's shared memory: the task
// lists of factor_solve_kernel (graph 0), spread over every warp of a co-resident grid,
// with a grid barrier where that kernel has a CTA barrier, so the factor is bitwise the
// same.  The barrier: CTA barrier, then thread 0 arrives on a global counter (the last
// arrival resets it and advances the generation) and waits for the generation to change,
// fenced on both sides so that every write before the barrier is seen after it on every
// SM; the wait has an iteration limit (sync->err, and the solve gives up).
constexpr unsigned long long kGridSpinLimit = 1ull << 24;  // ~1 s of 64-ns sleeps

// `extra` arrivals are expected beyond the grid's CTAs: 0 always, except in the test that
// makes every wait run out (no arrival completes the count).
__device__ bool grid_barrier(GridSync* gs, int* s_ok, unsigned extra) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &gs->gen;
    const unsigned g0 = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&gs->count, 1u) == gridDim.x - 1 + extra) {
      gs->count = 0;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      unsigned long long it = 0;
      while (*vgen == g0) {
        if (++it > kGridSpinLimit) {
          atomicExch(&gs->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)&gs->err) ok = 0;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// The global-memory solve of graph g by a group of `gsize` CTAs (this one is `grank`): the
// task lists of factor_solve_kernel spread over every warp of the group, with bar.sync()
// wherever that kernel has a CTA barrier, so the factor is bitwise the same.  `fail` is the
// graph's pair of level failure flags in global memory.  bar.sync() returns false when a
// bounded wait gave up (the grid barrier only): the graph then gets the zero update.
template <class Bar>
__device__ void solve_graph_global(const SolverPlan& P, int g, const double* __restrict__ A, double* Lg, double* Sg,
                                   const double* __restrict__ gvec, double* __restrict__ tau, double lambda,
                                   double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn, FactorKeep keep,
                                   int* fail2, int grank, int gsize, Bar& bar, double* s_xbuf) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gw = grank * kSolveWarps + warp, GW = gsize * kSolveWarps;
  const int gt = grank * kSolveThreads + tid, GT = gsize * kSolveThreads;
  const int* m = P.meta + kMetaCount * g;
  const int cbase = m[kMetaColBase], ncol = m[kMetaNCol], sbase = m[kMetaSlotBase], nslot = m[kMetaNSlot];
  const int nlev = m[kMetaNLvl];
  if (ncol == 0) {  // the same in every CTA of the group
    if (gt == 0) {
      ginfo[g].attempts = 1;
      ginfo[g].solved = 1;
      ginfo[g].done_ns = globaltimer_ns();
    }
    return;
  }
  SolveCtx C;
  C.L = Lg + (int64_t)sbase * 49;
  C.S = Sg + (int64_t)cbase * kColScratch;
  C.col_slot = P.col_slot + cbase + g;
  C.slot_row = P.slot_row + sbase;
  C.sched = P.sched + cbase;
  C.tri = P.tri + m[kMetaTriBase];
  C.utask = P.utask + m[kMetaUBase];
  C.ttask = P.ttask + m[kMetaTBase];
  C.lvl = P.lvl + 4 * m[kMetaLvlBase];
  C.slot_home = nullptr;
  C.col_home = nullptr;
  C.rank = 0;
  C.nranks = 1;
  const double* Ag = A + (int64_t)sbase * 49;
  const int* col_kf = P.col_kf + cbase;
  volatile int* vfail = fail2;

  int attempt = 0;
  bool ok = false, alive = true;
  double pow100 = 1.0;
  for (; attempt < max_attempts && alive; ++attempt, pow100 *= 100.0) {
    const double eps = eps0 * pow100;
    for (int64_t x = gt; x < (int64_t)nslot * 49; x += GT) C.L[x] = Ag[x];
    if (gt == 0) vfail[0] = 0;
    if (!(alive = bar.sync())) break;
    for (int x = gt; x < 7 * ncol; x += GT) {
      const int col = x / 7, k = x % 7;
      const int ds = C.col_slot[col];
      blk<false>(C, ds)[8 * k] += lambda * Ag[(int64_t)ds * 49 + 8 * k] + eps;
      y_of<false>(C, col)[k] = -gvec[7 * col_kf[col] + k];
    }
    if (!(alive = bar.sync())) break;
    bool failed = false;
    for (int lv = 0; lv < nlev; ++lv) {
      const int* L0 = C.lvl + 4 * lv;
      const int ncl = L0[4] - L0[0], nt = L0[7] - L0[3];
      const bool panel = nt == 0;
      const int nd = panel ? ncl : (ncl + 3) / 4;
      const int f0 = lv > 0 ? C.lvl[4 * (lv - 1) + 2] : 0, nf = lv > 0 ? L0[1] - f0 : 0;
      int* fail = fail2 + (lv & 1);
      if (panel && ncl == 1) {
        if (grank == 0 && warp < 4) {
          panel_factor4<false>(C, C.sched[L0[0]], warp, lane, s_xbuf, fail);
        } else {
          for (int i = gw - 4; i < 2 * nf; i += GW - 4) update_half<false>(C, C.utask[f0 + i / 2], i & 1, lane);
        }
      } else {
        for (int i = gw; i < nd + 2 * nf; i += GW) {
          if (i >= nd) update_half<false>(C, C.utask[f0 + (i - nd) / 2], (i - nd) & 1, lane);
          else if (panel) panel_factor<false>(C, C.sched[L0[0] + i], lane, fail);
          else diag_factor4<false>(C, C.sched + L0[0] + 4 * i, min(4, ncl - 4 * i), lane, fail);
        }
      }
      // the next level's flag: its last readers passed the previous barrier, its writers
      // start after this one
      if (gt == 0) vfail[(lv + 1) & 1] = 0;
      if (!(alive = bar.sync())) break;
      if (vfail[lv & 1]) {
        // every CTA has read the flag before any can reset it for the next attempt
        failed = true;
        alive = bar.sync();
        break;
      }
      if (!panel) {
        for (int x = gt; x < 7 * nt; x += GT) trsm_or_inverse<false>(C, L0[3], nt, 7 * nt, L0[0], x);
        if (!(alive = bar.sync())) break;
      }
      for (int x = gw; x < 2 * (L0[2] - L0[1]); x += GW) update_half<false>(C, C.utask[L0[1] + x / 2], x & 1, lane);
      // L_cc^{-1} of the level's columns (read only by the back substitution): the last
      // threads of the group, which the update tasks leave idle first
      for (int x = GT - 1 - gt; x < 7 * ncl; x += GT) trsm_or_inverse<false>(C, 0, 0, 0, L0[0], x);
      if (!(alive = bar.sync())) break;
    }
    if (!alive) break;
    if (!failed) {
      const int* L0 = C.lvl + 4 * (nlev - 1);  // far updates of the last level (none in an elimination tree)
      for (int x = gw; x < 2 * (L0[5] - L0[2]); x += GW) update_half<false>(C, C.utask[L0[2] + x / 2], x & 1, lane);
      if (!(alive = bar.sync())) break;
      ok = true;
      break;
    }
  }
  if (ok && alive) {
    for (int lv = nlev - 1; lv >= 0 && alive; --lv) {
      const int* L0 = C.lvl + 4 * lv;
      for (int q = L0[0] + gw; q < L0[4]; q += GW) backward_column<false>(C, C.sched[q], lane);
      alive = bar.sync();
    }
  }
  bool solved = ok && alive;
  for (int x = gt; x < 7 * ncol; x += GT) tau[7 * col_kf[x / 7] + x % 7] = solved ? y_of<false>(C, x / 7)[x % 7] : 0.0;
  if (solved && keep.L) {  // (the back substitution's last barrier ordered every write before these reads)
    for (int64_t x = gt; x < (int64_t)nslot * 49; x += GT) keep.L[(int64_t)sbase * 49 + x] = C.L[x];
    for (int64_t x = gt; x < (int64_t)ncol * kColScratch; x += GT) keep.S[(int64_t)cbase * kColScratch + x] = C.S[x];
  }
  // every CTA's tau is written before the stamp; a CTA whose last wait ran out zeroes its
  // part again (the others then run out too, or had already given up and written zeros)
  if (alive) alive = bar.sync();
  if (solved && !alive) {
    solved = false;
    for (int x = gt; x < 7 * ncol; x += GT) tau[7 * col_kf[x / 7] + x % 7] = 0.0;
  }
  if (gt == 0) {
    ginfo[g].attempts = solved ? attempt + 1 : max_attempts;
    ginfo[g].solved = solved ? 1 : 0;
    ginfo[g].done_ns = globaltimer_ns();
    if (!solved) atomicOr(warn, 1);
  }
}

struct GridBar {  // the bounded grid barrier of a cooperative launch
  GridSync* gs;
  int* s_ok;
  unsigned extra;
  __device__ bool sync() { return grid_barrier(gs, s_ok, extra); }
};
struct ClusterBar {  // the thread-block cluster's hardware barrier
  __device__ bool sync() {
    cooperative_groups::this_cluster().sync();
    return true;
  }
};
struct CtaBar {
  __device__ bool sync() {
    __syncthreads();
    return true;
  }
};

__global__ void __launch_bounds__(kSolveThreads, 1) factor_solve_grid_kernel(
    SolverPlan P, const double* __restrict__ A, double* Lg, double* Sg, const double* __restrict__ gvec,
    double* __restrict__ tau, double lambda, double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn,
    FactorKeep keep, GridSync* gs, unsigned extra) {
  __shared__ double s_xbuf[kPanelXchg];
  __shared__ int s_ok;
  GridBar bar{gs, &s_ok, extra};
  solve_graph_global(P, 0, A, Lg, Sg, gvec, tau, lambda, eps0, max_attempts, ginfo, warn, keep, gs->fail,
                     (int)blockIdx.x, (int)gridDim.x, bar, s_xbuf);
}

// ---- batches with large graphs: cluster groups (factor in global memory) ------------------
// One launch of clusters of kGroupCTAs CTAs.  CTA b runs the graphs gtask[b] = (list offset,
// count, rank in group, group size) of the list glist: a cluster whose CTAs all list the
// same large graph solves it together (group size kGroupCTAs, cluster barriers); any other
// CTA solves its own graphs one after the other (group size 1, CTA barriers).  Per graph
// two failure flags in gfail.
__global__ void __launch_bounds__(kSolveThreads, 1) factor_solve_group_kernel(
    SolverPlan P, const int4* __restrict__ gtask, const int32_t* __restrict__ glist, const double* __restrict__ A,
    double* Lg, double* Sg, const double* __restrict__ gvec, double* __restrict__ tau, double lambda, double eps0,
    int max_attempts, GraphInfoDev* ginfo, int* warn, FactorKeep keep, int* gfail) {
  __shared__ double s_xbuf[kPanelXchg];
  const int4 t = gtask[blockIdx.x];
  for (int k = 0; k < t.y; ++k) {
    const int g = glist[t.x + k];
    if (t.w > 1) {
      ClusterBar bar;
      solve_graph_global(P, g, A, Lg, Sg, gvec, tau, lambda, eps0, max_attempts, ginfo, warn, keep, gfail + 2 * g,
                         t.z, t.w, bar, s_xbuf);
    } else {
      CtaBar bar;
      solve_graph_global(P, g, A, Lg, Sg, gvec, tau, lambda, eps0, max_attempts, ginfo, warn, keep, gfail + 2 * g,
                         0, 1, bar, s_xbuf);
      __syncthreads();  // the next graph reuses the hand-over buffer
    }
  }
}

// ---- multi-SM solve: one cluster of C CTAs per graph (see ClusterPlan) ----------------
// Each CTA keeps its columns' blocks and scratch in its shared memory.  Per level: D of the
// CTA's columns with its far updates of the previous level, then its off-diagonal solves
// (both read only its own blocks), one cluster barrier (their results become visible to the
// other CTAs), the level's failure flag, then the CTA's near updates (sources read
// through the cluster window, destinations its own).  Backward substitution: one cluster
// barrier per level.  A CTA whose pivot fails writes the level's flag into every CTA's
// shared memory before the barrier, so after it each CTA reads only its own copy (no
// remote read on the common path) and all take the same decision; flags are
// double-buffered by level parity.
constexpr int kClusterThreads = 256;
constexpr int kClusterWarps = kClusterThreads / 32;

__global__ void __launch_bounds__(kClusterThreads, 1) factor_solve_cluster_kernel(
    SolverPlan P, ClusterPlan CP, const double* __restrict__ A, const double* __restrict__ gvec,
    double* __restrict__ tau, double lambda, double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn,
    FactorKeep keep) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ int s_fail[2];
  __shared__ double s_xbuf[kPanelXchg];
  const int rank = (int)cl.block_rank();
  const int g = blockIdx.x / CP.C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int* m = P.meta + kMetaCount * g;
  const int* cm = CP.cmeta + kCMetaCount * (g * CP.C + rank);
  const int cbase = m[kMetaColBase], ncol = m[kMetaNCol], sbase = m[kMetaSlotBase], nslot = m[kMetaNSlot];
  const int nlev = m[kMetaNLvl], ntri = cm[kCNTri];
  if (ncol == 0) {  // the whole cluster returns here (same graph)
    if (tid == 0 && rank == 0) {
      ginfo[g].attempts = 1;
      ginfo[g].solved = 1;
      ginfo[g].done_ns = globaltimer_ns();
    }
    return;
  }
  const int nsl = cm[kCNSlot], ncl = cm[kCNCol], nu = cm[kCNU], nt = cm[kCNT];
  unsigned char* q = dyn;
  SolveCtx C;
  // column scratch, then blocks: the same offsets in every CTA of the cluster
  C.S = carve<double>(q, (size_t)cm[kCNColMax] * kColScratch);
  C.L = carve<double>(q, (size_t)nsl * 49);
  int4* tri = carve<int4>(q, ntri);
  int4* ut = carve<int4>(q, nu);
  int2* tt = carve<int2>(q, nt);
  int* cs = carve<int>(q, ncl);
  int* lv = carve<int>(q, 4 * (nlev + 1));
  int* own = carve<int>(q, nsl);
  int* sh = carve<int>(q, nslot);
  int* ch = carve<int>(q, ncol);
  int* colslot = carve<int>(q, ncol + 1);
  int* srow = carve<int>(q, nslot);
  stage(tri, CP.ctri + cm[kCTri], ntri, tid, kClusterThreads);
  stage(ut, CP.cutask + cm[kCU], nu, tid, kClusterThreads);
  stage(tt, CP.cttask + cm[kCT], nt, tid, kClusterThreads);
  stage(cs, CP.csched + cm[kCSched], ncl, tid, kClusterThreads);
  stage(lv, CP.clvl + cm[kCLvl], 4 * (nlev + 1), tid, kClusterThreads);
  stage(own, CP.own_slot + cm[kCOwn], nsl, tid, kClusterThreads);
  stage(sh, CP.slot_home + sbase, nslot, tid, kClusterThreads);
  stage(ch, CP.col_home + cbase, ncol, tid, kClusterThreads);
  stage(colslot, P.col_slot + cbase + g, ncol + 1, tid, kClusterThreads);
  stage(srow, P.slot_row + sbase, nslot, tid, kClusterThreads);
  C.tri = tri; C.utask = ut; C.ttask = tt; C.col_slot = colslot; C.slot_row = srow; C.sched = cs; C.lvl = lv;
  C.slot_home = sh; C.col_home = ch; C.rank = rank; C.nranks = CP.C;
  // the block gather below takes its source addresses from `own`: the plan must have
  // landed (and be visible to every thread) before any address is formed from it
  async_wait_all();
  __syncthreads();
  // launched as a programmatic dependent of the assembly: the system is complete and
  // visible once the preceding grid has finished (returns at once without such a grid)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const double* Ag = A + (int64_t)sbase * 49;
  const int* col_kf = P.col_kf + cbase;

  int attempt = 0;
  bool ok = false;
  double pow100 = 1.0;
  for (; attempt < max_attempts; ++attempt, pow100 *= 100.0) {
    const double eps = eps0 * pow100;
    // this CTA's blocks of A (gathered by slot), damping and the forward right-hand side
    for (int64_t x = tid; x < (int64_t)nsl * 49; x += kClusterThreads) {
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(C.L + x);
      const double* src = Ag + (int64_t)own[x / 49] * 49 + x % 49;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    }
    async_wait_all();
    if (tid < 2) s_fail[tid] = 0;
    __syncthreads();
    for (int x = tid; x < 7 * ncl; x += kClusterThreads) {
      const int col = cs[x / 7], k = x % 7;
      const int ds = colslot[col];
      blk<true>(C, ds)[8 * k] += lambda * Ag[(int64_t)ds * 49 + 8 * k] + eps;
      y_of<true>(C, col)[k] = -gvec[7 * col_kf[col] + k];
    }
    cl.sync();  // every CTA's blocks are in place
    bool failed = false;
    for (int l = 0; l < nlev; ++l) {
      const int* L0 = lv + 4 * l;  // [own columns, near updates, far updates, off-diagonal tasks]
      // no off-diagonal solve tasks of this CTA at this level: its columns are factored as
      // whole panels (a panel level, or columns without off-diagonal blocks)
      const int ncl_l = L0[4] - L0[0], ntl = L0[7] - L0[3];
      const bool panel = ntl == 0;
      const int nd = panel ? ncl_l : (ncl_l + 3) / 4;
      const int f0 = l > 0 ? lv[4 * (l - 1) + 2] : 0, nf = l > 0 ? L0[1] - f0 : 0;
      if (panel && ncl_l == 1) {  // one column: spread over four warps, far updates on the rest
        if (warp < 4) panel_factor4<true>(C, cs[L0[0]], warp, lane, s_xbuf, &s_fail[l & 1]);
        else
          for (int i = warp - 4; i < 2 * nf; i += kClusterWarps - 4)
            update_half<true>(C, ut[f0 + i / 2], i & 1, lane);
      } else {
        for (int i = warp; i < nd + 2 * nf; i += kClusterWarps) {
          if (i >= nd) update_half<true>(C, ut[f0 + (i - nd) / 2], (i - nd) & 1, lane);
          else if (panel) panel_factor<true>(C, cs[L0[0] + i], lane, &s_fail[l & 1]);
          else diag_factor4<true>(C, cs + L0[0] + 4 * i, min(4, ncl_l - 4 * i), lane, &s_fail[l & 1]);
        }
      }
      if (!panel) {  // (a panel level's next barrier is the cluster barrier below)
        __syncthreads();
        for (int x = tid; x < 7 * ntl; x += kClusterThreads)
          trsm_or_inverse<true>(C, L0[3], ntl, 7 * ntl, L0[0], x);
      }
      // the next level's flag: its last writers (level l - 1) finished before the previous
      // barrier, its next ones (level l + 1) start after this one
      if (tid == 0) s_fail[(l + 1) & 1] = 0;
      cl.sync();
      // a failing CTA wrote this level's flag into every CTA before the barrier, so the
      // local copy is the OR over the cluster and every CTA takes the same decision
      if (s_fail[l & 1]) {
        cl.sync();
        failed = true;
        break;
      }
      for (int x = warp; x < 2 * (L0[2] - L0[1]); x += kClusterWarps)
        update_half<true>(C, ut[L0[1] + x / 2], x & 1, lane);
      // the level's L_cc^{-1} (read only by the back substitution), off the critical path:
      // threads of the last warps, which the update tasks leave idle first
      for (int x = kClusterThreads - 1 - tid; x < 7 * ncl_l; x += kClusterThreads)
        trsm_or_inverse<true>(C, 0, 0, 0, L0[0], x);
      __syncthreads();
    }
    if (!failed) {
      ok = true;
      break;
    }
  }
  if (ok) {
    // levels from kCTopLocal up hold rank 0's columns only: between them rank 0 needs a CTA
    // barrier, the other ranks nothing; from the level below on, one cluster barrier per level
    const int top_local = cm[kCTopLocal];
    for (int l = nlev - 1; l >= 0; --l) {
      const int* L0 = lv + 4 * l;
      for (int x = L0[0] + warp; x < L0[4]; x += kClusterWarps) backward_column<true>(C, cs[x], lane);
      if (l > top_local) {
        if (rank == 0) __syncthreads();  // the next level is rank 0's too
      } else {
        cl.sync();  // this level's solutions are read by the columns below it, on any rank
      }
    }
    for (int x = tid; x < 7 * ncl; x += kClusterThreads)
      tau[7 * col_kf[cs[x / 7]] + x % 7] = y_of<true>(C, cs[x / 7])[x % 7];
    if (keep.L) {  // this CTA's blocks and columns (its own shared memory only)
      for (int64_t x = tid; x < (int64_t)nsl * 49; x += kClusterThreads)
        keep.L[(int64_t)(sbase + own[x / 49]) * 49 + x % 49] = C.L[x];
      for (int x = tid; x < ncl * kColScratch; x += kClusterThreads) {
        const int col = cs[x / kColScratch];
        keep.S[(int64_t)(cbase + col) * kColScratch + x % kColScratch] =
            C.S[(int64_t)(ch[col] & 0xffffff) * kColScratch + x % kColScratch];
      }
    }
  } else {
    for (int x = tid; x < 7 * ncl; x += kClusterThreads) tau[7 * col_kf[cs[x / 7]] + x % 7] = 0.0;
  }
  if (tid == 0 && rank == 0) {
    ginfo[g].attempts = ok ? attempt + 1 : max_attempts;
    ginfo[g].solved = ok ? 1 : 0;
    if (!ok) atomicOr(warn, 1);
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
  if (tid == 0 && rank == 0) ginfo[g].done_ns = globaltimer_ns();  // every CTA's tau is written
}

// ---- solves with a kept factor ----------------------------------------------------------
// z = -(L L^T)^{-1} rhs with the blocks of L and the L_cc^{-1} a successful factorisation
// kept: the forward substitution level by level from the leaves, each column gathering
// its block row (z_c = L_cc^{-1} (z_c - sum_j L_cj z_j), j ascending), then the back
// substitution from the root (z_c = L_cc^{-T} (z_c - sum_r L_rc^T z_r)).  One CTA per
// graph with a CTA barrier between levels; the plan arrays and the working vector in
// shared memory when they fit, the factor read through the L2 (a kept factor is small).
// FP64 instructions occupy an SM sub-partition's FP64 unit for ~80 cycles each, so a level
// with more than kSubSpread columns packs four columns per warp (8 lanes each, one row per
// lane, the blocks of a column in sequence: ~9 FP64 instructions per column), and a narrow
// level gives each column a warp of its own (the row blocks four abreast, a shorter
// dependent chain of ~20 instructions).
constexpr int kSubSpread = 8;
constexpr int kSubAhead = 4;  // blocks whose loads a packed column issues before their FMAs

// one column per warp: lanes 7 b + i (b < 4) take row i of every fourth block of the row,
// the four partial sums meet by shuffles, lane q < 7 forms z_c[q] with row q of L_cc^{-1}
__device__ void substitute_forward_spread(const double* Lb, const double* Xb, int xs, const int* row_off, const int2* row_ent,
                                          double* Z, int col, int lane) {
  const int grp = lane / 7, i = lane % 7;
  const int r0 = row_off[col], nr = row_off[col + 1] - r0;
  double part = 0.0;
  if (grp < 4) {
    for (int b = grp; b < nr; b += 4) {
      const int2 e = row_ent[r0 + b];
      const double* B = Lb + (int64_t)e.x * 49 + 7 * i;
      const double* zj = Z + 7 * e.y;
      double p0 = B[0] * zj[0];
      double p1 = B[1] * zj[1];
      p0 = fma(B[2], zj[2], p0);
      p1 = fma(B[3], zj[3], p1);
      p0 = fma(B[4], zj[4], p0);
      p1 = fma(B[5], zj[5], p1);
      p0 = fma(B[6], zj[6], p0);
      part += p0 + p1;
    }
  }
  const double o1 = __shfl_sync(kFull, part, (i + 7) & 31);
  const double o2 = __shfl_sync(kFull, part, (i + 14) & 31);
  const double o3 = __shfl_sync(kFull, part, (i + 21) & 31);
  double* zc = Z + 7 * col;
  const double t = (lane < 7) ? zc[i] - ((part + o1) + (o2 + o3)) : 0.0;
  const double* X = Xb + (int64_t)col * xs;  // L_cc^{-1}, row-major
  double yq = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const double tr = __shfl_sync(kFull, t, r);
    if (lane < 7 && r <= i) yq = fma(X[7 * i + r], tr, yq);
  }
  __syncwarp();
  if (lane < 7) zc[i] = yq;
}

// the back substitution of one column per warp: the arithmetic of backward_column
__device__ void substitute_backward_spread(const double* Lb, const double* Xb, int xs, const int* col_slot,
                                           const int* slot_row, double* Z, int col, int lane) {
  const int grp = lane / 7, q = lane % 7;
  const int s_begin = col_slot[col] + 1, nb = col_slot[col + 1] - s_begin;
  double part = 0.0;
  if (grp < 4) {
    for (int b = grp; b < nb; b += 4) {
      const double* B = Lb + (int64_t)(s_begin + b) * 49;
      const double* xr = Z + 7 * slot_row[s_begin + b];
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
  double* zc = Z + 7 * col;
  const double t = (lane < 7) ? zc[q] - ((part + o1) + (o2 + o3)) : 0.0;
  const double* X = Xb + (int64_t)col * xs;
  double xq = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const double tr = __shfl_sync(kFull, t, r);
    if (lane < 7 && r >= q) xq = fma(X[7 * r + q], tr, xq);
  }
  __syncwarp();
  if (lane < 7) zc[q] = xq;
}

// four columns per warp: segment s = lane / 8 takes column cols[s] (s < ncols), its lane
// i < 7 row i.  s = sum_j L_cj z_j - z_c accumulates in one chain (so t = -s), then
// z_c = -L_cc^{-1} s with the segment's s_r by shuffles.
__device__ void substitute_forward_packed(const double* Lb, const double* Xb, int xs, const int* row_off, const int2* row_ent,
                                          double* Z, const int* cols, int ncols, int lane) {
  const int seg = lane >> 3, i = lane & 7;
  const bool act = seg < ncols && i < 7;
  const int col = cols[seg < ncols ? seg : 0];
  const double* X = Xb + (int64_t)col * xs + 7 * i;
  double xr[7];  // row i of L_cc^{-1}, loaded ahead of the chain
#pragma unroll
  for (int r = 0; r < 7; ++r) xr[r] = act && r <= i ? X[r] : 0.0;
  double sacc = 0.0;
  if (act) {
    sacc = -Z[7 * col + i];
    const int r0 = row_off[col], r1 = row_off[col + 1];
    for (int b0 = r0; b0 < r1; b0 += kSubAhead) {  // the loads of kSubAhead blocks, then their FMAs
      double bv[kSubAhead][7];
      int zo[kSubAhead];
#pragma unroll
      for (int u = 0; u < kSubAhead; ++u) {
        const int2 e = b0 + u < r1 ? row_ent[b0 + u] : make_int2(0, -1);
        zo[u] = 7 * e.y;
#pragma unroll
        for (int q = 0; q < 7; ++q) bv[u][q] = e.y >= 0 ? Lb[(int64_t)e.x * 49 + 7 * i + q] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kSubAhead; ++u)
        if (zo[u] >= 0)
#pragma unroll
          for (int q = 0; q < 7; ++q) sacc = fma(bv[u][q], Z[zo[u] + q], sacc);
    }
  }
  double y = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const double sr = __shfl_sync(kFull, sacc, (lane & ~7) | r);
    if (act && r <= i) y = fma(xr[r], sr, y);
  }
  __syncwarp();
  if (act) Z[7 * col + i] = -y;
}

__device__ void substitute_backward_packed(const double* Lb, const double* Xb, int xs, const int* col_slot,
                                           const int* slot_row, double* Z, const int* cols, int ncols, int lane) {
  const int seg = lane >> 3, q = lane & 7;
  const bool act = seg < ncols && q < 7;
  const int col = cols[seg < ncols ? seg : 0];
  const double* X = Xb + (int64_t)col * xs + q;
  double xc[7];  // column q of L_cc^{-1}, loaded ahead of the chain
#pragma unroll
  for (int r = 0; r < 7; ++r) xc[r] = act && r >= q ? X[7 * r] : 0.0;
  double sacc = 0.0;
  if (act) {
    sacc = -Z[7 * col + q];
    const int s0 = col_slot[col] + 1, s1 = col_slot[col + 1];
    for (int b0 = s0; b0 < s1; b0 += kSubAhead) {
      double bv[kSubAhead][7];
      int zo[kSubAhead];
#pragma unroll
      for (int u = 0; u < kSubAhead; ++u) {
        const bool has = b0 + u < s1;
        zo[u] = has ? 7 * slot_row[b0 + u] : -1;
#pragma unroll
        for (int i = 0; i < 7; ++i) bv[u][i] = has ? Lb[(int64_t)(b0 + u) * 49 + 7 * i + q] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kSubAhead; ++u)
        if (zo[u] >= 0)
#pragma unroll
          for (int i = 0; i < 7; ++i) sacc = fma(bv[u][i], Z[zo[u] + i], sacc);
    }
  }
  double x = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const double sr = __shfl_sync(kFull, sacc, (lane & ~7) | r);
    if (act && r >= q) x = fma(xc[r], sr, x);
  }
  __syncwarp();
  if (act) Z[7 * col + q] = -x;
}

// FSMEM (with SMEM): the kept blocks and L_cc^{-1} staged into shared memory as well.
template <bool SMEM, bool FSMEM>
__global__ void __launch_bounds__(kSolveThreads) factor_substitute_kernel(SolverPlan P, FactorKeep keep,
                                                                          const GraphInfoDev* __restrict__ rec,
                                                                          const double* __restrict__ rhs,
                                                                          double* __restrict__ out, double* zwork) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int* m = P.meta + kMetaCount * g;
  const int cbase = m[kMetaColBase], ncol = m[kMetaNCol], sbase = m[kMetaSlotBase], nslot = m[kMetaNSlot];
  const int nlev = m[kMetaNLvl];
  if (ncol == 0) return;
  const int* col_kf = P.col_kf + cbase;
  if (!rec[g].solved) {
    for (int x = tid; x < 7 * ncol; x += kSolveThreads) out[7 * col_kf[x / 7] + x % 7] = 0.0;
    return;
  }
  const double* Lb = keep.L + (int64_t)sbase * 49;
  const double* Sb = keep.S + (int64_t)cbase * kColScratch;
  const double* Xb = Sb + 14;  // L_cc^{-1} of column c at Xb + xs c
  int xs = kColScratch;
  const int* col_slot = P.col_slot + cbase + g;
  const int* slot_row = P.slot_row + sbase;
  const int* row_off = P.row_off + cbase + g;
  const int2* row_ent = P.row_ent + (sbase - cbase);
  const int* sched = P.sched + cbase;
  const int* lvl = P.lvl + 4 * m[kMetaLvlBase];
  // the kept factor was written iterations ago and has left the L2 since: bring all of it
  // back at once (one prefetch per 128-byte line) instead of level by level
  {
    const char* l0 = reinterpret_cast<const char*>(Lb);
    const char* s0 = reinterpret_cast<const char*>(Sb);
    const int64_t nl = ((int64_t)nslot * 49 * 8 + 127) / 128, ns = ((int64_t)ncol * kColScratch * 8 + 127) / 128;
    for (int64_t x = tid; x < nl + ns; x += kSolveThreads) {
      const char* p = x < nl ? l0 + 128 * x : s0 + 128 * (x - nl);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
  }
  double* Z;
  if (SMEM) {  // the layout of substitute_smem_bytes
    unsigned char* q = dyn;
    Z = carve<double>(q, (size_t)7 * ncol);
    int2* re = carve<int2>(q, nslot - ncol);
    int* ro = carve<int>(q, ncol + 1);
    int* cs = carve<int>(q, ncol + 1);
    int* sr = carve<int>(q, nslot);
    int* sc = carve<int>(q, ncol);
    int* lv = carve<int>(q, 4 * (nlev + 1));
    stage(re, row_ent, nslot - ncol, tid);
    stage(ro, row_off, ncol + 1, tid);
    stage(cs, col_slot, ncol + 1, tid);
    stage(sr, slot_row, nslot, tid);
    stage(sc, sched, ncol, tid);
    stage(lv, lvl, 4 * (nlev + 1), tid);
    row_ent = re; row_off = ro; col_slot = cs; slot_row = sr; sched = sc; lvl = lv;
    if (FSMEM) {
      double* Ls = carve<double>(q, (size_t)nslot * 49);
      double* Xs = carve<double>(q, (size_t)ncol * 49);
      stage(Ls, Lb, (int64_t)nslot * 49, tid);
      for (int x = tid; x < 49 * ncol; x += kSolveThreads) {
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(Xs + x);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(Xb + (int64_t)(x / 49) * kColScratch + x % 49)
                     : "memory");
      }
      Lb = Ls;
      Xb = Xs;
      xs = 49;
    }
  } else {
    Z = zwork + (int64_t)cbase * 7;
  }
  for (int x = tid; x < 7 * ncol; x += kSolveThreads) Z[x] = -rhs[7 * col_kf[x / 7] + x % 7];
  async_wait_all();
  __syncthreads();
  for (int lv = 0; lv < nlev; ++lv) {
    const int q0 = lvl[4 * lv], n = lvl[4 * lv + 4] - q0;
    if (n <= kSubSpread) {
      for (int q = warp; q < n; q += kSolveWarps)
        substitute_forward_spread(Lb, Xb, xs, row_off, row_ent, Z, sched[q0 + q], lane);
    } else {
      for (int q = 4 * warp; q < n; q += 4 * kSolveWarps)
        substitute_forward_packed(Lb, Xb, xs, row_off, row_ent, Z, sched + q0 + q, min(4, n - q), lane);
    }
    __syncthreads();
  }
  for (int lv = nlev - 1; lv >= 0; --lv) {
    const int q0 = lvl[4 * lv], n = lvl[4 * lv + 4] - q0;
    if (n <= kSubSpread) {
      for (int q = warp; q < n; q += kSolveWarps)
        substitute_backward_spread(Lb, Xb, xs, col_slot, slot_row, Z, sched[q0 + q], lane);
    } else {
      for (int q = 4 * warp; q < n; q += 4 * kSolveWarps)
        substitute_backward_packed(Lb, Xb, xs, col_slot, slot_row, Z, sched + q0 + q, min(4, n - q), lane);
    }
    __syncthreads();
  }
  for (int x = tid; x < 7 * ncol; x += kSolveThreads) out[7 * col_kf[x / 7] + x % 7] = Z[x];
}

}  // namespace

size_t factor_solve_max_smem() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  // static shared memory of the kernels: flags and the panel hand-over buffer
  const int reserve = 64 + (int)sizeof(double) * kPanelXchg;
  return optin > reserve ? (size_t)optin - reserve : 0;
}

int factor_solve_grid_ctas() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_solve_grid_kernel, kSolveThreads, 0) != cudaSuccess)
    return 0;
  return per_sm >= 1 ? sms : 0;  // one CTA per SM: co-resident by construction
}

cudaError_t launch_factor_solve_grid(int ctas, const SolverPlan& plan, const double* A, double* L, double* colscratch,
                                     const double* gvec, double* tau, double lambda, double eps0, int max_attempts,
                                     GraphInfoDev* ginfo, int* warn, GridSync* sync, cudaStream_t s,
                                     FactorKeep keep, unsigned extra_arrivals) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, factor_solve_grid_kernel, plan, A, L, colscratch, gvec, tau, lambda, eps0,
                            max_attempts, ginfo, warn, keep, sync, extra_arrivals);
}

// Test setting only: subtracts shift[g] from every diagonal entry of graph g's assembled
// system (one CTA per graph), so that a test can make the first attempts of the epsilon
// escalation fail by construction (an indefinite H - shift I) and check the retried
// factorisation against the oracle's on the same shifted system.
__global__ void diag_shift_kernel(SolverPlan P, double* __restrict__ A, const double* __restrict__ shift) {
  const int g = blockIdx.x;
  const double sh = shift[g];
  if (sh == 0.0) return;
  const int* m = P.meta + kMetaCount * g;
  const int cbase = m[kMetaColBase], ncol = m[kMetaNCol], sbase = m[kMetaSlotBase];
  const int* col_slot = P.col_slot + cbase + g;
  for (int x = threadIdx.x; x < 7 * ncol; x += blockDim.x)
    A[(int64_t)(sbase + col_slot[x / 7]) * 49 + 8 * (x % 7)] -= sh;
}

cudaError_t launch_diag_shift(int G, const SolverPlan& plan, double* A, const double* shift, cudaStream_t s) {
  if (G <= 0) return cudaSuccess;
  diag_shift_kernel<<<G, 256, 0, s>>>(plan, A, shift);
  return cudaGetLastError();
}

cudaError_t launch_factor_solve_group(int ctas, const SolverPlan& plan, const int4* gtask, const int32_t* glist,
                                      const double* A, double* L, double* colscratch, const double* gvec, double* tau,
                                      double lambda, double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn,
                                      int* gfail, cudaStream_t s, FactorKeep keep) {
  if (ctas <= 0 || ctas % kGroupCTAs) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)kGroupCTAs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, factor_solve_group_kernel, plan, gtask, glist, A, L, colscratch, gvec, tau, lambda,
                            eps0, max_attempts, ginfo, warn, keep, gfail);
}

// The dynamic shared memory limit of a solver kernel only grows: graphs alive at the same
// time plan different sizes, and each launch asks for its own graph's, which must stay
// within the limit whichever graph was created last.  Per kernel and device, the largest
// size set so far (setting a larger limit than a launch uses costs nothing).
constexpr int kMaxDevices = 64;
static std::mutex g_smem_attr_mu;
template <typename K>
cudaError_t grow_smem_limit(K kernel, size_t (&largest)[kMaxDevices], size_t smem_bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_smem_attr_mu);
  size_t* cur = (dev >= 0 && dev < kMaxDevices) ? &largest[dev] : nullptr;
  if (cur && smem_bytes <= *cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e == cudaSuccess && cur) *cur = smem_bytes;
  return e;
}
static size_t g_smem_substitute_f[kMaxDevices], g_smem_substitute[kMaxDevices], g_smem_solve[kMaxDevices],
    g_smem_cluster[kMaxDevices];

cudaError_t factor_substitute_prepare(size_t smem_bytes, bool factor_in_smem) {
  if (factor_in_smem) return grow_smem_limit(factor_substitute_kernel<true, true>, g_smem_substitute_f, smem_bytes);
  return grow_smem_limit(factor_substitute_kernel<true, false>, g_smem_substitute, smem_bytes);
}

cudaError_t launch_factor_substitute(int G, const SolverPlan& plan, FactorKeep keep, const GraphInfoDev* rec,
                                     const double* rhs, double* out, size_t smem_bytes, double* zwork, cudaStream_t s,
                                     bool factor_in_smem) {
  if (G <= 0) return cudaSuccess;
  if (!keep.L || !keep.S || (smem_bytes == 0 && !zwork)) return cudaErrorInvalidValue;
  if (smem_bytes && factor_in_smem)
    factor_substitute_kernel<true, true><<<G, kSolveThreads, smem_bytes, s>>>(plan, keep, rec, rhs, out, nullptr);
  else if (smem_bytes)
    factor_substitute_kernel<true, false><<<G, kSolveThreads, smem_bytes, s>>>(plan, keep, rec, rhs, out, nullptr);
  else
    factor_substitute_kernel<false, false><<<G, kSolveThreads, 0, s>>>(plan, keep, rec, rhs, out, zwork);
  return cudaGetLastError();
}

cudaError_t factor_solve_prepare(size_t smem_bytes) {
  return grow_smem_limit(factor_solve_kernel<true>, g_smem_solve, smem_bytes);
}

cudaError_t launch_factor_solve(int G, const SolverPlan& plan, bool smem, size_t smem_bytes, const double* A,
                                double* L, double* colscratch, const double* gvec, double* tau, double lambda,
                                double eps0, int max_attempts, GraphInfoDev* ginfo, int* warn, cudaStream_t s,
                                FactorKeep keep) {
  if (G <= 0) return cudaSuccess;
  if (smem) {
    factor_solve_kernel<true><<<G, kSolveThreads, smem_bytes, s>>>(plan, A, L, colscratch, gvec, tau, lambda, eps0,
                                                                   max_attempts, ginfo, warn, keep);
  } else {
    factor_solve_kernel<false><<<G, kSolveThreads, 0, s>>>(plan, A, L, colscratch, gvec, tau, lambda, eps0,
                                                           max_attempts, ginfo, warn, keep);
  }
  return cudaGetLastError();
}

}  // namespace como3r

namespace como3r {

cudaError_t factor_solve_cluster_prepare(size_t smem_bytes, int C) {
  cudaError_t e = grow_smem_limit(factor_solve_cluster_kernel, g_smem_cluster, smem_bytes);
  if (e == cudaSuccess && C > 8)
    e = cudaFuncSetAttribute(factor_solve_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

int factor_solve_cluster_max_active(size_t smem_bytes, int C) {
  if (factor_solve_cluster_prepare(smem_bytes, C) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, factor_solve_cluster_kernel, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_factor_solve_cluster(int G, const SolverPlan& plan, const ClusterPlan& cp, size_t smem_bytes,
                                        const double* A, const double* gvec, double* tau, double lambda, double eps0,
                                        int max_attempts, GraphInfoDev* ginfo, int* warn, cudaStream_t s,
                                        FactorKeep keep) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(G * cp.C));
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cp.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // may start before the preceding kernel (the assembly) finishes: it stages its plan
  // meanwhile and waits for that kernel before reading the system
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, factor_solve_cluster_kernel, plan, cp, A, gvec, tau, lambda, eps0, max_attempts,
                            ginfo, warn, keep);
}

}  // namespace como3r
