// Cross-agent candidate verification and gauge synchronisation (Sec. III-B, III-C):
// the bidirectional support gate min(nu_i, nu_j) >= nu_min and the similarity T* of
// Eq. (align) / Eq. (umeyama) that maps the moving component onto the reference one,
// with the endpoint transform T_i T_j^{-1} below nc_min correspondences.
//
// Candidate c = (i, j) comes with its two decoded match directions: for every pixel m of
// i the pixel of j (or -1), and for every pixel of j the pixel of i.  A match is
// high-confidence when c_m c_n >= q_min^2 (the exact product of the stored confidences;
// FP32 decides with a margin of a few ulps and defers the rare close calls to an exact
// FP64 product, so the decision equals the FP64 one) and both points are finite.
//
// K_align_reduce (HBM-bound; persistent warps over 2048-pixel items of either direction,
// four pixels per lane in flight: index loads, then every pixel load, then the sums): the
// streamed index row and pixel, the gathered pixel; counts of valid and high-confidence
// matches; for the forward direction the camera-frame moments of the high-confidence
// pairs, sum X_i, sum X_j, sum X_i X_j^T, sum |X_j|^2 -- FP32 per lane with Kahan
// compensation, TwoSum-compensated warp merges, one record per item (FP64 in the plain
// form).  Camera-frame coordinates keep the sums near the points' own scale; the world
// lift is linear, so it is applied to the moments afterwards:
//   x = s_i R_i X_i + t_i,  y = s_j R_j X_j + t_j,
//   A = (1/N) sum (x - xbar)(y - ybar)^T = s_i s_j R_i C R_j^T,  C = (1/N) sum X_i X_j^T - Xbar_i Xbar_j^T,
//   (1/N) sum |y - ybar|^2 = s_j^2 ((1/N) sum |X_j|^2 - |Xbar_j|^2).
// K_align_finish (one thread per candidate, FP64): sums the candidate's records in item
// order, the fractions nu, then A = U Lambda V^T by one-sided (Hestenes) Jacobi,
// S = diag(1, 1, det(U V^T)), R* = U S V^T, s* = tr(S Lambda) / var_y, t* = xbar - s* R* ybar;
// a cross-covariance of rank < 2 (sigma_2 <= 1e-12 sigma_1) leaves R* undetermined and takes
// the endpoint transform as well.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "../../include/como3r.h"
#include "como3r_internal.h"
#include "sim3.cuh"

namespace como3r {
namespace {

constexpr int kAlignItem = 2048;  // pixels per warp work item
constexpr int kSums = 16;         // Si[3], Sj[3], M[9] (M_ab = sum X_i,a X_j,b), Qj
constexpr int kAlignThreads = 256;

struct AlignDir {      // one match direction of a candidate: pixels of view a listed, matched into view b
  int64_t pa, pb;      // first pixel of a and of b in the packed points
  int64_t idx;         // first entry of this direction's match row
  int32_t na, nb;      // pixel counts
};
struct AlignCand {
  AlignDir dir[2];     // 0: i -> j (forward, moments), 1: j -> i (backward, count only)
  int32_t kf_i, kf_j;
  int32_t item0, item1;  // this candidate's items [item0, item1): forward items first
};
struct AlignItem {
  int32_t cand, dir, begin, end;
};
struct AlignRecord {   // per item: sums as (value, compensation) pairs, added in FP64 by the finish
  double v[kSums], c[kSums];
  long long n_valid, n_conf;
};

template <int DT, typename R>
__device__ __forceinline__ void load_point(const void* __restrict__ base, int64_t p, R& x, R& y, R& z, R& c) {
  if constexpr (DT == 0) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    x = (R)a.x; y = (R)a.y; z = (R)b.x; c = (R)b.y;
  } else if constexpr (DT == 1) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(base) + p);
    x = (R)v.x; y = (R)v.y; z = (R)v.z; c = (R)v.w;
  } else {
    const double2* q = reinterpret_cast<const double2*>(base) + 2 * p;
    const double2 a = __ldg(q), b = __ldg(q + 1);
    x = (R)a.x; y = (R)a.y; z = (R)b.x; c = (R)b.y;
  }
}

// c_a c_b >= q2 decided exactly.  FP32 operands (FP16 / FP32 storage): the rounded FP32
// product is within a relative 2^-24 of the exact one, so outside a +-2^-21 band around
// q2 its comparison is the exact one; inside, the exact FP64 product decides.
// The exact check stays out of line: if-converted into every lane, its FP64 multiply and
// conversions would occupy B300's narrow FP64 pipe on every match.
__device__ __noinline__ bool high_conf_exact(float ca, float cb, double q2) { return (double)ca * (double)cb >= q2; }
__device__ __forceinline__ bool high_conf(float ca, float cb, double q2, float q2f) {
  const float p = ca * cb;
  if (p > q2f * (1.f + 0x1p-21f)) return true;
  if (p < q2f * (1.f - 0x1p-21f)) return false;
  return high_conf_exact(ca, cb, q2);
}
__device__ __forceinline__ bool high_conf(double ca, double cb, double q2, float) { return ca * cb >= q2; }

template <typename R>
__device__ __forceinline__ bool finite4(R x, R y, R z, R c) {
  return isfinite(x) && isfinite(y) && isfinite(z) && isfinite(c);
}

// Kahan-compensated lane sums (FP32); FP64 adds plainly.
__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float yv = __fsub_rn(x, c);
  const float t = __fadd_rn(s, yv);
  c = __fsub_rn(__fsub_rn(t, s), yv);
  s = t;
}
__device__ __forceinline__ void kahan(double& s, double&, double x) { s += x; }

__device__ __forceinline__ float two_sum_f(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Warp total of (s + c) over the lanes as a (value, compensation) pair (TwoSum butterfly
// in FP32, both widened on the ALU: no FP64-pipe instruction in the pass).
__device__ __forceinline__ void warp_total(float s, float c, double& hi, double& lo) {
  float comp = c;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float rs = __shfl_xor_sync(0xffffffffu, s, off);
    const float rc = __shfl_xor_sync(0xffffffffu, comp, off);
    float err;
    s = two_sum_f(s, rs, err);
    comp = comp + rc + err;
  }
  hi = widen_f32(s);
  lo = widen_f32(comp);
}
__device__ __forceinline__ void warp_total(double s, double, double& hi, double& lo) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  hi = s;
  lo = 0.0;
}

// U pixels per lane in flight: index loads, then every pixel load, then the sums.
template <typename R, int DT, int U>
__global__ void __launch_bounds__(kAlignThreads, 2) align_reduce_kernel(
    const void* __restrict__ points, const int32_t* __restrict__ match_ij, const int32_t* __restrict__ match_ji,
    const AlignCand* __restrict__ cands, const AlignItem* __restrict__ items, int num_items, double q2,
    AlignRecord* __restrict__ rec, unsigned long long* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * kAlignThreads + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kAlignThreads) >> 5;
  const float q2f = (float)q2;
  for (int it = w0; it < num_items; it += nw) {
    const AlignItem item = items[it];
    const AlignDir d = cands[item.cand].dir[item.dir];
    const int32_t* __restrict__ idx = (item.dir == 0 ? match_ij : match_ji) + d.idx;
    R s[kSums], c[kSums];
#pragma unroll
    for (int k = 0; k < kSums; ++k) s[k] = c[k] = R(0);
    int n_valid = 0, n_conf = 0, n_bad = 0;
    for (int m0 = item.begin + lane; m0 < item.end; m0 += 32 * U) {
      int nn[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int m = m0 + 32 * u;
        nn[u] = m < item.end ? __ldg(idx + m) : -1;
        if (nn[u] < -1 || nn[u] >= d.nb) {  // out of range: counted as an error, never dereferenced
          ++n_bad;
          nn[u] = -1;
        }
      }
      R ax[U], ay[U], az[U], ac[U];
      R bx[U], by[U], bz[U], bc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (nn[u] >= 0) {
          load_point<DT, R>(points, d.pa + m0 + 32 * u, ax[u], ay[u], az[u], ac[u]);
          load_point<DT, R>(points, d.pb + nn[u], bx[u], by[u], bz[u], bc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (nn[u] < 0) continue;
        ++n_valid;
        bool hc;
        if constexpr (DT == 2 && sizeof(R) == 4) {  // FP64 storage: decide on the stored FP64 values
          const double* P = reinterpret_cast<const double*>(points);
          hc = high_conf(__ldg(P + 4 * (d.pa + m0 + 32 * u) + 3), __ldg(P + 4 * (d.pb + nn[u]) + 3), q2, q2f);
        } else {
          hc = high_conf(ac[u], bc[u], q2, q2f);
        }
        if (!(finite4(ax[u], ay[u], az[u], ac[u]) && finite4(bx[u], by[u], bz[u], bc[u]) && hc)) continue;
        ++n_conf;
        if (item.dir == 0) {
          kahan(s[0], c[0], ax[u]); kahan(s[1], c[1], ay[u]); kahan(s[2], c[2], az[u]);
          kahan(s[3], c[3], bx[u]); kahan(s[4], c[4], by[u]); kahan(s[5], c[5], bz[u]);
          kahan(s[6], c[6], ax[u] * bx[u]); kahan(s[7], c[7], ax[u] * by[u]); kahan(s[8], c[8], ax[u] * bz[u]);
          kahan(s[9], c[9], ay[u] * bx[u]); kahan(s[10], c[10], ay[u] * by[u]); kahan(s[11], c[11], ay[u] * bz[u]);
          kahan(s[12], c[12], az[u] * bx[u]); kahan(s[13], c[13], az[u] * by[u]); kahan(s[14], c[14], az[u] * bz[u]);
          kahan(s[15], c[15], bx[u] * bx[u] + by[u] * by[u] + bz[u] * bz[u]);
        }
      }
    }
    AlignRecord* r = rec + it;
    if (item.dir == 0) {
#pragma unroll
      for (int k = 0; k < kSums; ++k) {
        double hi, lo;
        warp_total(s[k], -c[k], hi, lo);  // a lane's Kahan total is s - c
        if (lane == k) {
          r->v[k] = hi;
          r->c[k] = lo;
        }
      }
    } else if (lane < kSums) {
      r->v[lane] = 0.0;
      r->c[lane] = 0.0;
    }
    const int tv = __reduce_add_sync(0xffffffffu, n_valid);
    const int tc = __reduce_add_sync(0xffffffffu, n_conf);
    const int tb = __reduce_add_sync(0xffffffffu, n_bad);
    if (lane == 0) {
      r->n_valid = tv;
      r->n_conf = tc;
      if (tb) atomicAdd(bad, (unsigned long long)tb);
    }
  }
}

// ---- FP64 3x3 helpers of the finishing kernel
__device__ __forceinline__ double det3(const double* M) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) + M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// A = U diag(sig) V^T, sig descending (one-sided Jacobi on the columns of A: rotations
// that make every column pair orthogonal, accumulated in V; then sig_k = |column k| and
// U's column k = column k / sig_k; a null column is completed to a right-handed basis).
__device__ void svd3(const double* A, double* U, double* sig, double* V) {
  double B[9];
  for (int k = 0; k < 9; ++k) B[k] = A[k];
  for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = 0; r < 3; ++r) {
          al += B[3 * r + p] * B[3 * r + p];
          be += B[3 * r + q] * B[3 * r + q];
          ga += B[3 * r + p] * B[3 * r + q];
        }
        if (ga == 0.0 || fabs(ga) <= 1e-300) continue;
        off = fmax(off, fabs(ga) / sqrt(al * be));
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < 3; ++r) {
          const double bp = B[3 * r + p], bq = B[3 * r + q];
          B[3 * r + p] = cs * bp - sn * bq;
          B[3 * r + q] = sn * bp + cs * bq;
          const double vp = V[3 * r + p], vq = V[3 * r + q];
          V[3 * r + p] = cs * vp - sn * vq;
          V[3 * r + q] = sn * vp + cs * vq;
        }
      }
    if (off < 1e-15) break;
  }
  double nrm[3];
  for (int k = 0; k < 3; ++k)
    nrm[k] = sqrt(B[k] * B[k] + B[3 + k] * B[3 + k] + B[6 + k] * B[6 + k]);
  int ord[3] = {0, 1, 2};  // descending
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (nrm[ord[b]] > nrm[ord[a]]) {
        const int t = ord[a];
        ord[a] = ord[b];
        ord[b] = t;
      }
  double Vs[9];
  for (int k = 0; k < 3; ++k) {
    const int o = ord[k];
    sig[k] = nrm[o];
    for (int r = 0; r < 3; ++r) {
      Vs[3 * r + k] = V[3 * r + o];
      U[3 * r + k] = nrm[o] > 0.0 ? B[3 * r + o] / nrm[o] : 0.0;
    }
  }
  for (int k = 0; k < 9; ++k) V[k] = Vs[k];
  if (!(sig[2] > 1e-300 * sig[0])) {  // third column: u0 x u1
    U[2] = U[3] * U[7] - U[6] * U[4];
    U[5] = U[6] * U[1] - U[0] * U[7];
    U[8] = U[0] * U[4] - U[3] * U[1];
  }
}

// Rotation matrix -> unit quaternion (x, y, z, w), w >= 0 (Shepperd's method: the square
// root is taken of the largest of 1 + trace and 1 + 2 R_kk - trace).
__device__ void rot_to_quat(const double* R, double* q) {
  const double tr = R[0] + R[4] + R[8];
  double x, y, z, w;
  if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
    const double r = sqrt(1.0 + tr), s = 0.5 / r;
    w = 0.5 * r; x = (R[7] - R[5]) * s; y = (R[2] - R[6]) * s; z = (R[3] - R[1]) * s;
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    const double r = sqrt(1.0 + 2.0 * R[0] - tr), s = 0.5 / r;
    x = 0.5 * r; w = (R[7] - R[5]) * s; y = (R[1] + R[3]) * s; z = (R[2] + R[6]) * s;
  } else if (R[4] >= R[8]) {
    const double r = sqrt(1.0 + 2.0 * R[4] - tr), s = 0.5 / r;
    y = 0.5 * r; w = (R[2] - R[6]) * s; x = (R[1] + R[3]) * s; z = (R[5] + R[7]) * s;
  } else {
    const double r = sqrt(1.0 + 2.0 * R[8] - tr), s = 0.5 / r;
    z = 0.5 * r; w = (R[3] - R[1]) * s; x = (R[2] + R[6]) * s; y = (R[5] + R[7]) * s;
  }
  const double sg = w < 0.0 ? -1.0 : 1.0;
  const double inv = sg / sqrt(x * x + y * y + z * z + w * w);
  q[0] = x * inv; q[1] = y * inv; q[2] = z * inv; q[3] = w * inv;
}

__global__ void align_finish_kernel(const AlignCand* __restrict__ cands, int C, const AlignRecord* __restrict__ rec,
                                    const double* __restrict__ poses, double nu_min, int nc_min,
                                    como3r_gauge_result* __restrict__ out) {
  const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= C) return;
  const AlignCand cd = cands[cidx];
  double S[kSums];
  for (int k = 0; k < kSums; ++k) S[k] = 0.0;
  long long nv[2] = {0, 0}, nc[2] = {0, 0};
  for (int it = cd.item0; it < cd.item1; ++it) {
    const AlignRecord& r = rec[it];
    const int dir = it < cd.item0 + (cd.dir[0].na + kAlignItem - 1) / kAlignItem ? 0 : 1;
    if (dir == 0)
      for (int k = 0; k < kSums; ++k) S[k] += r.v[k] + r.c[k];
    nv[dir] += r.n_valid;
    nc[dir] += r.n_conf;
  }
  como3r_gauge_result res;
  res.n_i = nc[0];
  res.n_j = nc[1];
  res.valid_i = nv[0];
  res.valid_j = nv[1];
  res.nu_i = (double)nc[0] / cd.dir[0].na;
  res.nu_j = (double)nc[1] / cd.dir[1].na;
  res.admitted = fmin(res.nu_i, res.nu_j) >= nu_min ? 1 : 0;
  // poses of i and j: (s R, t)
  const double* pi = poses + 8 * (int64_t)cd.kf_i;
  const double* pj = poses + 8 * (int64_t)cd.kf_j;
  double Ri[9], Rj[9];
  quat_to_rot(pi[3], pi[4], pi[5], pi[6], Ri);
  quat_to_rot(pj[3], pj[4], pj[5], pj[6], Rj);
  const double si = pi[7], sj = pj[7];
  double Rs[9], ss = 1.0, ts[3];
  int fallback = 1;
  const long long N = nc[0];
  if (N >= nc_min && N > 0) {
    const double iN = 1.0 / (double)N;
    const double Xi[3] = {S[0] * iN, S[1] * iN, S[2] * iN}, Xj[3] = {S[3] * iN, S[4] * iN, S[5] * iN};
    double Cc[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Cc[3 * a + b] = S[6 + 3 * a + b] * iN - Xi[a] * Xj[b];
    const double var_y = sj * sj * (S[15] * iN - (Xj[0] * Xj[0] + Xj[1] * Xj[1] + Xj[2] * Xj[2]));
    // A = s_i s_j R_i C R_j^T
    double T1[9], A[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        T1[3 * a + b] = Cc[3 * a] * Rj[3 * b] + Cc[3 * a + 1] * Rj[3 * b + 1] + Cc[3 * a + 2] * Rj[3 * b + 2];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        A[3 * a + b] = si * sj * (Ri[3 * a] * T1[b] + Ri[3 * a + 1] * T1[3 + b] + Ri[3 * a + 2] * T1[6 + b]);
    double U[9], sig[3], V[9];
    svd3(A, U, sig, V);
    if (sig[1] > 1e-12 * sig[0] && var_y > 0.0) {
      const double dsg = det3(U) * det3(V) < 0.0 ? -1.0 : 1.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          Rs[3 * a + b] = U[3 * a] * V[3 * b] + U[3 * a + 1] * V[3 * b + 1] + dsg * U[3 * a + 2] * V[3 * b + 2];
      ss = (sig[0] + sig[1] + dsg * sig[2]) / var_y;
      double xb[3], yb[3];
      for (int a = 0; a < 3; ++a) {
        xb[a] = si * (Ri[3 * a] * Xi[0] + Ri[3 * a + 1] * Xi[1] + Ri[3 * a + 2] * Xi[2]) + pi[a];
        yb[a] = sj * (Rj[3 * a] * Xj[0] + Rj[3 * a + 1] * Xj[1] + Rj[3 * a + 2] * Xj[2]) + pj[a];
      }
      for (int a = 0; a < 3; ++a)
        ts[a] = xb[a] - ss * (Rs[3 * a] * yb[0] + Rs[3 * a + 1] * yb[1] + Rs[3 * a + 2] * yb[2]);
      fallback = 0;
    } else {
      fallback = 2;
    }
  }
  if (fallback) {  // T_i T_j^{-1}: s = s_i / s_j, R = R_i R_j^T, t = t_i - s R t_j
    ss = si / sj;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        Rs[3 * a + b] = Ri[3 * a] * Rj[3 * b] + Ri[3 * a + 1] * Rj[3 * b + 1] + Ri[3 * a + 2] * Rj[3 * b + 2];
    for (int a = 0; a < 3; ++a)
      ts[a] = pi[a] - ss * (Rs[3 * a] * pj[0] + Rs[3 * a + 1] * pj[1] + Rs[3 * a + 2] * pj[2]);
  }
  res.fallback = fallback;
  double q[4];
  rot_to_quat(Rs, q);
  res.T[0] = ts[0]; res.T[1] = ts[1]; res.T[2] = ts[2];
  res.T[3] = q[0]; res.T[4] = q[1]; res.T[5] = q[2]; res.T[6] = q[3];
  res.T[7] = ss;
  out[cidx] = res;
}

// poses[k] <- T*[which[k]] poses[k] for which[k] >= 0 (left multiplication in Sim(3)).
__global__ void gauge_transport_kernel(double* __restrict__ poses, int N, const int32_t* __restrict__ which,
                                       const double* __restrict__ T, int C) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int c = which[k];
  if (c < 0 || c >= C) return;
  const double* g = T + 8 * (int64_t)c;
  double* p = poses + 8 * (int64_t)k;
  double Rg[9];
  quat_to_rot(g[3], g[4], g[5], g[6], Rg);
  const double t0 = p[0], t1 = p[1], t2 = p[2];
  for (int a = 0; a < 3; ++a) p[a] = g[7] * (Rg[3 * a] * t0 + Rg[3 * a + 1] * t1 + Rg[3 * a + 2] * t2) + g[a];
  // q' = q_g (x) q_k (Hamilton product, xyzw), renormalised
  const double gx = g[3], gy = g[4], gz = g[5], gw = g[6];
  const double x = p[3], y = p[4], z = p[5], w = p[6];
  double qx = gw * x + gx * w + gy * z - gz * y;
  double qy = gw * y - gx * z + gy * w + gz * x;
  double qz = gw * z + gx * y - gy * x + gz * w;
  double qw = gw * w - gx * x - gy * y - gz * z;
  const double inv = 1.0 / sqrt(qx * qx + qy * qy + qz * qz + qw * qw);
  p[3] = qx * inv; p[4] = qy * inv; p[5] = qz * inv; p[6] = qw * inv;
  p[7] = g[7] * p[7];
}

template <typename R, int U>
void launch_align_reduce_u(int dtype, int grid, cudaStream_t s, const void* points, const int32_t* mij,
                           const int32_t* mji, const AlignCand* cands, const AlignItem* items, int n_items, double q2,
                           AlignRecord* rec, unsigned long long* bad) {
  if (dtype == COMO3R_F16)
    align_reduce_kernel<R, 0, U><<<grid, kAlignThreads, 0, s>>>(points, mij, mji, cands, items, n_items, q2, rec, bad);
  else if (dtype == COMO3R_F32)
    align_reduce_kernel<R, 1, U><<<grid, kAlignThreads, 0, s>>>(points, mij, mji, cands, items, n_items, q2, rec, bad);
  else
    align_reduce_kernel<R, 2, U><<<grid, kAlignThreads, 0, s>>>(points, mij, mji, cands, items, n_items, q2, rec, bad);
}

// COMO3R_ALIGN_UNROLL = 1, 2 or 4 pixels in flight per lane (default 4).
template <typename R>
cudaError_t launch_align_reduce(int dtype, int grid, cudaStream_t s, const void* points, const int32_t* mij,
                                const int32_t* mji, const AlignCand* cands, const AlignItem* items, int n_items,
                                double q2, AlignRecord* rec, unsigned long long* bad) {
  const char* e = getenv("COMO3R_ALIGN_UNROLL");
  const int u = e ? atoi(e) : 4;
  if (u == 1) launch_align_reduce_u<R, 1>(dtype, grid, s, points, mij, mji, cands, items, n_items, q2, rec, bad);
  else if (u == 2) launch_align_reduce_u<R, 2>(dtype, grid, s, points, mij, mji, cands, items, n_items, q2, rec, bad);
  else launch_align_reduce_u<R, 4>(dtype, grid, s, points, mij, mji, cands, items, n_items, q2, rec, bad);
  return cudaGetLastError();
}

}  // namespace
}  // namespace como3r

using namespace como3r;

#define CKA(expr, where)                                           \
  do {                                                             \
    cudaError_t e_ = (expr);                                       \
    if (e_ != cudaSuccess) {                                       \
      cleanup();                                                   \
      return report_cuda_error(e_, where);                         \
    }                                                              \
  } while (0)

extern "C" int como3r_gauge_sync(const como3r_gauge_desc* d, void* cuda_stream, como3r_gauge_result* out,
                                 float* kernel_ms) {
  if (!d || !out) return report_error(COMO3R_ERR_INVALID_ARG, "desc and out must be non-NULL");
  const int C = d->num_candidates, N = d->num_kf;
  if (C < 0 || N < 0) return report_error(COMO3R_ERR_INVALID_ARG, "negative sizes");
  if (C == 0) return COMO3R_OK;
  if (!d->pix_off || !d->points_conf || !d->kf_i || !d->kf_j || !d->match_ij || !d->match_ji || !d->poses)
    return report_error(COMO3R_ERR_INVALID_ARG, "pix_off, points_conf, kf_i, kf_j, match_ij, match_ji and poses must be non-NULL");
  if (d->dtype < COMO3R_F16 || d->dtype > COMO3R_F64)
    return report_error(COMO3R_ERR_INVALID_ARG, "dtype must be COMO3R_F16, COMO3R_F32 or COMO3R_F64");
  if (d->mode != COMO3R_MIXED && d->mode != COMO3R_PLAIN_FP64)
    return report_error(COMO3R_ERR_INVALID_ARG, "mode must be COMO3R_MIXED or COMO3R_PLAIN_FP64");
  if (!(d->q_min >= 0.0) || !(d->nu_min >= 0.0) || d->nc_min < 0)
    return report_error(COMO3R_ERR_INVALID_ARG, "q_min and nu_min must be >= 0, nc_min >= 0");
  for (int k = 0; k < N; ++k)
    if (d->pix_off[k + 1] < d->pix_off[k] || d->pix_off[k + 1] - d->pix_off[k] >= (int64_t(1) << 31))
      return report_error(COMO3R_ERR_INVALID_ARG, "pix_off must be non-decreasing with < 2^31 pixels per keyframe");
  std::vector<AlignCand> cands(C);
  std::vector<AlignItem> items;
  int64_t off_ij = 0, off_ji = 0;
  for (int c = 0; c < C; ++c) {
    const int i = d->kf_i[c], j = d->kf_j[c];
    if (i < 0 || i >= N || j < 0 || j >= N || i == j)
      return report_error(COMO3R_ERR_INVALID_ARG, "candidate keyframes must be distinct ids in [0, num_kf)");
    AlignCand& cd = cands[c];
    const int32_t Pi = (int32_t)(d->pix_off[i + 1] - d->pix_off[i]);
    const int32_t Pj = (int32_t)(d->pix_off[j + 1] - d->pix_off[j]);
    if (Pi <= 0 || Pj <= 0) return report_error(COMO3R_ERR_INVALID_ARG, "candidate keyframes must have pixels");
    cd.dir[0] = AlignDir{d->pix_off[i], d->pix_off[j], off_ij, Pi, Pj};
    cd.dir[1] = AlignDir{d->pix_off[j], d->pix_off[i], off_ji, Pj, Pi};
    cd.kf_i = i;
    cd.kf_j = j;
    off_ij += Pi;
    off_ji += Pj;
    cd.item0 = (int32_t)items.size();
    for (int dir = 0; dir < 2; ++dir)
      for (int32_t b = 0; b < cd.dir[dir].na; b += kAlignItem)
        items.push_back(AlignItem{c, dir, b, std::min<int32_t>(b + kAlignItem, cd.dir[dir].na)});
    cd.item1 = (int32_t)items.size();
  }
  if (items.size() >= (size_t(1) << 31)) return report_error(COMO3R_ERR_UNSUPPORTED, "too many work items");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  AlignCand* d_c = nullptr;
  AlignItem* d_it = nullptr;
  AlignRecord* d_rec = nullptr;
  unsigned long long* d_bad = nullptr;
  double* d_poses = nullptr;
  como3r_gauge_result* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {  // stream-ordered frees (the pool keeps the memory for the next call)
    if (d_c) cudaFreeAsync(d_c, s);
    if (d_it) cudaFreeAsync(d_it, s);
    if (d_rec) cudaFreeAsync(d_rec, s);
    if (d_bad) cudaFreeAsync(d_bad, s);
    if (d_poses) cudaFreeAsync(d_poses, s);
    if (d_out) cudaFreeAsync(d_out, s);
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  const int n_items = (int)items.size();
  CKA(cudaMallocAsync(&d_c, sizeof(AlignCand) * C, s), "cudaMallocAsync");
  CKA(cudaMallocAsync(&d_it, sizeof(AlignItem) * n_items, s), "cudaMallocAsync");
  CKA(cudaMallocAsync(&d_rec, sizeof(AlignRecord) * n_items, s), "cudaMallocAsync");
  CKA(cudaMallocAsync(&d_bad, sizeof(unsigned long long), s), "cudaMallocAsync");
  CKA(cudaMallocAsync(&d_poses, sizeof(double) * 8 * (size_t)std::max(N, 1), s), "cudaMallocAsync");
  CKA(cudaMallocAsync(&d_out, sizeof(como3r_gauge_result) * C, s), "cudaMallocAsync");
  CKA(cudaMemcpyAsync(d_c, cands.data(), sizeof(AlignCand) * C, cudaMemcpyHostToDevice, s), "upload");
  CKA(cudaMemcpyAsync(d_it, items.data(), sizeof(AlignItem) * n_items, cudaMemcpyHostToDevice, s), "upload");
  CKA(cudaMemcpyAsync(d_poses, d->poses, sizeof(double) * 8 * (size_t)N, cudaMemcpyDefault, s), "poses");
  CKA(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), s), "memset");
  int dev = 0, sms = 148;
  CKA(cudaGetDevice(&dev), "device");
  CKA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device");
  const int warps_per_cta = kAlignThreads / 32;
  // persistent: two resident CTAs per SM, warps striding over the items
  const int grid = std::max(1, std::min(sms * 2, (n_items + warps_per_cta - 1) / warps_per_cta));
  const double q2 = d->q_min * d->q_min;
  if (kernel_ms) {
    CKA(cudaEventCreate(&e0), "event");
    CKA(cudaEventCreate(&e1), "event");
    CKA(cudaEventRecord(e0, s), "event");
  }
  if (d->mode == COMO3R_MIXED)
    CKA(launch_align_reduce<float>(d->dtype, grid, s, d->points_conf, d->match_ij, d->match_ji, d_c, d_it, n_items,
                                   q2, d_rec, d_bad),
        "align_reduce");
  else
    CKA(launch_align_reduce<double>(d->dtype, grid, s, d->points_conf, d->match_ij, d->match_ji, d_c, d_it, n_items,
                                    q2, d_rec, d_bad),
        "align_reduce");
  if (kernel_ms) CKA(cudaEventRecord(e1, s), "event");
  align_finish_kernel<<<(C + 63) / 64, 64, 0, s>>>(d_c, C, d_rec, d_poses, d->nu_min, d->nc_min, d_out);
  CKA(cudaGetLastError(), "align_finish");
  unsigned long long bad = 0;
  CKA(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s), "readback");
  CKA(cudaMemcpyAsync(out, d_out, sizeof(como3r_gauge_result) * C, cudaMemcpyDeviceToHost, s), "readback");
  CKA(cudaStreamSynchronize(s), "sync");
  if (kernel_ms) CKA(cudaEventElapsedTime(kernel_ms, e0, e1), "event");
  cleanup();
  if (bad) return report_error(COMO3R_ERR_INVALID_ARG, "match indices outside [-1, P) in a candidate's match rows");
  return COMO3R_OK;
}

extern "C" int como3r_gauge_transport(double* poses, int32_t num_kf, const int32_t* which, const double* T,
                                      int32_t num_candidates, void* cuda_stream) {
  if (num_kf < 0 || num_candidates < 0) return report_error(COMO3R_ERR_INVALID_ARG, "negative sizes");
  if (num_kf == 0) return COMO3R_OK;
  if (!poses || !which || (!T && num_candidates > 0))
    return report_error(COMO3R_ERR_INVALID_ARG, "poses, which and T must be non-NULL");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  gauge_transport_kernel<<<(num_kf + 127) / 128, 128, 0, s>>>(poses, num_kf, which, T, num_candidates);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_cuda_error(e, "gauge_transport");
  return COMO3R_OK;
}
