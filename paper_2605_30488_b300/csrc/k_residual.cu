// K1: per-match residual, whitening, Huber IRLS weights, 4x7 Jacobian and reduction of
// the relative-pose normal-equation blocks of every edge (Sec. III-A, III-D).
//
// Work is split into items (edge, [begin, end) of the streamed keyframe's pixels), each
// owned by one warp of a persistent grid.  Every lane accumulates its pixels (pixel
// m = begin + lane + 32 k: coalesced streams of match_idx and X_i, a gather of X_j[n])
// into 33 registers -- the 25 structurally nonzero entries of H_rel = sum J^T W J, the 7
// of g_rel = sum J^T W e, and the cost -- then the warp reduces them with shuffles and
// writes one partial record per item.  No CTA barrier, no shared memory, no atomics:
// results are bitwise reproducible and warps never wait for each other.
//
// Per match (m, n) of edge (i, j), with T_ij = (sR, t) and x = sR X_j,n + t:
//   d = ||x||, xh = x / d, e = [xh - psi(X_i,m); d - ||X_i,m||]          (Eq. residual)
//   q = sqrt(c_i,m c_j,n), r_c = sqrt(q) e_c / sigma_c, w_c = min(1, kappa / |r_c|),
//   W_c = w_c q / sigma_c^2, rho(r) = r^2/2 or kappa |r| - kappa^2/2       (Sec. III-A)
//   J = [Dpsi/Dx; Dd/Dx] [I, -[x]x, x]                                    (Eq. jacobian)
// which simplifies, with P = (I - xh xh^T) / d (so P[x]x = [x]x / d and P x = 0), to
//   ray rows   [P, -[xh]x, 0],   range row [xh^T, 0, d].
// So the (omega, zeta) block of H_rel vanishes and 25 of its 28 unique entries remain.
//
// MIXED mode: all of the above in FP32 (T_ij rounded from FP64 per edge), per-lane sums
// over <= chunk/32 matches, an error-free (TwoSum) compensated warp butterfly, and the
// record written as (sum, compensation) FP32 pairs that the per-edge reduction adds in
// FP64 (B300's FP64 pipe is slow, so no FP64 instruction runs in this kernel).
// PLAIN mode: FP64 throughout, record of FP64 values.
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "como3r_internal.h"

namespace como3r {
namespace {

constexpr int kAcc = 32;  // H (25) + g (7) reduced by the butterfly; the cost separately

template <typename R>
struct Consts {
  R isr, isd, ivr, ivd, kappa, half_kappa;
};

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
template <typename R> __device__ __forceinline__ R kInfinity();
template <> __device__ __forceinline__ float kInfinity<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double kInfinity<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

// Square root of a non-negative value (0 -> 0); FP32 through the reciprocal square root.
__device__ __forceinline__ float nn_sqrt(float v) { return v > 0.f ? v * rsqrtf(v) : 0.f; }
__device__ __forceinline__ double nn_sqrt(double v) { return sqrt(v); }

// ---- pixel loads: (x, y, z, c) in the storage type, widened to R
template <int DT, typename R>
__device__ __forceinline__ void load_px(const void* __restrict__ base, int64_t p, R& x, R& y, R& z, R& c) {
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

template <typename R>
struct Acc {
  R v[kAcc];  // [0..24] H_rel unique entries, [25..31] g_rel
  R E;
  int skipped;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < kAcc; ++k) v[k] = R(0);
    E = R(0);
    skipped = 0;
  }
};

// One match: residual, robust weights, Jacobian rows, accumulation (see file header).
template <typename R>
__device__ __forceinline__ void accumulate(R xi, R yi, R zi, R ci, R xj, R yj, R zj, R cj, const R* T,
                                           const Consts<R>& k, Acc<R>& acc) {
  const R x0 = fma(T[0], xj, fma(T[1], yj, fma(T[2], zj, T[9])));
  const R x1 = fma(T[3], xj, fma(T[4], yj, fma(T[5], zj, T[10])));
  const R x2 = fma(T[6], xj, fma(T[7], yj, fma(T[8], zj, T[11])));
  const R d2 = fma(x0, x0, fma(x1, x1, x2 * x2));
  const R di2 = fma(xi, xi, fma(yi, yi, zi * zi));
  const R cc = ci * cj;
  const R th2 = R(1e-24), inf = kInfinity<R>();
  const bool ok = (d2 > th2) & (d2 < inf) & (di2 > th2) & (di2 < inf) & (cc >= R(0)) & (cc < inf);
  if (!ok) {
    ++acc.skipped;
    return;
  }
  const R rd = rsq(d2), d = d2 * rd;
  const R rdi = rsq(di2), di = di2 * rdi;
  const R a = x0 * rd, b = x1 * rd, c = x2 * rd;  // xh
  const R e0 = fma(-xi, rdi, a), e1 = fma(-yi, rdi, b), e2 = fma(-zi, rdi, c), e3 = d - di;
  const R q = nn_sqrt(cc);
  const R sq = nn_sqrt(q);
  const R sr = sq * k.isr, sd = sq * k.isd;
  const R r0 = sr * e0, r1 = sr * e1, r2 = sr * e2, r3 = sd * e3;
  const R a0 = fabs(r0), a1 = fabs(r1), a2 = fabs(r2), a3 = fabs(r3);
  const bool i0 = a0 <= k.kappa, i1 = a1 <= k.kappa, i2 = a2 <= k.kappa, i3 = a3 <= k.kappa;
  const R w0 = i0 ? R(1) : qdiv(k.kappa, a0);
  const R w1 = i1 ? R(1) : qdiv(k.kappa, a1);
  const R w2 = i2 ? R(1) : qdiv(k.kappa, a2);
  const R w3 = i3 ? R(1) : qdiv(k.kappa, a3);
  const R rho0 = i0 ? R(0.5) * r0 * r0 : k.kappa * (a0 - k.half_kappa);
  const R rho1 = i1 ? R(0.5) * r1 * r1 : k.kappa * (a1 - k.half_kappa);
  const R rho2 = i2 ? R(0.5) * r2 * r2 : k.kappa * (a2 - k.half_kappa);
  const R rho3 = i3 ? R(0.5) * r3 * r3 : k.kappa * (a3 - k.half_kappa);
  acc.E += (rho0 + rho1) + (rho2 + rho3);
  const R qr = q * k.ivr;
  const R u0 = w0 * qr, u1 = w1 * qr, u2 = w2 * qr, u3 = w3 * q * k.ivd;  // W_c
  const R f0 = u0 * e0, f1 = u1 * e1, f2 = u2 * e2, f3 = u3 * e3;        // W_c e_c
  // P = (I - xh xh^T) / d, symmetric
  const R p00 = fma(-a, a, R(1)) * rd, p11 = fma(-b, b, R(1)) * rd, p22 = fma(-c, c, R(1)) * rd;
  const R p01 = -a * b * rd, p02 = -a * c * rd, p12 = -b * c * rd;
  // weighted ray rows  wk_l = u_k P_kl
  const R w00 = u0 * p00, w01 = u0 * p01, w02 = u0 * p02;
  const R w10 = u1 * p01, w11 = u1 * p11, w12 = u1 * p12;
  const R w20 = u2 * p02, w21 = u2 * p12, w22 = u2 * p22;
  const R ua = u3 * a, ub = u3 * b, uc = u3 * c;
  R* h = acc.v;
  // (v, v): sum_k u_k P_kl P_km + u3 xh_l xh_m
  h[0] = fma(w00, p00, fma(w10, p01, fma(w20, p02, fma(ua, a, h[0]))));
  h[1] = fma(w00, p01, fma(w10, p11, fma(w20, p12, fma(ua, b, h[1]))));
  h[2] = fma(w00, p02, fma(w10, p12, fma(w20, p22, fma(ua, c, h[2]))));
  h[3] = fma(w01, p01, fma(w11, p11, fma(w21, p12, fma(ub, b, h[3]))));
  h[4] = fma(w01, p02, fma(w11, p12, fma(w21, p22, fma(ub, c, h[4]))));
  h[5] = fma(w02, p02, fma(w12, p12, fma(w22, p22, fma(uc, c, h[5]))));
  // (v, omega): sum_k u_k P_kl S_km with S = -[xh]x:
  //   S_0 = (0, c, -b), S_1 = (-c, 0, a), S_2 = (b, -a, 0)
  h[6] = fma(-c, w10, fma(b, w20, h[6]));
  h[7] = fma(c, w00, fma(-a, w20, h[7]));
  h[8] = fma(-b, w00, fma(a, w10, h[8]));
  h[9] = fma(-c, w11, fma(b, w21, h[9]));
  h[10] = fma(c, w01, fma(-a, w21, h[10]));
  h[11] = fma(-b, w01, fma(a, w11, h[11]));
  h[12] = fma(-c, w12, fma(b, w22, h[12]));
  h[13] = fma(c, w02, fma(-a, w22, h[13]));
  h[14] = fma(-b, w02, fma(a, w12, h[14]));
  // (omega, omega): sum_k u_k S_kl S_km
  const R cc2 = c * c, bb2 = b * b, aa2 = a * a;
  h[15] = fma(u1, cc2, fma(u2, bb2, h[15]));
  h[16] = fma(-u2 * a, b, h[16]);
  h[17] = fma(-u1 * a, c, h[17]);
  h[18] = fma(u0, cc2, fma(u2, aa2, h[18]));
  h[19] = fma(-u0 * b, c, h[19]);
  h[20] = fma(u0, bb2, fma(u1, aa2, h[20]));
  // (v, zeta) and (zeta, zeta): range row only
  const R ud = u3 * d;
  h[21] = fma(ud, a, h[21]);
  h[22] = fma(ud, b, h[22]);
  h[23] = fma(ud, c, h[23]);
  h[24] = fma(ud, d, h[24]);
  // g_rel = sum_c W_c e_c J_c
  h[25] = fma(f0, p00, fma(f1, p01, fma(f2, p02, fma(f3, a, h[25]))));
  h[26] = fma(f0, p01, fma(f1, p11, fma(f2, p12, fma(f3, b, h[26]))));
  h[27] = fma(f0, p02, fma(f1, p12, fma(f2, p22, fma(f3, c, h[27]))));
  h[28] = fma(-c, f1, fma(b, f2, h[28]));
  h[29] = fma(c, f0, fma(-a, f2, h[29]));
  h[30] = fma(-b, f0, fma(a, f1, h[30]));
  h[31] = fma(f3, d, h[31]);
}

// Error-free transformation: s + err == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Warp butterfly ("transpose") reduction of 32 values per lane: at each of the 5 levels a
// lane keeps one half of its values and sends the other half to its partner, so after it
// lane l holds the warp total of value l.  The FP32 variant carries TwoSum compensation.
__device__ __forceinline__ void warp_transpose_reduce(float (&v)[kAcc], float (&comp)[kAcc], int lane) {
#pragma unroll
  for (int k = 0; k < kAcc; ++k) comp[k] = 0.f;
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int off = 16 >> lvl;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < off; ++k) {
      const float send_v = upper ? v[k] : v[k + off];
      const float keep_v = upper ? v[k + off] : v[k];
      const float send_c = upper ? comp[k] : comp[k + off];
      const float keep_c = upper ? comp[k + off] : comp[k];
      const float rv = __shfl_xor_sync(0xffffffffu, send_v, off);
      const float rc = __shfl_xor_sync(0xffffffffu, send_c, off);
      float err;
      v[k] = two_sum(keep_v, rv, err);
      comp[k] = keep_c + rc + err;
    }
  }
}

__device__ __forceinline__ void warp_transpose_reduce(double (&v)[kAcc], double (&comp)[kAcc], int lane) {
#pragma unroll
  for (int k = 0; k < kAcc; ++k) comp[k] = 0.0;
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int off = 16 >> lvl;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < off; ++k) {
      const double send_v = upper ? v[k] : v[k + off];
      const double keep_v = upper ? v[k + off] : v[k];
      v[k] = keep_v + __shfl_xor_sync(0xffffffffu, send_v, off);
    }
  }
}

// Compensated warp sum of one value: returns the sum, `c` receives the compensation.
__device__ __forceinline__ float warp_sum_pair(float x, float& c) {
  c = 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float rx = __shfl_xor_sync(0xffffffffu, x, off);
    const float rc = __shfl_xor_sync(0xffffffffu, c, off);
    float err;
    x = two_sum(x, rx, err);
    c = c + rc + err;
  }
  return x;
}
__device__ __forceinline__ double warp_sum_pair(double x, double& c) {
  c = 0.0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Partial record of one item: kPartial slots of 8 bytes.  Slots 0..31 hold the 32
// butterfly accumulators, 32 the cost, 33 the skipped-match count, 34..35 zero.  MIXED
// writes each slot as float2 (sum, compensation), PLAIN as one double.
__device__ __forceinline__ void store_slot(float2* rec, int k, float v, float c) { rec[k] = make_float2(v, c); }
__device__ __forceinline__ void store_slot(double* rec, int k, double v, double c) { rec[k] = v + c; }

// One group of UNROLL pixels per lane: match indices, then the two packed pixels.
template <typename R, int U>
struct Group {
  int n[U];
  R xi[U], yi[U], zi[U], ci[U], xj[U], yj[U], zj[U], cj[U];
};

template <typename R, int U>
__device__ __forceinline__ void load_indices(int (&n)[U], const int32_t* __restrict__ idx, int m0, int end) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int m = m0 + 32 * u;
    n[u] = (m < end) ? __ldg(idx + m) : -1;
  }
}

template <int DT, typename R, int U>
__device__ __forceinline__ void load_pixels(Group<R, U>& G, const void* __restrict__ points, int64_t pix_i,
                                            int64_t pix_j, int m0) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (G.n[u] >= 0) {
      load_px<DT, R>(points, pix_i + m0 + 32 * u, G.xi[u], G.yi[u], G.zi[u], G.ci[u]);
      load_px<DT, R>(points, pix_j + G.n[u], G.xj[u], G.yj[u], G.zj[u], G.cj[u]);
    }
  }
}

template <typename R, int U>
__device__ __forceinline__ void accumulate_group(const Group<R, U>& G, const R* T, const Consts<R>& k, Acc<R>& acc) {
#pragma unroll
  for (int u = 0; u < U; ++u)
    if (G.n[u] >= 0) accumulate<R>(G.xi[u], G.yi[u], G.zi[u], G.ci[u], G.xj[u], G.yj[u], G.zj[u], G.cj[u], T, k, acc);
}

template <typename R, int DT, int BLOCK, int MINB, int UNROLL, bool PIPE>
__global__ void __launch_bounds__(BLOCK, MINB) residual_reduce_kernel(
    const void* __restrict__ points, const int32_t* __restrict__ midx, const Item* __restrict__ items,
    int num_items, const EdgeStatic* __restrict__ es, const double* __restrict__ T64,
    const float* __restrict__ T32, RobustParams rp, void* __restrict__ partials) {
  using Slot = typename std::conditional<sizeof(R) == 4, float2, double>::type;
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * BLOCK) >> 5;
  Consts<R> k;
  k.isr = (R)rp.inv_sigma_ray; k.isd = (R)rp.inv_sigma_dist;
  k.ivr = (R)rp.inv_var_ray; k.ivd = (R)rp.inv_var_dist;
  k.kappa = (R)rp.kappa; k.half_kappa = (R)(0.5 * rp.kappa);

  for (int it = gwarp; it < num_items; it += nwarps) {
    const Item item = items[it];
    const int64_t pix_i = es[item.edge].pix_i, pix_j = es[item.edge].pix_j;
    const int32_t* __restrict__ idx = midx + es[item.edge].idx_off;
    R T[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      if constexpr (sizeof(R) == 4) T[q] = T32[16 * item.edge + q];
      else T[q] = T64[12 * item.edge + q];
    }
    Acc<R> acc;
    acc.zero();
    constexpr int STEP = 32 * UNROLL;
    if constexpr (!PIPE) {
      // plain loop: indices, then both pixels, then the arithmetic of this group
      for (int g0 = item.begin; g0 < item.end; g0 += STEP) {
        Group<R, UNROLL> G;
        load_indices<R, UNROLL>(G.n, idx, g0 + lane, item.end);
        load_pixels<DT, R, UNROLL>(G, points, pix_i, pix_j, g0 + lane);
        accumulate_group<R, UNROLL>(G, T, k, acc);
      }
    } else {
      // software pipeline over groups: while group g is computed, the pixels of g+1 and
      // the match indices of g+2 are in flight (two register groups, ping-pong)
      Group<R, UNROLL> A, B;
      int g0 = item.begin;
      load_indices<R, UNROLL>(A.n, idx, g0 + lane, item.end);
      load_pixels<DT, R, UNROLL>(A, points, pix_i, pix_j, g0 + lane);
      load_indices<R, UNROLL>(B.n, idx, g0 + STEP + lane, item.end);
      while (g0 < item.end) {
        load_pixels<DT, R, UNROLL>(B, points, pix_i, pix_j, g0 + STEP + lane);
        int nA[UNROLL];
        load_indices<R, UNROLL>(nA, idx, g0 + 2 * STEP + lane, item.end);
        accumulate_group<R, UNROLL>(A, T, k, acc);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) A.n[u] = nA[u];
        g0 += STEP;
        if (g0 >= item.end) break;
        load_pixels<DT, R, UNROLL>(A, points, pix_i, pix_j, g0 + STEP + lane);
        int nB[UNROLL];
        load_indices<R, UNROLL>(nB, idx, g0 + 2 * STEP + lane, item.end);
        accumulate_group<R, UNROLL>(B, T, k, acc);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) B.n[u] = nB[u];
        g0 += STEP;
      }
    }
    // ---- warp reduction: compensated butterfly, lane l ends with accumulator l
    R comp[kAcc];
    warp_transpose_reduce(acc.v, comp, lane);
    R Ec = R(0);
    const R Ev = warp_sum_pair(acc.E, Ec);
    const int sk = __reduce_add_sync(0xffffffffu, acc.skipped);
    Slot* rec = reinterpret_cast<Slot*>(partials) + (int64_t)it * kPartial;
    store_slot(rec, lane, acc.v[0], comp[0]);
    if (lane == 0) {
      store_slot(rec, kAcc, Ev, Ec);
      store_slot(rec, kAcc + 1, (R)sk, R(0));
      store_slot(rec, kAcc + 2, R(0), R(0));
      store_slot(rec, kAcc + 3, R(0), R(0));
    }
  }
}

// Launch configurations the autotuner chooses from (256-thread CTAs):
//   0  plain loop, 2 pixels per lane per group, natural register budget
//   1  software-pipelined loop, 1 pixel per lane per group
//   2  software-pipelined loop, 2 pixels per lane per group
//   3  software-pipelined loop, 1 pixel per lane, register budget for 3 CTAs per SM
// FP64 runs configurations 0 and 1 only.
constexpr int kK1Block = 256;
constexpr int kK1Cfgs = 4;

template <typename R, int DT>
const void* pick_cfg(int cfg) {
  switch (cfg) {
    case 0: return reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 1, 2, false>);
    case 1: return reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 1, 1, true>);
    case 2: return sizeof(R) == 4 ? reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 1, 2, true>) : nullptr;
    case 3: return sizeof(R) == 4 ? reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 3, 1, true>) : nullptr;
    default: return nullptr;
  }
}

const void* pick_kernel(int mode, int dtype, int cfg) {
  if (mode == 1) {
    switch (dtype) {
      case 0: return pick_cfg<float, 0>(cfg);
      case 1: return pick_cfg<float, 1>(cfg);
      case 2: return pick_cfg<float, 2>(cfg);
    }
  } else {
    switch (dtype) {
      case 0: return pick_cfg<double, 0>(cfg);
      case 1: return pick_cfg<double, 1>(cfg);
      case 2: return pick_cfg<double, 2>(cfg);
    }
  }
  return nullptr;
}

}  // namespace

int residual_reduce_num_cfgs(int mode) { return mode == 1 ? kK1Cfgs : 2; }

int residual_reduce_block() { return kK1Block; }

int residual_reduce_max_blocks_per_sm(int mode, int dtype, int cfg) {
  const void* f = pick_kernel(mode, dtype, cfg);
  if (!f) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kK1Block, 0) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_residual_reduce(int mode, int dtype, int cfg, int grid, const void* points,
                                   const int32_t* midx, const Item* items, int num_items,
                                   const EdgeStatic* es, const double* T64, const float* T32,
                                   RobustParams rp, void* partials, cudaStream_t s) {
  const void* f = pick_kernel(mode, dtype, cfg);
  if (!f) return cudaErrorInvalidValue;
  if (num_items <= 0) return cudaSuccess;
  void* args[] = {(void*)&points, (void*)&midx, (void*)&items, (void*)&num_items, (void*)&es,
                  (void*)&T64, (void*)&T32, (void*)&rp, (void*)&partials};
  return cudaLaunchKernel(f, dim3(grid), dim3(kK1Block), args, 0, s);
}

}  // namespace como3r
