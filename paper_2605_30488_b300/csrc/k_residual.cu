// K1: per-match residual, whitening, Huber IRLS weights, 4x7 Jacobian and reduction of
// the relative-pose normal-equation blocks of every edge (Sec. III-A, III-D).
//
// Work is split into items (edge, [begin, end) of the streamed keyframe's pixels), each
// owned by one warp of a persistent grid.  Every lane accumulates its pixels (pixel
// m = begin + lane + 32 k: coalesced streams of match_idx and X_i, a gather of X_j[n])
// into 34 registers -- the 25 structurally nonzero entries of H_rel = sum J^T W J, the 7
// of g_rel = sum J^T W e, and the cost with the error of its FP32 sum (the cost terms are
// all non-negative, so a lane's long sum would otherwise drift by ~1e-5 relative over a
// few thousand matches) -- then the warp reduces them with shuffles and
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
  R isr, isd, ivr, ivd, kappa, half_kappa, kivr, kivd;  // kivr = kappa / sigma_r^2, kivd = kappa / sigma_d^2
};

template <typename R>
__device__ __forceinline__ Consts<R> make_consts(const RobustParams& rp) {
  Consts<R> k;
  if constexpr (sizeof(R) == 4) {  // the host-rounded FP32 copies: no FP64 conversion in the kernel
    k.isr = rp.f_inv_sigma_ray; k.isd = rp.f_inv_sigma_dist;
    k.ivr = rp.f_inv_var_ray; k.ivd = rp.f_inv_var_dist;
    k.kappa = rp.f_kappa; k.half_kappa = 0.5f * rp.f_kappa;
    k.kivr = rp.f_kappa_inv_var_ray; k.kivd = rp.f_kappa_inv_var_dist;
  } else {
    k.isr = rp.inv_sigma_ray; k.isd = rp.inv_sigma_dist;
    k.ivr = rp.inv_var_ray; k.ivd = rp.inv_var_dist;
    k.kappa = rp.kappa; k.half_kappa = 0.5 * rp.kappa;
    k.kivr = rp.kappa * rp.inv_var_ray; k.kivd = rp.kappa * rp.inv_var_dist;
  }
  return k;
}

// FP32: hardware approximations with denormals flushed (inputs here are far from the
// denormal range; relative error ~2^-22, well inside the mixed form's 1e-5 tolerance)
__device__ __forceinline__ float rsq(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
template <typename R> __device__ __forceinline__ R kInfinity();
template <> __device__ __forceinline__ float kInfinity<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double kInfinity<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

// Square root of a non-negative value (0 -> 0).
__device__ __forceinline__ float nn_sqrt(float v) {  // hardware approximation (sqrt(0) = 0)
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
  return y;
}
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
  R E;        // sum of the Huber costs rho(r_c) of the lane's matches
  R Ec;       // its compensation (FP32: error-free Fast2Sum terms; FP64: unused, 0)
  int skipped;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < kAcc; ++k) v[k] = R(0);
    E = R(0);
    Ec = R(0);
    skipped = 0;
  }
};

// E + x with its rounding error kept in Ec (both non-negative: Fast2Sum on the larger
// and the smaller operand is error-free); FP64 adds plainly.
__device__ __forceinline__ void add_cost(float& E, float& Ec, float x) {
  const float hi = fmaxf(E, x), lo = fminf(E, x);
  const float s = __fadd_rn(hi, lo);
  Ec = __fadd_rn(Ec, __fsub_rn(lo, __fsub_rn(s, hi)));
  E = s;
}
__device__ __forceinline__ void add_cost(double& E, double&, double x) { E += x; }

// One match: residual, robust weights, Jacobian rows, accumulation (see file header).
// x = sR X_j + t from the edge's transform: FP64 holds sR itself, the FP32 copy sR - I (its
// entries small for the near-identity relative poses of neighbouring keyframes, so their
// rounding, shared by all of the edge's matches, is small), with X_j added back.
template <typename R>
__device__ __forceinline__ void transform_point(const R* T, R xj, R yj, R zj, R& x0, R& x1, R& x2) {
  x0 = fma(T[0], xj, fma(T[1], yj, fma(T[2], zj, T[9])));
  x1 = fma(T[3], xj, fma(T[4], yj, fma(T[5], zj, T[10])));
  x2 = fma(T[6], xj, fma(T[7], yj, fma(T[8], zj, T[11])));
  if constexpr (sizeof(R) == 4) {
    x0 += xj;
    x1 += yj;
    x2 += zj;
  }
}

template <typename R>
__device__ __forceinline__ void accumulate(R xi, R yi, R zi, R ci, R xj, R yj, R zj, R cj, const R* T,
                                           const Consts<R>& k, Acc<R>& acc) {
  R x0, x1, x2;
  transform_point<R>(T, xj, yj, zj, x0, x1, x2);
  const R d2 = fma(x0, x0, fma(x1, x1, x2 * x2));
  const R di2 = fma(xi, xi, fma(yi, yi, zi * zi));
  const R cc = ci * cj;
  // skip degenerate or non-finite matches: both squared ranges in (1e-24, inf), c_i c_j in
  // [0, inf); NaN fails every comparison
  const R th2 = R(1e-24), inf = kInfinity<R>();
  const bool ok = (fmin(d2, di2) > th2) & (fmax(fmax(d2, di2), cc) < inf) & (cc >= R(0));
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
  // Huber: W_c = w_c q / sigma_c^2 with w = min(1, kappa / |r|), formed as
  // min(q / sigma^2, (kappa q / sigma^2) / |r|), exact (q / sigma^2) inside the threshold
  // (kappa / 0 = inf gives the inside value; q = 0 gives 0); with m = min(|r|, kappa),
  // rho(r) = m (|r| - m / 2) on both branches (r^2 / 2 inside, kappa |r| - kappa^2 / 2 outside)
  const R a0 = fabs(r0), a1 = fabs(r1), a2 = fabs(r2), a3 = fabs(r3);
  const R m0 = fmin(a0, k.kappa), m1 = fmin(a1, k.kappa), m2 = fmin(a2, k.kappa), m3 = fmin(a3, k.kappa);
  // rho(r_c) = m_c (|r_c| - m_c / 2) on both branches
  const R mh = R(-0.5);
  // the lane's cost sum runs over at most 64 matches between compensated folds, like H
  acc.E += fma(m0, fma(mh, m0, a0), fma(m1, fma(mh, m1, a1), fma(m2, fma(mh, m2, a2), m3 * fma(mh, m3, a3))));
  const R qr = q * k.ivr, qkr = q * k.kivr, qd = q * k.ivd, qkd = q * k.kivd;
  const R u0 = fmin(qr, qkr * rcp(a0)), u1 = fmin(qr, qkr * rcp(a1)), u2 = fmin(qr, qkr * rcp(a2));
  const R u3 = fmin(qd, qkd * rcp(a3));  // W_c
  const R f0 = u0 * e0, f1 = u1 * e1, f2 = u2 * e2, f3 = u3 * e3;        // W_c e_c
  // P = (I - xh xh^T) / d, symmetric
  const R ard = a * rd, brd = b * rd, crd = c * rd;
  const R p00 = fma(-ard, a, rd), p11 = fma(-brd, b, rd), p22 = fma(-crd, c, rd);
  const R p01 = -ard * b, p02 = -ard * c, p12 = -brd * c;
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

// ---- two matches per lane in packed FP32x2 arithmetic (sm_100+ FFMA2 / FMUL2 / FADD2)
// Element .x is match A, .y is match B; every operation is the scalar one of accumulate()
// applied to both elements, so each element's rounding is unchanged while the FP32
// instruction count of the arithmetic roughly halves.  Accumulators stay separate per
// element (AccPair) and are added when the record is written.
struct AccPair {
  float2 v[kAcc];
  float2 E, Ec;  // Huber cost sums and their compensations, per element
  int skipped;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < kAcc; ++k) v[k] = make_float2(0.f, 0.f);
    E = Ec = make_float2(0.f, 0.f);
    skipped = 0;
  }
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// A pair of matches (either may be a padding or degenerate slot: its inputs are replaced
// by a benign point with zero confidence, so it contributes exactly zero).
__device__ __forceinline__ void accumulate_pair(float2 xi, float2 yi, float2 zi, float2 ci, float2 xj, float2 yj,
                                                float2 zj, float2 cj, bool useA, bool useB, const float* T,
                                                const Consts<float>& k, AccPair& acc) {
  // T holds sR - I (see transform_point): X_j added back
  const float2 x0 = add2(xj, fma2(f2(T[0]), xj, fma2(f2(T[1]), yj, fma2(f2(T[2]), zj, f2(T[9])))));
  const float2 x1 = add2(yj, fma2(f2(T[3]), xj, fma2(f2(T[4]), yj, fma2(f2(T[5]), zj, f2(T[10])))));
  const float2 x2 = add2(zj, fma2(f2(T[6]), xj, fma2(f2(T[7]), yj, fma2(f2(T[8]), zj, f2(T[11])))));
  float2 d2 = fma2(x0, x0, fma2(x1, x1, mul2(x2, x2)));
  float2 di2 = fma2(xi, xi, fma2(yi, yi, mul2(zi, zi)));
  float2 cc = mul2(ci, cj);
  const float th2 = 1e-24f, inf = kInfinity<float>();
  const bool okA = useA && (fminf(d2.x, di2.x) > th2) & (fmaxf(fmaxf(d2.x, di2.x), cc.x) < inf) & (cc.x >= 0.f);
  const bool okB = useB && (fminf(d2.y, di2.y) > th2) & (fmaxf(fmaxf(d2.y, di2.y), cc.y) < inf) & (cc.y >= 0.f);
  acc.skipped += (useA && !okA) + (useB && !okB);
  if (!okA && !okB) return;
  // a slot that does not contribute: unit ranges, zero confidence -> every term is 0
  float2 XI = xi, YI = yi, ZI = zi;
  if (!okA) { d2.x = 1.f; di2.x = 1.f; cc.x = 0.f; XI.x = 1.f; YI.x = 0.f; ZI.x = 0.f; }
  if (!okB) { d2.y = 1.f; di2.y = 1.f; cc.y = 0.f; XI.y = 1.f; YI.y = 0.f; ZI.y = 0.f; }
  const float2 X0 = f2(okA ? x0.x : 1.f, okB ? x0.y : 1.f);
  const float2 X1 = f2(okA ? x1.x : 0.f, okB ? x1.y : 0.f);
  const float2 X2 = f2(okA ? x2.x : 0.f, okB ? x2.y : 0.f);
  const float2 rd = f2(rsq(d2.x), rsq(d2.y)), d = mul2(d2, rd);
  const float2 rdi = f2(rsq(di2.x), rsq(di2.y)), di = mul2(di2, rdi);
  const float2 a = mul2(X0, rd), b = mul2(X1, rd), c = mul2(X2, rd);
  const float2 e0 = fma2(neg2(XI), rdi, a), e1 = fma2(neg2(YI), rdi, b), e2 = fma2(neg2(ZI), rdi, c);
  const float2 e3 = add2(d, neg2(di));
  const float2 q = f2(nn_sqrt(cc.x), nn_sqrt(cc.y));
  const float2 sq = f2(nn_sqrt(q.x), nn_sqrt(q.y));
  const float2 sr = mul2(sq, f2(k.isr)), sd = mul2(sq, f2(k.isd));
  const float2 r0 = mul2(sr, e0), r1 = mul2(sr, e1), r2 = mul2(sr, e2), r3 = mul2(sd, e3);
  const float2 a0 = f2(fabsf(r0.x), fabsf(r0.y)), a1 = f2(fabsf(r1.x), fabsf(r1.y));
  const float2 a2 = f2(fabsf(r2.x), fabsf(r2.y)), a3 = f2(fabsf(r3.x), fabsf(r3.y));
  const float2 m0 = f2(fminf(a0.x, k.kappa), fminf(a0.y, k.kappa)), m1 = f2(fminf(a1.x, k.kappa), fminf(a1.y, k.kappa));
  const float2 m2 = f2(fminf(a2.x, k.kappa), fminf(a2.y, k.kappa)), m3 = f2(fminf(a3.x, k.kappa), fminf(a3.y, k.kappa));
  {
    const float2 h = f2(-0.5f);
    const float2 rho = fma2(m0, fma2(h, m0, a0), fma2(m1, fma2(h, m1, a1), fma2(m2, fma2(h, m2, a2),
                                                                            mul2(m3, fma2(h, m3, a3)))));
    add_cost(acc.E.x, acc.Ec.x, rho.x);
    add_cost(acc.E.y, acc.Ec.y, rho.y);
  }
  // W_c = min(q / sigma_c^2, (kappa q / sigma_c^2) / |r_c|), as in accumulate()
  const float2 qr = mul2(q, f2(k.ivr)), qkr = mul2(q, f2(k.kivr)), qd = mul2(q, f2(k.ivd)), qkd = mul2(q, f2(k.kivd));
  const float2 t0 = mul2(qkr, f2(rcp(a0.x), rcp(a0.y))), t1 = mul2(qkr, f2(rcp(a1.x), rcp(a1.y)));
  const float2 t2 = mul2(qkr, f2(rcp(a2.x), rcp(a2.y))), t3 = mul2(qkd, f2(rcp(a3.x), rcp(a3.y)));
  const float2 u0 = f2(fminf(qr.x, t0.x), fminf(qr.y, t0.y)), u1 = f2(fminf(qr.x, t1.x), fminf(qr.y, t1.y));
  const float2 u2 = f2(fminf(qr.x, t2.x), fminf(qr.y, t2.y)), u3 = f2(fminf(qd.x, t3.x), fminf(qd.y, t3.y));
  const float2 g0 = mul2(u0, e0), g1 = mul2(u1, e1), g2 = mul2(u2, e2), g3 = mul2(u3, e3);
  const float2 ard = mul2(a, rd), brd = mul2(b, rd), crd = mul2(c, rd);
  const float2 p00 = fma2(neg2(ard), a, rd), p11 = fma2(neg2(brd), b, rd), p22 = fma2(neg2(crd), c, rd);
  const float2 p01 = mul2(neg2(ard), b), p02 = mul2(neg2(ard), c), p12 = mul2(neg2(brd), c);
  const float2 w00 = mul2(u0, p00), w01 = mul2(u0, p01), w02 = mul2(u0, p02);
  const float2 w10 = mul2(u1, p01), w11 = mul2(u1, p11), w12 = mul2(u1, p12);
  const float2 w20 = mul2(u2, p02), w21 = mul2(u2, p12), w22 = mul2(u2, p22);
  const float2 ua = mul2(u3, a), ub = mul2(u3, b), uc = mul2(u3, c);
  float2* h = acc.v;
  h[0] = fma2(w00, p00, fma2(w10, p01, fma2(w20, p02, fma2(ua, a, h[0]))));
  h[1] = fma2(w00, p01, fma2(w10, p11, fma2(w20, p12, fma2(ua, b, h[1]))));
  h[2] = fma2(w00, p02, fma2(w10, p12, fma2(w20, p22, fma2(ua, c, h[2]))));
  h[3] = fma2(w01, p01, fma2(w11, p11, fma2(w21, p12, fma2(ub, b, h[3]))));
  h[4] = fma2(w01, p02, fma2(w11, p12, fma2(w21, p22, fma2(ub, c, h[4]))));
  h[5] = fma2(w02, p02, fma2(w12, p12, fma2(w22, p22, fma2(uc, c, h[5]))));
  const float2 na = neg2(a), nb = neg2(b), nc = neg2(c);
  h[6] = fma2(nc, w10, fma2(b, w20, h[6]));
  h[7] = fma2(c, w00, fma2(na, w20, h[7]));
  h[8] = fma2(nb, w00, fma2(a, w10, h[8]));
  h[9] = fma2(nc, w11, fma2(b, w21, h[9]));
  h[10] = fma2(c, w01, fma2(na, w21, h[10]));
  h[11] = fma2(nb, w01, fma2(a, w11, h[11]));
  h[12] = fma2(nc, w12, fma2(b, w22, h[12]));
  h[13] = fma2(c, w02, fma2(na, w22, h[13]));
  h[14] = fma2(nb, w02, fma2(a, w12, h[14]));
  const float2 cc2 = mul2(c, c), bb2 = mul2(b, b), aa2 = mul2(a, a);
  h[15] = fma2(u1, cc2, fma2(u2, bb2, h[15]));
  h[16] = fma2(neg2(mul2(u2, a)), b, h[16]);
  h[17] = fma2(neg2(mul2(u1, a)), c, h[17]);
  h[18] = fma2(u0, cc2, fma2(u2, aa2, h[18]));
  h[19] = fma2(neg2(mul2(u0, b)), c, h[19]);
  h[20] = fma2(u0, bb2, fma2(u1, aa2, h[20]));
  const float2 ud = mul2(u3, d);
  h[21] = fma2(ud, a, h[21]);
  h[22] = fma2(ud, b, h[22]);
  h[23] = fma2(ud, c, h[23]);
  h[24] = fma2(ud, d, h[24]);
  h[25] = fma2(g0, p00, fma2(g1, p01, fma2(g2, p02, fma2(g3, a, h[25]))));
  h[26] = fma2(g0, p01, fma2(g1, p11, fma2(g2, p12, fma2(g3, b, h[26]))));
  h[27] = fma2(g0, p02, fma2(g1, p12, fma2(g2, p22, fma2(g3, c, h[27]))));
  h[28] = fma2(nc, g1, fma2(b, g2, h[28]));
  h[29] = fma2(c, g0, fma2(na, g2, h[29]));
  h[30] = fma2(nb, g0, fma2(a, g1, h[30]));
  h[31] = fma2(g3, d, h[31]);
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

// The same butterfly without compensation (mid-run folds: five rounded additions per value,
// bounded error; the running totals they feed are compensated).
template <typename R>
__device__ __forceinline__ void warp_transpose_reduce_plain(R (&v)[kAcc], int lane) {
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int off = 16 >> lvl;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < off; ++k) {
      const R send_v = upper ? v[k] : v[k + off];
      const R keep_v = upper ? v[k + off] : v[k];
      v[k] = keep_v + __shfl_xor_sync(0xffffffffu, send_v, off);
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

// Plain warp sum (the lanes' cost compensations: tiny, so their own rounding is moot).
__device__ __forceinline__ float warp_sum_plain(float x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}
__device__ __forceinline__ double warp_sum_plain(double) { return 0.0; }

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

// ---- bounded compensated runs
// A lane sums at most kFoldGroups groups (at most one match of each) in plain FP32
// registers; then the warp folds them: the compensated butterfly leaves in lane l the warp
// total of accumulator l, which TwoSum adds to the lane's running pair (s, c), the
// rounding error going to c.  So no FP32 sum runs over more than 64 terms per lane and
// everything above the lane is compensated; a record holds the (s, c) pairs.  FP64 folds
// with plain additions.
constexpr int kFoldGroups = 64;

template <typename R>
struct Folded {
  R s, c;      // lane l: warp total of accumulator l over the folded matches, s + c
  R es, ec;    // every lane: the warp's Huber cost over the folded matches, es + ec
  int groups;  // groups summed in the lanes' registers since the last fold (warp-uniform)
  __device__ __forceinline__ void zero() {
    s = R(0);
    c = R(0);
    es = R(0);
    ec = R(0);
    groups = 0;
  }
};

__device__ __forceinline__ void two_sum_into(float& s, float& c, float v, float cv) {
  float err;
  const float t = two_sum(s, v, err);
  c = c + cv + err;
  s = t;
}
__device__ __forceinline__ void two_sum_into(double& s, double&, double v, double cv) { s += v + cv; }
__device__ __forceinline__ void fold_add(Folded<float>& f, float v, float cv) { two_sum_into(f.s, f.c, v, cv); }
__device__ __forceinline__ void fold_add(Folded<double>& f, double v, double cv) { f.s += v + cv; }

// The lanes' cost sums (and, for the packed variant, their compensations) into the folded
// cost: a compensated warp sum added by TwoSum.
template <typename R>
__device__ __forceinline__ void fold_cost(Acc<R>& acc, Folded<R>& f) {
  R ec = R(0);
  const R ev = warp_sum_pair(acc.E, ec);
  ec += warp_sum_plain(acc.Ec);
  two_sum_into(f.es, f.ec, ev, ec);
  acc.E = R(0);
  acc.Ec = R(0);
}

// The final fold of a record: compensated butterfly.
template <typename R>
__device__ __forceinline__ void fold(Acc<R>& acc, Folded<R>& f, int lane) {
  R comp[kAcc];
  warp_transpose_reduce(acc.v, comp, lane);
  fold_add(f, acc.v[0], comp[0]);
  fold_cost(acc, f);
#pragma unroll
  for (int k = 0; k < kAcc; ++k) acc.v[k] = R(0);
  f.groups = 0;
}

// A mid-run fold: plain butterfly (its five additions per value round the warp's partial
// totals of at most 64 matches per lane), compensated accumulation into (s, c).
template <typename R>
__device__ __forceinline__ void fold_mid(Acc<R>& acc, Folded<R>& f, int lane) {
  warp_transpose_reduce_plain(acc.v, lane);
  fold_add(f, acc.v[0], R(0));
  fold_cost(acc, f);
#pragma unroll
  for (int k = 0; k < kAcc; ++k) acc.v[k] = R(0);
  f.groups = 0;
}

// Before `g` more groups are summed: fold first when the lanes' runs would exceed the bound.
template <typename R>
__device__ __forceinline__ void fold_before(Acc<R>& acc, Folded<R>& f, int g, int lane) {
  if (f.groups > 0 && f.groups + g > kFoldGroups) fold_mid(acc, f, lane);
  f.groups += g;
}

// Writes the warp's record `it`: the folded accumulators when `flush` (last item of a run of
// items of one edge owned by this warp), zeros otherwise (the per-edge reduction adds all
// records of an edge, so folding items into one record is exact).
template <typename R>
__device__ __forceinline__ void write_record(Acc<R>& acc, Folded<R>& f, void* partials, int it, bool flush,
                                             int lane) {
  using Slot = typename std::conditional<sizeof(R) == 4, float2, double>::type;
  Slot* rec = reinterpret_cast<Slot*>(partials) + (int64_t)it * kPartial;
  if (!flush) {
    store_slot(rec, lane, R(0), R(0));
    if (lane < kPartial - kAcc) store_slot(rec, kAcc + lane, R(0), R(0));
    return;
  }
  fold(acc, f, lane);
  const int sk = __reduce_add_sync(0xffffffffu, acc.skipped);
  store_slot(rec, lane, f.s, f.c);
  if (lane == 0) {
    store_slot(rec, kAcc, f.es, f.ec);
    store_slot(rec, kAcc + 1, (R)sk, R(0));
    store_slot(rec, kAcc + 2, R(0), R(0));
    store_slot(rec, kAcc + 3, R(0), R(0));
  }
  acc.zero();
  f.zero();
}

// This warp's run of items and its first record index (-1: one record per item).
__device__ __forceinline__ void warp_range(const WarpSched& ws, int gwarp, int nwarps, int num_items, int& it0,
                                           int& it1, int& seg) {
  if (ws.start) {
    it0 = ws.start[gwarp];
    it1 = ws.start[gwarp + 1];
    seg = ws.seg[gwarp];
  } else {
    const int per = (num_items + nwarps - 1) / nwarps;
    it0 = min(gwarp * per, num_items);
    it1 = min(it0 + per, num_items);
    seg = -1;
  }
}

template <typename R>
__device__ __forceinline__ void finish_item(Acc<R>& acc, Folded<R>& f, void* partials, int it, int& seg, bool flush,
                                            int lane) {
  if (seg < 0) {
    write_record(acc, f, partials, it, flush, lane);
  } else if (flush) {
    write_record(acc, f, partials, seg, true, lane);
    ++seg;
  }
}

template <typename R, int DT, int BLOCK, int MINB, int UNROLL, bool PIPE>
__global__ void __launch_bounds__(BLOCK, MINB) residual_reduce_kernel(
    const void* __restrict__ points, const int32_t* __restrict__ midx, const Item* __restrict__ items,
    int num_items, const EdgeStatic* __restrict__ es, const double* __restrict__ T64,
    const float* __restrict__ T32, RobustParams rp, void* __restrict__ partials, WarpSched ws) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * BLOCK) >> 5;
  const Consts<R> k = make_consts<R>(rp);

  // each warp owns a contiguous run of items and reduces once per edge
  int it0, it1, seg;
  warp_range(ws, gwarp, nwarps, num_items, it0, it1, seg);
  Acc<R> acc;
  acc.zero();
  Folded<R> f;
  f.zero();
  for (int it = it0; it < it1; ++it) {
    const Item item = items[it];
    const int64_t pix_i = es[item.edge].pix_i, pix_j = es[item.edge].pix_j;
    const int32_t* __restrict__ idx = midx + es[item.edge].idx_off;
    R T[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      if constexpr (sizeof(R) == 4) T[q] = T32[16 * item.edge + q];
      else T[q] = T64[12 * item.edge + q];
    }
    constexpr int STEP = 32 * UNROLL;
    if constexpr (!PIPE) {
      // plain loop: indices, then both pixels, then the arithmetic of this group
      for (int g0 = item.begin; g0 < item.end; g0 += STEP) {
        Group<R, UNROLL> G;
        load_indices<R, UNROLL>(G.n, idx, g0 + lane, item.end);
        load_pixels<DT, R, UNROLL>(G, points, pix_i, pix_j, g0 + lane);
        fold_before(acc, f, UNROLL, lane);
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
        fold_before(acc, f, UNROLL, lane);
        accumulate_group<R, UNROLL>(A, T, k, acc);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) A.n[u] = nA[u];
        g0 += STEP;
        if (g0 >= item.end) break;
        load_pixels<DT, R, UNROLL>(A, points, pix_i, pix_j, g0 + STEP + lane);
        int nB[UNROLL];
        load_indices<R, UNROLL>(nB, idx, g0 + 2 * STEP + lane, item.end);
        fold_before(acc, f, UNROLL, lane);
        accumulate_group<R, UNROLL>(B, T, k, acc);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) B.n[u] = nB[u];
        g0 += STEP;
      }
    }
    // ---- warp reduction (compensated butterfly) at the end of each edge run
    finish_item(acc, f, partials, it, seg, it + 1 == it1 || items[it + 1].edge != item.edge, lane);
  }
}

// ---- shared-memory-staged variant (cp.async) -----------------------------------------
// Each warp owns a slice of shared memory: two buffers of match indices (the current item
// and the prefetched next one, kAsyncChunk entries each) and a ring of kRing pixel
// groups (32 lanes x streamed + gathered pixel).  The item's list of valid matches
// (entry = n << 10 | m) is precompacted when the schedule is built, or, without a list,
// compacted by the warp in place once its index row has landed (ballot + prefix count),
// so every lane of the arithmetic works on a real match although a third of the
// streamed pixels typically have none.  The pixels of the compacted matches then flow
// through the ring: lane l only ever reads ring slots it filled itself, so the ring needs
// no warp synchronisation, and kRing groups of both pixel loads stay in flight per warp
// without costing registers.
constexpr int kAsyncChunk = 1024;
constexpr int kRing = 4;
constexpr int kK1Block = 256;
constexpr int kK1Warps = kK1Block / 32;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int DT> struct PixBytes;
template <> struct PixBytes<0> { static constexpr int v = 8; };
template <> struct PixBytes<1> { static constexpr int v = 16; };
template <> struct PixBytes<2> { static constexpr int v = 32; };

template <int DT>
__device__ __forceinline__ void copy_px(unsigned char* dst, const void* base, int64_t p) {
  const unsigned char* src = static_cast<const unsigned char*>(base) + p * PixBytes<DT>::v;
  if constexpr (DT == 0) cp_async8(dst, src);
  else if constexpr (DT == 1) cp_async16(dst, src);
  else {
    cp_async16(dst, src);
    cp_async16(dst + 16, src + 16);
  }
}

template <int DT, typename R>
__device__ __forceinline__ void read_px(const unsigned char* s, R& x, R& y, R& z, R& c) {
  if constexpr (DT == 0) {
    const uint2 v = *reinterpret_cast<const uint2*>(s);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    x = (R)a.x; y = (R)a.y; z = (R)b.x; c = (R)b.y;
  } else if constexpr (DT == 1) {
    const float4 v = *reinterpret_cast<const float4*>(s);
    x = (R)v.x; y = (R)v.y; z = (R)v.z; c = (R)v.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(s), b = *reinterpret_cast<const double2*>(s + 16);
    x = (R)a.x; y = (R)a.y; z = (R)b.x; c = (R)b.y;
  }
}

static_assert(kAsyncChunk == kCompactSlot, "valid-match list slots hold one 1024-pixel item");

// copies an item's precompacted valid-match list (cnt packed entries, slot 16-byte aligned)
// into buf (all lanes; 16-byte pieces, 4-byte tail)
__device__ __forceinline__ void prefetch_packed(int32_t* buf, const uint32_t* __restrict__ src, int cnt, int lane) {
  const int n16 = cnt & ~3;
  for (int q = 4 * lane; q < n16; q += 128) cp_async16(buf + q, src + q);
  for (int q = n16 + lane; q < cnt; q += 32) cp_async4(buf + q, src + q);
}

// copies the match indices of `item` into buf (all lanes; 16-byte pieces, 4-byte tail)
__device__ __forceinline__ void prefetch_indices(int32_t* buf, const int32_t* __restrict__ idx, const Item& item,
                                                 int lane) {
  const int n = item.end - item.begin;
  const int n16 = n & ~3;
  for (int q = 4 * lane; q < n16; q += 128) cp_async16(buf + q, idx + item.begin + q);
  for (int q = n16 + lane; q < n; q += 32) cp_async4(buf + q, idx + item.begin + q);
}

// cp.async of one packed pixel to a shared-memory address given as a 32-bit shared-space
// address (no generic-to-shared conversion per copy)
template <int DT>
__device__ __forceinline__ void copy_px_s(uint32_t dst, const unsigned char* src) {
  if constexpr (DT == 0) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
  } else if constexpr (DT == 1) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16), "l"(src + 16) : "memory");
  }
}

template <typename R, int DT, bool PAIR>
__global__ void __launch_bounds__(256, PAIR ? 1 : 2) residual_reduce_async_kernel(
    const void* __restrict__ points, const int32_t* __restrict__ midx, const Item* __restrict__ items,
    int num_items, const EdgeStatic* __restrict__ es, const double* __restrict__ T64,
    const float* __restrict__ T32, RobustParams rp, void* __restrict__ partials, WarpSched ws) {
  constexpr int PX = PixBytes<DT>::v;
  constexpr int kWarpBytes = 2 * kAsyncChunk * 4 + kRing * 32 * 2 * PX;
  constexpr int kSlotBytes = 32 * 2 * PX;  // one ring slot: 32 lanes x (streamed, gathered) pixel
  static_assert((kRing & (kRing - 1)) == 0, "ring depth is a power of two");
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned char* mine = smem + (size_t)warp * kWarpBytes;
  int32_t* ibuf[2] = {reinterpret_cast<int32_t*>(mine), reinterpret_cast<int32_t*>(mine) + kAsyncChunk};
  unsigned char* ring = mine + 2 * kAsyncChunk * 4 + lane * 2 * PX;  // + slot * kSlotBytes
  const uint32_t ring_s = smem_addr(ring);
  const int gwarp = (blockIdx.x * 256 + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * 256) >> 5;
  const Consts<R> k = make_consts<R>(rp);

  // each warp owns a contiguous run of items and reduces once per edge
  int it0, it1, seg;
  warp_range(ws, gwarp, nwarps, num_items, it0, it1, seg);
  int b = 0;
  // with precompacted valid-match lists the index rows are not read at all
  const bool pre = ws.compact != nullptr;
  int cnt_cur = 0, cnt_next = 0;
  if (it0 < it1) {
    const Item first = items[it0];
    if (pre) {
      cnt_cur = ws.counts[it0];
      prefetch_packed(ibuf[0], ws.compact + (int64_t)it0 * kCompactSlot, cnt_cur, lane);
    } else {
      prefetch_indices(ibuf[0], midx + es[first.edge].idx_off, first, lane);
    }
  }
  cp_commit();
  Acc<R> acc;
  acc.zero();
  Folded<R> f;
  f.zero();
  AccPair pacc;  // PAIR only
  if constexpr (PAIR) pacc.zero();
  // PAIR: the packed accumulators are folded through acc (their two elements added first)
  auto fold_pairs = [&]() {
    if constexpr (PAIR) {
#pragma unroll
      for (int q = 0; q < kAcc; ++q) {
        acc.v[q] = pacc.v[q].x + pacc.v[q].y;
        pacc.v[q] = make_float2(0.f, 0.f);
      }
      fold_mid(acc, f, lane);
    }
  };
  for (int it = it0; it < it1; ++it, b ^= 1) {
    const Item item = items[it];
    const int next = it + 1;
    if (next < it1) {
      if (pre) {
        cnt_next = ws.counts[next];
        prefetch_packed(ibuf[b ^ 1], ws.compact + (int64_t)next * kCompactSlot, cnt_next, lane);
      } else {
        const Item itn = items[next];
        prefetch_indices(ibuf[b ^ 1], midx + es[itn.edge].idx_off, itn, lane);
      }
    }
    cp_commit();
    cp_wait<1>();  // this item's indices (all but the group just committed)
    __syncwarp();
    // the item's streamed and gathered keyframes as byte pointers (pixel offsets are added
    // per match as 32-bit multiples of the pixel size)
    const unsigned char* src_i =
        static_cast<const unsigned char*>(points) + (es[item.edge].pix_i + item.begin) * PX;
    const unsigned char* src_j = static_cast<const unsigned char*>(points) + es[item.edge].pix_j * PX;
    const int32_t* cur = ibuf[b];
    R T[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      if constexpr (sizeof(R) == 4) T[q] = T32[16 * item.edge + q];
      else T[q] = T64[12 * item.edge + q];
    }
    const int n_pix = item.end - item.begin;
    int nvalid = 0;
    if (pre) {
      nvalid = cnt_cur;  // the list is in the buffer already
      cnt_cur = cnt_next;
    } else {
      // compact the valid matches of the item in place (writes never reach unread entries)
      int32_t* curw = ibuf[b];
      const unsigned below = (1u << lane) - 1u;
      for (int g0 = 0; g0 < n_pix; g0 += 32) {
        const int m = g0 + lane;
        const int n = m < n_pix ? cur[m] : -1;
        const unsigned mask = __ballot_sync(0xffffffffu, n >= 0);
        if (n >= 0) curw[nvalid + __popc(mask & below)] = (int32_t)(((uint32_t)n << 10) | (uint32_t)m);
        nvalid += __popc(mask);
      }
      __syncwarp();
    }
    const int ngroups = (nvalid + 31) >> 5;
    if constexpr (PAIR) {
      if (f.groups > 0 && f.groups + ngroups > kFoldGroups) fold_pairs();
      f.groups += ngroups;
    } else {
      fold_before(acc, f, ngroups, lane);
    }
    // this lane's list entry of group gidx (entries past the list issue nothing)
    auto issue = [&](int gidx) {
      const int e = 32 * gidx + lane;
      if (e < nvalid) {
        const uint32_t v = (uint32_t)cur[e];
        const uint32_t slot = ring_s + (uint32_t)(gidx & (kRing - 1)) * kSlotBytes;
        copy_px_s<DT>(slot, src_i + (v & 1023u) * PX);
        copy_px_s<DT>(slot + PX, src_j + (v >> 10) * PX);
      }
      cp_commit();
    };
#pragma unroll
    for (int s0 = 0; s0 < kRing; ++s0) issue(s0);
    if constexpr (!PAIR) {
      for (int gidx = 0; gidx < ngroups; ++gidx) {
        cp_wait<kRing - 1>();
        if (32 * gidx + lane < nvalid) {
          const unsigned char* slot = ring + (size_t)(gidx & (kRing - 1)) * kSlotBytes;
          R xi, yi, zi, ci, xj, yj, zj, cj;
          read_px<DT, R>(slot, xi, yi, zi, ci);
          read_px<DT, R>(slot + PX, xj, yj, zj, cj);
          accumulate<R>(xi, yi, zi, ci, xj, yj, zj, cj, T, k, acc);
        }
        issue(gidx + kRing);
      }
    } else {
      // two groups per step: the lane's matches of groups g and g + 1 as one packed pair
      for (int gidx = 0; gidx < ngroups; gidx += 2) {
        cp_wait<kRing - 2>();
        const bool useA = 32 * gidx + lane < nvalid, useB = 32 * (gidx + 1) + lane < nvalid;
        float xiA = 0.f, yiA = 0.f, ziA = 0.f, ciA = 0.f, xjA = 0.f, yjA = 0.f, zjA = 0.f, cjA = 0.f;
        float xiB = 0.f, yiB = 0.f, ziB = 0.f, ciB = 0.f, xjB = 0.f, yjB = 0.f, zjB = 0.f, cjB = 0.f;
        if (useA) {
          const unsigned char* slot = ring + (size_t)(gidx & (kRing - 1)) * kSlotBytes;
          read_px<DT, float>(slot, xiA, yiA, ziA, ciA);
          read_px<DT, float>(slot + PX, xjA, yjA, zjA, cjA);
        }
        if (useB) {
          const unsigned char* slot = ring + (size_t)((gidx + 1) & (kRing - 1)) * kSlotBytes;
          read_px<DT, float>(slot, xiB, yiB, ziB, ciB);
          read_px<DT, float>(slot + PX, xjB, yjB, zjB, cjB);
        }
        if (useA || useB)
          accumulate_pair(f2(xiA, xiB), f2(yiA, yiB), f2(ziA, ziB), f2(ciA, ciB), f2(xjA, xjB), f2(yjA, yjB),
                          f2(zjA, zjB), f2(cjA, cjB), useA, useB, T, k, pacc);
        issue(gidx + kRing);
        issue(gidx + kRing + 1);
      }
    }
    cp_wait<0>();
    __syncwarp();  // the index buffer of this item is reused two items later
    const bool flush = it + 1 == it1 || items[it + 1].edge != item.edge;
    if constexpr (PAIR) {
      // fold the two elements of the packed accumulators (only read when flushing)
      if (flush) {
        fold_pairs();
        float err;
        acc.E = two_sum(pacc.E.x, pacc.E.y, err);
        acc.Ec = pacc.Ec.x + pacc.Ec.y + err;
        acc.skipped = pacc.skipped;
        pacc.zero();
      }
    }
    finish_item(acc, f, partials, it, seg, flush, lane);
  }
  cp_wait<0>();
}

template <int DT>
constexpr int async_smem_bytes() { return 8 * (2 * kAsyncChunk * 4 + kRing * 32 * 2 * PixBytes<DT>::v); }

// ---- TMA-staged variant (bulk asynchronous copies into a CTA ring) -------------------
// CTA-level items of kAsyncChunk pixels.  Thread 0 streams each item's match indices and
// streamed pixels (both contiguous) into a kTmaStages-deep shared-memory ring with bulk
// copies (cp.async.bulk), whose completion an mbarrier counts in bytes: tens of KB per CTA
// in flight at the cost of two instructions, none per lane.  The eight warps take four
// interleaved 32-pixel groups of each item; while a warp computes item q from shared
// memory, its gathers of item q + 1 (cp.async, one per valid match, into a per-warp double
// buffer) are in flight, so the gather latency overlaps the arithmetic and holds no
// registers.  A warp releases the stage on a second mbarrier after item q; thread 0
// refills it with the item kTmaStages ahead.  The CTA reduces
// (warp butterflies, then FP64 across warps in warp order) once per run of items of one
// edge.  Every mbarrier wait is bounded: a wait that gives up is counted in
// g_k1_stalls and the kernel finishes without that stage's data (the result is then
// wrong and the count says so); it never hangs.
constexpr int kTmaCfg = 5;
constexpr int kTmaStages = 3;
constexpr long long kSpinLimit = 1LL << 24;
__device__ unsigned int g_k1_stalls = 0;

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Polls the phase of the given parity; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long spin = 0; spin < kSpinLimit; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// This CTA's run of items and its first record index (-1: one record per item).
__device__ __forceinline__ void cta_range(const WarpSched& ws, int num_items, int& it0, int& it1, int& seg) {
  if (ws.start) {
    it0 = ws.start[blockIdx.x];
    it1 = ws.start[blockIdx.x + 1];
    seg = ws.seg[blockIdx.x];
  } else {
    const int per = (num_items + gridDim.x - 1) / gridDim.x;
    it0 = min((int)blockIdx.x * per, num_items);
    it1 = min(it0 + per, num_items);
    seg = -1;
  }
}

// CTA-wide record of the accumulators (all threads call it; `flush` is CTA-uniform).
template <typename R>
__device__ __forceinline__ void cta_record(Acc<R>& acc, Folded<R>& f, void* partials, int rec_idx, bool flush,
                                           double (*red)[kAcc + 2], int tid, int lane, int warp) {
  using Slot = typename std::conditional<sizeof(R) == 4, float2, double>::type;
  Slot* rec = reinterpret_cast<Slot*>(partials) + (int64_t)rec_idx * kPartial;
  if (!flush) {
    if (tid < kPartial) store_slot(rec, tid, R(0), R(0));
    return;
  }
  fold(acc, f, lane);
  const R Ev = f.es, Ec = f.ec;
  const int sk = __reduce_add_sync(0xffffffffu, acc.skipped);
  red[warp][lane] = (double)f.s + (double)f.c;
  f.zero();
  if (lane == 0) {
    red[warp][kAcc] = (double)Ev + (double)Ec;
    red[warp][kAcc + 1] = (double)sk;
  }
  acc.zero();
  __syncthreads();
  if (tid < kPartial) {
    double sum = 0.0;
    if (tid < kAcc + 2)
#pragma unroll
      for (int w = 0; w < kK1Warps; ++w) sum += red[w][tid];
    if constexpr (sizeof(R) == 4) {
      const float hi = (float)sum;
      rec[tid] = make_float2(hi, (float)(sum - (double)hi));
    } else {
      rec[tid] = sum;
    }
  }
  __syncthreads();
}

template <typename R, int DT>
__global__ void __launch_bounds__(256, 2) residual_reduce_tma_kernel(
    const void* __restrict__ points, const int32_t* __restrict__ midx, const Item* __restrict__ items,
    int num_items, const EdgeStatic* __restrict__ es, const double* __restrict__ T64,
    const float* __restrict__ T32, RobustParams rp, void* __restrict__ partials, WarpSched ws) {
  constexpr int PX = PixBytes<DT>::v;
  constexpr int kIdxBytes = kAsyncChunk * 4;
  constexpr int kStageBytes = kIdxBytes + kAsyncChunk * PX;
  static_assert(kAsyncChunk == 4 * 32 * kK1Warps, "four 32-pixel groups per warp and item");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kTmaStages], empty_bar[kTmaStages];
  __shared__ double red[kK1Warps][kAcc + 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int it0, it1, seg;
  cta_range(ws, num_items, it0, it1, seg);
  const int n_local = it1 - it0;
  if (tid == 0) {
    for (int q = 0; q < kTmaStages; ++q) {
      mbar_init(&full_bar[q], 1);
      mbar_init(&empty_bar[q], kK1Warps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const Consts<R> k = make_consts<R>(rp);
  // thread 0: bulk copies of local item q into stage q % kTmaStages
  auto issue = [&](int q) {
    const Item item = items[it0 + q];
    const EdgeStatic& e = es[item.edge];
    const uint32_t n = (uint32_t)(item.end - item.begin);
    unsigned char* base = smem + (size_t)(q % kTmaStages) * kStageBytes;
    uint64_t* bar = &full_bar[q % kTmaStages];
    mbar_expect_tx(bar, n * (4u + (uint32_t)PX));
    bulk_copy(base, midx + e.idx_off + item.begin, n * 4u, bar);
    bulk_copy(base + kIdxBytes, static_cast<const unsigned char*>(points) + (e.pix_i + item.begin) * PX,
              n * (uint32_t)PX, bar);
  };
  // gathered pixels of items q (buffer q & 1) and q + 1: per warp 4 groups x 32 lanes, each
  // lane's own slots (written by its cp.async, read only by itself)
  unsigned char* gbuf = smem + (size_t)kTmaStages * kStageBytes;
  auto gslot = [&](int b, int u) -> unsigned char* {
    return gbuf + ((size_t)((b * kK1Warps + warp) * 4 + u) * 32 + lane) * PX;
  };
  // groups interleaved across warps (warp w: groups w, w + 8, w + 16, w + 24), so a band of
  // valid columns spreads over all warps of the CTA
  auto gather = [&](int q) {
    const Item item = items[it0 + q];
    const int64_t pix_j = es[item.edge].pix_j;
    const int32_t* sidx = reinterpret_cast<const int32_t*>(smem + (size_t)(q % kTmaStages) * kStageBytes);
    const int n_pix = item.end - item.begin;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int m = 32 * (warp + kK1Warps * u) + lane;
      const int n = m < n_pix ? sidx[m] : -1;
      if (n >= 0) copy_px<DT>(gslot(q & 1, u), points, pix_j + n);
    }
  };
  if (tid == 0)
    for (int q = 0; q < kTmaStages && q < n_local; ++q) issue(q);
  bool landed_cur = n_local > 0 && mbar_wait(&full_bar[0], 0u);
  if (landed_cur) gather(0);
  cp_commit();
  Acc<R> acc;
  acc.zero();
  Folded<R> f;
  f.zero();
  for (int q = 0; q < n_local; ++q) {
    const int st = q % kTmaStages;
    const uint32_t parity = (uint32_t)(q / kTmaStages) & 1u;
    const int it = it0 + q;
    const Item item = items[it];
    if (!landed_cur && lane == 0) atomicAdd(&g_k1_stalls, 1u);
    // the gathers of item q + 1 fly while item q is computed
    bool landed_next = false;
    if (q + 1 < n_local) {
      landed_next = mbar_wait(&full_bar[(q + 1) % kTmaStages], (uint32_t)((q + 1) / kTmaStages) & 1u);
      if (landed_next) gather(q + 1);
    }
    cp_commit();
    cp_wait<1>();  // item q's gathers have landed (all groups but the newest)
    R T[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) {
      if constexpr (sizeof(R) == 4) T[t] = T32[16 * item.edge + t];
      else T[t] = T64[12 * item.edge + t];
    }
    fold_before(acc, f, 4, lane);  // at most four matches per lane per item
    if (landed_cur) {
      const int32_t* sidx = reinterpret_cast<const int32_t*>(smem + (size_t)st * kStageBytes);
      const unsigned char* sxi = smem + (size_t)st * kStageBytes + kIdxBytes;
      const int n_pix = item.end - item.begin;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = 32 * (warp + kK1Warps * u) + lane;
        if (m < n_pix && sidx[m] >= 0) {
          R xi, yi, zi, ci, xj, yj, zj, cj;
          read_px<DT, R>(sxi + (size_t)m * PX, xi, yi, zi, ci);
          read_px<DT, R>(gslot(q & 1, u), xj, yj, zj, cj);
          accumulate<R>(xi, yi, zi, ci, xj, yj, zj, cj, T, k, acc);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_bar[st]);  // this warp no longer reads the stage
    if (tid == 0 && q + kTmaStages < n_local) {
      if (mbar_wait(&empty_bar[st], parity)) issue(q + kTmaStages);
      else atomicAdd(&g_k1_stalls, 1u);  // not refilled: the waits for it give up too
    }
    landed_cur = landed_next;
    const bool flush = it + 1 == it1 || items[it + 1].edge != item.edge;
    if (seg < 0) {
      cta_record(acc, f, partials, it, flush, red, tid, lane, warp);
    } else if (flush) {
      cta_record(acc, f, partials, seg, true, red, tid, lane, warp);
      ++seg;
    }
  }
  cp_wait<0>();
}

template <int DT>
constexpr int tma_smem_bytes() {
  return kTmaStages * (kAsyncChunk * 4 + kAsyncChunk * PixBytes<DT>::v) + 2 * kAsyncChunk * PixBytes<DT>::v;
}

// Launch configurations the autotuner chooses from (256-thread CTAs):
//   0  plain loop, 2 pixels per lane per group, natural register budget
//   1  software-pipelined loop, 1 pixel per lane per group
//   2  software-pipelined loop, 2 pixels per lane per group
//   3  software-pipelined loop, 1 pixel per lane, register budget for 3 CTAs per SM
//   4  shared-memory-staged loop (cp.async ring) over warp-compacted valid matches; work
//      items of exactly 1024 pixels, only when every match-index row starts 16-byte
//      aligned and every keyframe has at most 2^22 pixels
//   5  TMA-staged CTA ring (bulk copies of index rows and streamed pixels), FP32 compute
//      on FP16 / FP32 storage; the same item and alignment conditions as 4
//   6  as 4 with two matches per lane in packed FP32x2 arithmetic (FP32 compute only)
// FP64 has configurations 0, 1 and 4.
constexpr int kK1Cfgs = 7;
constexpr int kPairCfg = 6;
constexpr int kAsyncCfg = 4;

template <typename R, int DT>
const void* pick_cfg(int cfg) {
  if (cfg == 0) return reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 1, 2, false>);
  if (cfg == 1) return reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 1, 1, true>);
  if constexpr (sizeof(R) == 4) {
    if (cfg == 2) return reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 1, 2, true>);
    if (cfg == 3) return reinterpret_cast<const void*>(&residual_reduce_kernel<R, DT, kK1Block, 3, 1, true>);
  }
  if (cfg == kAsyncCfg) return reinterpret_cast<const void*>(&residual_reduce_async_kernel<R, DT, false>);
  if constexpr (sizeof(R) == 4) {
    if (cfg == kPairCfg) return reinterpret_cast<const void*>(&residual_reduce_async_kernel<R, DT, true>);
  }
  if constexpr (sizeof(R) == 4 && DT < 2) {
    if (cfg == kTmaCfg) return reinterpret_cast<const void*>(&residual_reduce_tma_kernel<R, DT>);
  }
  return nullptr;
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

int residual_reduce_num_cfgs(int mode) { return kK1Cfgs; }

int residual_reduce_cfg_chunk(int cfg) {
  return (cfg == kAsyncCfg || cfg == kTmaCfg || cfg == kPairCfg) ? kAsyncChunk : 0;
}

static size_t cfg_smem(int dtype, int cfg) {
  if (cfg == kTmaCfg) return dtype == 0 ? tma_smem_bytes<0>() : tma_smem_bytes<1>();
  if (cfg != kAsyncCfg && cfg != kPairCfg) return 0;
  return dtype == 0 ? async_smem_bytes<0>() : (dtype == 1 ? async_smem_bytes<1>() : async_smem_bytes<2>());
}

cudaError_t residual_reduce_prepare() {
  // opt the shared-memory-staged variants into more than 48 KB of dynamic shared memory
  cudaError_t e = cudaSuccess;
  for (int mode = 0; mode < 2; ++mode)
    for (int d = 0; d < 3 && e == cudaSuccess; ++d)
      e = cudaFuncSetAttribute(pick_kernel(mode, d, kAsyncCfg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)cfg_smem(d, kAsyncCfg));
  for (int d = 0; d < 2 && e == cudaSuccess; ++d)
    e = cudaFuncSetAttribute(pick_kernel(1, d, kTmaCfg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cfg_smem(d, kTmaCfg));
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaFuncSetAttribute(pick_kernel(1, d, kPairCfg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cfg_smem(d, kPairCfg));
  return e;
}

int residual_reduce_block() { return kK1Block; }

int residual_reduce_workers_per_cta(int cfg) { return cfg == kTmaCfg ? 1 : kK1Block / 32; }

unsigned int residual_reduce_stalls() {
  unsigned int v = 0;
  cudaMemcpyFromSymbol(&v, g_k1_stalls, sizeof(v));
  return v;
}

void residual_reduce_cost_weights(int cfg, int& wv, int& wp) {
  // first candidates of the autotuner (measured on the 2x40 workload): cfg 0-3 pay one
  // memory round trip per 32-pixel group whether it holds matches or not; cfg 4 and 5
  // prefetch whole index rows, so valid matches weigh more
  wp = 1;
  wv = (cfg == kAsyncCfg || cfg == kPairCfg) ? 3 : (cfg == kTmaCfg ? 1 : 0);
}

int residual_reduce_max_blocks_per_sm(int mode, int dtype, int cfg) {
  const void* f = pick_kernel(mode, dtype, cfg);
  if (!f) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kK1Block, cfg_smem(dtype, cfg)) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_residual_reduce(int mode, int dtype, int cfg, int grid, const void* points,
                                   const int32_t* midx, const Item* items, int num_items,
                                   const EdgeStatic* es, const double* T64, const float* T32,
                                   RobustParams rp, void* partials, WarpSched ws, cudaStream_t s) {
  const void* f = pick_kernel(mode, dtype, cfg);
  if (!f) return cudaErrorInvalidValue;
  if (num_items <= 0) return cudaSuccess;
  void* args[] = {(void*)&points, (void*)&midx, (void*)&items, (void*)&num_items, (void*)&es,
                  (void*)&T64, (void*)&T32, (void*)&rp, (void*)&partials, (void*)&ws};
  return cudaLaunchKernel(f, dim3(grid), dim3(kK1Block), args, cfg_smem(dtype, cfg), s);
}

}  // namespace como3r
