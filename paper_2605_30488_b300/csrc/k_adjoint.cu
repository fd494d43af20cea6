// Adjoint of the refined cost: gradient of L(theta) = E_global(T^K(theta), theta) with
// respect to per-pixel log-range l_p (X_p = exp(l_p) psi(X_p)) and confidence c_p, where
// T^K are the poses after K Gauss-Newton iterations (Sec. III-D) and theta feeds the
// pose-depth alternation of Sec. III-E.
//
// Reverse mode through the iterations.  Iteration k maps T^k to T^{k+1} = Exp(tau_k) T^k
// with tau_k = -A_k^{-1} g_k, A_k = H_k + eps_k I (the attempt that succeeded forward).
// With a_{k+1} the adjoint of T^{k+1} in left-perturbation coordinates:
//   tau_bar = phi1(ad_tau)^T a_{k+1}            (left Jacobian of Exp, phi1(X) = sum X^n/(n+1)!)
//   a' = exp(ad_tau)^T a_{k+1}                  (Exp(tau) Exp(d) = Exp(Ad_{Exp tau} d) Exp(tau))
//   u = A_k^{-1} tau_bar                        (one more solve with the same factor)
//   phi(T, theta) = -(u^T g(T, theta) + u^T H(T, theta) tau_k), u and tau_k held fixed
//   a_k = a' + d phi / dT^k,   theta_bar += d phi / d theta,
// starting from a_K = dE/dT^K = g(T^K) and theta_bar = dE/dtheta at fixed T^K (the
// envelope term).  Per match, with W_c = w(r_c) q / sigma_c^2 and J_c the Jacobian row of
// the relative pose (file k_residual.cu's simplified form), u^T g + u^T H tau is
//   F = sum_matches sum_c W_c a_c (e_c + b_c),  a = J u~,  b = J tau~,
// u~ = Ad_{T_i^{-1}} (u_j - u_i), tau~ = Ad_{T_i^{-1}} (tau_j - tau_i) per edge.  The match
// kernel differentiates F by hand (reverse mode) with respect to the transformed point x,
// the streamed range ||X_i||, q and (linearly) u~, tau~; it scatters the pixel derivatives
// and reduces the edge's dF/dxi (relative pose), dF/du~, dF/dtau~.  The edge kernel chains
// them to the keyframes: dF/dd_j = Ad^T F_xi; dF/dd_i = -Ad^T F_xi + ad_{du}^T Ad^T F_u~ +
// ad_{dtau}^T Ad^T F_tau~ (Ad_{T_i^{-1}} itself moves with T_i: d(Ad w) = Ad ad_w d_i).
#include <cuda_fp16.h>

#include <cstdint>

#include "como3r_internal.h"

namespace como3r {
namespace {

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

template <typename R> __device__ __forceinline__ R inf_of();
template <> __device__ __forceinline__ float inf_of<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double inf_of<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

template <typename R>
struct V3 {
  R x, y, z;
};
template <typename R> __device__ __forceinline__ V3<R> v3(R x, R y, R z) { return {x, y, z}; }
template <typename R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R> __device__ __forceinline__ V3<R> axpy(R s, V3<R> a, V3<R> b) {
  return {s * a.x + b.x, s * a.y + b.y, s * a.z + b.z};
}
template <typename R> __device__ __forceinline__ V3<R> scale(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }

constexpr int kAdjRec = kAdjointRecord;  // per item: dF/dxi (7), dF/du~ (7), dF/dtau~ (7)

template <typename R>
struct AdjConsts {
  R isr, isd, ivr, ivd, kappa;
};

// The constants in the compute type (FP32 ones rounded on the host).
template <typename R>
AdjConsts<R> adj_consts(const RobustParams& rp) {
  if constexpr (sizeof(R) == 4)
    return AdjConsts<R>{rp.f_inv_sigma_ray, rp.f_inv_sigma_dist, rp.f_inv_var_ray, rp.f_inv_var_dist, rp.f_kappa};
  else
    return AdjConsts<R>{rp.inv_sigma_ray, rp.inv_sigma_dist, rp.inv_var_ray, rp.inv_var_dist, rp.kappa};
}

// Pixel-gradient accumulation: FP32 atomics into the caller's float arrays (MIXED), FP64
// atomics into double accumulators (PLAIN).
__device__ __forceinline__ void acc_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void acc_add(double* p, double v) { atomicAdd(p, v); }

// Reciprocal, reciprocal square root and square root: in FP32 the hardware approximations
// (about 2 ulp; the mixed form's gradients are checked at 1e-5), in FP64 exact.
__device__ __forceinline__ float a_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double a_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float a_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double a_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float a_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double a_sqrt(double x) { return sqrt(x); }

// The reverse pass of one match (m of keyframe i, n of keyframe j): adds its terms to the
// item's F and scatters its four pixel derivatives.
template <typename R, bool PHI>
__device__ __forceinline__ void adjoint_one(R xi, R yi, R zi, R ci, R xj, R yj, R zj, R cj, const R (&T)[12],
                                            const AdjConsts<R>& k, V3<R> uv, V3<R> uw, R uz, V3<R> tv, V3<R> tw,
                                            R tz, R out_scale, R* __restrict__ gl, R* __restrict__ gc, int64_t pi,
                                            int64_t pj, R (&F)[kAdjRec]) {
  const R inf = inf_of<R>(), th2 = R(1e-24);
  // sR X_j = dx / dl_j (the FP32 copy of the transform holds sR - I: X_j added back)
  V3<R> sx = v3(T[0] * xj + T[1] * yj + T[2] * zj, T[3] * xj + T[4] * yj + T[5] * zj,
                T[6] * xj + T[7] * yj + T[8] * zj);
  if constexpr (sizeof(R) == 4) sx = v3(sx.x + xj, sx.y + yj, sx.z + zj);
  const V3<R> x = v3(sx.x + T[9], sx.y + T[10], sx.z + T[11]);
  const R d2 = dot(x, x), di2 = xi * xi + yi * yi + zi * zi, cc = ci * cj;
  const bool ok = (fmin(d2, di2) > th2) & (fmax(fmax(d2, di2), cc) < inf) & (cc >= R(0));
  if (!ok) return;  // skipped forward too
  const R rd = a_rsqrt(d2), d = d2 * rd, rdi = a_rsqrt(di2), di = di2 * rdi;
  const V3<R> xh = scale(rd, x);
  const R e0 = xh.x - xi * rdi, e1 = xh.y - yi * rdi, e2 = xh.z - zi * rdi, e3 = d - di;
  const R q = a_sqrt(cc), sq = a_sqrt(q);
  const R sr = sq * k.isr, sd = sq * k.isd;
  const R r0 = sr * e0, r1 = sr * e1, r2 = sr * e2, r3 = sd * e3;
  const R a0 = fabs(r0), a1 = fabs(r1), a2 = fabs(r2), a3 = fabs(r3);
  const bool o0 = a0 > k.kappa, o1 = a1 > k.kappa, o2 = a2 > k.kappa, o3 = a3 > k.kappa;
  const R w0 = o0 ? k.kappa * a_rcp(a0) : R(1);
  const R w1 = o1 ? k.kappa * a_rcp(a1) : R(1);
  const R w2 = o2 ? k.kappa * a_rcp(a2) : R(1);
  const R w3 = o3 ? k.kappa * a_rcp(a3) : R(1);
  V3<R> xhb;       // d/d xh
  R db, eb3;       // d/d d, d/d e_d
  R dci, dcj;      // d/d c_i, d/d c_j
  if (!PHI) {
    // f = sum_c rho(r_c): rho' = w r
    const R rb0 = w0 * r0, rb1 = w1 * r1, rb2 = w2 * r2, rb3 = w3 * r3;
    xhb = v3(rb0 * sr, rb1 * sr, rb2 * sr);
    eb3 = rb3 * sd;
    db = eb3;
    // dq/dc_i = q / (2 c_i) and dr_c/dq = r_c / (2q): df/dc_i = sum_c w_c r_c^2 / (4 c_i)
    const R s4 = R(0.25) * (rb0 * r0 + rb1 * r1 + rb2 * r2 + rb3 * r3);
    dci = ci > R(0) ? s4 * a_rcp(ci) : R(0);
    dcj = cj > R(0) ? s4 * a_rcp(cj) : R(0);
  } else {
    const R W0 = w0 * q * k.ivr, W1 = w1 * q * k.ivr, W2 = w2 * q * k.ivr, W3 = w3 * q * k.ivd;
    // a = J u~ (ray rows P u_v + u_w x xh, range row xh.u_v + d u_z), b = J tau~
    const R al = dot(xh, uv), be = dot(xh, tv);
    const V3<R> av = scale(rd, axpy(-al, xh, uv)), bv = scale(rd, axpy(-be, xh, tv));
    const V3<R> ar = axpy(R(1), av, cross(uw, xh)), br = axpy(R(1), bv, cross(tw, xh));
    const R ad = al + d * uz, bd = be + d * tz;
    const R s0 = e0 + br.x, s1 = e1 + br.y, s2 = e2 + br.z, s3 = e3 + bd;
    const R h0 = ar.x * s0, h1 = ar.y * s1, h2 = ar.z * s2, h3 = ad * s3;
    // W depends on q directly and through r (outer Huber region: w = kappa / |r|)
    const R qb = (o0 ? R(0.5) : R(1)) * h0 * w0 * k.ivr + (o1 ? R(0.5) : R(1)) * h1 * w1 * k.ivr +
                 (o2 ? R(0.5) : R(1)) * h2 * w2 * k.ivr + (o3 ? R(0.5) : R(1)) * h3 * w3 * k.ivd;
    const R eb0 = W0 * ar.x - (o0 ? h0 * W0 * a_rcp(r0) * sr : R(0));
    const R eb1 = W1 * ar.y - (o1 ? h1 * W1 * a_rcp(r1) * sr : R(0));
    const R eb2 = W2 * ar.z - (o2 ? h2 * W2 * a_rcp(r2) * sr : R(0));
    eb3 = W3 * ad - (o3 ? h3 * W3 * a_rcp(r3) * sd : R(0));
    const V3<R> abr = v3(W0 * s0, W1 * s1, W2 * s2), bbr = v3(W0 * ar.x, W1 * ar.y, W2 * ar.z);
    const R ab3 = W3 * s3, bb3 = W3 * ad;
    xhb = v3(eb0, eb1, eb2);
    db = eb3;
    // through a_ray = (u_v - xh al) / d + u_w x xh and a_d = al + d u_z
    db += -rd * dot(abr, av) + ab3 * uz;
    xhb = axpy(-al * rd, abr, xhb);
    xhb = axpy(-rd * dot(abr, xh) + ab3, uv, xhb);
    xhb = axpy(R(1), cross(abr, uw), xhb);
    // the same through b with tau~
    db += -rd * dot(bbr, bv) + bb3 * tz;
    xhb = axpy(-be * rd, bbr, xhb);
    xhb = axpy(-rd * dot(bbr, xh) + bb3, tv, xhb);
    xhb = axpy(R(1), cross(bbr, tw), xhb);
    const R hq = R(0.5) * qb * q;
    dci = ci > R(0) ? hq * a_rcp(ci) : R(0);
    dcj = cj > R(0) ? hq * a_rcp(cj) : R(0);
    // dF/du~ = sum_c abar_c J_c, dF/dtau~ = sum_c bbar_c J_c with
    // sum_c beta_c J_c = [P beta_r + beta_d xh, xh x beta_r, beta_d d]
    const V3<R> pa = axpy(ab3, xh, scale(rd, axpy(-dot(xh, abr), xh, abr)));
    const V3<R> ca = cross(xh, abr);
    const V3<R> pb = axpy(bb3, xh, scale(rd, axpy(-dot(xh, bbr), xh, bbr)));
    const V3<R> cb = cross(xh, bbr);
    F[7] += pa.x; F[8] += pa.y; F[9] += pa.z; F[10] += ca.x; F[11] += ca.y; F[12] += ca.z; F[13] += ab3 * d;
    F[14] += pb.x; F[15] += pb.y; F[16] += pb.z; F[17] += cb.x; F[18] += cb.y; F[19] += cb.z; F[20] += bb3 * d;
  }
  // xh = x / d, d = ||x||: x_bar = (xh_bar - xh (xh . xh_bar)) / d + d_bar xh
  const V3<R> xb = axpy(db, xh, scale(rd, axpy(-dot(xh, xhb), xh, xhb)));
  if (PHI) {
    const V3<R> xc = cross(x, xb);
    F[0] += xb.x; F[1] += xb.y; F[2] += xb.z; F[3] += xc.x; F[4] += xc.y; F[5] += xc.z; F[6] += dot(xb, x);
  }
  // dl_j: dx/dl_j = sR X_j; dl_i: d||X_i||/dl_i = ||X_i|| and e_d = d - ||X_i||
  acc_add(gl + pj, out_scale * dot(xb, sx));
  acc_add(gl + pi, -out_scale * eb3 * di);
  acc_add(gc + pi, out_scale * dci);
  acc_add(gc + pj, out_scale * dcj);
}

// One warp per work item (edge, pixel range).  Without match lists the lanes stride the
// item's streamed pixels (a pixel without a match idles its lane); with K1's precompacted
// valid-match lists (entry (n << 10) | pixel offset, built with the schedule) the lanes
// take the valid matches only, so every lane works and the index rows are not read.
template <typename R, int DT, bool PHI, bool LIST>
__global__ void __launch_bounds__(256) adjoint_match_kernel(
    const void* __restrict__ points, const int32_t* __restrict__ midx, const Item* __restrict__ items, int num_items,
    const EdgeStatic* __restrict__ es, const double* __restrict__ T64, const float* __restrict__ T32,
    const R* __restrict__ evec, AdjConsts<R> k, R out_scale, R* __restrict__ gl, R* __restrict__ gc,
    double* __restrict__ rec, const int32_t* __restrict__ counts, const uint32_t* __restrict__ compact) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < num_items; it += nwarps) {
    const Item item = items[it];
    const EdgeStatic e = es[item.edge];
    R T[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) {
      if constexpr (sizeof(R) == 4) T[t] = T32[16 * item.edge + t];
      else T[t] = T64[12 * item.edge + t];
    }
    V3<R> uv{}, uw{}, tv{}, tw{};
    R uz = R(0), tz = R(0);
    if (PHI) {
      const R* ev = evec + 16 * item.edge;
      uv = v3(ev[0], ev[1], ev[2]); uw = v3(ev[3], ev[4], ev[5]); uz = ev[6];
      tv = v3(ev[7], ev[8], ev[9]); tw = v3(ev[10], ev[11], ev[12]); tz = ev[13];
    }
    R F[kAdjRec];
#pragma unroll
    for (int q = 0; q < kAdjRec; ++q) F[q] = R(0);
    const int64_t base_i = e.pix_i + item.begin;
    // software pipeline: while one match per lane is differentiated, the pixels of the next
    // and the index (list entry) of the one after are in flight.  Without lists an entry is
    // the pixel offset itself with n from the index row, -1 where there is no match.
    const int32_t* idx = midx + e.idx_off + item.begin;
    const uint32_t* list = LIST ? compact + (int64_t)it * kCompactSlot : nullptr;
    const int cnt = LIST ? counts[it] : item.end - item.begin;
    auto entry = [&](int q, int& m, int& n) {
      if (q >= cnt) {
        m = 0;
        n = -1;
      } else if constexpr (LIST) {
        const uint32_t v = __ldg(list + q);
        m = (int)(v & 1023u);
        n = (int)(v >> 10);
      } else {
        m = q;
        n = __ldg(idx + q);
      }
    };
    int mA, nA, mB, nB;
    entry(lane, mA, nA);
    entry(lane + 32, mB, nB);
    R ax = 0, ay = 0, az = 0, ac = 0, bx = 0, by = 0, bz = 0, bc = 0;
    if (nA >= 0) {
      load_point<DT, R>(points, base_i + mA, ax, ay, az, ac);
      load_point<DT, R>(points, e.pix_j + nA, bx, by, bz, bc);
    }
    for (int q0 = 0; q0 < cnt; q0 += 32) {
      R nax = 0, nay = 0, naz = 0, nac = 0, nbx = 0, nby = 0, nbz = 0, nbc = 0;
      if (nB >= 0) {
        load_point<DT, R>(points, base_i + mB, nax, nay, naz, nac);
        load_point<DT, R>(points, e.pix_j + nB, nbx, nby, nbz, nbc);
      }
      int mC, nC;
      entry(q0 + 64 + lane, mC, nC);
      const int m = mA, n = nA;
      const R xi = ax, yi = ay, zi = az, ci = ac, xj = bx, yj = by, zj = bz, cj = bc;
      mA = mB; nA = nB;
      mB = mC; nB = nC;
      ax = nax; ay = nay; az = naz; ac = nac; bx = nbx; by = nby; bz = nbz; bc = nbc;
      if (n >= 0)
        adjoint_one<R, PHI>(xi, yi, zi, ci, xj, yj, zj, cj, T, k, uv, uw, uz, tv, tw, tz, out_scale, gl, gc,
                            base_i + m, e.pix_j + n, F);
    }
    if (PHI) {
#pragma unroll
      for (int q = 0; q < kAdjRec; ++q) {
        R v = F[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        F[q] = v;
      }
      R mine = R(0);
#pragma unroll
      for (int q = 0; q < kAdjRec; ++q)
        if (lane == q) mine = F[q];
      if (lane < kAdjRec) rec[(int64_t)it * kAdjRec + lane] = (double)mine;
    }
  }
}

// Per edge (one warp; an FP64 warp instruction holds its SM sub-partition's FP64 unit
// ~80 cycles however many lanes it uses, so work is spread over lanes): Ad-rotated adjoint and step differences for the match kernel,
// u~ = Ad (u_j - u_i), tau~ = Ad (tau_j - tau_i), stored in R (16 per edge).
template <typename R>
__global__ void adjoint_edge_prep_kernel(const EdgeStatic* __restrict__ es, int E, const double* __restrict__ Ad,
                                         const double* __restrict__ u, const double* __restrict__ tau,
                                         R* __restrict__ evec) {
  __shared__ double d[14];  // u_j - u_i, tau_j - tau_i
  const int e = blockIdx.x, lane = threadIdx.x;
  if (e >= E) return;
  const int i = es[e].i, j = es[e].j;
  if (lane < 14) {
    const double* src = lane < 7 ? u : tau;
    const int k = lane % 7;
    d[lane] = src[7 * j + k] - src[7 * i + k];
  }
  __syncwarp();
  if (lane < 14) {
    const int r = lane % 7, base = lane < 7 ? 0 : 7;
    const double* A = Ad + 49 * (int64_t)e + 7 * r;
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < 7; ++c) acc = fma(A[c], d[base + c], acc);
    evec[16 * e + lane] = (R)acc;
  } else if (lane < 16) {
    evec[16 * e + lane] = R(0);
  }
}

// Component k of ad_xi^T y for xi = (v, w, z) with ad_xi = [[w^ + z I, v^, -v], [0, w^, 0], [0, 0, 0]]:
// (w^ + z I)^T y_v = y_v x w + z y_v, (v^)^T y_v + (w^)^T y_w = y_v x v + y_w x w, -v . y_v.
__device__ __forceinline__ double ad_transpose_component(const double* xi, const double* y, int k) {
  const double v0 = xi[0], v1 = xi[1], v2 = xi[2], w0 = xi[3], w1 = xi[4], w2 = xi[5], z = xi[6];
  const double y0 = y[0], y1 = y[1], y2 = y[2], q0 = y[3], q1 = y[4], q2 = y[5];
  switch (k) {
    case 0: return (y1 * w2 - y2 * w1) + z * y0;
    case 1: return (y2 * w0 - y0 * w2) + z * y1;
    case 2: return (y0 * w1 - y1 * w0) + z * y2;
    case 3: return (y1 * v2 - y2 * v1) + (q1 * w2 - q2 * w1);
    case 4: return (y2 * v0 - y0 * v2) + (q2 * w0 - q0 * w2);
    case 5: return (y0 * v1 - y1 * v0) + (q0 * w1 - q1 * w0);
    default: return -(v0 * y0 + v1 * y1 + v2 * y2);
  }
}

// Per edge (kAdjEdgeThreads threads): FP64 sum of the item records in a fixed order (warp w
// of W sums items w, w + W, ... of slot `lane`, four loads ahead; the W partial sums are
// then added pairwise), then the keyframe terms out[e][0..6] = dF/dd_i, out[e][7..13] =
// dF/dd_j, one component per lane (an FP64 instruction holds its SM sub-partition ~80
// cycles however few lanes it uses, so a component per lane is a short chain).
// (Eight warps: 10.19 -> 10.15 ms for the vjp of the 2 x 40 workload against four; sixteen
// measured the same as eight.)
constexpr int kAdjEdgeThreads = 256;
__global__ void __launch_bounds__(kAdjEdgeThreads) adjoint_edge_kernel(
    const double* __restrict__ rec, const int32_t* __restrict__ item_off, int E, const EdgeStatic* __restrict__ es,
    const double* __restrict__ Ad, const double* __restrict__ u, const double* __restrict__ tau,
    double* __restrict__ out) {
  constexpr int W = kAdjEdgeThreads / 32;
  __shared__ double part[W][kAdjRec], F[kAdjRec], y[kAdjRec], d[14], pq[14];
  const int e = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (e >= E) return;
  const int i = es[e].i, j = es[e].j;
  if (lane < kAdjRec) {
    const int i0 = item_off[e] + warp, i1 = item_off[e + 1];
    double f = 0.0;
    int it = i0;
    for (; it + 3 * W < i1; it += 4 * W) {
      const double r0 = rec[(int64_t)it * kAdjRec + lane], r1 = rec[(int64_t)(it + W) * kAdjRec + lane];
      const double r2 = rec[(int64_t)(it + 2 * W) * kAdjRec + lane], r3 = rec[(int64_t)(it + 3 * W) * kAdjRec + lane];
      f = (((f + r0) + r1) + r2) + r3;
    }
    for (; it < i1; it += W) f += rec[(int64_t)it * kAdjRec + lane];
    part[warp][lane] = f;
  } else if (warp == 0 && lane - kAdjRec < 7) {
    const int k = lane - kAdjRec;
    d[k] = u[7 * j + k] - u[7 * i + k];
  }
  if (warp == 1 && lane < 7) d[7 + lane] = tau[7 * j + lane] - tau[7 * i + lane];
  __syncthreads();
  if (warp != 0) return;
  if (lane < kAdjRec) {
    double q[W];
#pragma unroll
    for (int w = 0; w < W; ++w) q[w] = part[w][lane];
#pragma unroll
    for (int h = 1; h < W; h *= 2)
#pragma unroll
      for (int w = 0; w + h < W; w += 2 * h) q[w] += q[w + h];
    F[lane] = q[0];
  }
  __syncwarp();
  // y = [Ad^T F_xi, Ad^T F_u~, Ad^T F_tau~]
  if (lane < kAdjRec) {
    const int c = lane % 7, base = lane - c;
    const double* A = Ad + 49 * (int64_t)e;
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < 7; ++r) acc = fma(A[7 * r + c], F[base + r], acc);
    y[lane] = acc;
  }
  __syncwarp();
  // ad_(u~_j - u~_i)^T y_u~ (lanes 0..6) and ad_(tau_j - tau_i)^T y_tau~ (lanes 7..13)
  if (lane < 14) pq[lane] = lane < 7 ? ad_transpose_component(d, y + 7, lane) : ad_transpose_component(d + 7, y + 14, lane - 7);
  __syncwarp();
  if (lane < 7) {
    out[14 * e + lane] = -y[lane] + pq[lane] + pq[7 + lane];
    out[14 * e + 7 + lane] = y[lane];
  }
}

// C = A B for 7x7 row-major matrices in shared memory, one entry per thread of a 64-thread
// block (entries 49..63 idle): every FP64 instruction holds its SM sub-partition's FP64
// unit for ~80 cycles, so two warps (two sub-partitions) halve the product's time on one
// warp.  C may alias A or B; all 64 threads call it.
__device__ __forceinline__ void block_mat7_mul(const double* A, const double* B, double* C, int tid) {
  double c = 0.0;
  if (tid < 49) {
    const int r = tid / 7, q = tid % 7;
#pragma unroll
    for (int k = 0; k < 7; ++k) c = fma(A[7 * r + k], B[7 * k + q], c);
  }
  __syncthreads();
  if (tid < 49) C[tid] = c;
  __syncthreads();
}

// Terms of the phi1 series below: with ||X||_inf <= 1/2 the remainder after X^14 / 15! is
// below (1/2)^15 / 16! ~ 1.5e-18, under FP64 rounding.
constexpr int kPhiTerms = 14;

// Per keyframe (two warps): a' = exp(ad_tau)^T a and rhs = -phi1(ad_tau)^T a (so the solve
// returns u = A^{-1} tau_bar); frozen keyframes get zeros.  exp and phi1 of X = ad_tau by
// scaling and squaring (Higham, 2005): X / 2^s with ||X / 2^s||_inf <= 1/2, the Taylor
// series of phi1 to X^14 / 15! (Horner), exp = I + X phi1, then s doublings
// phi1(2X) = phi1(X)(exp(X) + I)/2, exp(2X) = exp(X)^2.
__global__ void __launch_bounds__(64) adjoint_keyframe_kernel(const double* __restrict__ a,
                                                              const double* __restrict__ tau,
                                                              const uint8_t* __restrict__ frozen, int N,
                                                              double* __restrict__ a_out, double* __restrict__ rhs) {
  __shared__ double X[49], P[49], E[49];
  __shared__ int s_sq;
  const int kf = blockIdx.x, tid = threadIdx.x;
  if (kf >= N) return;
  if (frozen[kf]) {
    if (tid < 7) a_out[7 * kf + tid] = rhs[7 * kf + tid] = 0.0;
    return;
  }
  const double* t = tau + 7 * kf;
  const bool ent = tid < 49;
  const int r = tid / 7, c = tid % 7;
  const double id = (ent && r == c) ? 1.0 : 0.0;
  // ad_tau = [[w^ + z I, v^, -v], [0, w^, 0], [0, 0, 0]]
  if (ent) {
    auto skew = [&](const double* w, int i, int k) -> double {
      if (i == k) return 0.0;
      if (i == 0) return k == 1 ? -w[2] : w[1];
      if (i == 1) return k == 0 ? w[2] : -w[0];
      return k == 0 ? -w[1] : w[0];
    };
    double v = 0.0;
    if (r < 3 && c < 3) v = skew(t + 3, r, c) + (r == c ? t[6] : 0.0);
    else if (r < 3 && c < 6) v = skew(t, r, c - 3);
    else if (r < 3) v = -t[r];
    else if (r < 6 && c >= 3 && c < 6) v = skew(t + 3, r - 3, c - 3);
    X[tid] = v;
  }
  __syncthreads();
  // infinity norm (max row sum) in warp 0, then the number of halvings
  if (tid < 32) {
    double rs = 0.0;
    if (tid < 7)
#pragma unroll
      for (int k = 0; k < 7; ++k) rs += fabs(X[7 * tid + k]);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) rs = fmax(rs, __shfl_xor_sync(0xffffffffu, rs, off));
    if (tid == 0) {
      int sq = 0;
      while (rs > 0.5 && sq < 64) {
        rs *= 0.5;
        ++sq;
      }
      s_sq = sq;
    }
  }
  __syncthreads();
  const int sq = s_sq;
  if (ent) {
    X[tid] *= ldexp(1.0, -sq);
    P[tid] = id;
  }
  __syncthreads();
#pragma unroll
  for (int n = kPhiTerms; n >= 1; --n) {  // P <- I + X P / (n + 1)
    block_mat7_mul(X, P, P, tid);
    if (ent) P[tid] = fma(P[tid], 1.0 / (double)(n + 1), id);
    __syncthreads();
  }
  block_mat7_mul(X, P, E, tid);
  if (ent) E[tid] += id;
  __syncthreads();
  for (int s2 = 0; s2 < sq; ++s2) {
    if (ent) E[tid] += id;  // E + I
    __syncthreads();
    block_mat7_mul(P, E, P, tid);
    if (ent) {
      P[tid] *= 0.5;
      E[tid] -= id;
    }
    __syncthreads();
    block_mat7_mul(E, E, E, tid);
  }
  const double* ak = a + 7 * kf;
  if (tid < 14) {
    const int q = tid % 7;
    const double* M = tid < 7 ? E : P;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) acc = fma(M[7 * k + q], ak[k], acc);
    if (tid < 7) a_out[7 * kf + q] = acc;
    else rhs[7 * kf + q] = -acc;
  }
}

// Per keyframe: a = a' - sum over its edges of dF/dd (phi = -F), in the fixed list order
// of the assembly (entries edge * 2 + [keyframe is the streamed side i]); or, when
// `a_prime` is null, the start a = scale g(T^K).  Frozen keyframes get zeros.
__global__ void adjoint_gather_kernel(const double* __restrict__ a_prime, const double* __restrict__ edge_out,
                                      const int32_t* __restrict__ kf_contrib_off,
                                      const int32_t* __restrict__ kf_contrib, const uint8_t* __restrict__ frozen,
                                      int N, const double* __restrict__ gvec, double scale, double* __restrict__ a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= 7 * N) return;
  const int kf = x / 7, k = x % 7;
  if (frozen[kf]) {
    a[x] = 0.0;
    return;
  }
  if (!a_prime) {
    a[x] = scale * gvec[x];
    return;
  }
  double s = a_prime[x];
  for (int q = kf_contrib_off[kf]; q < kf_contrib_off[kf + 1]; ++q) {
    const int c = kf_contrib[q];
    s -= edge_out[14 * (c >> 1) + ((c & 1) ? 0 : 7) + k];
  }
  a[x] = s;
}

__global__ void to_float_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    dst[x] = (float)src[x];
}

// X_p = exp(l_p) r_p, confidence c_p, packed (x, y, z, c) in the storage type.
template <int DT>
__global__ void points_from_logdepth_kernel(const float* __restrict__ rays, const float* __restrict__ logdepth,
                                            const float* __restrict__ conf, int64_t n, void* __restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float s = expf(logdepth[p]);
    const float x = s * rays[3 * p], y = s * rays[3 * p + 1], z = s * rays[3 * p + 2], c = conf[p];
    if constexpr (DT == 0) {
      __half2* o = reinterpret_cast<__half2*>(out) + 2 * p;
      o[0] = __floats2half2_rn(x, y);
      o[1] = __floats2half2_rn(z, c);
    } else if constexpr (DT == 1) {
      reinterpret_cast<float4*>(out)[p] = make_float4(x, y, z, c);
    } else {
      double* o = reinterpret_cast<double*>(out) + 4 * p;
      o[0] = (double)x; o[1] = (double)y; o[2] = (double)z; o[3] = (double)c;
    }
  }
}

// Unit ray, log-range and confidence of every stored point (inverse of the above; a
// point with zero or non-finite range gets ray 0 and log-range -inf).
template <int DT>
__global__ void rays_from_points_kernel(const void* __restrict__ points, int64_t n, float* __restrict__ rays,
                                        float* __restrict__ logdepth, float* __restrict__ conf) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double x, y, z, c;
    load_point<DT, double>(points, p, x, y, z, c);
    const double r = sqrt(x * x + y * y + z * z);
    const bool ok = r > 0.0 && r < 1e300;
    rays[3 * p] = ok ? (float)(x / r) : 0.f;
    rays[3 * p + 1] = ok ? (float)(y / r) : 0.f;
    rays[3 * p + 2] = ok ? (float)(z / r) : 0.f;
    logdepth[p] = ok ? (float)log(r) : -__int_as_float(0x7f800000);
    conf[p] = (float)c;
  }
}

int grid_for(int64_t n, int block) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + block - 1) / block;
  return (int)(need < (int64_t)sms * 8 ? (need > 0 ? need : 1) : (int64_t)sms * 8);
}

}  // namespace

cudaError_t launch_adjoint_match(int mode, int dtype, bool phi, const void* points, const int32_t* midx,
                                 const Item* items, int num_items, const EdgeStatic* es, const double* T64,
                                 const float* T32, const void* evec, RobustParams rp, double out_scale, void* gl,
                                 void* gc, double* rec, const int32_t* counts, const uint32_t* compact, cudaStream_t s) {
  if (num_items == 0) return cudaSuccess;
  const int block = 256;
  const int grid = grid_for((int64_t)num_items * 32, block);
  const bool list = counts && compact;
#define COMO3R_ADJ2(R, DT, PHI, LIST)                                                                            \
  adjoint_match_kernel<R, DT, PHI, LIST><<<grid, block, 0, s>>>(points, midx, items, num_items, es, T64, T32,     \
                                                                (const R*)evec, k, (R)out_scale, (R*)gl, (R*)gc, \
                                                                rec, counts, compact)
#define COMO3R_ADJ(R, DT)                                                                                       \
  do {                                                                                                        \
    const AdjConsts<R> k = adj_consts<R>(rp);                                                                 \
    if (phi) {                                                                                                \
      if (list) COMO3R_ADJ2(R, DT, true, true);                                                              \
      else COMO3R_ADJ2(R, DT, true, false);                                                                   \
    } else {                                                                                                  \
      if (list) COMO3R_ADJ2(R, DT, false, true);                                                             \
      else COMO3R_ADJ2(R, DT, false, false);                                                                  \
    }                                                                                                         \
  } while (0)
  if (mode == 1) {
    if (dtype == 0) COMO3R_ADJ(float, 0);
    else if (dtype == 1) COMO3R_ADJ(float, 1);
    else COMO3R_ADJ(float, 2);
  } else {
    if (dtype == 0) COMO3R_ADJ(double, 0);
    else if (dtype == 1) COMO3R_ADJ(double, 1);
    else COMO3R_ADJ(double, 2);
  }
#undef COMO3R_ADJ2
#undef COMO3R_ADJ
  return cudaGetLastError();
}

cudaError_t launch_adjoint_edge_prep(int mode, const EdgeStatic* es, int E, const double* Ad, const double* u,
                                     const double* tau, void* evec, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  if (mode == 1)
    adjoint_edge_prep_kernel<float><<<E, 32, 0, s>>>(es, E, Ad, u, tau, (float*)evec);
  else
    adjoint_edge_prep_kernel<double><<<E, 32, 0, s>>>(es, E, Ad, u, tau, (double*)evec);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_edge(const double* rec, const int32_t* item_off, int E, const EdgeStatic* es,
                                const double* Ad, const double* u, const double* tau, double* out, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  adjoint_edge_kernel<<<E, kAdjEdgeThreads, 0, s>>>(rec, item_off, E, es, Ad, u, tau, out);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_keyframe(const double* a, const double* tau, const uint8_t* frozen, int N, double* a_out,
                                    double* rhs, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  adjoint_keyframe_kernel<<<N, 64, 0, s>>>(a, tau, frozen, N, a_out, rhs);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gather(const double* a_prime, const double* edge_out, const int32_t* kf_contrib_off,
                                  const int32_t* kf_contrib, const uint8_t* frozen, int N, const double* gvec,
                                  double scale, double* a, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  adjoint_gather_kernel<<<(7 * N + 127) / 128, 128, 0, s>>>(a_prime, edge_out, kf_contrib_off, kf_contrib, frozen,
                                                            N, gvec, scale, a);
  return cudaGetLastError();
}

cudaError_t launch_to_float(const double* src, float* dst, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  to_float_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_points_from_logdepth(int dtype, const float* rays, const float* logdepth, const float* conf,
                                        int64_t n, void* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = grid_for(n, 256);
  if (dtype == 0) points_from_logdepth_kernel<0><<<grid, 256, 0, s>>>(rays, logdepth, conf, n, out);
  else if (dtype == 1) points_from_logdepth_kernel<1><<<grid, 256, 0, s>>>(rays, logdepth, conf, n, out);
  else points_from_logdepth_kernel<2><<<grid, 256, 0, s>>>(rays, logdepth, conf, n, out);
  return cudaGetLastError();
}

cudaError_t launch_rays_from_points(int dtype, const void* points, int64_t n, float* rays, float* logdepth,
                                    float* conf, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = grid_for(n, 256);
  if (dtype == 0) rays_from_points_kernel<0><<<grid, 256, 0, s>>>(points, n, rays, logdepth, conf);
  else if (dtype == 1) rays_from_points_kernel<1><<<grid, 256, 0, s>>>(points, n, rays, logdepth, conf);
  else rays_from_points_kernel<2><<<grid, 256, 0, s>>>(points, n, rays, logdepth, conf);
  return cudaGetLastError();
}

}  // namespace como3r
