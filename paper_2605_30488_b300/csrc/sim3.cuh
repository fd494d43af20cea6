// FP64 Sim(3) device math: quaternion to rotation, the coefficients of the left Exp and
// the retraction.
//
// A pose is stored (tx, ty, tz, qx, qy, qz, qw, s) and means T = [s R(q) t; 0 1], which
// maps camera coordinates into the world frame (Sec. III-A).  Tangent vectors are
// tau = (v, omega, zeta) and act by the left perturbation T <- Exp(tau) T (Sec. III-D).
#pragma once
#include <cuda_runtime.h>

namespace como3r {

__device__ __forceinline__ void quat_to_rot(double x, double y, double z, double w, double* R) {
  const double n2 = x * x + y * y + z * z + w * w;
  const double inv = rsqrt(n2);
  x *= inv; y *= inv; z *= inv; w *= inv;
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - z * w);
  R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w);
  R[7] = 2.0 * (y * z + x * w);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Coefficients of W = A I + B [w]x + C [w]x^2 = int_0^1 e^{u zeta} R(u omega) du, the
// translation part of Exp(tau) = [[e^zeta R(omega), W v], [0, 1]]:
//   A = int e^{u zeta} du,  B = int e^{u zeta} sin(u theta)/theta du,
//   C = int e^{u zeta} (1 - cos(u theta))/theta^2 du.
// Expanding e^{u zeta}, sin and cos in powers of u and integrating term by term:
//   A = sum_a zeta^a / (a+1)!
//   B = sum_{a,b} zeta^a (-theta^2)^b / (a! (2b+1)! (a+2b+2))
//   C = sum_{a, b>=1} zeta^a (-theta^2)^(b-1) / (a! (2b)! (a+2b+1)).
// Near the origin (theta^2 + zeta^2 < 1e-2) these series are summed to total degree 12
// (truncation below 1e-17); elsewhere the closed forms of the integrals are used.
struct ExpSeriesTables {
  double A[13];
  double B[13][7];
  double C[14][7];
};
__host__ __device__ constexpr ExpSeriesTables build_exp_series_tables() {
  ExpSeriesTables t{};
  double f[16] = {};
  f[0] = 1.0;
  for (int k = 1; k < 16; ++k) f[k] = f[k - 1] / (double)k;
  for (int a = 0; a <= 12; ++a) {
    t.A[a] = f[a + 1];
    for (int b = 0; b < 7; ++b) t.B[a][b] = (a + 2 * b <= 12) ? f[a] * f[2 * b + 1] / (double)(a + 2 * b + 2) : 0.0;
  }
  for (int a = 0; a <= 13; ++a)
    for (int b = 1; b <= 7; ++b) t.C[a][b - 1] = (a + 2 * b <= 13) ? f[a] * f[2 * b] / (double)(a + 2 * b + 1) : 0.0;
  return t;
}
static __constant__ ExpSeriesTables kExpSeries = build_exp_series_tables();
// the same tables in global memory, for lane-dependent indexing (a constant-cache access
// with different addresses across a warp is serialised)
static __device__ const ExpSeriesTables kExpSeriesG = build_exp_series_tables();

// A, B, C and e^zeta.  Near the origin the series are evaluated in Horner form: for every
// power a of zeta the polynomial in theta^2 is an independent chain, then one chain in
// zeta combines them, and e^zeta = 1 + zeta A (exact to rounding there).  An FP64 warp
// instruction on this GPU holds its SM sub-partition's FP64 unit ~80 cycles, so the
// instruction count matters.
__device__ __forceinline__ void exp_coefficients(double theta2, double zeta, double& A, double& B, double& C,
                                                 double& ez) {
  const double rho2 = theta2 + zeta * zeta;
  if (rho2 < 1e-2) {
    const double x = -theta2;
    double beta[13], gamma[14];
#pragma unroll
    for (int a = 0; a <= 13; ++a) {
      double pb = 0.0, pc = 0.0;
#pragma unroll
      for (int b = 6; b >= 0; --b) {
        if (a <= 12 && a + 2 * b <= 12) pb = fma(pb, x, kExpSeries.B[a][b]);
        if (a + 2 * (b + 1) <= 13) pc = fma(pc, x, kExpSeries.C[a][b]);
      }
      if (a <= 12) beta[a] = pb;
      gamma[a] = pc;
    }
    A = kExpSeries.A[12];
    B = beta[12];
    C = gamma[13];
#pragma unroll
    for (int a = 11; a >= 0; --a) {
      A = fma(A, zeta, kExpSeries.A[a]);
      B = fma(B, zeta, beta[a]);
    }
#pragma unroll
    for (int a = 12; a >= 0; --a) C = fma(C, zeta, gamma[a]);
    ez = fma(zeta, A, 1.0);
    return;
  }
  ez = exp(zeta);
  A = (fabs(zeta) > 1e-12) ? expm1(zeta) / zeta : 1.0 + 0.5 * zeta;
  if (theta2 > 1e-24) {
    const double th = sqrt(theta2);
    double sn, cs;
    sincos(th, &sn, &cs);
    B = (ez * (zeta * sn - th * cs) + th) / (th * rho2);
    C = (A - (ez * (zeta * cs + th * sn) - zeta) / rho2) / theta2;
  } else {
    // theta -> 0 limits of B and C (here |zeta| >= 0.1)
    B = (ez * (zeta - 1.0) + 1.0) / (zeta * zeta);
    C = (ez * (zeta * zeta - 2.0 * zeta + 2.0) - 2.0) / (2.0 * zeta * zeta * zeta);
  }
}

// exp_coefficients evaluated by a whole warp (all lanes call it with the same arguments
// and receive the same results).  Near the origin lane a < 14 evaluates the polynomial in
// theta^2 that multiplies zeta^a, scales it by zeta^a (binary powering) and a fixed-order
// shuffle tree sums the terms: ~40 instructions per warp instead of ~150 on one lane.
__device__ __forceinline__ void exp_coefficients_warp(double theta2, double zeta, int lane, double& A, double& B,
                                                      double& C, double& ez) {
  const double rho2 = theta2 + zeta * zeta;
  if (rho2 < 1e-2) {
    const double x = -theta2;
    const int a = lane < 14 ? lane : 13;
    double pb = 0.0, pc = 0.0;
#pragma unroll
    for (int b = 6; b >= 0; --b) {
      const double cb = (a <= 12 && a + 2 * b <= 12) ? kExpSeriesG.B[a < 13 ? a : 12][b] : 0.0;
      const double cc = (a + 2 * (b + 1) <= 13) ? kExpSeriesG.C[a][b] : 0.0;
      pb = fma(pb, x, cb);
      pc = fma(pc, x, cc);
    }
    double za = 1.0, base = zeta;
#pragma unroll
    for (int i = 0, e = a; i < 4; ++i, e >>= 1) {
      if (e & 1) za *= base;
      base *= base;
    }
    double tA = lane < 13 ? za * kExpSeriesG.A[a < 13 ? a : 12] : 0.0;
    double tB = lane < 13 ? za * pb : 0.0;
    double tC = lane < 14 ? za * pc : 0.0;
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      tA += __shfl_xor_sync(0xffffffffu, tA, off);
      tB += __shfl_xor_sync(0xffffffffu, tB, off);
      tC += __shfl_xor_sync(0xffffffffu, tC, off);
    }
    A = __shfl_sync(0xffffffffu, tA, 0);
    B = __shfl_sync(0xffffffffu, tB, 0);
    C = __shfl_sync(0xffffffffu, tC, 0);
    ez = fma(zeta, A, 1.0);
    return;
  }
  exp_coefficients(theta2, zeta, A, B, C, ez);
}

// Rotation of a quaternion that is unit by construction (no renormalisation).
__device__ __forceinline__ void unit_quat_to_rot(double x, double y, double z, double w, double* R) {
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - z * w);
  R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w);
  R[7] = 2.0 * (y * z + x * w);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// pose <- Exp(tau) pose given the coefficients A, B, C, e^zeta of exp_coefficients.
// s' = e^zeta s, q' = q_omega (x) q (renormalised), t' = e^zeta R(omega) t + W v.
__device__ __forceinline__ void retract_left_with(const double* tau, double* pose, double A, double B, double C,
                                                  double ez) {
  const double v0 = tau[0], v1 = tau[1], v2 = tau[2];
  const double w0 = tau[3], w1 = tau[4], w2 = tau[5];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  double k, qw;  // quaternion of the rotation by omega: (k omega, qw), k = sin(theta/2)/theta
  if (th2 < 1e-2) {
    // sin(h)/(2h) and cos(h) with h = theta/2 < 0.05: Taylor series in y = -h^2 to h^12
    const double y = -0.25 * th2;
    k = fma(fma(fma(fma(fma(y, 1.0 / 39916800.0, 1.0 / 362880.0), y, 1.0 / 5040.0), y, 1.0 / 120.0), y, 1.0 / 6.0), y,
            1.0);
    k *= 0.5;
    qw = fma(fma(fma(fma(fma(fma(y, 1.0 / 479001600.0, 1.0 / 3628800.0), y, 1.0 / 40320.0), y, 1.0 / 720.0), y,
                     1.0 / 24.0),
                 y, 0.5),
             y, 1.0);
  } else {
    const double th = sqrt(th2);
    double sn, cs;
    sincos(0.5 * th, &sn, &cs);
    k = sn / th;
    qw = cs;
  }
  const double ax = k * w0, ay = k * w1, az = k * w2;
  double Rw[9];
  unit_quat_to_rot(ax, ay, az, qw, Rw);
  // W v = A v + B (w x v) + C (w x (w x v))
  const double c1[3] = {w1 * v2 - w2 * v1, w2 * v0 - w0 * v2, w0 * v1 - w1 * v0};
  const double c2[3] = {w1 * c1[2] - w2 * c1[1], w2 * c1[0] - w0 * c1[2], w0 * c1[1] - w1 * c1[0]};
  const double vv[3] = {v0, v1, v2};
  const double t0 = pose[0], t1 = pose[1], t2 = pose[2];
  double tn[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double Rt = Rw[3 * r] * t0 + Rw[3 * r + 1] * t1 + Rw[3 * r + 2] * t2;
    tn[r] = ez * Rt + A * vv[r] + B * c1[r] + C * c2[r];
  }
  // Hamilton product q_omega (x) q, both stored (x, y, z, w)
  const double bx = pose[3], by = pose[4], bz = pose[5], bw = pose[6];
  const double nx = qw * bx + bw * ax + (ay * bz - az * by);
  const double ny = qw * by + bw * ay + (az * bx - ax * bz);
  const double nz = qw * bz + bw * az + (ax * by - ay * bx);
  const double nw = qw * bw - (ax * bx + ay * by + az * bz);
  const double inv = rsqrt(nx * nx + ny * ny + nz * nz + nw * nw);
  pose[0] = tn[0]; pose[1] = tn[1]; pose[2] = tn[2];
  pose[3] = nx * inv; pose[4] = ny * inv; pose[5] = nz * inv; pose[6] = nw * inv;
  pose[7] = ez * pose[7];
}

// pose <- Exp(tau) pose as retract_left_with, eight lanes at once: lanes 0..2 the
// translation rows, lane 3 the scale, lanes 4..7 the quaternion (x, y, z, w).  Every lane
// runs the same straight-line code on lane-selected operands (an FP64 warp instruction costs
// the same whatever the lane count, so the update takes ~1/2 of the one-lane version's
// instructions).  R(omega) t = t + 2 (qw u + a x u), u = a x t, for the unit quaternion
// (a, qw) of omega.  All 32 lanes must call it (shuffles); lanes >= 8 write nothing.
__device__ __forceinline__ void retract_left_warp(const double* tau, double* pose, double A, double B, double C,
                                                  double ez, int lane) {
  const double v[3] = {tau[0], tau[1], tau[2]};
  const double w[3] = {tau[3], tau[4], tau[5]};
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double k, qw;  // quaternion of the rotation by omega: (k omega, qw), k = sin(theta/2)/theta
  if (th2 < 1e-2) {
    // the two series of retract_left_with in y = -theta^2/4, term for term: 2k on even
    // lanes, qw on odd lanes
    const double y = -0.25 * th2;
    const bool odd = lane & 1;
    double sr = odd ? 1.0 / 479001600.0 : 0.0;
    sr = fma(sr, y, odd ? 1.0 / 3628800.0 : 1.0 / 39916800.0);
    sr = fma(sr, y, odd ? 1.0 / 40320.0 : 1.0 / 362880.0);
    sr = fma(sr, y, odd ? 1.0 / 720.0 : 1.0 / 5040.0);
    sr = fma(sr, y, odd ? 1.0 / 24.0 : 1.0 / 120.0);
    sr = fma(sr, y, odd ? 0.5 : 1.0 / 6.0);
    sr = fma(sr, y, 1.0);
    k = 0.5 * __shfl_sync(0xffffffffu, sr, 0);
    qw = __shfl_sync(0xffffffffu, sr, 1);
  } else {
    const double th = sqrt(th2);
    double sn, cs;
    sincos(0.5 * th, &sn, &cs);
    k = sn / th;
    qw = cs;
  }
  const double a[3] = {k * w[0], k * w[1], k * w[2]};
  const double t[3] = {pose[0], pose[1], pose[2]};
  const double b[4] = {pose[3], pose[4], pose[5], pose[6]};
  // translation row r (lanes 0..2; other lanes compute row lane % 3 and drop it)
  const int r = lane % 3, r1 = r == 2 ? 0 : r + 1, r2 = r == 0 ? 2 : r - 1;
  const double u[3] = {a[1] * t[2] - a[2] * t[1], a[2] * t[0] - a[0] * t[2], a[0] * t[1] - a[1] * t[0]};
  const double axu = a[r1] * u[r2] - a[r2] * u[r1];
  const double rt = fma(2.0, fma(qw, u[r], axu), t[r]);
  const double c1[3] = {w[1] * v[2] - w[2] * v[1], w[2] * v[0] - w[0] * v[2], w[0] * v[1] - w[1] * v[0]};
  const double c2 = w[r1] * c1[r2] - w[r2] * c1[r1];
  const double tn = fma(C, c2, fma(B, c1[r], fma(A, v[r], ez * rt)));
  // Hamilton product q_omega (x) q, component c = lane - 4 (lanes 4..7), as one chain of
  // lane-selected products: qw b_c + b_w a_c + a_{c+1} b_{c+2} - a_{c+2} b_{c+1} for x, y, z
  // and qw b_w - a . b for w
  const int c = (lane - 4) & 3, cc = c < 3 ? c : 0, c1i = cc == 2 ? 0 : cc + 1, c2i = cc == 0 ? 2 : cc - 1;
  const bool isw = c == 3;
  double n = qw * (isw ? b[3] : b[cc]);
  n = fma(isw ? -a[0] : b[3], isw ? b[0] : a[cc], n);
  n = fma(isw ? -a[1] : a[c1i], isw ? b[1] : b[c2i], n);
  n = fma(isw ? -a[2] : -a[c2i], isw ? b[2] : b[c1i], n);
  double n2 = n * n;  // |q'|^2 over lanes 4..7
  n2 += __shfl_xor_sync(0xffffffffu, n2, 1);
  n2 += __shfl_xor_sync(0xffffffffu, n2, 2);
  const double qn = n * rsqrt(n2);
  __syncwarp();  // every lane has read the pose before lanes 0..7 overwrite it
  if (lane < 3) pose[lane] = tn;
  else if (lane == 3) pose[7] = ez * pose[7];
  else if (lane < 8) pose[lane - 1] = qn;
}

// pose <- Exp(tau) pose (one thread).
__device__ __forceinline__ void retract_left(const double* tau, double* pose) {
  const double th2 = tau[3] * tau[3] + tau[4] * tau[4] + tau[5] * tau[5];
  double A, B, C, ez;
  exp_coefficients(th2, tau[6], A, B, C, ez);
  retract_left_with(tau, pose, A, B, C, ez);
}

}  // namespace como3r
