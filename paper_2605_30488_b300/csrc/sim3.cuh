// FP64 Sim(3) device math: pose loading, relative poses, Ad of an inverse, left Exp.
//
// A pose is stored (tx, ty, tz, qx, qy, qz, qw, s) and means T = [s R(q) t; 0 1], which
// maps camera coordinates into the world frame (Sec. III-A).  Tangent vectors are
// tau = (v, omega, zeta) and act by the left perturbation T <- Exp(tau) T (Sec. III-D).
#pragma once
#include <cuda_runtime.h>

namespace como3r {

struct Sim3d {
  double R[9];  // rotation, row-major
  double s;     // scale
  double t[3];  // translation
};

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

__device__ __forceinline__ void load_pose(const double* p, Sim3d& T) {
  T.t[0] = p[0]; T.t[1] = p[1]; T.t[2] = p[2];
  quat_to_rot(p[3], p[4], p[5], p[6], T.R);
  T.s = p[7];
}

// T_ij = T_i^{-1} T_j: sR_ij = (s_j / s_i) R_i^T R_j, t_ij = R_i^T (t_j - t_i) / s_i.
__device__ __forceinline__ void relative_pose(const Sim3d& Ti, const Sim3d& Tj, double* sR, double* t) {
  const double si_inv = 1.0 / Ti.s;
  const double sij = Tj.s * si_inv;
  const double dt[3] = {Tj.t[0] - Ti.t[0], Tj.t[1] - Ti.t[1], Tj.t[2] - Ti.t[2]};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // (R_i^T R_j)[r][c] = sum_k R_i[k][r] R_j[k][c]
      sR[3 * r + c] = sij * (Ti.R[r] * Tj.R[c] + Ti.R[3 + r] * Tj.R[3 + c] + Ti.R[6 + r] * Tj.R[6 + c]);
    }
    t[r] = si_inv * (Ti.R[r] * dt[0] + Ti.R[3 + r] * dt[1] + Ti.R[6 + r] * dt[2]);
  }
}

// Ad of T^{-1} for T = (s R, t): T^{-1} = (s' R', t') with s' = 1/s, R' = R^T,
// t' = -R^T t / s, and Ad_(s'R', t') = [[s'R', [t']x R', -t'], [0, R', 0], [0, 0, 1]]
// (tau = (v, omega, zeta); from T hat(tau) T^{-1} = hat(Ad tau)).  Row-major 7x7.
__device__ __forceinline__ void adjoint_of_inverse(const Sim3d& T, double* Ad) {
  const double sp = 1.0 / T.s;
  double Rp[9], tp[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Rp[3 * r + c] = T.R[3 * c + r];
#pragma unroll
  for (int r = 0; r < 3; ++r) tp[r] = -sp * (Rp[3 * r] * T.t[0] + Rp[3 * r + 1] * T.t[1] + Rp[3 * r + 2] * T.t[2]);
#pragma unroll
  for (int k = 0; k < 49; ++k) Ad[k] = 0.0;
  const double tx[9] = {0.0, -tp[2], tp[1], tp[2], 0.0, -tp[0], -tp[1], tp[0], 0.0};  // [t']x
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ad[7 * r + c] = sp * Rp[3 * r + c];
      Ad[7 * r + 3 + c] = tx[3 * r] * Rp[c] + tx[3 * r + 1] * Rp[3 + c] + tx[3 * r + 2] * Rp[6 + c];
      Ad[7 * (3 + r) + 3 + c] = Rp[3 * r + c];
    }
    Ad[7 * r + 6] = -tp[r];
  }
  Ad[48] = 1.0;
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

__device__ __forceinline__ void exp_coefficients(double theta2, double zeta, double& A, double& B, double& C) {
  const double rho2 = theta2 + zeta * zeta;
  if (rho2 < 1e-2) {
    A = 0.0; B = 0.0; C = 0.0;
    double za = 1.0;  // zeta^a
#pragma unroll
    for (int a = 0; a <= 13; ++a) {
      if (a <= 12) A += za * kExpSeries.A[a];
      double tb = 1.0;  // (-theta^2)^b for B, (-theta^2)^(b'-1) with b' = b+1 for C
#pragma unroll
      for (int b = 0; b < 7; ++b) {
        if (a <= 12 && a + 2 * b <= 12) B += za * tb * kExpSeries.B[a][b];
        if (a + 2 * (b + 1) <= 13) C += za * tb * kExpSeries.C[a][b];
        tb *= -theta2;
      }
      za *= zeta;
    }
    return;
  }
  const double ez = exp(zeta);
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

// pose <- Exp(tau) pose.  s' = e^zeta s, q' = q_omega (x) q (renormalised),
// t' = e^zeta R(omega) t + W v.
__device__ __forceinline__ void retract_left(const double* tau, double* pose) {
  const double v0 = tau[0], v1 = tau[1], v2 = tau[2];
  const double w0 = tau[3], w1 = tau[4], w2 = tau[5];
  const double zeta = tau[6];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  double A, B, C;
  exp_coefficients(th2, zeta, A, B, C);
  double k, qw;  // quaternion of the rotation by omega: (k omega, qw)
  if (th2 > 1e-16) {
    const double th = sqrt(th2);
    double sn, cs;
    sincos(0.5 * th, &sn, &cs);
    k = sn / th;
    qw = cs;
  } else {
    k = 0.5 - th2 / 48.0;
    qw = 1.0 - th2 / 8.0;
  }
  const double ax = k * w0, ay = k * w1, az = k * w2;
  double Rw[9];
  quat_to_rot(ax, ay, az, qw, Rw);
  const double ez = exp(zeta);
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

}  // namespace como3r
