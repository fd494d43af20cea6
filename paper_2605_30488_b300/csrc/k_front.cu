// Front-end kernels (Sec. III-A): projective ray matching and confidence-weighted fusion.
//
// Matching: for every queried point x (keyframe k's pointmap predicted in frame f's
// camera), p* = argmin_p |psi([X^f_f]_p) - psi(x)|^2 on f's ray image, found by a
// deterministic descent over pixels: from a start pixel, move to the best of the 8
// neighbours (fixed order, strictly smaller distance, first in order on ties) while it
// improves, at most max_steps moves.  Every distance is FP32 with each operation correctly
// rounded in one fixed order,
//   n = sqrt((x0 x0 + x1 x1) + x2 x2), psi = x / n,  d = ((a0-b0)^2 + (a1-b1)^2) + (a2-b2)^2,
// (no contraction into FMAs), so the integer result is reproducible on any IEEE machine.
// A query whose point is not finite or has zero norm, or whose final distance exceeds
// 2 - 2 cos(max_angle) (rounded to FP32), gets -1; pixels of f whose ray is not finite are
// never entered.  ray_image_kernel writes f's rays once (12 B + pad per pixel; they stay
// in L2 while the queries walk); match_kernel is one thread per query.
//
// Fusion (Eq. fusion): X_k <- (C_k X_k + C_f (T_kf X_f)) / (C_k + C_f), C_k <- C_k + C_f,
// one thread per pixel, in the storage type's precision (FP32 or FP64); como3r_fuse_packed
// fuses many keyframes (each with its own T_kf) in one launch, pixel for pixel the same.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdint>

#include "../../include/como3r.h"
#include "como3r_internal.h"

namespace como3r {
namespace {

__device__ __forceinline__ void load_xyz_f32(const void* base, int dtype, int64_t p, float& x, float& y, float& z) {
  if (dtype == COMO3R_F16) {
    const uint2 v = reinterpret_cast<const uint2*>(base)[p];
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    x = a.x; y = a.y; z = b.x;
  } else if (dtype == COMO3R_F32) {
    const float4 v = reinterpret_cast<const float4*>(base)[p];
    x = v.x; y = v.y; z = v.z;
  } else {
    const double* q = reinterpret_cast<const double*>(base) + 4 * p;
    x = __double2float_rn(q[0]); y = __double2float_rn(q[1]); z = __double2float_rn(q[2]);
  }
}

// psi(x) in FP32, fixed order, each operation correctly rounded; NaN for a bad point.
__device__ __forceinline__ float4 ray_f32(float x, float y, float z) {
  const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z)));
  float4 r = make_float4(__fdiv_rn(x, n), __fdiv_rn(y, n), __fdiv_rn(z, n), 0.f);
  if (!(isfinite(r.x) && isfinite(r.y) && isfinite(r.z) && n > 0.f)) r = make_float4(NAN, NAN, NAN, 0.f);
  return r;
}

__device__ __forceinline__ float ray_dist(float4 a, float4 b) {
  const float d0 = __fsub_rn(a.x, b.x), d1 = __fsub_rn(a.y, b.y), d2 = __fsub_rn(a.z, b.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
}

__global__ void ray_image_kernel(const void* __restrict__ pts, int dtype, int64_t n, float4* __restrict__ rays) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float x, y, z;
    load_xyz_f32(pts, dtype, p, x, y, z);
    rays[p] = ray_f32(x, y, z);
  }
}

__global__ void match_kernel(const float4* __restrict__ rays, int H, int W, const void* __restrict__ query, int dtype,
                             int Q, const int32_t* __restrict__ init, int max_steps, float dmax,
                             int32_t* __restrict__ out, float* __restrict__ dist) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Q) return;
  float x, y, z;
  load_xyz_f32(query, dtype, t, x, y, z);
  const float4 q = ray_f32(x, y, z);
  const int P = H * W;
  int cur = init ? init[t] : t % P;
  cur = cur < 0 ? 0 : (cur >= P ? P - 1 : cur);
  float dcur = ray_dist(__ldg(rays + cur), q);
  if (isnan(dcur)) dcur = INFINITY;
  const bool okq = !isnan(q.x);
  if (okq) {
    for (int step = 0; step < max_steps; ++step) {
      const int cy = cur / W, cx = cur - cy * W;
      float best = dcur;
      int bidx = cur;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int dy = k < 3 ? -1 : (k < 5 ? 0 : 1);
        const int dx = k < 3 ? k - 1 : (k < 5 ? (k == 3 ? -1 : 1) : k - 6);
        const int ny = cy + dy, nx = cx + dx;
        if (ny < 0 || ny >= H || nx < 0 || nx >= W) continue;
        const int c = ny * W + nx;
        const float d = ray_dist(__ldg(rays + c), q);
        if (d < best) {  // NaN compares false
          best = d;
          bidx = c;
        }
      }
      if (bidx == cur) break;
      cur = bidx;
      dcur = best;
    }
  }
  out[t] = (okq && dcur <= dmax) ? cur : -1;
  if (dist) dist[t] = dcur;
}

// One pixel of the fusion; m = (s R row-major, t) of T_kf in the storage precision.
template <typename T, typename V4>
__device__ __forceinline__ void fuse_pixel(V4* __restrict__ canon, const V4* __restrict__ pred, int64_t p,
                                           const T (&m)[12]) {
  V4 a = canon[p];
  const V4 b = pred[p];
  const T y0 = m[0] * b.x + m[1] * b.y + m[2] * b.z + m[9];
  const T y1 = m[3] * b.x + m[4] * b.y + m[5] * b.z + m[10];
  const T y2 = m[6] * b.x + m[7] * b.y + m[8] * b.z + m[11];
  const T c = a.w + b.w;
  a.x = (a.w * a.x + b.w * y0) / c;
  a.y = (a.w * a.y + b.w * y1) / c;
  a.z = (a.w * a.z + b.w * y2) / c;
  a.w = c;
  canon[p] = a;
}

template <typename T>
struct FuseOne {
  T m[12];
};

template <typename T, typename V4>
__global__ void fuse_kernel(V4* __restrict__ canon, const V4* __restrict__ pred, int64_t n, FuseOne<T> f) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    fuse_pixel<T, V4>(canon, pred, p, f.m);
}

// Many keyframes per launch: blockIdx.y is the keyframe within the batch, blockIdx.x strides
// over its pixels; the transforms and offsets travel as kernel parameters.
constexpr int kFuseBatch = 128;
template <typename T>
struct FuseBatch {
  int64_t off[kFuseBatch + 1];
  T m[kFuseBatch][12];
};

template <typename T, typename V4>
__global__ void fuse_packed_kernel(V4* __restrict__ canon, const V4* __restrict__ pred, FuseBatch<T> b) {
  const int q = blockIdx.y;
  const int64_t p1 = b.off[q + 1];
  T m[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) m[k] = b.m[q][k];
  for (int64_t p = b.off[q] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1;
       p += (int64_t)gridDim.x * blockDim.x)
    fuse_pixel<T, V4>(canon, pred, p, m);
}

int grid_for_n(int64_t n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t g = (n + 255) / 256;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), (int64_t)sms * 16);
}

}  // namespace
}  // namespace como3r

using namespace como3r;

extern "C" int como3r_project_match(const como3r_match_desc* d, int32_t* match, float* dist, void* cuda_stream) {
  if (!d || !match) return report_error(COMO3R_ERR_INVALID_ARG, "desc and match must be non-NULL");
  if (d->H <= 0 || d->W <= 0 || (int64_t)d->H * d->W >= (int64_t(1) << 31) || d->num_queries < 0 ||
      d->max_steps < 0 || !(d->max_angle >= 0.0))
    return report_error(COMO3R_ERR_INVALID_ARG, "bad sizes, max_steps or max_angle");
  if (d->dtype < COMO3R_F16 || d->dtype > COMO3R_F64)
    return report_error(COMO3R_ERR_INVALID_ARG, "dtype must be COMO3R_F16, COMO3R_F32 or COMO3R_F64");
  if (d->num_queries == 0) return COMO3R_OK;
  if (!d->frame_points || !d->query_points)
    return report_error(COMO3R_ERR_INVALID_ARG, "frame_points and query_points must be non-NULL");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int64_t P = (int64_t)d->H * d->W;
  float4* rays = nullptr;
  cudaError_t e = cudaMallocAsync(&rays, sizeof(float4) * P, s);
  if (e) return report_cuda_error(e, "cudaMallocAsync");
  ray_image_kernel<<<grid_for_n(P), 256, 0, s>>>(d->frame_points, d->dtype, P, rays);
  const float dmax = (float)(2.0 - 2.0 * cos(d->max_angle));
  match_kernel<<<(d->num_queries + 127) / 128, 128, 0, s>>>(rays, d->H, d->W, d->query_points, d->dtype,
                                                             d->num_queries, d->init, d->max_steps, dmax, match, dist);
  e = cudaGetLastError();
  cudaFreeAsync(rays, s);
  if (e) return report_cuda_error(e, "project_match");
  return COMO3R_OK;
}

namespace {

// T_kf = (t, q, s) -> (s R row-major, t) in FP64 on the host, then rounded to the storage
// precision; false for a zero (or non-finite) quaternion.
template <typename T>
bool fuse_transform(const double* T_kf, T (&m)[12]) {
  const double qx = T_kf[3], qy = T_kf[4], qz = T_kf[5], qw = T_kf[6];
  const double nq = std::sqrt(qx * qx + qy * qy + qz * qz + qw * qw);
  if (!(nq > 0.0)) return false;
  const double x = qx / nq, y = qy / nq, z = qz / nq, w = qw / nq, sc = T_kf[7];
  const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                       2 * (x * y + z * w),     1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                       2 * (x * z - y * w),     2 * (y * z + x * w),     1 - 2 * (x * x + y * y)};
  for (int k = 0; k < 9; ++k) m[k] = (T)(sc * R[k]);
  for (int k = 0; k < 3; ++k) m[9 + k] = (T)T_kf[k];
  return true;
}

template <typename T, typename V4>
int fuse_packed_typed(void* canon, const void* pred, const int64_t* pix_off, const double* T_kf, int n,
                      cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int q0 = 0; q0 < n; q0 += kFuseBatch) {
    const int nb = std::min(kFuseBatch, n - q0);
    FuseBatch<T> b{};
    int64_t longest = 0;
    for (int q = 0; q <= nb; ++q) b.off[q] = pix_off[q0 + q];
    for (int q = 0; q < nb; ++q) {
      if (!fuse_transform<T>(T_kf + 8 * (int64_t)(q0 + q), b.m[q]))
        return report_error(COMO3R_ERR_INVALID_ARG, "a T_kf has a zero quaternion");
      longest = std::max(longest, b.off[q + 1] - b.off[q]);
    }
    if (longest == 0) continue;
    // about four resident waves of 256-thread blocks over the batch, at most one block per
    // 256 pixels of the longest keyframe
    const int64_t want = std::max<int64_t>(1, (int64_t)sms * 16 / nb);
    const int gx = (int)std::min<int64_t>(want, (longest + 255) / 256);
    fuse_packed_kernel<T, V4><<<dim3(gx, nb), 256, 0, s>>>(static_cast<V4*>(canon), static_cast<const V4*>(pred), b);
    const cudaError_t e = cudaGetLastError();
    if (e) return report_cuda_error(e, "fuse_packed");
  }
  return COMO3R_OK;
}

}  // namespace

extern "C" int como3r_fuse(void* canon, const void* pred, int64_t num_pixels, int32_t dtype, const double* T_kf,
                           void* cuda_stream) {
  if (num_pixels < 0) return report_error(COMO3R_ERR_INVALID_ARG, "num_pixels must be >= 0");
  if (num_pixels == 0) return COMO3R_OK;
  if (!canon || !pred || !T_kf) return report_error(COMO3R_ERR_INVALID_ARG, "canon, pred and T_kf must be non-NULL");
  if (dtype != COMO3R_F32 && dtype != COMO3R_F64)
    return report_error(COMO3R_ERR_UNSUPPORTED, "fusion keeps a running average: FP32 or FP64 storage");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int g = grid_for_n(num_pixels);
  if (dtype == COMO3R_F32) {
    FuseOne<float> f;
    if (!fuse_transform<float>(T_kf, f.m)) return report_error(COMO3R_ERR_INVALID_ARG, "T_kf has a zero quaternion");
    fuse_kernel<float, float4><<<g, 256, 0, s>>>(static_cast<float4*>(canon), static_cast<const float4*>(pred),
                                                  num_pixels, f);
  } else {
    FuseOne<double> f;
    if (!fuse_transform<double>(T_kf, f.m)) return report_error(COMO3R_ERR_INVALID_ARG, "T_kf has a zero quaternion");
    fuse_kernel<double, double4><<<g, 256, 0, s>>>(static_cast<double4*>(canon), static_cast<const double4*>(pred),
                                                    num_pixels, f);
  }
  const cudaError_t e = cudaGetLastError();
  if (e) return report_cuda_error(e, "fuse");
  return COMO3R_OK;
}

extern "C" int como3r_fuse_packed(void* canon, const void* pred, const int64_t* pix_off, const double* T_kf,
                                  int32_t n, int32_t dtype, void* cuda_stream) {
  if (n < 0 || !pix_off) return report_error(COMO3R_ERR_INVALID_ARG, "n must be >= 0 and pix_off non-NULL");
  if (pix_off[0] != 0) return report_error(COMO3R_ERR_INVALID_ARG, "pix_off[0] must be 0");
  for (int q = 0; q < n; ++q)
    if (pix_off[q + 1] < pix_off[q]) return report_error(COMO3R_ERR_INVALID_ARG, "pix_off must be non-decreasing");
  if (n == 0 || pix_off[n] == 0) return COMO3R_OK;
  if (!canon || !pred || !T_kf) return report_error(COMO3R_ERR_INVALID_ARG, "canon, pred and T_kf must be non-NULL");
  if (dtype != COMO3R_F32 && dtype != COMO3R_F64)
    return report_error(COMO3R_ERR_UNSUPPORTED, "fusion keeps a running average: FP32 or FP64 storage");
  // every transform is checked before the first launch, so a rejected call leaves canon untouched
  for (int q = 0; q < n; ++q) {
    double m[12];
    if (!fuse_transform<double>(T_kf + 8 * (int64_t)q, m))
      return report_error(COMO3R_ERR_INVALID_ARG, "a T_kf has a zero quaternion");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (dtype == COMO3R_F32) return fuse_packed_typed<float, float4>(canon, pred, pix_off, T_kf, n, s);
  return fuse_packed_typed<double, double4>(canon, pred, pix_off, T_kf, n, s);
}
