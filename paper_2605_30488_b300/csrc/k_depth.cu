// Terminal segment-level structure refinement (Sec. III-E): one log-scale eta_g per
// segment, X_p(eta_g) = |X_p,init| exp(eta_g) psi(X_p,init) (Eq. depth_parameter), the
// robust 3-D point residual sqrt(q) [T_ij X_j,n(eta) - X_i,m(eta)]_c / sigma_point over
// the graph's matches (Eq. depth_data), the boundary and prior terms (Eq. depth_total),
// and the Jacobi-style damped Newton update: per segment the diagonal of the data normal
// matrix (J_g = -X_i,m and J_h = s_ij R_ij X_j,n chain-ruled through eta, each scaled by
// sqrt(q) / sigma_point; the cross term J_g^T W J_h dropped), the diagonal of the
// boundary pairs, lambda_prior, the full gradient, and delta = -g / ((1 + lambda_lm) H)
// clipped to |delta| <= eta_max; segments of fixed keyframes stay.
//
// Setup (host, once): the pristine snapshot of the graph's pointmaps becomes per-pixel
// records (the snapshot point and its confidence: X(eta) = e^eta X_init, with e^eta per
// segment; the effective segment), the boundary pairs
// (g, h, Delta_gh) and their per-segment lists.  Per iteration:
//   depth_match_kernel (HBM-bound): persistent warps over the graph's work items, each
//     lane taking four consecutive pixels (two in FP64) with all their loads in flight;
//     a lane first adds its pixels' (g, H) contributions per side in two (segment, g, H)
//     slots (consecutive pixels mostly share a segment), then runs of lanes with the same
//     segment are reduced (segmented warp reduction: the streamed pixels of a warp are
//     contiguous, the gathered ones shifted, so runs are long) and the run's head adds
//     them with one FP64 atomic each -- one warp-level reduction per side per 128 pixels;
//   depth_update_kernel (one thread per segment, FP64): boundary and prior terms, the
//     damped clipped step into the other eta buffer (Jacobi: every step reads the same eta).
// MIXED does the per-match arithmetic in FP32 (hardware exp / reciprocal square root /
// reciprocal approximations), PLAIN_FP64 in FP64; accumulators are FP64.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "../../include/como3r.h"
#include "como3r_internal.h"
#include "plan.h"

namespace como3r {
namespace {

constexpr int kDepthThreads = 256;

template <typename R> struct Rec;
template <> struct Rec<float> { using T = float4; };
template <> struct Rec<double> { using T = double4; };

// Segmented sum over runs of equal keys in consecutive lanes: returns, in the first lane of
// every run, the run's total (other lanes: partial sums, unused).  In the kernel's
// arithmetic type (FP32 in the mixed form: at most 32 terms per run).
template <typename R>
__device__ __forceinline__ void run_sums(int key, R& a, R& b, int lane, bool& head) {
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned after = heads & ~((2u << lane) - 1u);  // heads above this lane
  const int end = after ? __ffs(after) - 2 : 31;        // last lane of this lane's run
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R oa = __shfl_down_sync(0xffffffffu, a, off);
    const R ob = __shfl_down_sync(0xffffffffu, b, off);
    if (lane + off <= end) {
      a += oa;
      b += ob;
    }
  }
}

// A run head's FP64 atomics (executed in L2); FP32 values are widened on the ALU, so the
// SM's FP64 pipe stays free.
__device__ __forceinline__ void seg_add(double* __restrict__ gsum, double* __restrict__ hsum, int k, float a,
                                        float b) {
  atomicAdd(gsum + k, widen_f32(a));
  atomicAdd(hsum + k, widen_f32(b));
}
__device__ __forceinline__ void seg_add(double* __restrict__ gsum, double* __restrict__ hsum, int k, double a,
                                        double b) {
  atomicAdd(gsum + k, a);
  atomicAdd(hsum + k, b);
}

// FP32: hardware approximations (relative error ~2^-22, far inside the mixed form's 1e-5);
// FP64: the exact functions.  (e^eta is computed once per segment by the update kernel.)
__device__ __forceinline__ float rsq_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// c^(1/4) of c >= 0 (0 -> 0)
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float qroot(float c) { return sqrt_approx(sqrt_approx(c)); }
__device__ __forceinline__ double qroot(double c) { return sqrt(sqrt(c)); }
__device__ __forceinline__ float huber_w(float r, float kappa) { return fminf(1.f, kappa * rcp_approx(fabsf(r))); }
__device__ __forceinline__ double huber_w(double r, double kappa) {
  const double a = fabs(r);
  return a <= kappa ? 1.0 : kappa / a;
}
template <typename R>
__device__ __forceinline__ R huber_rho(R r, R kappa) {
  const R a = fabs(r);
  return a <= kappa ? R(0.5) * r * r : kappa * a - R(0.5) * kappa * kappa;
}

// A lane's two (segment, g, H) accumulation slots of one side: a value goes to the slot
// holding its segment, else to a free slot, else straight to the atomics (a third
// segment among a lane's few consecutive pixels is rare).
template <typename R>
struct Slots {
  int ka = -1, kb = -1;
  R ga = R(0), ha = R(0), gb = R(0), hb = R(0);
  __device__ __forceinline__ void add(int k, R g, R h, double* gsum, double* hsum) {
    if (k < 0) return;
    if (k == ka || ka < 0) {
      ka = k;
      ga += g;
      ha += h;
    } else if (k == kb || kb < 0) {
      kb = k;
      gb += g;
      hb += h;
    } else {
      seg_add(gsum, hsum, k, g, h);
    }
  }
  // warp-level: runs of lanes with the same segment add once per run (the second slot
  // only when some lane uses it)
  __device__ __forceinline__ void flush(int lane, double* gsum, double* hsum) {
    bool head;
    run_sums(ka, ga, ha, lane, head);
    if (head && ka >= 0) seg_add(gsum, hsum, ka, ga, ha);
    if (__any_sync(0xffffffffu, kb >= 0)) {
      run_sums(kb, gb, hb, lane, head);
      if (head && kb >= 0) seg_add(gsum, hsum, kb, gb, hb);
    }
  }
};

// LIST: the items' precompacted valid-match lists of the residual kernel (entry
// (n << 10) | pixel offset in the item, in pixel order) replace the index rows, so every
// lane takes matches only (a lane's four entries are consecutive, so its streamed pixels
// are still mostly one segment) and the index rows are not read.
template <typename R, bool LIST>
__global__ void __launch_bounds__(kDepthThreads, 2) depth_match_kernel(
    const typename Rec<R>::T* __restrict__ rec, const int32_t* __restrict__ seg,
    const int32_t* __restrict__ midx, const Item* __restrict__ items, int num_items,
    const EdgeStatic* __restrict__ es, const double* __restrict__ T64, const float* __restrict__ T32,
    const R* __restrict__ scale, double kscale, double kappa_d, double* __restrict__ gsum,
    double* __restrict__ hsum, double* __restrict__ cost, const int32_t* __restrict__ counts,
    const uint32_t* __restrict__ compact) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * kDepthThreads + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kDepthThreads) >> 5;
  constexpr int kDepthUnroll = sizeof(R) == 4 ? 4 : 2;  // pixels per lane in flight (FP64 records are twice as wide)
  const R kappa = (R)kappa_d, ks = (R)kscale;
  double lane_cost = 0.0;
  for (int it = w0; it < num_items; it += nw) {
    const Item item = items[it];
    const EdgeStatic e = es[item.edge];
    R item_cost = R(0);  // this lane's Huber costs of the item (<= 64 terms)
    R T[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      if constexpr (sizeof(R) == 4) T[q] = T32[16 * item.edge + q];
      else T[q] = T64[12 * item.edge + q];
    }
    const int32_t* idx = midx + e.idx_off;
    // the item's entries: pixels (index rows) or valid matches (lists)
    const uint32_t* list = LIST ? compact + (int64_t)it * kCompactSlot : nullptr;
    const int q_begin = LIST ? 0 : item.begin, q_end = LIST ? counts[it] : item.end;
    // a lane's entries of one chunk: one 16-byte load when the four are in range and
    // aligned, else one by one (-1 past the end); mm = the streamed pixel (offset from the
    // keyframe's first pixel), nn = the gathered one
    auto load_idx = [&](int qb, int (&mm)[kDepthUnroll], int (&nn)[kDepthUnroll]) {
      if constexpr (LIST) {
        if (qb + 3 < q_end) {  // list slots start 16-byte aligned
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(list + qb));
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int u = 0; u < kDepthUnroll; ++u) {
            mm[u] = item.begin + (int)(w[u] & 1023u);
            nn[u] = (int)(w[u] >> 10);
          }
          return;
        }
#pragma unroll
        for (int u = 0; u < kDepthUnroll; ++u) {
          const uint32_t w = qb + u < q_end ? __ldg(list + qb + u) : 0u;
          mm[u] = item.begin + (int)(w & 1023u);
          nn[u] = qb + u < q_end ? (int)(w >> 10) : -1;
        }
      } else {
        if constexpr (kDepthUnroll == 4) {
          if (qb + 3 < q_end && (reinterpret_cast<uintptr_t>(idx + qb) & 15u) == 0) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(idx + qb));
            nn[0] = v.x; nn[1] = v.y; nn[2] = v.z; nn[3] = v.w;
#pragma unroll
            for (int u = 0; u < kDepthUnroll; ++u) mm[u] = qb + u;
            return;
          }
        }
#pragma unroll
        for (int u = 0; u < kDepthUnroll; ++u) {
          mm[u] = qb + u;
          nn[u] = qb + u < q_end ? __ldg(idx + qb + u) : -1;
        }
      }
    };
    // each lane takes kDepthUnroll consecutive entries of the item (streamed loads of a lane
    // are (nearly) contiguous; its pixels mostly share one segment, so they add up in the
    // lane); the next chunk's entries are in flight while this chunk's records are gathered
    int nxt_m[kDepthUnroll], nxt_n[kDepthUnroll];
    load_idx(q_begin + kDepthUnroll * lane, nxt_m, nxt_n);
    for (int q0 = q_begin; q0 < q_end; q0 += 32 * kDepthUnroll) {
      const int qb = q0 + kDepthUnroll * lane;
      int mm[kDepthUnroll], nn[kDepthUnroll];
#pragma unroll
      for (int u = 0; u < kDepthUnroll; ++u) {
        mm[u] = nxt_m[u];
        nn[u] = nxt_n[u];
      }
      if (q0 + 32 * kDepthUnroll < q_end) load_idx(qb + 32 * kDepthUnroll, nxt_m, nxt_n);
      typename Rec<R>::T ri[kDepthUnroll], rj[kDepthUnroll];
      int si[kDepthUnroll], sj[kDepthUnroll];
#pragma unroll
      for (int u = 0; u < kDepthUnroll; ++u) {
        si[u] = sj[u] = -1;
        if (nn[u] >= 0) {
          const int64_t pi = e.pix_i + mm[u], pj = e.pix_j + nn[u];
          ri[u] = rec[pi];
          rj[u] = rec[pj];
          si[u] = __ldg(seg + pi);
          sj[u] = __ldg(seg + pj);
        }
      }
      Slots<R> side_i, side_j;
#pragma unroll
      for (int u = 0; u < kDepthUnroll; ++u) {
        if (nn[u] < 0) continue;  // every valid match adds to the objective; sides with a segment to (g, H)
        // X(eta) = |X_init| e^eta psi(X_init) = e^eta X_init; e^eta per segment
        const R di = si[u] >= 0 ? __ldg(scale + si[u]) : R(1);
        const R dj = sj[u] >= 0 ? __ldg(scale + sj[u]) : R(1);
        const R xi0 = di * ri[u].x, xi1 = di * ri[u].y, xi2 = di * ri[u].z;
        const R xj0 = dj * rj[u].x, xj1 = dj * rj[u].y, xj2 = dj * rj[u].z;
        // s R X_j (the FP32 copy of the transform holds sR - I: X_j added back)
        R a0 = fma(T[0], xj0, fma(T[1], xj1, T[2] * xj2));
        R a1 = fma(T[3], xj0, fma(T[4], xj1, T[5] * xj2));
        R a2 = fma(T[6], xj0, fma(T[7], xj1, T[8] * xj2));
        if constexpr (sizeof(R) == 4) {
          a0 += xj0;
          a1 += xj1;
          a2 += xj2;
        }
        const R y0 = a0 + T[9], y1 = a1 + T[10], y2 = a2 + T[11];
        const R cc = ri[u].w * rj[u].w;
        const R nx2 = fma(xi0, xi0, fma(xi1, xi1, xi2 * xi2)), ny2 = fma(y0, y0, fma(y1, y1, y2 * y2));
        const bool ok = isfinite(nx2) && isfinite(ny2) && isfinite(cc) && nx2 > R(1e-24) && ny2 > R(1e-24) &&
                        cc >= R(0);
        if (!ok) continue;
        const R k = qroot(cc) * ks;
        const R r0 = k * (y0 - xi0), r1 = k * (y1 - xi1), r2 = k * (y2 - xi2);
        const R w0 = huber_w(r0, kappa), w1 = huber_w(r1, kappa), w2 = huber_w(r2, kappa);
        item_cost += huber_rho(r0, kappa) + huber_rho(r1, kappa) + huber_rho(r2, kappa);
        // J_g = -k X_i, J_h = k s R X_j
        const R g0 = -k * xi0, g1 = -k * xi1, g2 = -k * xi2;
        const R h0 = k * a0, h1 = k * a1, h2 = k * a2;
        side_i.add(si[u], w0 * r0 * g0 + w1 * r1 * g1 + w2 * r2 * g2, w0 * g0 * g0 + w1 * g1 * g1 + w2 * g2 * g2,
                   gsum, hsum);
        side_j.add(sj[u], w0 * r0 * h0 + w1 * r1 * h1 + w2 * r2 * h2, w0 * h0 * h0 + w1 * h1 * h1 + w2 * h2 * h2,
                   gsum, hsum);
      }
      side_i.flush(lane, gsum, hsum);
      side_j.flush(lane, gsum, hsum);
    }
    if constexpr (sizeof(R) == 4) lane_cost += widen_f32(item_cost);
    else lane_cost += item_cost;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lane_cost += __shfl_xor_sync(0xffffffffu, lane_cost, off);
  if (lane == 0 && lane_cost != 0.0) atomicAdd(cost, lane_cost);
}

// One thread per segment: boundary and prior terms, the damped clipped Jacobi step (eta
// read from eta_in, written to eta_out), the objective's boundary / prior parts, and the
// accumulators reset for the next iteration.
__global__ void depth_update_kernel(int M, const uint8_t* __restrict__ movable, const uint8_t* __restrict__ active,
                                    const int32_t* __restrict__ poff, const int32_t* __restrict__ pother,
                                    const double* __restrict__ pdelta, const double* __restrict__ eta_in,
                                    double* __restrict__ eta_out, float* __restrict__ scale32_out,
                                    double* __restrict__ scale64_out,
                                    double* __restrict__ gsum,
                                    double* __restrict__ hsum, double lambda_smooth, double lambda_prior,
                                    double lambda_lm, double eta_max, int apply, double* __restrict__ cost) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const double es = eta_in[s];
  double g = gsum[s], h = hsum[s], e = 0.0;
  if (active[s]) {
    for (int q = poff[s]; q < poff[s + 1]; ++q) {
      // pdelta is Delta oriented from this segment to the other one
      const double res = es - eta_in[pother[q]] + pdelta[q];
      g += lambda_smooth * res;
      h += lambda_smooth;
      if (s < pother[q]) e += 0.5 * lambda_smooth * res * res;  // each pair once
    }
    g += lambda_prior * es;
    h += lambda_prior;
    e += 0.5 * lambda_prior * es * es;
  }
  double step = 0.0;
  if (apply && movable[s] && h > 0.0) step = fmin(eta_max, fmax(-eta_max, -g / ((1.0 + lambda_lm) * h)));
  eta_out[s] = es + step;
  if (scale32_out) scale32_out[s] = expf((float)(es + step));
  if (scale64_out) scale64_out[s] = exp(es + step);
  gsum[s] = 0.0;
  hsum[s] = 0.0;
  if (e != 0.0) atomicAdd(cost, e);
}

__global__ void eta_to_scale_kernel(const double* __restrict__ a, float* __restrict__ b32, double* __restrict__ b64,
                                    int M) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  if (b32) b32[s] = expf((float)a[s]);
  if (b64) b64[s] = exp(a[s]);
}

// Refined pointmap in the graph's storage type: X = exp(logd + eta) psi for pixels of a
// segment, the snapshot point otherwise; the confidence is copied.
template <typename R, int DT>
__global__ void depth_points_kernel(const typename Rec<R>::T* __restrict__ rec, const int32_t* __restrict__ seg,
                                    const double* __restrict__ eta, const void* __restrict__ src, int64_t n,
                                    void* __restrict__ dst) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int s = seg[p];
    if constexpr (DT == 0) {
      uint2 v = reinterpret_cast<const uint2*>(src)[p];
      if (s >= 0) {
        const typename Rec<R>::T r = rec[p];
        const double d = exp(eta[s]);
        const __half2 a = __floats2half2_rn((float)(d * r.x), (float)(d * r.y));
        const float cz = __half2float(reinterpret_cast<const __half2*>(&v.y)->y);
        const __half2 b = __floats2half2_rn((float)(d * r.z), cz);
        v.x = *reinterpret_cast<const unsigned*>(&a);
        v.y = *reinterpret_cast<const unsigned*>(&b);
      }
      reinterpret_cast<uint2*>(dst)[p] = v;
    } else if constexpr (DT == 1) {
      float4 v = reinterpret_cast<const float4*>(src)[p];
      if (s >= 0) {
        const typename Rec<R>::T r = rec[p];
        const double d = exp(eta[s]);
        v.x = (float)(d * r.x); v.y = (float)(d * r.y); v.z = (float)(d * r.z);
      }
      reinterpret_cast<float4*>(dst)[p] = v;
    } else {
      const double2* q = reinterpret_cast<const double2*>(src) + 2 * p;
      double2 a = q[0], b = q[1];
      if (s >= 0) {
        const typename Rec<R>::T r = rec[p];
        const double d = exp(eta[s]);
        a.x = d * r.x; a.y = d * r.y; b.x = d * r.z;
      }
      double2* o = reinterpret_cast<double2*>(dst) + 2 * p;
      o[0] = a;
      o[1] = b;
    }
  }
}

double host_half(uint16_t h) {
  const uint32_t sgn = (h >> 15) & 1u, ex = (h >> 10) & 31u, man = h & 1023u;
  double v;
  if (ex == 0) v = std::ldexp((double)man, -24);
  else if (ex == 31) v = man ? NAN : INFINITY;
  else v = std::ldexp((double)(man | 1024u), (int)ex - 25);
  return sgn ? -v : v;
}

}  // namespace

struct DepthState {
  int mode = COMO3R_MIXED, dtype = COMO3R_F32;
  int64_t npix = 0;
  int M = 0, n_active = 0, n_pairs = 0;
  void* rec = nullptr;        // float4 / double4 [npix]: snapshot point (x, y, z), confidence
  int32_t* seg = nullptr;     // [npix] effective global segment or -1
  uint8_t* movable = nullptr; // [M]
  uint8_t* active = nullptr;  // [M]
  int32_t* poff = nullptr;    // [M + 1] pair lists per segment
  int32_t* pother = nullptr;  // [2 n_pairs]
  double* pdelta = nullptr;   // [2 n_pairs] Delta oriented from the list's segment
  double *eta[2] = {nullptr, nullptr}, *gsum = nullptr, *hsum = nullptr, *cost = nullptr;
  float* sc32[2] = {nullptr, nullptr};   // e^eta, FP32, read by the mixed-form match pass
  double* sc64[2] = {nullptr, nullptr};  // e^eta, FP64, read by the plain-form match pass
  double sigma_point = 0.05, lambda_smooth = 1.0, lambda_prior = 1.0, lambda_lm = 0.05, eta_max = 0.5;
  std::vector<void*> allocs;
};

void depth_free(DepthState* st) {
  if (!st) return;
  for (void* p : st->allocs) cudaFree(p);
  delete st;
}

namespace {
template <typename T>
cudaError_t dmalloc(DepthState* st, T** p, size_t n) {
  const cudaError_t e = cudaMalloc(p, sizeof(T) * std::max<size_t>(n, 1));
  if (e == cudaSuccess) st->allocs.push_back(*p);
  return e;
}
}  // namespace

int depth_setup(const HostPlan& p, const void* points, int dtype, int mode, const int32_t* labels_any,
                const como3r_depth_desc* d, cudaStream_t s, DepthState** out, int64_t* num_segments) {
  const int64_t npix = p.total_px;
  // host copies of the points and labels (one-off setup)
  const size_t bpp = dtype == COMO3R_F16 ? 8 : dtype == COMO3R_F32 ? 16 : 32;
  std::vector<unsigned char> raw((size_t)npix * bpp);
  std::vector<int32_t> lab((size_t)npix);
  cudaError_t e = cudaMemcpyAsync(raw.data(), points, raw.size(), cudaMemcpyDefault, s);
  if (!e) e = cudaMemcpyAsync(lab.data(), labels_any, sizeof(int32_t) * lab.size(), cudaMemcpyDefault, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return report_cuda_error(e, "depth setup readback");
  auto px = [&](int64_t q, double* v) {
    if (dtype == COMO3R_F16) {
      const uint16_t* h = reinterpret_cast<const uint16_t*>(raw.data()) + 4 * q;
      for (int c = 0; c < 4; ++c) v[c] = host_half(h[c]);
    } else if (dtype == COMO3R_F32) {
      const float* f = reinterpret_cast<const float*>(raw.data()) + 4 * q;
      for (int c = 0; c < 4; ++c) v[c] = f[c];
    } else {
      const double* f = reinterpret_cast<const double*>(raw.data()) + 4 * q;
      for (int c = 0; c < 4; ++c) v[c] = f[c];
    }
  };
  std::vector<double> logd((size_t)npix), cf((size_t)npix), xyz((size_t)npix * 3);
  std::vector<uint8_t> fin((size_t)npix);
  for (int64_t q = 0; q < npix; ++q) {
    double v[4];
    px(q, v);
    for (int c = 0; c < 3; ++c) xyz[3 * q + c] = v[c];
    const double dd = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const bool ok = std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]) && std::isfinite(v[3]) &&
                    dd > 1e-12;
    fin[q] = ok;
    logd[q] = ok ? std::log(dd) : NAN;
    cf[q] = v[3];
  }
  std::vector<int32_t> eff((size_t)npix, -1);
  std::vector<uint8_t> movable, active;
  std::unordered_map<uint64_t, std::pair<double, int64_t>> pairs;
  int M = 0;
  for (int k = 0; k < p.N; ++k) {
    const int64_t a0 = p.pix_off[k], n = p.pix_off[k + 1] - a0;
    int Mk = 0;
    for (int64_t q = 0; q < n; ++q) Mk = std::max(Mk, lab[a0 + q] + 1);
    std::vector<int64_t> cnt(Mk, 0);
    for (int64_t q = 0; q < n; ++q) {
      const int L = lab[a0 + q];
      if (L >= 0 && fin[a0 + q] && cf[a0 + q] >= d->c_min) ++cnt[L];
    }
    for (int64_t q = 0; q < n; ++q) {
      const int L = lab[a0 + q];
      if (L >= 0 && fin[a0 + q] && cf[a0 + q] >= d->c_min && cnt[L] >= d->min_pixels) eff[a0 + q] = M + L;
    }
    for (int L = 0; L < Mk; ++L) {
      active.push_back(cnt[L] >= d->min_pixels);
      movable.push_back(cnt[L] >= d->min_pixels && !p.frozen[k]);
    }
    // 4-adjacent boundary pairs of the keyframe
    int g = 0;
    while (g + 1 < (int)p.kf_offset.size() && p.kf_offset[g + 1] <= k) ++g;
    const int W = p.width[g];
    for (int64_t q = 0; q < n; ++q) {
      const int32_t a = eff[a0 + q];
      if (a < 0) continue;
      const int64_t nb[2] = {(q % W) + 1 < W ? q + 1 : -1, q + W < n ? q + W : -1};
      for (int t = 0; t < 2; ++t) {
        if (nb[t] < 0) continue;
        const int32_t b = eff[a0 + nb[t]];
        if (b < 0 || b == a) continue;
        const int32_t lo = std::min(a, b), hi = std::max(a, b);
        const double diff = a < b ? logd[a0 + q] - logd[a0 + nb[t]] : logd[a0 + nb[t]] - logd[a0 + q];
        auto& acc = pairs[((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi];
        acc.first += diff;
        acc.second += 1;
      }
    }
    M += Mk;
  }
  // per-segment pair lists (each pair in both lists, Delta oriented from the list's segment)
  std::vector<std::vector<std::pair<int32_t, double>>> lists(M);
  std::vector<std::pair<uint64_t, std::pair<double, int64_t>>> sorted(pairs.begin(), pairs.end());
  std::sort(sorted.begin(), sorted.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  for (const auto& kv : sorted) {
    const int32_t lo = (int32_t)(kv.first >> 32), hi = (int32_t)(kv.first & 0xffffffffu);
    const double delta = kv.second.first / (double)kv.second.second;  // logd(lo side) - logd(hi side)
    lists[lo].push_back({hi, delta});
    lists[hi].push_back({lo, -delta});
  }
  std::vector<int32_t> poff(M + 1, 0), pother;
  std::vector<double> pdelta;
  for (int sgi = 0; sgi < M; ++sgi) {
    poff[sgi + 1] = poff[sgi] + (int32_t)lists[sgi].size();
    for (const auto& x : lists[sgi]) {
      pother.push_back(x.first);
      pdelta.push_back(x.second);
    }
  }
  DepthState* st = new DepthState();
  st->mode = mode;
  st->dtype = dtype;
  st->npix = npix;
  st->M = M;
  st->n_pairs = (int)sorted.size();
  st->sigma_point = d->sigma_point;
  st->lambda_smooth = d->lambda_smooth;
  st->lambda_prior = d->lambda_prior;
  st->lambda_lm = d->lambda_lm;
  st->eta_max = d->eta_max;
  for (uint8_t a : active) st->n_active += a;
  const bool f32 = mode == COMO3R_MIXED;
  // per pixel the snapshot point and its confidence (a degenerate point becomes NaN, so
  // every match touching it fails the per-match test)
  std::vector<unsigned char> recb((size_t)npix * (f32 ? 16 : 32));
  for (int64_t q = 0; q < npix; ++q) {
    const double r[4] = {fin[q] ? xyz[3 * q] : NAN, fin[q] ? xyz[3 * q + 1] : NAN, fin[q] ? xyz[3 * q + 2] : NAN,
                         cf[q]};
    if (f32) {
      float* o = reinterpret_cast<float*>(recb.data()) + 4 * q;
      for (int c = 0; c < 4; ++c) o[c] = (float)r[c];
    } else {
      double* o = reinterpret_cast<double*>(recb.data()) + 4 * q;
      for (int c = 0; c < 4; ++c) o[c] = r[c];
    }
  }
  unsigned char* rec_d = nullptr;
  if ((e = dmalloc(st, &rec_d, recb.size())) ||
      (e = dmalloc(st, &st->seg, (size_t)npix)) || (e = dmalloc(st, &st->movable, (size_t)M)) ||
      (e = dmalloc(st, &st->active, (size_t)M)) || (e = dmalloc(st, &st->poff, (size_t)M + 1)) ||
      (e = dmalloc(st, &st->pother, pother.size())) || (e = dmalloc(st, &st->pdelta, pdelta.size())) ||
      (e = dmalloc(st, &st->eta[0], (size_t)M)) || (e = dmalloc(st, &st->eta[1], (size_t)M)) ||
      (e = dmalloc(st, &st->sc32[0], (size_t)M)) || (e = dmalloc(st, &st->sc32[1], (size_t)M)) ||
      (e = dmalloc(st, &st->sc64[0], (size_t)M)) || (e = dmalloc(st, &st->sc64[1], (size_t)M)) ||
      (e = dmalloc(st, &st->gsum, (size_t)M)) || (e = dmalloc(st, &st->hsum, (size_t)M)) ||
      (e = dmalloc(st, &st->cost, 1))) {
    depth_free(st);
    return report_cuda_error(e, "depth setup allocation");
  }
  st->rec = rec_d;
  e = cudaMemcpyAsync(rec_d, recb.data(), recb.size(), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(st->seg, eff.data(), sizeof(int32_t) * npix, cudaMemcpyHostToDevice, s);
  if (!e && M) e = cudaMemcpyAsync(st->movable, movable.data(), M, cudaMemcpyHostToDevice, s);
  if (!e && M) e = cudaMemcpyAsync(st->active, active.data(), M, cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(st->poff, poff.data(), sizeof(int32_t) * (M + 1), cudaMemcpyHostToDevice, s);
  if (!e && !pother.empty())
    e = cudaMemcpyAsync(st->pother, pother.data(), sizeof(int32_t) * pother.size(), cudaMemcpyHostToDevice, s);
  if (!e && !pdelta.empty())
    e = cudaMemcpyAsync(st->pdelta, pdelta.data(), sizeof(double) * pdelta.size(), cudaMemcpyHostToDevice, s);
  if (!e && M) e = cudaMemsetAsync(st->gsum, 0, sizeof(double) * M, s);
  if (!e && M) e = cudaMemsetAsync(st->hsum, 0, sizeof(double) * M, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) {
    depth_free(st);
    return report_cuda_error(e, "depth setup upload");
  }
  *out = st;
  if (num_segments) *num_segments = M;
  return COMO3R_OK;
}

int depth_run(DepthState* st, const HostPlan& p, const Item* items, int num_items, const EdgeStatic* es,
              const int32_t* midx, const int32_t* counts, const uint32_t* compact, const double* T64,
              const float* T32, double kappa, int sms, double* eta_io, int iters, double* cost_trace,
              void* points_out, const void* points_src, float* match_ms, cudaStream_t s) {
  const int M = st->M;
  cudaError_t e = cudaSuccess;
  if (M) e = cudaMemcpyAsync(st->eta[0], eta_io, sizeof(double) * M, cudaMemcpyDefault, s);
  if (!e && M) {
    const bool f32 = st->mode == COMO3R_MIXED;
    eta_to_scale_kernel<<<(M + 255) / 256, 256, 0, s>>>(st->eta[0], f32 ? st->sc32[0] : nullptr,
                                                        f32 ? nullptr : st->sc64[0], M);
    e = cudaGetLastError();
  }
  const int grid = std::max(1, std::min(sms * 2, (num_items + 7) / 8));
  const double kscale = 1.0 / st->sigma_point;
  std::vector<double> trace((size_t)iters + 1, 0.0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms_tot = 0.f;
  if (match_ms && !e) e = cudaEventCreate(&e0);
  if (match_ms && !e) e = cudaEventCreate(&e1);
  int cur = 0;
  for (int k = 0; k <= iters && !e; ++k) {
    e = cudaMemsetAsync(st->cost, 0, sizeof(double), s);
    if (!e && match_ms) e = cudaEventRecord(e0, s);
    if (!e) {
      const bool list = counts && compact;
#define COMO3R_DEPTH(R, V, SC, LIST)                                                                          \
  depth_match_kernel<R, LIST><<<grid, kDepthThreads, 0, s>>>(static_cast<const V*>(st->rec), st->seg, midx,   \
                                                              items, num_items, es, T64, T32, SC, kscale, kappa, \
                                                              st->gsum, st->hsum, st->cost, counts, compact)
      if (st->mode == COMO3R_MIXED) {
        if (list) COMO3R_DEPTH(float, float4, st->sc32[cur], true);
        else COMO3R_DEPTH(float, float4, st->sc32[cur], false);
      } else {
        if (list) COMO3R_DEPTH(double, double4, st->sc64[cur], true);
        else COMO3R_DEPTH(double, double4, st->sc64[cur], false);
      }
#undef COMO3R_DEPTH
      e = cudaGetLastError();
    }
    if (!e && match_ms) e = cudaEventRecord(e1, s);
    // the last pass only evaluates the objective at the final eta
    if (!e && M)
      depth_update_kernel<<<(M + 127) / 128, 128, 0, s>>>(M, st->movable, st->active, st->poff, st->pother,
                                                           st->pdelta, st->eta[cur], st->eta[cur ^ 1],
                                                           st->mode == COMO3R_MIXED ? st->sc32[cur ^ 1] : nullptr,
                                                           st->mode == COMO3R_MIXED ? nullptr : st->sc64[cur ^ 1],
                                                           st->gsum,
                                                           st->hsum, st->lambda_smooth, st->lambda_prior,
                                                           st->lambda_lm, st->eta_max, k < iters ? 1 : 0, st->cost);
    if (!e) e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(&trace[k], st->cost, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!e && match_ms) {
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
      ms_tot += ms;
    }
    if (k < iters) cur ^= 1;
  }
  if (!e && M) e = cudaMemcpyAsync(eta_io, st->eta[cur], sizeof(double) * M, cudaMemcpyDefault, s);
  if (!e && points_out) {
    const int pg = (int)std::min<int64_t>((st->npix + 255) / 256, (int64_t)sms * 16);
    if (st->mode == COMO3R_MIXED) {
      const float4* r = static_cast<const float4*>(st->rec);
      if (st->dtype == COMO3R_F16) depth_points_kernel<float, 0><<<pg, 256, 0, s>>>(r, st->seg, st->eta[cur], points_src, st->npix, points_out);
      else if (st->dtype == COMO3R_F32) depth_points_kernel<float, 1><<<pg, 256, 0, s>>>(r, st->seg, st->eta[cur], points_src, st->npix, points_out);
      else depth_points_kernel<float, 2><<<pg, 256, 0, s>>>(r, st->seg, st->eta[cur], points_src, st->npix, points_out);
    } else {
      const double4* r = static_cast<const double4*>(st->rec);
      if (st->dtype == COMO3R_F16) depth_points_kernel<double, 0><<<pg, 256, 0, s>>>(r, st->seg, st->eta[cur], points_src, st->npix, points_out);
      else if (st->dtype == COMO3R_F32) depth_points_kernel<double, 1><<<pg, 256, 0, s>>>(r, st->seg, st->eta[cur], points_src, st->npix, points_out);
      else depth_points_kernel<double, 2><<<pg, 256, 0, s>>>(r, st->seg, st->eta[cur], points_src, st->npix, points_out);
    }
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e) return report_cuda_error(e, "depth refine");
  if (cost_trace) std::memcpy(cost_trace, trace.data(), sizeof(double) * trace.size());
  if (match_ms) *match_ms = ms_tot / (float)(iters + 1);
  return COMO3R_OK;
}

}  // namespace como3r
