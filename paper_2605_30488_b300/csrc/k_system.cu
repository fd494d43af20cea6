// FP64 kernels around K1: edge preparation (T_ij, Ad), per-edge reduction of the K1
// partials with the Ad sandwich (Sec. III-D: DT_ij/DT_i = -Ad_{T_i^{-1}},
// DT_ij/DT_j = +Ad_{T_i^{-1}}), block-sparse assembly in a fixed order, dense export,
// Sim(3) retraction, and the create-time check of the match indices.
#include <cstdint>

#include "como3r_internal.h"
#include "sim3.cuh"

namespace como3r {
namespace {

// ---- K0: per edge T_ij (FP64 and its FP32 rounding) and Ad_{T_i^{-1}}
__global__ void edge_prep_kernel(const double* __restrict__ poses, const EdgeStatic* __restrict__ es, int E,
                                 double* __restrict__ T64, float* __restrict__ T32, double* __restrict__ Ad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  Sim3d Ti, Tj;
  load_pose(poses + 8 * es[e].i, Ti);
  load_pose(poses + 8 * es[e].j, Tj);
  double sR[9], t[3];
  relative_pose(Ti, Tj, sR, t);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    T64[12 * e + k] = sR[k];
    T32[16 * e + k] = (float)sR[k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T64[12 * e + 9 + k] = t[k];
    T32[16 * e + 9 + k] = (float)t[k];
  }
#pragma unroll
  for (int k = 12; k < 16; ++k) T32[16 * e + k] = 0.f;
  double A[49];
  adjoint_of_inverse(Ti, A);
#pragma unroll
  for (int k = 0; k < 49; ++k) Ad[49 * e + k] = A[k];
}

// Index of entry (r, c) of the 7x7 H_rel among the 25 unique entries kept by K1, or -1
// for the structurally zero (omega, zeta) entries.
__device__ __forceinline__ int hrel_index(int r, int c) {
  if (r > c) { const int t = r; r = c; c = t; }
  if (c < 3) return r * 3 - r * (r - 1) / 2 + (c - r);                 // (v, v)
  if (r < 3 && c < 6) return 6 + 3 * r + (c - 3);                       // (v, omega)
  if (r < 3 && c == 6) return 21 + r;                                   // (v, zeta)
  if (r >= 3 && c < 6) {                                                // (omega, omega)
    const int a = r - 3, b = c - 3;
    return 15 + a * 3 - a * (a - 1) / 2 + (b - a);
  }
  if (r == 6 && c == 6) return 24;                                      // (zeta, zeta)
  return -1;                                                            // (omega, zeta)
}

// ---- K2: per edge, fixed-order FP64 sum of its item records, then
// M_e = Ad^T H_rel Ad (= H_jj = H_ii = -H_ij) and b_e = Ad^T g_rel (= g_j = -g_i).
// Eight groups of 36 threads each sum every eighth record; the group sums are then added
// in group order, so the result is independent of scheduling.
constexpr int kReduceGroups = 8;
constexpr int kReduceThreads = kReduceGroups * kPartial;  // 288

__device__ __forceinline__ double slot_value(const float2* rec, int k) {
  const float2 v = rec[k];
  return (double)v.x + (double)v.y;
}
__device__ __forceinline__ double slot_value(const double* rec, int k) { return rec[k]; }

template <typename Slot>
__global__ void __launch_bounds__(kReduceThreads) edge_reduce_kernel(
    const Slot* __restrict__ partials, const int32_t* __restrict__ item_off, const double* __restrict__ Ad_all,
    double* __restrict__ edge_M, double* __restrict__ edge_b, double* __restrict__ edge_cost,
    double* __restrict__ edge_skip, double* __restrict__ edge_rec, const long long* __restrict__ edge_valid) {
  const int e = blockIdx.x, t = threadIdx.x;
  __shared__ double red[kReduceGroups][kPartial];
  __shared__ double acc[kPartial];
  __shared__ double H[49], Ad[49], T1[49], g[7];
  const int i0 = item_off[e], i1 = item_off[e + 1];
  {
    const int grp = t / kPartial, a = t % kPartial;
    double s = 0.0;
    for (int it = i0 + grp; it < i1; it += kReduceGroups) s += slot_value(partials + (int64_t)it * kPartial, a);
    red[grp][a] = s;
  }
  if (t < 49) Ad[t] = Ad_all[49 * e + t];
  __syncthreads();
  if (t < kPartial) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kReduceGroups; ++q) s += red[q][t];
    acc[t] = s;
  }
  __syncthreads();
  if (t < 49) {
    const int k = hrel_index(t / 7, t % 7);
    H[t] = k >= 0 ? acc[k] : 0.0;
  }
  if (t < 7) g[t] = acc[kHUnique + t];
  __syncthreads();
  if (t < 49) {
    const int r = t / 7, c = t % 7;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) s += H[7 * r + k] * Ad[7 * k + c];
    T1[t] = s;
  }
  __syncthreads();
  if (t < 49) {
    const int r = t / 7, c = t % 7;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) s += Ad[7 * k + r] * T1[7 * k + c];
    edge_M[49 * e + t] = s;
    if (edge_rec) edge_rec[(int64_t)kEdgeRec * e + t] = H[t];
  } else if (t < 56) {
    const int r = t - 49;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) s += Ad[7 * k + r] * g[k];
    edge_b[7 * e + r] = s;
    if (edge_rec) edge_rec[(int64_t)kEdgeRec * e + t] = g[r];
  } else if (t == 56) {
    edge_cost[e] = acc[32];
    edge_skip[e] = acc[33];
    if (edge_rec) {
      double* rec = edge_rec + (int64_t)kEdgeRec * e;
      rec[56] = acc[32];
      rec[57] = (double)edge_valid[e];
      rec[58] = acc[33];
#pragma unroll
      for (int k = 59; k < kEdgeRec; ++k) rec[k] = 0.0;
    }
  }
}

// ---- assembly: slots of the factor pattern, per-keyframe gradients, per-graph cost.
// Contributions are encoded edge * 2 + negate and summed in list (edge) order.
__global__ void __launch_bounds__(64) assemble_kernel(int num_slots, const int32_t* __restrict__ slot_contrib_off,
                                                      const int32_t* __restrict__ slot_contrib,
                                                      const double* __restrict__ edge_M, double* __restrict__ A, int N,
                                                      const int32_t* __restrict__ kf_contrib_off,
                                                      const int32_t* __restrict__ kf_contrib,
                                                      const double* __restrict__ edge_b, double* __restrict__ gvec,
                                                      int G, const int32_t* __restrict__ edge_offset,
                                                      const double* __restrict__ edge_cost,
                                                      const double* __restrict__ edge_skip, GraphInfoDev* ginfo,
                                                      double* cost_hist, const int* iter_counter, int* warn) {
  const int b = blockIdx.x, t = threadIdx.x;
  if (b < num_slots) {
    if (t >= 49) return;
    double s = 0.0;
    for (int q = slot_contrib_off[b]; q < slot_contrib_off[b + 1]; ++q) {
      const int c = slot_contrib[q];
      const double v = edge_M[49 * (c >> 1) + t];
      s += (c & 1) ? -v : v;
    }
    A[49 * (int64_t)b + t] = s;
  } else if (b < num_slots + N) {
    const int k = b - num_slots;
    if (t >= 7) return;
    double s = 0.0;
    for (int q = kf_contrib_off[k]; q < kf_contrib_off[k + 1]; ++q) {
      const int c = kf_contrib[q];
      const double v = edge_b[7 * (c >> 1) + t];
      s += (c & 1) ? -v : v;
    }
    gvec[7 * k + t] = s;
  } else {
    const int it = iter_counter ? *iter_counter : 0;
    for (int g = t; g < G; g += blockDim.x) {
      double c = 0.0, sk = 0.0;
      for (int e = edge_offset[g]; e < edge_offset[g + 1]; ++e) {
        c += edge_cost[e];
        sk += edge_skip[e];
      }
      ginfo[g].cost = c;
      ginfo[g].skipped = (long long)sk;
      if (cost_hist) cost_hist[(int64_t)it * G + g] = c;
      if (sk > 0.0) atomicOr(warn, 2);
    }
  }
}

__global__ void export_dense_kernel(int num_slots, const int32_t* __restrict__ slot_kf_r,
                                    const int32_t* __restrict__ slot_kf_c, const double* __restrict__ A, int N,
                                    const double* __restrict__ gvec, double* __restrict__ H_out,
                                    double* __restrict__ g_out) {
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t n = 7 * (int64_t)N;
  if (b < num_slots) {
    if (t >= 49 || !H_out) return;
    const int r = t / 7, c = t % 7;
    const int64_t kr = slot_kf_r[b], kc = slot_kf_c[b];
    const double v = A[49 * (int64_t)b + t];
    H_out[(7 * kr + r) * n + 7 * kc + c] = v;
    if (kr != kc) H_out[(7 * kc + c) * n + 7 * kr + r] = v;
  } else if (g_out) {
    for (int64_t x = t; x < n; x += blockDim.x) g_out[x] = gvec[x];
  }
}

__global__ void retract_kernel(const double* __restrict__ tau, double* __restrict__ poses,
                               const uint8_t* __restrict__ frozen, int N, int* iter_counter) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0 && iter_counter) *iter_counter += 1;
  if (k >= N) return;
  if (frozen && frozen[k]) return;
  const double* t = tau + 7 * k;
  // a zero update leaves the pose bitwise unchanged (no renormalisation)
  if (t[0] == 0.0 && t[1] == 0.0 && t[2] == 0.0 && t[3] == 0.0 && t[4] == 0.0 && t[5] == 0.0 && t[6] == 0.0) return;
  double p[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) p[q] = poses[8 * k + q];
  retract_left(tau + 7 * k, p);
#pragma unroll
  for (int q = 0; q < 8; ++q) poses[8 * k + q] = p[q];
}

// Counts entries outside [-1, P_j) (any edge) and valid entries per edge.
__global__ void check_matches_kernel(const int32_t* __restrict__ midx, const EdgeStatic* __restrict__ es,
                                     unsigned long long* bad, long long* edge_valid) {
  const int e = blockIdx.x;
  const EdgeStatic s = es[e];
  const int32_t* idx = midx + s.idx_off;
  long long valid = 0;
  unsigned long long nbad = 0;
  for (int m = threadIdx.x; m < s.npix_i; m += blockDim.x) {
    const int32_t n = idx[m];
    if (n < -1 || n >= s.npix_j) ++nbad;
    else if (n >= 0) ++valid;
  }
  for (int off = 16; off > 0; off >>= 1) {
    valid += __shfl_xor_sync(0xffffffffu, valid, off);
    nbad += __shfl_xor_sync(0xffffffffu, nbad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (valid) atomicAdd((unsigned long long*)&edge_valid[e], (unsigned long long)valid);
    if (nbad) atomicAdd(bad, nbad);
  }
}

}  // namespace

cudaError_t launch_edge_prep(const double* poses, const EdgeStatic* es, int E, double* T64, float* T32,
                             double* Ad, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  edge_prep_kernel<<<(E + 63) / 64, 64, 0, s>>>(poses, es, E, T64, T32, Ad);
  return cudaGetLastError();
}

cudaError_t launch_edge_reduce(int mode, const void* partials, const int32_t* item_off, int E, const double* Ad,
                               double* edge_M, double* edge_b, double* edge_cost, double* edge_skip,
                               double* edge_rec, const long long* edge_valid, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  if (mode == 1)
    edge_reduce_kernel<float2><<<E, kReduceThreads, 0, s>>>(static_cast<const float2*>(partials), item_off, Ad,
                                                            edge_M, edge_b, edge_cost, edge_skip, edge_rec,
                                                            edge_valid);
  else
    edge_reduce_kernel<double><<<E, kReduceThreads, 0, s>>>(static_cast<const double*>(partials), item_off, Ad,
                                                            edge_M, edge_b, edge_cost, edge_skip, edge_rec,
                                                            edge_valid);
  return cudaGetLastError();
}

cudaError_t launch_assemble(int num_slots, const int32_t* slot_contrib_off, const int32_t* slot_contrib,
                            const double* edge_M, double* A, int N, const int32_t* kf_contrib_off,
                            const int32_t* kf_contrib, const double* edge_b, double* gvec, int G,
                            const int32_t* edge_offset, const double* edge_cost, const double* edge_skip,
                            GraphInfoDev* ginfo, double* cost_hist, const int* iter_counter, int* warn,
                            cudaStream_t s) {
  assemble_kernel<<<num_slots + N + 1, 64, 0, s>>>(num_slots, slot_contrib_off, slot_contrib, edge_M, A, N,
                                                   kf_contrib_off, kf_contrib, edge_b, gvec, G, edge_offset,
                                                   edge_cost, edge_skip, ginfo, cost_hist, iter_counter, warn);
  return cudaGetLastError();
}

cudaError_t launch_export_dense(int num_slots, const int32_t* slot_kf_r, const int32_t* slot_kf_c,
                                const double* A, int N, const double* gvec, double* H_out, double* g_out,
                                cudaStream_t s) {
  export_dense_kernel<<<num_slots + 1, 64, 0, s>>>(num_slots, slot_kf_r, slot_kf_c, A, N, gvec, H_out, g_out);
  return cudaGetLastError();
}

cudaError_t launch_retract(const double* tau, double* poses, const uint8_t* frozen, int N, int* iter_counter,
                           cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  retract_kernel<<<(N + 63) / 64, 64, 0, s>>>(tau, poses, frozen, N, iter_counter);
  return cudaGetLastError();
}

cudaError_t launch_check_matches(const int32_t* midx, const EdgeStatic* es, int E, unsigned long long* bad,
                                 long long* edge_valid, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  check_matches_kernel<<<E, 256, 0, s>>>(midx, es, bad, edge_valid);
  return cudaGetLastError();
}

}  // namespace como3r
