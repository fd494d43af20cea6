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
// One warp per edge, SIMD across lanes: lanes 0 and 1 expand the two quaternions, lanes
// 0..11 form the twelve entries of T_ij and all lanes the 49 entries of Ad.  (An FP64 warp
// instruction holds its SM sub-partition's FP64 unit ~80 cycles whatever its lane count,
// so the instruction count of a warp is its duration.)
__global__ void edge_prep_kernel(const double* __restrict__ poses, const EdgeStatic* __restrict__ es, int E,
                                 double* __restrict__ T64, float* __restrict__ T32, double* __restrict__ Ad) {
  __shared__ double sh[2][13];  // R (row-major), t, s of keyframe i (row 0) and j (row 1)
  const int e = blockIdx.x, lane = threadIdx.x;
  if (e >= E) return;
  if (lane < 2) {
    const double* p = poses + 8 * (lane == 0 ? es[e].i : es[e].j);
    double R[9];
    quat_to_rot(p[3], p[4], p[5], p[6], R);
#pragma unroll
    for (int q = 0; q < 9; ++q) sh[lane][q] = R[q];
    sh[lane][9] = p[0];
    sh[lane][10] = p[1];
    sh[lane][11] = p[2];
    sh[lane][12] = p[7];
  }
  __syncwarp();
  const double* Ri = sh[0];
  const double* Rj = sh[1];
  const double si_inv = 1.0 / Ri[12];
  // T_ij = T_i^{-1} T_j: sR_ij = (s_j / s_i) R_i^T R_j, t_ij = R_i^T (t_j - t_i) / s_i
  if (lane < 12) {
    const int r = lane < 9 ? lane / 3 : lane - 9;
    double b0, b1, b2, f;
    if (lane < 9) {
      const int c = lane % 3;
      b0 = Rj[c]; b1 = Rj[3 + c]; b2 = Rj[6 + c];
      f = Rj[12] * si_inv;
    } else {
      b0 = Rj[9] - Ri[9]; b1 = Rj[10] - Ri[10]; b2 = Rj[11] - Ri[11];
      f = si_inv;
    }
    const double v = f * fma(Ri[r], b0, fma(Ri[3 + r], b1, Ri[6 + r] * b2));
    T64[12 * e + lane] = v;
    // the FP32 copy holds sR_ij - I: relative poses of neighbouring keyframes are close to
    // the identity, so its entries are small and their rounding error (the only error of
    // the transform shared by all of an edge's matches) is roughly ten times smaller than
    // that of sR_ij itself; the kernels add X_j back in FP32
    T32[16 * e + lane] = (float)(lane < 9 && lane % 4 == 0 ? v - 1.0 : v);
  } else if (lane < 16) {
    T32[16 * e + lane] = 0.f;
  }
  // Ad_{T_i^{-1}} with T_i^{-1} = (s' R', t'), s' = 1/s_i, R' = R_i^T, t' = -R_i^T t_i / s_i:
  // [[s' R', [t']x R', -t'], [0, R', 0], [0, 0, 1]]
  double tp[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) tp[r] = -si_inv * fma(Ri[r], Ri[9], fma(Ri[3 + r], Ri[10], Ri[6 + r] * Ri[11]));
  for (int x = lane; x < 49; x += 32) {
    const int r = x / 7, c = x % 7;
    double v = 0.0;
    if (r < 3 && c < 3) {
      v = si_inv * Ri[3 * c + r];
    } else if (r < 3 && c < 6) {
      // ([t']x R')[r][c'] = sum_k [t']x[r][k] R_i[c'][k]
      const int cc = c - 3;
      const double t0 = r == 0 ? 0.0 : (r == 1 ? tp[2] : -tp[1]);
      const double t1 = r == 0 ? -tp[2] : (r == 1 ? 0.0 : tp[0]);
      const double t2 = r == 0 ? tp[1] : (r == 1 ? -tp[0] : 0.0);
      v = fma(t0, Ri[3 * cc], fma(t1, Ri[3 * cc + 1], t2 * Ri[3 * cc + 2]));
    } else if (r < 3) {
      v = -tp[r];
    } else if (r < 6 && c >= 3 && c < 6) {
      v = Ri[3 * (c - 3) + (r - 3)];
    } else if (r == 6 && c == 6) {
      v = 1.0;
    }
    Ad[49 * e + x] = v;
  }
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
  // the solver launched after this kernel may start now: it stages its static plan and
  // waits for this grid's completion (griddepcontrol.wait) before it reads A or g
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
  } else if (b < num_slots + N + G) {
    // cost and skipped matches of graph g: strided partial sums, then a fixed-order tree
    // (bitwise reproducible; a single thread's chain of FP64 adds is ~70 cycles per edge)
    __shared__ double sc[64], ss[64];
    const int g = b - num_slots - N;
    double c = 0.0, sk = 0.0;
    for (int e = edge_offset[g] + t; e < edge_offset[g + 1]; e += 64) {
      c += edge_cost[e];
      sk += edge_skip[e];
    }
    sc[t] = c;
    ss[t] = sk;
    __syncthreads();
    for (int h = 32; h > 0; h >>= 1) {
      if (t < h) {
        sc[t] += sc[t + h];
        ss[t] += ss[t + h];
      }
      __syncthreads();
    }
    if (t == 0) {
      const int it = iter_counter ? *iter_counter : 0;
      ginfo[g].cost = sc[0];
      ginfo[g].skipped = (long long)ss[0];
      if (cost_hist) cost_hist[(int64_t)it * G + g] = sc[0];
      if (ss[0] > 0.0) atomicOr(warn, 2);
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

// One keyframe per warp: the warp evaluates the series coefficients together, and lanes
// 0..7 apply the update, one pose entry each (see edge_prep_kernel on FP64 instruction
// counts).
__global__ void retract_kernel(const double* __restrict__ tau, double* __restrict__ poses,
                               const uint8_t* __restrict__ frozen, int N, int* iter_counter) {
  const int k = blockIdx.x, lane = threadIdx.x;
  if (k == 0 && lane == 0 && iter_counter) *iter_counter += 1;
  if (k >= N) return;
  if (frozen && frozen[k]) return;
  const double* t = tau + 7 * k;
  // a zero update leaves the pose bitwise unchanged (no renormalisation)
  if (t[0] == 0.0 && t[1] == 0.0 && t[2] == 0.0 && t[3] == 0.0 && t[4] == 0.0 && t[5] == 0.0 && t[6] == 0.0) return;
  const double th2 = t[3] * t[3] + t[4] * t[4] + t[5] * t[5];
  double A, B, C, ez;
  exp_coefficients_warp(th2, t[6], lane, A, B, C, ez);
  retract_left_warp(t, poses + 8 * k, A, B, C, ez, lane);
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
  edge_prep_kernel<<<E, 32, 0, s>>>(poses, es, E, T64, T32, Ad);
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
  assemble_kernel<<<num_slots + N + G, 64, 0, s>>>(num_slots, slot_contrib_off, slot_contrib, edge_M, A, N,
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
  retract_kernel<<<N, 32, 0, s>>>(tau, poses, frozen, N, iter_counter);
  return cudaGetLastError();
}

// One device-clock stamp into *out (marks the start of a timed call on its stream).
__global__ void stamp_kernel(long long* out) { *out = globaltimer_ns(); }

cudaError_t launch_stamp(long long* out, cudaStream_t s) {
  stamp_kernel<<<1, 1, 0, s>>>(out);
  return cudaGetLastError();
}

cudaError_t launch_check_matches(const int32_t* midx, const EdgeStatic* es, int E, unsigned long long* bad,
                                 long long* edge_valid, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  check_matches_kernel<<<E, 256, 0, s>>>(midx, es, bad, edge_valid);
  return cudaGetLastError();
}

}  // namespace como3r
