// como3r_linearize_noalloc: per-edge linearisation that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// linearisation: real-time loops that must not stall on the allocator, and host
// frameworks that own the whole device memory budget and forbid side allocations.  For
// them this file keeps every intermediate buffer of the linearisation -- per-edge
// relative poses and adjoints, the residual kernel's work list and per-item records, the
// per-edge reduction outputs -- in one file-scope device array of fixed size, so the
// call needs only the caller's inputs and output.
//
// The array lives as long as the library is loaded, on every device that loads it.  Its
// device address is looked up once per device with cudaGetSymbolAddress (host code may
// not use the array's name as a device pointer).  All calls share it: a call overwrites
// what the previous one left, and calls whose GPU work overlaps (other streams, other
// host threads) race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/como3r.h"
#include "como3r_internal.h"

namespace como3r {
namespace {

constexpr int kMaxEdges = COMO3R_NOALLOC_MAX_EDGES;
constexpr int kMaxItems = COMO3R_NOALLOC_MAX_ITEMS;
constexpr int kMaxGraphs = COMO3R_NOALLOC_MAX_GRAPHS;
constexpr int kMaxDevices = 64;
constexpr int kMinChunk = 1024;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffEs = 0;
constexpr size_t kOffItems = align256(kOffEs + sizeof(EdgeStatic) * kMaxEdges);
constexpr size_t kOffItemOff = align256(kOffItems + sizeof(Item) * kMaxItems);
constexpr size_t kOffT64 = align256(kOffItemOff + sizeof(int32_t) * (kMaxEdges + 1));
constexpr size_t kOffT32 = align256(kOffT64 + sizeof(double) * 12 * kMaxEdges);
constexpr size_t kOffAd = align256(kOffT32 + sizeof(float) * 16 * kMaxEdges);
constexpr size_t kOffRecords = align256(kOffAd + sizeof(double) * 49 * kMaxEdges);
constexpr size_t kOffM = align256(kOffRecords + sizeof(double) * kPartial * kMaxItems);
constexpr size_t kOffB = align256(kOffM + sizeof(double) * 49 * kMaxEdges);
constexpr size_t kOffCost = align256(kOffB + sizeof(double) * 7 * kMaxEdges);
constexpr size_t kOffSkip = align256(kOffCost + sizeof(double) * kMaxEdges);
constexpr size_t kOffValid = align256(kOffSkip + sizeof(double) * kMaxEdges);
constexpr size_t kOffBad = align256(kOffValid + sizeof(long long) * kMaxEdges);
constexpr size_t kScratchBytes = align256(kOffBad + sizeof(unsigned long long));
static_assert(kScratchBytes <= COMO3R_NOALLOC_SCRATCH_BYTES, "scratch exceeds its documented size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host staging of the work description (static storage; the entry point is not reentrant).
static EdgeStatic h_es[kMaxEdges];
static Item h_items[kMaxItems];
static int32_t h_item_off[kMaxEdges + 1];
static int64_t h_graph_px[kMaxGraphs + 1];
static unsigned long long h_bad;

static unsigned char* g_scratch_dev[kMaxDevices];
static std::mutex g_setup_mutex;

// Device address of the scratch on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool positive(double x) { return x > 0.0 && x < 1e300; }

int invalid(const char* why) { return report_error(COMO3R_ERR_INVALID_ARG, why); }

}  // namespace
}  // namespace como3r

using namespace como3r;

extern "C" int como3r_linearize_noalloc(const como3r_graph_desc* d, const double* poses, double* edge_out,
                                        void* cuda_stream) {
  if (!d || !poses || !edge_out) return invalid("desc, poses and edge_out must not be NULL");
  const int G = d->num_graphs;
  if (G < 1 || G > kMaxGraphs) return invalid("num_graphs must be in [1, COMO3R_NOALLOC_MAX_GRAPHS]");
  if (!d->kf_offset || !d->height || !d->width || !d->edge_offset || !d->edge_i || !d->edge_j || !d->points_conf)
    return invalid("a required array of the description is NULL");
  if (d->copy_inputs || (d->mode != COMO3R_PLAIN_FP64 && d->mode != COMO3R_MIXED) || d->dtype < COMO3R_F16 ||
      d->dtype > COMO3R_F64 || !positive(d->sigma_ray) || !positive(d->sigma_dist) || !positive(d->huber_k))
    return invalid("copy_inputs must be 0; mode, dtype, sigma_ray, sigma_dist and huber_k must be valid");
  if (d->kf_offset[0] != 0 || d->edge_offset[0] != 0) return invalid("kf_offset[0] and edge_offset[0] must be 0");
  const int E = d->edge_offset[G];
  if (E < 0 || E > kMaxEdges) return invalid("more edges than COMO3R_NOALLOC_MAX_EDGES");  // beyond the scratch
  if (E == 0) return COMO3R_OK;
  if (!d->match_idx) return invalid("match_idx is NULL");
  // pixel layout: graph g's keyframes each hold height[g] * width[g] pixels
  h_graph_px[0] = 0;
  for (int g = 0; g < G; ++g) {
    if (d->kf_offset[g + 1] <= d->kf_offset[g] || d->edge_offset[g + 1] < d->edge_offset[g])
      return invalid("kf_offset must increase and edge_offset must not decrease");
    if (d->height[g] <= 0 || d->width[g] <= 0 || (int64_t)d->height[g] * d->width[g] >= (int64_t(1) << 30))
      return invalid("height and width must be positive with fewer than 2^30 pixels");
    h_graph_px[g + 1] = h_graph_px[g] + (int64_t)(d->kf_offset[g + 1] - d->kf_offset[g]) * d->height[g] * d->width[g];
  }
  int64_t streamed = 0, idx_off = 0;
  for (int g = 0; g < G; ++g) {
    const int k0 = d->kf_offset[g], k1 = d->kf_offset[g + 1];
    const int32_t P = d->height[g] * d->width[g];
    for (int e = d->edge_offset[g]; e < d->edge_offset[g + 1]; ++e) {
      const int i = d->edge_i[e], j = d->edge_j[e];
      if (i < k0 || i >= k1 || j < k0 || j >= k1 || i == j)
        return invalid("edge endpoints must be two different keyframes of the edge's graph");
      EdgeStatic s{};
      s.pix_i = h_graph_px[g] + (int64_t)(i - k0) * P;
      s.pix_j = h_graph_px[g] + (int64_t)(j - k0) * P;
      s.idx_off = idx_off;
      s.i = i;
      s.j = j;
      s.npix_i = P;
      s.npix_j = P;
      h_es[e] = s;
      idx_off += P;
      streamed += P;
    }
  }
  // smallest chunk (a multiple of kMinChunk) whose items fit the scratch
  int64_t chunk = kMinChunk;
  const int64_t room = kMaxItems - E;
  if (room <= 0) return invalid("more edges than the work-item table holds");
  while ((streamed + chunk - 1) / chunk > room) chunk += kMinChunk;
  int n_items = 0;
  h_item_off[0] = 0;
  for (int e = 0; e < E; ++e) {
    for (int64_t b = 0; b < h_es[e].npix_i; b += chunk) {
      if (n_items >= kMaxItems) return invalid("more work items than COMO3R_NOALLOC_MAX_ITEMS");
      h_items[n_items++] = Item{e, (int32_t)b, (int32_t)std::min<int64_t>(b + chunk, h_es[e].npix_i), 0};
    }
    h_item_off[e + 1] = n_items;
  }
  if (!device_pointer(d->points_conf) || !device_pointer(d->match_idx) || !device_pointer(poses) ||
      !device_pointer(edge_out))
    return invalid("points_conf, match_idx, poses and edge_out must be device memory");
  if (reinterpret_cast<uintptr_t>(d->points_conf) % 16 || reinterpret_cast<uintptr_t>(d->match_idx) % 4)
    return invalid("points_conf must be 16-byte and match_idx 4-byte aligned");

  unsigned char* base = nullptr;
  if (cudaError_t e = scratch_address(&base)) return report_cuda_error(e, "scratch address");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  auto* es = reinterpret_cast<EdgeStatic*>(base + kOffEs);
  auto* items = reinterpret_cast<Item*>(base + kOffItems);
  auto* item_off = reinterpret_cast<int32_t*>(base + kOffItemOff);
  auto* T64 = reinterpret_cast<double*>(base + kOffT64);
  auto* T32 = reinterpret_cast<float*>(base + kOffT32);
  auto* Ad = reinterpret_cast<double*>(base + kOffAd);
  void* records = base + kOffRecords;
  auto* M = reinterpret_cast<double*>(base + kOffM);
  auto* B = reinterpret_cast<double*>(base + kOffB);
  auto* cost = reinterpret_cast<double*>(base + kOffCost);
  auto* skip = reinterpret_cast<double*>(base + kOffSkip);
  auto* valid = reinterpret_cast<long long*>(base + kOffValid);
  auto* bad = reinterpret_cast<unsigned long long*>(base + kOffBad);

  cudaError_t err = cudaMemcpyAsync(es, h_es, sizeof(EdgeStatic) * E, cudaMemcpyHostToDevice, s);
  if (!err) err = cudaMemcpyAsync(items, h_items, sizeof(Item) * n_items, cudaMemcpyHostToDevice, s);
  if (!err) err = cudaMemcpyAsync(item_off, h_item_off, sizeof(int32_t) * (E + 1), cudaMemcpyHostToDevice, s);
  // counters the kernels accumulate into must start at zero (the scratch keeps old values)
  if (!err) err = cudaMemsetAsync(valid, 0, sizeof(long long) * E, s);
  if (!err) err = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
  if (!err) err = launch_check_matches(d->match_idx, es, E, bad, valid, s);
  if (!err) err = cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s);
  if (!err) err = cudaStreamSynchronize(s);
  if (err) return report_cuda_error(err, "linearize_noalloc match check");
  if (h_bad) return invalid("a match index lies outside [-1, P_j)");

  const RobustParams rp = make_robust_params(d->sigma_ray, d->sigma_dist, d->huber_k);
  int dev = 0, sms = 1;
  if (cudaError_t e = cudaGetDevice(&dev)) return report_cuda_error(e, "cudaGetDevice");
  if (cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return report_cuda_error(e, "attribute");
  const int occ = std::max(1, residual_reduce_max_blocks_per_sm(d->mode, d->dtype, 0));
  const int warps_per_cta = residual_reduce_block() / 32;
  const int grid = std::max(1, std::min(sms * occ, (n_items + warps_per_cta - 1) / warps_per_cta));
  err = launch_edge_prep(poses, es, E, T64, T32, Ad, s);
  if (!err) err = launch_residual_reduce(d->mode, d->dtype, 0, grid, d->points_conf, d->match_idx, items, n_items, es,
                                         T64, T32, rp, records, WarpSched{nullptr, nullptr}, s);
  if (!err) err = launch_edge_reduce(d->mode, records, item_off, E, Ad, M, B, cost, skip, edge_out, valid, s);
  return err ? report_cuda_error(err, "linearize_noalloc") : COMO3R_OK;
}
