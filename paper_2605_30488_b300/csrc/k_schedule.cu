// Work balance of K1 across the warps of its persistent grid.
//
// The valid-match count of a work item varies from zero (outside an edge's overlap) to
// the item size, so equal item counts per warp leave some SMs with several times the
// arithmetic of others, while a loop that is bound by one memory round trip per group
// of pixels costs the same for empty and full groups.  Every warp (or CTA) gets a
// contiguous run of items whose cost (wv x valid matches + wp x pixels scanned, weights
// chosen per launch configuration) is 1/W of the total, and writes one record per run of
// items of one edge ("segment").  Segments are numbered in warp order, so the
// records of an edge are contiguous and the per-edge reduction sums them in a fixed order.
// The schedule depends only on the match indices, so it is rebuilt on the device (no host
// synchronisation) when they change, not per iteration.
#include <cstdint>

#include "como3r_internal.h"

namespace como3r {
namespace {

constexpr int kBalanceThreads = 1024;

// Valid matches of every item (one warp per item); with `compact`, also the item's list of
// valid matches in pixel order, packed (n << 10) | (pixel offset in the item), at
// compact + it * kCompactSlot (items of at most kCompactSlot pixels, n < 2^22).
__global__ void count_item_valid_kernel(const int32_t* __restrict__ midx, const EdgeStatic* __restrict__ es,
                                        const Item* __restrict__ items, int num_items, int32_t* __restrict__ counts,
                                        uint32_t* __restrict__ compact) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int it = w0; it < num_items; it += nw) {
    const Item item = items[it];
    const int32_t* idx = midx + es[item.edge].idx_off;
    uint32_t* out = (compact && item.end - item.begin <= kCompactSlot) ? compact + (int64_t)it * kCompactSlot : nullptr;
    int c = 0;
    for (int g0 = item.begin; g0 < item.end; g0 += 32) {
      const int m = g0 + lane;
      const int n = m < item.end ? __ldg(idx + m) : -1;
      const unsigned mask = __ballot_sync(0xffffffffu, n >= 0);
      if (out && n >= 0) out[c + __popc(mask & below)] = ((uint32_t)n << 10) | (uint32_t)(m - item.begin);
      c += __popc(mask);
    }
    if (lane == 0) counts[it] = c;
  }
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ long long block_exclusive_scan(long long v, long long* sh, long long& excl) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < kBalanceThreads; off <<= 1) {
    const long long a = t >= off ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += a;
    __syncthreads();
  }
  excl = sh[t] - v;
  const long long total = sh[kBalanceThreads - 1];
  __syncthreads();
  return total;
}

// Largest w in [0, n] with a[w] <= x (a non-decreasing, a[0] <= x).
__device__ int upper_bound_minus1(const int32_t* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One CTA: prefix sums of item costs (into cum[0..num_items]), warp starts by cost
// quantiles, segment bases per warp and the first segment of every edge.
__global__ void __launch_bounds__(kBalanceThreads) balance_kernel(const int32_t* __restrict__ counts,
                                                                   const Item* __restrict__ items, int num_items,
                                                                   const int32_t* __restrict__ item_off, int E, int W,
                                                                   int wv, int wp,
                                                                   long long* __restrict__ cum,
                                                                   int32_t* __restrict__ start,
                                                                   int32_t* __restrict__ seg,
                                                                   int32_t* __restrict__ seg_off) {
  __shared__ long long sh[kBalanceThreads];
  const int t = threadIdx.x;
  long long carry = 0;
  for (int base = 0; base < num_items; base += kBalanceThreads) {
    const int i = base + t;
    const long long c =
        i < num_items ? (long long)wv * counts[i] + (long long)wp * (items[i].end - items[i].begin) : 0;
    long long ex;
    const long long tot = block_exclusive_scan(c, sh, ex);
    if (i < num_items) cum[i] = carry + ex;
    carry += tot;
  }
  if (t == 0) cum[num_items] = carry;
  __syncthreads();
  const long long total = carry;
  // start[w] = first item whose exclusive prefix reaches total * w / W
  for (int w = t; w <= W; w += kBalanceThreads) {
    int s;
    if (w == 0) s = 0;
    else if (w == W) s = num_items;
    else {
      const long long target = (long long)((__int128)total * w / W);
      int lo = 0, hi = num_items;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cum[mid] < target) lo = mid + 1;
        else hi = mid;
      }
      s = lo;
    }
    start[w] = s;
  }
  __syncthreads();
  // segments: distinct edges of each warp's run (items are ordered by edge and every edge
  // has at least one item, so the count is last edge - first edge + 1)
  long long carry_s = 0;
  for (int base = 0; base < W; base += kBalanceThreads) {
    const int w = base + t;
    long long n = 0;
    if (w < W && start[w + 1] > start[w]) n = items[start[w + 1] - 1].edge - items[start[w]].edge + 1;
    long long ex;
    const long long tot = block_exclusive_scan(n, sh, ex);
    if (w < W) seg[w] = (int32_t)(carry_s + ex);
    carry_s += tot;
  }
  __syncthreads();
  for (int e = t; e <= E; e += kBalanceThreads) {
    if (e == E) {
      seg_off[E] = (int32_t)carry_s;
    } else {
      const int i = item_off[e];
      const int w = upper_bound_minus1(start, W, i);
      seg_off[e] = seg[w] + (e - items[start[w]].edge);
    }
  }
}

}  // namespace

cudaError_t launch_schedule(const int32_t* midx, const EdgeStatic* es, const Item* items, int num_items,
                            const int32_t* item_off, int E, int W, int wv, int wp, int32_t* counts, long long* cum,
                            int32_t* start, int32_t* seg, int32_t* seg_off, uint32_t* compact, cudaStream_t s) {
  if (num_items <= 0 || W <= 0) return cudaErrorInvalidValue;
  int blocks = (num_items + 7) / 8;
  if (blocks > 1184) blocks = 1184;
  count_item_valid_kernel<<<blocks, 256, 0, s>>>(midx, es, items, num_items, counts, compact);
  balance_kernel<<<1, kBalanceThreads, 0, s>>>(counts, items, num_items, item_off, E, W, wv, wp, cum, start, seg,
                                                seg_off);
  return cudaGetLastError();
}

}  // namespace como3r
