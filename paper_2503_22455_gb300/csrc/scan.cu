// Device-wide exclusive prefix sum of int32 flags (deterministic, three passes).
// Used by every compaction in the set-up: crossings, affected nodes, irregular
// Shortley-Weller nodes.
#include "kernels.cuh"

namespace iim {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;          // elements per thread
constexpr int kScanTile = kScanBlock * kScanItems;

__global__ void k_scan_tile_sums(const int* __restrict__ in, int64_t len, int* __restrict__ sums) {
  __shared__ int red[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanBlock + threadIdx.x;
    if (i < len) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
  }
}

// single block: exclusive scan of the tile sums in place; total -> *total
__global__ void k_scan_sums(int* __restrict__ sums, int nt, int* __restrict__ total) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nt; base += kScanBlock) {
    int i = base + threadIdx.x;
    int v = i < nt ? sums[i] : 0;
    int x = v;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int incl = x + (wid > 0 ? wsum[wid - 1] : 0);
    if (i < nt) sums[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_tiles(const int* __restrict__ in, int64_t len, const int* __restrict__ sums,
                             int* __restrict__ out) {
  __shared__ int wsum[32];
  __shared__ int carry;
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (threadIdx.x == 0) carry = sums[blockIdx.x];
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanBlock + threadIdx.x;
    int v = i < len ? in[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int incl = x + (wid > 0 ? wsum[wid - 1] : 0);
    if (i < len) out[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry += incl;
    __syncthreads();
  }
}

int64_t scan_scratch_ints(int64_t len) { return (len + kScanTile - 1) / kScanTile + 1; }

void scan_exclusive(const int* in, int* out, int64_t len, int* total, int* scratch, cudaStream_t s) {
  if (len <= 0) {
    cudaMemsetAsync(total, 0, sizeof(int), s);
    return;
  }
  int nt = (int)((len + kScanTile - 1) / kScanTile);
  IIM_LAUNCH(k_scan_tile_sums, nt, kScanBlock, 0, s, in, len, scratch);
  IIM_LAUNCH(k_scan_sums, 1, kScanBlock, 0, s, scratch, nt, total);
  IIM_LAUNCH(k_scan_tiles, nt, kScanBlock, 0, s, in, len, scratch, out);
}

}  // namespace iim
