// scan_kernels.cuh -- exclusive prefix sum of u32 arrays (the prefix sums of
// the level bucket sort, the radix sorts and the particle segment split,
// Sec. 2.2 and Sec. 4).  The kernels have internal linkage so that every
// translation unit that includes this header carries its own copy.
#pragma once
#include <cstdint>

namespace amr {
namespace {

// exclusive scan of u32, 1024 items per block
constexpr int kScanItems = 1024;
constexpr int kScanBlock = kScanItems;

__global__ void k_scan_block(uint32_t *__restrict__ data, int64_t n, uint32_t *__restrict__ sums) {
  __shared__ uint32_t s[kScanBlock];
  __shared__ uint32_t wsum[8];
  const int64_t base = blockIdx.x * int64_t(kScanBlock);
  for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x) {
    const int64_t t = base + q;
    s[q] = t < n ? data[t] : 0u;
  }
  __syncthreads();
  // each of the 256 threads owns 4 items; warp scans of the thread sums by
  // shuffles, then the 8 warp totals
  const int q0 = threadIdx.x * 4, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t a0 = s[q0], a1 = s[q0 + 1], a2 = s[q0 + 2], a3 = s[q0 + 3];
  const uint32_t tot = a0 + a1 + a2 + a3;
  uint32_t x = tot;  // inclusive within the warp
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t wpre = 0;
  for (int k = 0; k < w; ++k) wpre += wsum[k];
  const uint32_t excl = wpre + x - tot;
  s[q0] = excl;
  s[q0 + 1] = excl + a0;
  s[q0 + 2] = excl + a0 + a1;
  s[q0 + 3] = excl + a0 + a1 + a2;
  if (threadIdx.x == 255) sums[blockIdx.x] = wpre + x;
  __syncthreads();
  for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x) {
    const int64_t t = base + q;
    if (t < n) data[t] = s[q];
  }
}

__global__ void k_scan_add(uint32_t *__restrict__ data, int64_t n, const uint32_t *__restrict__ sums) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) data[t] += sums[t / kScanBlock];
}

// the second pass when there are at most kScanFlat blocks: block b + 1 adds
// the sum of the block totals before it, which it forms itself (no scan of
// the totals, one launch less)
constexpr int64_t kScanFlat = 4096;
__global__ void k_scan_add_flat(uint32_t *__restrict__ data, int64_t n, const uint32_t *__restrict__ sums) {
  const int64_t b = blockIdx.x + 1;
  uint32_t acc = 0;
  for (int64_t q = threadIdx.x; q < b; q += blockDim.x) acc += sums[q];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
  __shared__ uint32_t part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  uint32_t off = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) off += part[w];
  const int64_t base = b * int64_t(kScanBlock);
  for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x) {
    const int64_t t = base + q;
    if (t < n) data[t] += off;
  }
}

}  // namespace
}  // namespace amr
