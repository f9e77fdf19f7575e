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
  const int64_t base = blockIdx.x * int64_t(kScanBlock);
  for (int q = threadIdx.x; q < kScanBlock; q += blockDim.x) {
    const int64_t t = base + q;
    s[q] = t < n ? data[t] : 0u;
  }
  __syncthreads();
  // each of the 256 threads owns 4 items; Hillis-Steele over the thread sums
  const int q0 = threadIdx.x * 4;
  uint32_t a0 = s[q0], a1 = s[q0 + 1], a2 = s[q0 + 2], a3 = s[q0 + 3];
  const uint32_t tot = a0 + a1 + a2 + a3;
  __shared__ uint32_t part[256];
  part[threadIdx.x] = tot;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const uint32_t x = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += x;
    __syncthreads();
  }
  const uint32_t excl = part[threadIdx.x] - tot;
  s[q0] = excl;
  s[q0 + 1] = excl + a0;
  s[q0 + 2] = excl + a0 + a1;
  s[q0 + 3] = excl + a0 + a1 + a2;
  if (threadIdx.x == 255) sums[blockIdx.x] = part[255];
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

}  // namespace
}  // namespace amr
