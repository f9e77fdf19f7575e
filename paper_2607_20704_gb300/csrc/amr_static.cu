// amr_static.cu -- amr_cfl_dt_static: the CFL time-step reduction of a
// single-level block of cells with its scratch in fixed device storage, for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where no device allocation may happen --
// inside a process whose device memory is pre-reserved by another runtime's
// pool (so cudaMalloc fails or would steal from it), in a real-time loop
// that must never touch the allocator, or from an allocator-less host
// environment.  Such a caller owns its input and output buffers and needs
// the library to bring its own scratch.
//
// The scratch lives in file-scope __device__ arrays below.  Every GPU that
// loads the library holds them until the process exits (512 KiB + 8 bytes
// per device).  Host code never dereferences their names: the device
// address is taken once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernel.  The addresses are kept for the
// life of the process; a cudaDeviceReset invalidates them (and the library's
// module), so a caller that resets a device does not call this entry point
// again in that process.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>

#include "amr.h"

void amr_set_error_text(const char *text);

namespace {

constexpr int kBlock = 256;
constexpr int64_t kMaxBlocks = 65536;  // one partial maximum per block
constexpr int kMaxDevices = 64;

// per-block maxima, then the count of finished blocks (must start at zero)
static __device__ __align__(256) double g_block_max[kMaxBlocks];
static __device__ __align__(256) unsigned int g_blocks_done;

struct DeviceScratch {
  double *block_max = nullptr;
  unsigned int *done = nullptr;
  bool ready = false;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_lock;

amr_status set_error(amr_status s, const char *msg) {
  amr_set_error_text(msg);
  return s;
}

// One thread per cell: sum_d (|u_d| + c) in FP64; block maximum to the
// scratch; the last block to finish reduces the block maxima in index order
// and writes dt = cfl dx / max.  A non-finite cell makes dt NaN.
__global__ void k_cfl_static(const double *__restrict__ U, int64_t n, int64_t stride, double dx,
                             double gamma, double cfl, double smallr, double smallp,
                             double *block_max, unsigned int *done, double *dt_out) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  double s = 0.0;
  if (t < n) {
    const double u0 = U[t], u1 = U[stride + t], u2 = U[2 * stride + t], u3 = U[3 * stride + t],
                 u4 = U[4 * stride + t];
    const double r = fmax(u0, smallr);
    const double vx = u1 / r, vy = u2 / r, vz = u3 / r;
    const double ek = 0.5 * r * ((vx * vx + vy * vy) + vz * vz);
    const double p = fmax((gamma - 1.0) * (u4 - ek), r * smallp);
    const double cs = sqrt(gamma * p / r);
    s = ((fabs(vx) + cs) + (fabs(vy) + cs)) + (fabs(vz) + cs);
    // each input tested on its own: a sum of large finite values may overflow
    if (!isfinite(s) || !isfinite(u0) || !isfinite(u1) || !isfinite(u2) || !isfinite(u3) ||
        !isfinite(u4))
      s = __longlong_as_double(0x7FF8000000000000ll);
  }
  __shared__ double wmax[kBlock / 32];
  __shared__ bool last;
  // fmax drops a NaN operand, so carry "non-finite" as +inf through the max
  if (s != s) s = __longlong_as_double(0x7FF0000000000000ll);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = wmax[0];
    for (int w = 1; w < kBlock / 32; ++w) m = fmax(m, wmax[w]);
    block_max[blockIdx.x] = m;
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double m = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) m = fmax(m, __ldcg(block_max + b));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kBlock / 32; ++w) m = fmax(m, wmax[w]);
    m = fmax(m, wmax[0]);
    *dt_out = isinf(m) ? __longlong_as_double(0x7FF8000000000000ll) : cfl * dx / m;
    *done = 0u;  // leave the counter cleared for the next call as well
  }
}

}  // namespace

extern "C" amr_status amr_cfl_dt_static(const double *U, int64_t n_cells, int64_t stride,
                                        int level, double gamma, double cfl, double smallr,
                                        double smallc, double *dt_out, void *stream) {
  if (!U || !dt_out) return set_error(AMR_EINVAL, "amr_cfl_dt_static: NULL device pointer");
  if (n_cells < 1 || n_cells > AMR_CFL_STATIC_MAX_CELLS) {
    char msg[160];
    snprintf(msg, sizeof msg, "amr_cfl_dt_static: n_cells = %lld outside [1, %lld] (fixed scratch size)",
             (long long)n_cells, (long long)AMR_CFL_STATIC_MAX_CELLS);
    return set_error(AMR_EINVAL, msg);
  }
  if (stride < n_cells) return set_error(AMR_EINVAL, "amr_cfl_dt_static: stride < n_cells");
  if (level < 0 || level > 30) return set_error(AMR_EINVAL, "amr_cfl_dt_static: level outside [0, 30]");
  if (!(gamma > 1.0) || !(cfl > 0.0) || !(smallr > 0.0) || !(smallc > 0.0))
    return set_error(AMR_EINVAL, "amr_cfl_dt_static: gamma > 1, cfl > 0, smallr > 0, smallc > 0 required");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error(AMR_ECUDA, "amr_cfl_dt_static: no current CUDA device");
  DeviceScratch sc;
  {
    std::lock_guard<std::mutex> g(g_scratch_lock);
    DeviceScratch &d = g_scratch[dev];
    if (!d.ready) {  // first call on this device: look up the scratch addresses
      void *pm = nullptr, *pd = nullptr;
      if (cudaGetSymbolAddress(&pm, g_block_max) != cudaSuccess ||
          cudaGetSymbolAddress(&pd, g_blocks_done) != cudaSuccess) {
        cudaGetLastError();
        return set_error(AMR_ECUDA, "amr_cfl_dt_static: cudaGetSymbolAddress failed");
      }
      d.block_max = static_cast<double *>(pm);
      d.done = static_cast<unsigned int *>(pd);
      d.ready = true;
    }
    sc = d;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(sc.done, 0, sizeof(unsigned int), s) != cudaSuccess) {
    cudaGetLastError();
    return set_error(AMR_ECUDA, "amr_cfl_dt_static: clearing the block counter failed");
  }
  const unsigned blocks = unsigned((n_cells + kBlock - 1) / kBlock);
  k_cfl_static<<<blocks, kBlock, 0, s>>>(U, n_cells, stride, ldexp(1.0, -level), gamma, cfl,
                                         smallr, smallc * smallc / gamma, sc.block_max, sc.done,
                                         dt_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof msg, "amr_cfl_dt_static: launch failed: %s", cudaGetErrorString(e));
    return set_error(AMR_ECUDA, msg);
  }
  return AMR_OK;
}
