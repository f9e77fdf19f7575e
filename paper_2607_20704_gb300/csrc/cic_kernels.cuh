// cic_kernels.cuh -- particle mass deposition by Cloud-in-Cell on a periodic
// n^3 grid (paper Sec. 4, mass deposition), in FP64 or FP32.
//
// Shifted stencil: along each axis s = x n - 1/2, i0 = floor(s), f = s - i0;
// the particle gives m (wx wy wz) n^3 to the 8 cells (i0 + cx, j0 + cy,
// k0 + cz), wx = 1 - f for cx = 0 and f for cx = 1 (the `medium' stencil:
// only the 2^3 cells with non-zero weight).  The cell (i0, j0, k0) is the
// particle's source cell; particles are sorted by the Hilbert index of their
// source cell so that particles of one source cell are contiguous.
//
//   sort      source-cell Hilbert keys, then a stable LSD radix sort of
//             (key, particle) pairs, tiles of 2048 items staged through
//             shared memory so that every digit's run is written contiguously;
//             then the particle arrays are gathered into the sorted order.
//   atomic    one thread per particle; lanes of a warp that share a source
//             cell add their 8 contributions by a segmented shuffle reduction
//             and the segment's first lane issues 8 atomic adds (the paper's
//             medium kernel: warp combining + atomicAdd).
//   segment   deterministic: segment starts by a prefix sum over the sorted
//             keys; one thread per source-cell segment sums its particles'
//             8 contributions in particle order; one thread per grid cell
//             gathers the 8 segment sums that reach it, in stencil order
//             (the paper's small kernel: prefix sums and one update per
//             segment and stencil offset).  The result depends only on the
//             particles and their order, not on the launch or on timing.
//
// Every grid index is masked by n - 1 (n a power of two), so that no position,
// even a non-finite one, addresses outside the grid.
#pragma once
#include "amr_internal.cuh"
#include "scan_kernels.cuh"

namespace amr {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 items per tile

// source cell and weights along one axis; x n is exact for n a power of two
template <class T>
__device__ __forceinline__ int cic_axis(T x, int n, T &w0, T &w1) {
  const T s = x * T(n) - T(0.5);
  const T fl = floor(s);
  w1 = s - fl;
  w0 = T(1) - w1;
  return int(fl) & (n - 1);
}

__device__ __forceinline__ uint32_t grid_at(int n, int i, int j, int k) {
  const int m = n - 1;
  return uint32_t(i & m) + uint32_t(n) * (uint32_t(j & m) + uint32_t(n) * uint32_t(k & m));
}

// the 8 contributions of one particle, corner c = cx + 2 cy + 4 cz
template <class T>
__device__ __forceinline__ void cic_weights(T x, T y, T z, T ms, int n, int &i, int &j, int &k,
                                            T w[8]) {
  T wx[2], wy[2], wz[2];
  i = cic_axis(x, n, wx[0], wx[1]);
  j = cic_axis(y, n, wy[0], wy[1]);
  k = cic_axis(z, n, wz[0], wz[1]);
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = ms * ((wx[c & 1] * wy[(c >> 1) & 1]) * wz[c >> 2]);
}

// ---------------------------------------------------------------------------
// sort
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_part_keys(int64_t np, int n, int bits, const T *__restrict__ x,
                            const T *__restrict__ y, const T *__restrict__ z,
                            uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= np) return;
  T w0, w1;
  const int i = cic_axis(x[t], n, w0, w1), j = cic_axis(y[t], n, w0, w1),
            k = cic_axis(z[t], n, w0, w1);
  key[t] = uint32_t(hilbert_index(uint32_t(i), uint32_t(j), uint32_t(k), bits));
  val[t] = uint32_t(t);
}

// per-tile digit counts, table[d * ntiles + tile]
__global__ void __launch_bounds__(kSortThreads) k_psort_hist(const uint32_t *__restrict__ keys,
                                                             int64_t np, int shift, int nbits,
                                                             uint32_t *__restrict__ table,
                                                             int64_t ntiles) {
  __shared__ uint32_t hist[256];
  const int ndig = 1 << nbits;
  const int lane = threadIdx.x & 31;
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * int64_t(kSortTile);
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t t = base + r * kSortThreads + threadIdx.x;
    const unsigned dig = t < np ? (keys[t] >> shift) & unsigned(ndig - 1) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
    if (dig != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&hist[dig], unsigned(__popc(peers)));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) table[int64_t(d) * ntiles + blockIdx.x] = hist[d];
}

// stable scatter of one tile: ranks in item order (rounds, then warps, then
// lanes), the tile staged in shared memory in digit order, then written out
// so that consecutive threads write consecutive places of a digit's run.
// offs = exclusive scan of the table, with offs[ndig * ntiles] = np.
__global__ void __launch_bounds__(kSortThreads) k_psort_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t np, int shift, int nbits, const uint32_t *__restrict__ offs,
    int64_t ntiles) {
  __shared__ uint32_t skey[kSortTile], sval[kSortTile];
  __shared__ uint32_t wcnt[kSortThreads / 32][256], wpre[kSortThreads / 32][256];
  __shared__ uint32_t lstart[256], run[256], part[kSortThreads];
  const int ndig = 1 << nbits;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = blockIdx.x * int64_t(kSortTile);
  const int nt = int(np - base < kSortTile ? np - base : kSortTile);
  // digit counts of this tile from the scanned table, then their exclusive
  // scan over the digits (one digit per thread; ndig <= 256)
  const int d0 = threadIdx.x;
  uint32_t cnt = 0;
  if (d0 < ndig) {
    const int64_t e = int64_t(d0) * ntiles + blockIdx.x;
    cnt = offs[e + 1] - offs[e];
  }
  part[threadIdx.x] = cnt;
  for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
  __syncthreads();
  for (int off = 1; off < kSortThreads; off <<= 1) {
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  lstart[threadIdx.x] = part[threadIdx.x] - cnt;
  run[threadIdx.x] = part[threadIdx.x] - cnt;
  __syncthreads();
  for (int r = 0; r < kSortRounds; ++r) {
    const int q = r * kSortThreads + threadIdx.x;
    const bool valid = q < nt;
    const uint32_t k = valid ? kin[base + q] : 0u;
    const uint32_t v = valid ? vin[base + q] : 0u;
    const unsigned dig = valid ? (k >> shift) & unsigned(ndig - 1) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < ndig) {
      uint32_t acc = run[threadIdx.x];
      for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t c = wcnt[w][threadIdx.x];
        if (c) {
          wpre[w][threadIdx.x] = acc;
          acc += c;
          wcnt[w][threadIdx.x] = 0;
        }
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    if (valid) {
      const uint32_t lp = wpre[warp][dig] + rank;
      skey[lp] = k;
      sval[lp] = v;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nt; q += kSortThreads) {
    const uint32_t k = skey[q];
    const unsigned dig = (k >> shift) & unsigned(ndig - 1);
    const int64_t dst = int64_t(offs[int64_t(dig) * ntiles + blockIdx.x]) + (q - int64_t(lstart[dig]));
    kout[dst] = k;
    vout[dst] = sval[q];
  }
}

// particle arrays into the sorted order
template <class T>
__global__ void k_part_gather(int64_t np, const uint32_t *__restrict__ perm, const T *__restrict__ x,
                              const T *__restrict__ y, const T *__restrict__ z,
                              const T *__restrict__ m, const uint32_t *__restrict__ id,
                              T *__restrict__ x2, T *__restrict__ y2, T *__restrict__ z2,
                              T *__restrict__ m2, uint32_t *__restrict__ id2) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= np) return;
  const uint32_t p = perm[t];
  x2[t] = x[p];
  y2[t] = y[p];
  z2[t] = z[p];
  m2[t] = m[p];
  id2[t] = id[p];
}

// ---------------------------------------------------------------------------
// atomic deposit (warp combining of equal source cells)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_cic_atomic(int64_t np, int n, T scale, const T *__restrict__ x,
                                                    const T *__restrict__ y, const T *__restrict__ z,
                                                    const T *__restrict__ m, T *__restrict__ rho) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  const bool valid = t < np;
  T w[8];
  int i = 0, j = 0, k = 0;
  uint32_t cell = 0xFFFFFFFFu;
  if (valid) {
    cic_weights(x[t], y[t], z[t], m[t] * scale, n, i, j, k, w);
    cell = grid_at(n, i, j, k);
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) w[c] = T(0);
  }
  // segments: runs of equal source cells among the warp's lanes
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, cell, 1);
  const unsigned heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != cell);
  if (heads != 0xFFFFFFFFu) {
    const unsigned above = heads & ~((2u << lane) - 1u);  // heads after this lane (lane 31: none)
    const unsigned next = above ? unsigned(__ffs(above) - 1) : 32u;
    const unsigned len = ((heads >> lane) & 1u) ? next - lane : 0u;
    const unsigned maxrun = __reduce_max_sync(0xFFFFFFFFu, len);
    // backward segmented inclusive scan: the head lane ends with its
    // segment's total
    for (unsigned off = 1; off < maxrun; off <<= 1) {
      const bool take = lane + off < next;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const T o = __shfl_down_sync(0xFFFFFFFFu, w[c], off);
        if (take) w[c] += o;
      }
    }
  }
  if (valid && ((heads >> lane) & 1u)) {
#pragma unroll
    for (int c = 0; c < 8; ++c) atomicAdd(&rho[grid_at(n, i + (c & 1), j + ((c >> 1) & 1), k + (c >> 2))], w[c]);
  }
}

// ---------------------------------------------------------------------------
// deterministic deposit (segment sums)
// ---------------------------------------------------------------------------
__global__ void k_seg_heads(int64_t np, const uint32_t *__restrict__ key, uint32_t *__restrict__ flag) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= np) return;
  flag[q] = (q == 0 || key[q] != key[q - 1]) ? 1u : 0u;
}

// start[s] of every segment s (scan = exclusive scan of the head flags);
// start[S] = np and *nseg = S, written by the last particle's thread
__global__ void k_seg_starts(int64_t np, const uint32_t *__restrict__ key, const uint32_t *__restrict__ scan,
                             uint32_t *__restrict__ start, uint32_t *__restrict__ nseg) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= np) return;
  const bool head = q == 0 || key[q] != key[q - 1];
  if (head) start[scan[q]] = uint32_t(q);
  if (q == np - 1) {
    const uint32_t S = scan[q] + (head ? 1u : 0u);
    start[S] = uint32_t(np);
    *nseg = S;
  }
}

// one thread per segment: the 8 sums of its particles' contributions, in
// particle order, into sums[c * cap + s]; the segment's source cell maps to s
template <class T>
__global__ void k_seg_sum(int64_t cap, int n, T scale, const uint32_t *__restrict__ nseg,
                          const uint32_t *__restrict__ start, const T *__restrict__ x,
                          const T *__restrict__ y, const T *__restrict__ z, const T *__restrict__ m,
                          T *__restrict__ sums, int32_t *__restrict__ cellmap) {
  const int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (s >= int64_t(*nseg)) return;
  const uint32_t q0 = start[s], q1 = start[s + 1];
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = T(0);
  int i = 0, j = 0, k = 0;
  for (uint32_t q = q0; q < q1; ++q) {
    T w[8];
    cic_weights(x[q], y[q], z[q], m[q] * scale, n, i, j, k, w);
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += w[c];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) sums[c * cap + s] = acc[c];
  cellmap[grid_at(n, i, j, k)] = int32_t(s);
}

// one thread per grid cell: rho = the sums of the (up to) 8 segments whose
// stencils reach the cell, in stencil order c = 0..7
template <class T>
__global__ void k_seg_gather(int n, int64_t cap, const int32_t *__restrict__ cellmap,
                             const T *__restrict__ sums, T *__restrict__ rho) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= int64_t(n) * n * n) return;
  const int i = int(t & (n - 1)), j = int((t / n) & (n - 1)), k = int(t / (int64_t(n) * n));
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int32_t s = cellmap[grid_at(n, i - (c & 1), j - ((c >> 1) & 1), k - (c >> 2))];
    if (s >= 0) acc += sums[c * cap + s];
  }
  rho[t] = acc;
}

// ---------------------------------------------------------------------------
// host <-> device helpers of the particle handle
// ---------------------------------------------------------------------------
// the entry past the digit table: 0, so that its exclusive scan ends with np
__global__ void k_table_end(uint32_t *table, int64_t at) { table[at] = 0u; }

template <class T>
__global__ void k_from_double(int64_t n, const double *__restrict__ a, T *__restrict__ b) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) b[t] = T(a[t]);
}

template <class T>
__global__ void k_to_double(int64_t n, const T *__restrict__ a, double *__restrict__ b) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) b[t] = double(a[t]);
}

__global__ void k_iota(int64_t n, uint32_t *id) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) id[t] = uint32_t(t);
}

}  // namespace
}  // namespace amr
