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

// Grid of the deposition: n = 2^bits cells per axis; fn = n in the state type.
template <class T>
struct CicGrid {
  int n, bits;
  T fn, scale;  // scale = n^3 (mass -> density), exact
};

// floor(x 2^k) for a double 0 <= x < 1, from its bits on the integer pipe
// (GB300 runs FP64 at 1/64 of the FP32 rate, so the deposition keeps its
// FP64 instruction count low).  Out-of-range inputs give some value that the
// callers mask into the grid.
__device__ __forceinline__ int floor_scaled(double x, int k) {
  const uint64_t u = uint64_t(__double_as_longlong(x));
  const int E = int(u >> 52) & 0x7FF;
  const uint64_t M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = 1075 - E - k;
  if (E == 0 || sh >= 64) return 0;
  if (sh <= 0) return 0x7FFFFFFF;
  return int(M >> sh);
}

// (2 i + 1) / 2 as a double, built on the integer pipe (|2 i + 1| < 2^31)
__device__ __forceinline__ double half_odd(int i) {
  const int k = 2 * i + 1;
  const uint32_t a = uint32_t(k < 0 ? -k : k);
  const int lz = __clz(a);
  const int e = 31 - lz;                              // a = 1.frac 2^e
  const uint32_t frac = e ? (a << (lz + 1)) : 0u;     // bits below the leading one, left aligned
  const uint32_t hi = (uint32_t(k < 0) << 31) | (uint32_t(1022 + e) << 20) | (frac >> 12);
  return __hiloint2double(int(hi), int(frac << 20));
}

// source cell along one axis: floor(x n - 1/2), unmasked
template <class T>
__device__ __forceinline__ int cic_cell(T x, const CicGrid<T> &g) {
  return int(floor(x * g.fn - T(0.5)));
}
template <>
__device__ __forceinline__ int cic_cell<double>(double x, const CicGrid<double> &g) {
  // floor(x n - 1/2) = floor((floor(2 x n) - 1) / 2)
  return (floor_scaled(x, g.bits + 1) - 1) >> 1;
}

// source cell (masked into the grid) and weights along one axis:
// s = x n - 1/2, i0 = floor(s), w1 = f = s - i0, w0 = 1 - f
template <class T>
__device__ __forceinline__ int cic_axis(T x, const CicGrid<T> &g, T &w0, T &w1) {
  const T s = x * g.fn - T(0.5);
  const T fl = floor(s);
  w1 = s - fl;
  w0 = T(1) - w1;
  return int(fl) & (g.n - 1);
}
template <>
__device__ __forceinline__ int cic_axis<double>(double x, const CicGrid<double> &g, double &w0,
                                                double &w1) {
  // x n and x n - 1/2 - i0 are exact, so one FMA gives the same f as
  // (x n - 1/2) - floor(x n - 1/2)
  const int i0 = cic_cell(x, g);
  w1 = fma(x, g.fn, -half_odd(i0));
  w0 = 1.0 - w1;
  return i0 & (g.n - 1);
}

__device__ __forceinline__ uint32_t grid_at(int n, int i, int j, int k) {
  const int m = n - 1;
  return uint32_t(i & m) + uint32_t(n) * (uint32_t(j & m) + uint32_t(n) * uint32_t(k & m));
}

// the 8 contributions ((m n^3 wx) wy) wz of one particle, corner
// c = cx + 2 cy + 4 cz; (i, j, k) its source cell
template <class T>
__device__ __forceinline__ void cic_weights(T x, T y, T z, T m, const CicGrid<T> &g, int &i, int &j,
                                            int &k, T w[8]) {
  T wx[2], wy[2], wz[2];
  i = cic_axis(x, g, wx[0], wx[1]);
  j = cic_axis(y, g, wy[0], wy[1]);
  k = cic_axis(z, g, wz[0], wz[1]);
  const T ms = m * g.scale;
  T a[2], b[4];
#pragma unroll
  for (int cx = 0; cx < 2; ++cx) a[cx] = ms * wx[cx];
#pragma unroll
  for (int q = 0; q < 4; ++q) b[q] = a[q & 1] * wy[q >> 1];
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = b[c & 3] * wz[c >> 2];
}

// Sums of the lanes' w over runs of lanes (`runs`: bit L set where a run
// starts at lane L; bit 0 always set): a backward segmented scan that leaves
// each run's total in its first lane.  The tree depends only on the run
// lengths, so equal inputs give equal sums.
template <class T>
__device__ __forceinline__ void warp_run_sums(T w[8], unsigned runs, unsigned lane) {
  const unsigned above = runs & ~((2u << lane) - 1u);  // run starts after this lane
  const unsigned next = above ? unsigned(__ffs(above) - 1) : 32u;
  const unsigned len = ((runs >> lane) & 1u) ? next - lane : 0u;
  const unsigned maxrun = __reduce_max_sync(0xFFFFFFFFu, len);
  for (unsigned off = 1; off < maxrun; off <<= 1) {
    const bool take = lane + off < next;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const T o = __shfl_down_sync(0xFFFFFFFFu, w[c], off);
      if (take) w[c] += o;
    }
  }
}

// The 8 sums over all 32 lanes, reduce-scatter style (9 additions per lane
// instead of 40): afterwards lane L holds the total of component L >> 2.
template <class T>
__device__ __forceinline__ T warp_total_scatter(const T w[8], unsigned lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  T h[4], q[2];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const T send = b4 ? w[c] : w[c + 4];
    const T keep = b4 ? w[c + 4] : w[c];
    h[c] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T send = b3 ? h[c] : h[c + 2];
    const T keep = b3 ? h[c + 2] : h[c];
    q[c] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
  }
  T v = (b2 ? q[1] : q[0]) + __shfl_xor_sync(0xFFFFFFFFu, b2 ? q[0] : q[1], 4);
  v += __shfl_xor_sync(0xFFFFFFFFu, v, 2);
  v += __shfl_xor_sync(0xFFFFFFFFu, v, 1);
  return v;
}

// ---------------------------------------------------------------------------
// sort
// ---------------------------------------------------------------------------
// 3-D Hilbert index of (x, y, z) < 2^BITS (BITS <= 10), x most significant:
// the same curve as hilbert_index (Skilling's transposed construction),
// unrolled and branch-free: the conditional exchanges become masks, the
// Gray-code step a suffix XOR, and the bit interleave magic-number spreads.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  return (v | (v << 2)) & 0x09249249u;
}

template <int BITS>
__device__ __forceinline__ uint32_t hilbert_index_u32(uint32_t a0, uint32_t a1, uint32_t a2) {
#pragma unroll
  for (int b = BITS - 1; b >= 1; --b) {
    const uint32_t m = (1u << b) - 1u;
    a0 ^= (0u - ((a0 >> b) & 1u)) & m;
    const uint32_t s1 = 0u - ((a1 >> b) & 1u);
    const uint32_t t1 = (a0 ^ a1) & m & ~s1;
    a0 ^= (m & s1) | t1;
    a1 ^= t1;
    const uint32_t s2 = 0u - ((a2 >> b) & 1u);
    const uint32_t t2 = (a0 ^ a2) & m & ~s2;
    a0 ^= (m & s2) | t2;
    a2 ^= t2;
  }
  a1 ^= a0;
  a2 ^= a1;
  uint32_t g = a2 >> 1;  // g_i = XOR of the bits of a2 above i
  g ^= g >> 1;
  g ^= g >> 2;
  g ^= g >> 4;
  g ^= g >> 8;
  a0 ^= g;
  a1 ^= g;
  a2 ^= g;
  return (spread3(a0) << 2) | (spread3(a1) << 1) | spread3(a2);
}

template <class T, int BITS>
__global__ void k_part_keys(int64_t np, CicGrid<T> g, const T *__restrict__ x, const T *__restrict__ y,
                            const T *__restrict__ z, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ val) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= np) return;
  const uint32_t m = uint32_t(g.n - 1);
  const uint32_t i = uint32_t(cic_cell(x[t], g)) & m, j = uint32_t(cic_cell(y[t], g)) & m,
                 k = uint32_t(cic_cell(z[t], g)) & m;
  key[t] = hilbert_index_u32<BITS>(i, j, k);
  val[t] = uint32_t(t);
}

// per-tile digit counts, tile-major: table[tile * ndig + d]; digits of up to 8 bits
constexpr int kSortBins = 256;

__global__ void __launch_bounds__(kSortThreads) k_psort_hist(const uint32_t *__restrict__ keys,
                                                             int64_t np, int shift, int nbits,
                                                             uint32_t *__restrict__ table,
                                                             int64_t ntiles) {
  __shared__ uint32_t hist[kSortBins];
  const int ndig = 1 << nbits;
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * int64_t(kSortTile);
  unsigned dk[kSortRounds];  // all loads of the tile in flight at once
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t t = base + r * kSortThreads + threadIdx.x;
    dk[r] = t < np ? __ldcs(keys + t) : 0xFFFFFFFFu;
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r)
    if (dk[r] != 0xFFFFFFFFu) atomicAdd(&hist[(dk[r] >> shift) & unsigned(ndig - 1)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) table[int64_t(blockIdx.x) * ndig + d] = hist[d];
}

// Offsets of the scatter from the tile-major counts cnt[tile][d]: per digit,
// an exclusive prefix over tiles inside chunks of kScanChunk tiles (pref),
// then the chunks' exclusive prefix per digit (base[chunk][d]), then the
// digits' bases (dbase[d]); a tile's run of digit d starts at
// pref[tile][d] + base[tile / kScanChunk][d] + dbase[d].  The counts, the
// prefixes and the scatter's reads all run along the digits (coalesced).
constexpr int kScanChunk = 32;

__global__ void k_psort_chunks(const uint32_t *__restrict__ cnt, int64_t ntiles, int ndig,
                               uint32_t *__restrict__ pref, uint32_t *__restrict__ base) {
  const int d = threadIdx.x;
  if (d >= ndig) return;
  const int64_t t0 = blockIdx.x * int64_t(kScanChunk);
  const int64_t t1 = t0 + kScanChunk < ntiles ? t0 + kScanChunk : ntiles;
  uint32_t run = 0;
  for (int64_t t = t0; t < t1; ++t) {
    const uint32_t c = cnt[t * ndig + d];
    pref[t * ndig + d] = run;
    run += c;
  }
  base[int64_t(blockIdx.x) * ndig + d] = run;  // the chunk's total, for now
}

// one block per digit: exclusive scan of the digit's chunk totals (in place)
// and the digit's total
__global__ void __launch_bounds__(kSortThreads) k_psort_digit_scan(uint32_t *__restrict__ base, int64_t nchunks,
                                                                  int ndig, uint32_t *__restrict__ dtot) {
  __shared__ uint32_t part[kSortThreads];
  const int d = blockIdx.x;
  const int64_t per = (nchunks + kSortThreads - 1) / kSortThreads;
  const int64_t c0 = threadIdx.x * per, c1 = c0 + per < nchunks ? c0 + per : nchunks;
  uint32_t sum = 0;
  for (int64_t c = c0; c < c1; ++c) sum += base[c * ndig + d];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < kSortThreads; off <<= 1) {
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (int64_t c = c0; c < c1; ++c) {
    const uint32_t x = base[c * ndig + d];
    base[c * ndig + d] = run;
    run += x;
  }
  if (threadIdx.x == kSortThreads - 1) dtot[d] = part[kSortThreads - 1];
}

// one block: the digits' bases, the exclusive scan of their totals (in place)
__global__ void __launch_bounds__(kSortThreads) k_psort_digit_base(uint32_t *__restrict__ dtot, int ndig) {
  __shared__ uint32_t part[kSortThreads];
  const int d = threadIdx.x;
  const uint32_t x = d < ndig ? dtot[d] : 0u;
  part[d] = x;
  __syncthreads();
  for (int off = 1; off < kSortThreads; off <<= 1) {
    const uint32_t v = d >= off ? part[d - off] : 0u;
    __syncthreads();
    part[d] += v;
    __syncthreads();
  }
  if (d < ndig) dtot[d] = part[d] - x;
}

// stable scatter of one tile: ranks in item order (rounds, then warps, then
// lanes), the tile staged in shared memory in digit order, then written out
// so that consecutive threads write consecutive places of a digit's run.
__global__ void __launch_bounds__(kSortThreads) k_psort_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t np, int shift, int nbits, const uint32_t *__restrict__ cnt,
    const uint32_t *__restrict__ pref, const uint32_t *__restrict__ cbase, const uint32_t *__restrict__ dbase) {
  __shared__ uint32_t skey[kSortTile], sval[kSortTile];
  __shared__ uint32_t wcnt[kSortThreads / 32][256], wpre[kSortThreads / 32][256];
  __shared__ uint32_t lstart[256], run[256], part[kSortThreads];
  const int ndig = 1 << nbits;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = blockIdx.x * int64_t(kSortTile);
  const int nt = int(np - base < kSortTile ? np - base : kSortTile);
  // digit counts and global offsets of this tile, then the counts'
  // exclusive scan over the digits (one digit per thread; ndig <= 256)
  __shared__ uint32_t goff[256];
  const int d0 = threadIdx.x;
  uint32_t cnt_d = 0;
  if (d0 < ndig) {
    const int64_t e = int64_t(blockIdx.x) * ndig + d0;
    cnt_d = cnt[e];
    goff[d0] = pref[e] + cbase[int64_t(blockIdx.x / kScanChunk) * ndig + d0] + dbase[d0];
  }
  part[threadIdx.x] = cnt_d;
  for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
  __syncthreads();
  for (int off = 1; off < kSortThreads; off <<= 1) {
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  lstart[threadIdx.x] = part[threadIdx.x] - cnt_d;
  run[threadIdx.x] = part[threadIdx.x] - cnt_d;
  uint32_t kr[kSortRounds], vr[kSortRounds];  // all loads of the tile in flight at once
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int q = r * kSortThreads + threadIdx.x;
    kr[r] = q < nt ? __ldcs(kin + base + q) : 0u;
    vr[r] = q < nt ? __ldcs(vin + base + q) : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int q = r * kSortThreads + threadIdx.x;
    const bool valid = q < nt;
    const uint32_t k = kr[r];
    const uint32_t v = vr[r];
    const unsigned dig = valid ? (k >> shift) & unsigned(ndig - 1) : 0xFFFFFFFFu;
    const unsigned peers = digit_peers(dig, nbits, valid);
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
    const int64_t dst = int64_t(goff[dig]) + (q - int64_t(lstart[dig]));
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
__global__ void __launch_bounds__(256) k_cic_atomic(int64_t np, CicGrid<T> g, const T *__restrict__ x,
                                                    const T *__restrict__ y, const T *__restrict__ z,
                                                    const T *__restrict__ m, T *__restrict__ rho) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  const bool valid = t < np;
  T w[8];
  int i = 0, j = 0, k = 0;
  uint32_t cell = 0xFFFFFFFFu;
  if (valid) {
    cic_weights(x[t], y[t], z[t], m[t], g, i, j, k, w);
    cell = grid_at(g.n, i, j, k);
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) w[c] = T(0);
  }
  // runs of equal source cells among the warp's lanes
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, cell, 1);
  const unsigned runs = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != cell);
  if (runs == 1u) {
    // one source cell for the whole warp (or no particle at all): lanes
    // 0, 4, .., 28 add one component each
    if (cell == 0xFFFFFFFFu) return;
    const T v = warp_total_scatter(w, lane);
    if ((lane & 3) == 0) {
      const int c = int(lane >> 2);
      atomicAdd(&rho[grid_at(g.n, i + (c & 1), j + ((c >> 1) & 1), k + (c >> 2))], v);
    }
    return;
  }
  // Partial runs: FP32 sums them before its atomics; FP64, whose additions
  // cost 1/64 of the FP32 rate on GB300, lets every particle add its own 8
  // contributions (L2 absorbs the extra atomics).
  const bool combine = sizeof(T) == 4;
  if (combine && runs != 0xFFFFFFFFu) warp_run_sums(w, runs, lane);
  if (valid && (!combine || ((runs >> lane) & 1u))) {
#pragma unroll
    for (int c = 0; c < 8; ++c) atomicAdd(&rho[grid_at(g.n, i + (c & 1), j + ((c >> 1) & 1), k + (c >> 2))], w[c]);
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

// Per particle, in aligned groups of 32 (one warp each): the contributions
// summed over each run of equal source cells inside the group (fixed shuffle
// tree).  A run that starts segment s writes its sums to sums[c * cap + s]
// and maps its source cell to s; the run at the start of group G that
// continues a segment from earlier groups writes them to carry[c * ngroups + G].
template <class T>
__global__ void __launch_bounds__(256) k_seg_partial(int64_t np, CicGrid<T> g, const uint32_t *__restrict__ key,
                                                     const uint32_t *__restrict__ scan, const T *__restrict__ x,
                                                     const T *__restrict__ y, const T *__restrict__ z,
                                                     const T *__restrict__ m, int64_t cap, int64_t ngroups,
                                                     T *__restrict__ sums, T *__restrict__ carry,
                                                     int32_t *__restrict__ cellmap) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  const bool valid = t < np;
  T w[8];
  int i = 0, j = 0, k = 0;
  uint32_t kk = 0xFFFFFFFFu;
  bool head = false;
  if (valid) {
    cic_weights(x[t], y[t], z[t], m[t], g, i, j, k, w);
    kk = key[t];
    head = t == 0 || key[t - 1] != kk;
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) w[c] = T(0);
  }
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, kk, 1);
  const unsigned runs = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != kk);
  if (runs == 1u) {
    // the whole group is one run: reduce-scatter, lane 4c writes component c
    if (kk == 0xFFFFFFFFu) return;
    const T v = warp_total_scatter(w, lane);
    const bool head0 = __shfl_sync(0xFFFFFFFFu, head, 0);
    if ((lane & 3) == 0) {
      const int c = int(lane >> 2);
      if (head0)
        sums[c * cap + int64_t(scan[t - lane])] = v;
      else
        carry[c * ngroups + (t >> 5)] = v;
    }
    if (lane == 0 && head0) cellmap[grid_at(g.n, i, j, k)] = int32_t(scan[t]);
    return;
  }
  if (runs != 0xFFFFFFFFu) warp_run_sums(w, runs, lane);
  if (!valid) return;
  if (head) {
    const int64_t s = scan[t];
#pragma unroll
    for (int c = 0; c < 8; ++c) sums[c * cap + s] = w[c];
    cellmap[grid_at(g.n, i, j, k)] = int32_t(s);
  } else if (lane == 0) {
    const int64_t G = t >> 5;
#pragma unroll
    for (int c = 0; c < 8; ++c) carry[c * ngroups + G] = w[c];
  }
}

// Per segment that spans groups: add the carries of its later groups, in
// group order.
template <class T>
__global__ void k_seg_carry(const uint32_t *__restrict__ nseg, const uint32_t *__restrict__ start, int64_t cap,
                            int64_t ngroups, const T *__restrict__ carry, T *__restrict__ sums) {
  const int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (s >= int64_t(*nseg)) return;
  const int64_t g0 = int64_t(start[s]) >> 5, g1 = (int64_t(start[s + 1]) - 1) >> 5;
  if (g1 == g0) return;
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = sums[c * cap + s];
  for (int64_t G = g0 + 1; G <= g1; ++G) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += carry[c * ngroups + G];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) sums[c * cap + s] = acc[c];
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
