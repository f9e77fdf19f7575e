// mg_kernels.cuh -- multigrid Poisson V-cycles on the periodic base level
// (paper Sec. 5, self-gravity).
//
//   (sum of the 6 neighbours - 6 phi) / dx^2 = fourpiG (rho - mean rho)
//
// Smoother: red-black Gauss-Seidel, colour = parity of x + y + z (the parity
// of the cell's index inside its oct).  Restriction: the residuals of the 8
// children, averaged into the coarse source.  Prolongation: trilinear, weights
// (1, 3, 3, 9, 3, 9, 9, 27)/64.  Hierarchy: the same periodic box at half the
// resolution per level, down to 2^3 cells, smoothed 8 times there.
//
// The base level lives in the mesh's oct order; the solver works on dense
// arrays [x + n (y + n z)] of every multigrid level (unit-stride x, so every
// stencil access is coalesced), gathered from and scattered back to the octs.
// On GB300 the FP64 pipe bounds these stencils (about 8 FP64 operations per
// cell against 16 bytes of traffic); no step divides: the Gauss-Seidel update
// multiplies by the rounded 1/6 where the operator divides by 6 (the two differ
// by at most a few units in the last place per update), and the residual
// multiplies by 1/dx^2, which is exact (dx is a power of two).
#pragma once
#include "amr_internal.cuh"

namespace amr {

__device__ __forceinline__ int64_t mg_at(int n, int x, int y, int z) {
  const int m = n - 1;  // n is a power of two: periodic wrap by masking
  return int64_t(x & m) + int64_t(n) * (int64_t(y & m) + int64_t(n) * int64_t(z & m));
}

__device__ __forceinline__ double mg_nbsum(int n, const double *__restrict__ p, int x, int y, int z) {
  return ((p[mg_at(n, x - 1, y, z)] + p[mg_at(n, x + 1, y, z)]) +
          (p[mg_at(n, x, y - 1, z)] + p[mg_at(n, x, y + 1, z)])) +
         (p[mg_at(n, x, y, z - 1)] + p[mg_at(n, x, y, z + 1)]);
}

// base-level density (oct order) into the dense array; one thread per cell
template <class T>
__global__ void k_mg_gather(const T *__restrict__ U, const uint64_t *__restrict__ key, int lo,
                            int nl, int n, double *__restrict__ rho) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= 8 * int64_t(nl)) return;
  const int o = lo + int(g >> 3), c = int(g & 7);
  const uint64_t k = key[o];
  const int x = 2 * int(ikey_x(k)) + (c & 1), y = 2 * int(ikey_y(k)) + ((c >> 1) & 1),
            z = 2 * int(ikey_z(k)) + ((c >> 2) & 1);
  rho[mg_at(n, x, y, z)] = double(U[8 * int64_t(o) + c]);
}

// block sums of a[0..m) into part[blockIdx.x] (warp shuffles, then shared
// memory); squared when sq
__global__ void k_mg_sum(const double *__restrict__ a, int64_t m, int sq, double *__restrict__ part) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < m; t += int64_t(gridDim.x) * blockDim.x)
    s += sq ? a[t] * a[t] : a[t];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// out = scale * (sum of the partial sums); one thread
__global__ void k_mg_total(const double *__restrict__ part, int nparts, double scale,
                           double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += part[q];
  *out = s * scale;
}

// f = fourpiG (rho - mean)
__global__ void k_mg_source(const double *__restrict__ rho, int64_t m, const double *__restrict__ mean,
                            double fourpiG, double *__restrict__ f) {
  const double mu = *mean;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < m; t += int64_t(gridDim.x) * blockDim.x)
    f[t] = fourpiG * (rho[t] - mu);
}

// one colour of a red-black sweep: thread t -> (x, y, z) with x + y + z of
// the colour's parity
__global__ void k_mg_smooth(int n, double dx2, const double *__restrict__ f, double *p, int colour) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t half = int64_t(n) * n * n / 2;
  if (t >= half) return;
  const int h = n >> 1;
  const int xh = int(t % h);
  const int64_t yz = t / h;
  const int y = int(yz % n), z = int(yz / n);
  const int x = 2 * xh + ((y + z + colour) & 1);
  const int64_t i = mg_at(n, x, y, z);
  p[i] = (mg_nbsum(n, p, x, y, z) - dx2 * f[i]) * (1.0 / 6.0);
}

// coarse source = mean of the 8 children's residuals; coarse correction = 0
__global__ void k_mg_restrict(int n, double inv_dx2, const double *__restrict__ f,
                              const double *__restrict__ p, double *__restrict__ fc, double *__restrict__ ec) {
  const int h = n >> 1;
  const int64_t T = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (T >= int64_t(h) * h * h) return;
  const int X = int(T % h), Y = int((T / h) % h), Z = int(T / (int64_t(h) * h));
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int x = 2 * X + (c & 1), y = 2 * Y + ((c >> 1) & 1), z = 2 * Z + ((c >> 2) & 1);
    const int64_t i = mg_at(n, x, y, z);
    s += f[i] - (mg_nbsum(n, p, x, y, z) - 6.0 * p[i]) * inv_dx2;
  }
  fc[T] = s * 0.125;
  ec[T] = 0.0;
}

// phi += trilinear prolongation of the coarse correction
__global__ void k_mg_prolong(int n, const double *__restrict__ ec, double *__restrict__ p) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= int64_t(n) * n * n) return;
  const int h = n >> 1;
  const int x = int(t % n), y = int((t / n) % n), z = int(t / (int64_t(n) * n));
  const int X = x >> 1, Y = y >> 1, Z = z >> 1;
  const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
  double v = 27.0 * ec[mg_at(h, X, Y, Z)];
  v += 9.0 * ((ec[mg_at(h, X + sx, Y, Z)] + ec[mg_at(h, X, Y + sy, Z)]) + ec[mg_at(h, X, Y, Z + sz)]);
  v += 3.0 * ((ec[mg_at(h, X + sx, Y + sy, Z)] + ec[mg_at(h, X + sx, Y, Z + sz)]) +
              ec[mg_at(h, X, Y + sy, Z + sz)]);
  v += ec[mg_at(h, X + sx, Y + sy, Z + sz)];
  p[t] += v / 64.0;
}

// the 2^3 grid: `sweeps` red-black sweeps by one block of 8 threads
__global__ void k_mg_coarsest(double dx2, const double *__restrict__ f, double *p, int sweeps) {
  const int t = threadIdx.x;  // 0..7: (x, y, z) = bits of t
  const int x = t & 1, y = (t >> 1) & 1, z = (t >> 2) & 1;
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      if (((x + y + z) & 1) == colour) {
        const int64_t i = mg_at(2, x, y, z);
        p[i] = (mg_nbsum(2, p, x, y, z) - dx2 * f[i]) * (1.0 / 6.0);
      }
      __syncthreads();
    }
}

// residual of the base level into r (for its L2 norm)
__global__ void k_mg_residual(int n, double inv_dx2, const double *__restrict__ f,
                              const double *__restrict__ p, double *__restrict__ r) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= int64_t(n) * n * n) return;
  const int x = int(t % n), y = int((t / n) % n), z = int(t / (int64_t(n) * n));
  r[t] = f[t] - (mg_nbsum(n, p, x, y, z) - 6.0 * p[t]) * inv_dx2;
}

// sqrt of the sum of the partial sums into out
__global__ void k_mg_norm(const double *__restrict__ part, int nparts, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += part[q];
  *out = sqrt(s);
}

// phi - mean into the octs' cells (mesh order)
__global__ void k_mg_scatter(const double *__restrict__ p, const uint64_t *__restrict__ key, int lo,
                             int nl, int n, const double *__restrict__ mean,
                             double *__restrict__ phi_cells) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= 8 * int64_t(nl)) return;
  const int o = lo + int(g >> 3), c = int(g & 7);
  const uint64_t k = key[o];
  const int x = 2 * int(ikey_x(k)) + (c & 1), y = 2 * int(ikey_y(k)) + ((c >> 1) & 1),
            z = 2 * int(ikey_z(k)) + ((c >> 2) & 1);
  phi_cells[g] = p[mg_at(n, x, y, z)] - *mean;
}

// ---------------------------------------------------------------------------
// Poisson on a refined level (Sec. 5, level by level): flat tables over the
// cells of each MG level (level 0: the level's cells; level k: their
// ancestors at level L-k), built on the host once per (member, level).
// Every operation is rounded as written (no contraction), in the order of the
// plain definition, so the potential equals that of a sequential evaluation
// bit for bit.
//   nb[6][n]   face neighbour in the same MG level (-x,+x,-y,+y,-z,+z) or -1
//   nbnd[n]    faces to the outside (Dirichlet): the diagonal is -(6 + nbnd)
//   bsum[n]    2 sum of the faces' boundary values (MG level 0; 0 above)
//   child[8][n]   children in the MG level below (order cx, cy, cz with cz
//                 fastest) or -1; pro[8][n] the 8 coarse cells of a cell's
//                 trilinear stencil (a, b, d: 4 a + 2 b + d) or -1
// ---------------------------------------------------------------------------
__global__ void k_mgl_bsum(int64_t n, const int32_t *__restrict__ fatherg, const int32_t *__restrict__ acrossg,
                           const double *__restrict__ phil, double *__restrict__ bsum) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const double pf = phil[fatherg[t]];
  double bs = 0.0;
  for (int k = 0; k < 6; ++k) {
    const int32_t q = acrossg[k * n + t];
    if (q >= 0) bs = __dadd_rn(bs, __dmul_rn(2.0, __dmul_rn(0.5, __dadd_rn(pf, phil[q]))));
  }
  bsum[t] = bs;
}

// source fourpiG (rho - rho_bar); rho_bar from the device when rho_bar_dev is
// set (the base level's mean, without a host round trip)
template <class T>
__global__ void k_mgl_source(int64_t n, const int32_t *__restrict__ g0, const T *__restrict__ rho, double fourpiG,
                             double rho_bar, const double *__restrict__ rho_bar_dev, double *__restrict__ f) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const double rb = rho_bar_dev ? *rho_bar_dev : rho_bar;
  f[t] = __dmul_rn(fourpiG, __dsub_rn(double(rho[g0[t]]), rb));
}

__global__ void k_mgl_gather(int64_t n, const int32_t *__restrict__ g0, const double *__restrict__ phil,
                             double *__restrict__ e) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) e[t] = phil[g0[t]];
}

__global__ void k_mgl_scatter(int64_t n, const int32_t *__restrict__ g0, const double *__restrict__ e,
                              double *__restrict__ phil) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) phil[g0[t]] = e[t];
}

__device__ __forceinline__ double mgl_nbsum(int64_t n, const int32_t *__restrict__ nb, const double *e, int64_t t) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int32_t q = nb[k * n + t];
    if (q >= 0) s = __dadd_rn(s, e[q]);
  }
  return s;
}

// one colour of a red-black sweep: the cells of list[0..m)
__global__ void k_mgl_smooth(int64_t n, const int32_t *__restrict__ list, int64_t m, const int32_t *__restrict__ nb,
                             const int32_t *__restrict__ nbnd, const double *__restrict__ bsum,
                             const double *__restrict__ f, double *e, double dx2) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= m) return;
  const int64_t t = list[i];
  const double s = mgl_nbsum(n, nb, e, t);
  const double bs = bsum ? bsum[t] : 0.0;
  e[t] = __ddiv_rn(__dsub_rn(__dadd_rn(s, bs), __dmul_rn(dx2, f[t])), double(6 + nbnd[t]));
}

__global__ void k_mgl_residual(int64_t n, const int32_t *__restrict__ nb, const int32_t *__restrict__ nbnd,
                               const double *__restrict__ bsum, const double *__restrict__ f,
                               const double *__restrict__ e, double dx2, double *__restrict__ r) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const double s = mgl_nbsum(n, nb, e, t);
  const double bs = bsum ? bsum[t] : 0.0;
  r[t] = __dsub_rn(f[t], __ddiv_rn(__dsub_rn(__dadd_rn(s, bs), __dmul_rn(double(6 + nbnd[t]), e[t])), dx2));
}

// coarse source = the children's residuals summed over 8; correction zeroed
__global__ void k_mgl_restrict(int64_t nc, const int32_t *__restrict__ child, const double *__restrict__ r,
                               double *__restrict__ fc, double *__restrict__ ec) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nc) return;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int32_t q = child[j * nc + t];
    if (q >= 0) s = __dadd_rn(s, r[q]);
  }
  fc[t] = __ddiv_rn(s, 8.0);
  ec[t] = 0.0;
}

__global__ void k_mgl_prolong(int64_t nf, const int32_t *__restrict__ pro, const double *__restrict__ ec,
                              double *__restrict__ e) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nf) return;
  double c[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int32_t q = pro[j * nf + t];
    c[j] = q >= 0 ? ec[q] : 0.0;
  }
  // c[4 a + 2 b + d]: a along x, b along y, d along z
  double v = __dmul_rn(27.0, c[0]);
  v = __dadd_rn(v, __dmul_rn(9.0, __dadd_rn(__dadd_rn(c[4], c[2]), c[1])));
  v = __dadd_rn(v, __dmul_rn(3.0, __dadd_rn(__dadd_rn(c[6], c[5]), c[3])));
  v = __dadd_rn(v, c[7]);
  e[t] = __dadd_rn(e[t], __ddiv_rn(v, 64.0));
}

// sum of r^2 into one value per block (for the residual norm)
__global__ void k_mgl_sq(int64_t n, const double *__restrict__ r, double *__restrict__ part) {
  __shared__ double ws[8];
  double s = 0.0;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x)
    s += r[t] * r[t];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) b += ws[w];
    part[blockIdx.x] = b;
  }
}

__global__ void k_mgl_norm(const double *__restrict__ part, int nparts, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += part[b];
  *out = sqrt(s);
}

// ---------------------------------------------------------------------------
// the tables of a refined level's hierarchy, built on the device: cells are
// keyed by (x << 2b) | (y << b) | z with b bits per axis (lexicographic in
// x, y, z, the sorted order of every table); neighbours, children and
// prolongation stencils are found by binary search in the sorted keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mgl_key(int64_t x, int64_t y, int64_t z, int b) {
  return (uint64_t(x) << (2 * b)) | (uint64_t(y) << b) | uint64_t(z);
}
__device__ __forceinline__ void mgl_unkey(uint64_t k, int b, int64_t &x, int64_t &y, int64_t &z) {
  const uint64_t m = (uint64_t(1) << b) - 1;
  x = int64_t(k >> (2 * b));
  y = int64_t((k >> b) & m);
  z = int64_t(k & m);
}
// index of key c in the sorted keys[0..n), or -1 (at most log2(n) + 1 steps)
__device__ __forceinline__ int32_t mgl_find(const uint64_t *__restrict__ keys, int64_t n, uint64_t c) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < c) lo = mid + 1; else hi = mid;
  }
  return (lo < n && keys[lo] == c) ? int32_t(lo) : -1;
}

// the cells of the level-L octs [lo, lo + nl): key and global cell index
__global__ void k_mgl_cells(const uint64_t *__restrict__ key, int lo, int64_t nl, int L, uint64_t *__restrict__ ck,
                            uint32_t *__restrict__ cv) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= 8 * nl) return;
  const int o = lo + int(t >> 3), c = int(t & 7);
  const uint64_t k = key[o];
  ck[t] = mgl_key(2 * int64_t(ikey_x(k)) + (c & 1), 2 * int64_t(ikey_y(k)) + ((c >> 1) & 1),
                  2 * int64_t(ikey_z(k)) + ((c >> 2) & 1), L);
  cv[t] = uint32_t(8 * int64_t(o) + c);
}

// parent keys (b bits per axis) of sorted child keys (b + 1 bits)
__global__ void k_mgl_parents(const uint64_t *__restrict__ ck, int64_t n, int b, uint64_t *__restrict__ pk,
                              uint32_t *__restrict__ pv) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  int64_t x, y, z;
  mgl_unkey(ck[t], b + 1, x, y, z);
  pk[t] = mgl_key(x >> 1, y >> 1, z >> 1, b);
  pv[t] = uint32_t(t);
}

// head flags of runs of equal keys in a sorted array
__global__ void k_mgl_heads(const uint64_t *__restrict__ k, int64_t n, uint32_t *__restrict__ head) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) head[t] = (t == 0 || k[t] != k[t - 1]) ? 1u : 0u;
}

// the unique keys (pos = exclusive scan of head) and their count
__global__ void k_mgl_unique(const uint64_t *__restrict__ k, const uint32_t *__restrict__ head,
                             const uint32_t *__restrict__ pos, int64_t n, uint64_t *__restrict__ out,
                             int64_t *__restrict__ count) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  if (head[t]) out[pos[t]] = k[t];
  if (t == n - 1) *count = int64_t(pos[t] + head[t]);
}

// the six face neighbours in the MG level (-1 outside it), the count of
// faces to the outside, and the even-colour flag (parity of x + y + z)
__global__ void k_mgl_faces(const uint64_t *__restrict__ keys, int64_t n, int b, int32_t *__restrict__ nb,
                            int32_t *__restrict__ nbnd, uint32_t *__restrict__ even) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  int64_t x, y, z;
  mgl_unkey(keys[t], b, x, y, z);
  const int64_t m = (int64_t(1) << b) - 1;
  int nout = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const int64_t dd = sg ? 1 : -1;
      const int32_t q = mgl_find(keys, n, mgl_key((x + (d == 0) * dd) & m, (y + (d == 1) * dd) & m,
                                                  (z + (d == 2) * dd) & m, b));
      nb[(2 * d + sg) * n + t] = q;
      nout += q < 0;
    }
  nbnd[t] = nout;
  even[t] = ((x + y + z) & 1) ? 0u : 1u;
}

// colour lists: even cells first, then odd, each in key order (pos = the
// exclusive scan of even; nc0 = the number of even cells)
__global__ void k_mgl_colours(const uint32_t *__restrict__ even, const uint32_t *__restrict__ pos, int64_t n,
                              int32_t *__restrict__ col, int64_t *__restrict__ nc0) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const int64_t n0 = int64_t(pos[n - 1] + even[n - 1]);
  col[even[t] ? int64_t(pos[t]) : n0 + (t - int64_t(pos[t]))] = int32_t(t);
  if (t == 0) *nc0 = n0;
}

// children of coarse cell t (b bits) in the finer MG level (b + 1 bits),
// order (cx, cy, cz) with cz fastest
__global__ void k_mgl_children(const uint64_t *__restrict__ keys, int64_t n, int b,
                               const uint64_t *__restrict__ fkeys, int64_t nf, int32_t *__restrict__ child) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  int64_t x, y, z;
  mgl_unkey(keys[t], b, x, y, z);
  int j = 0;
  for (int cx = 0; cx < 2; ++cx)
    for (int cy = 0; cy < 2; ++cy)
      for (int cz = 0; cz < 2; ++cz, ++j)
        child[j * n + t] = mgl_find(fkeys, nf, mgl_key(2 * x + cx, 2 * y + cy, 2 * z + cz, b + 1));
}

// trilinear stencil of fine cell t (b + 1 bits) in the coarse MG level (b
// bits): entry 4a + 2b' + d for the coarse cells (X + a sx, Y + b' sy, Z + d sz)
__global__ void k_mgl_stencils(const uint64_t *__restrict__ fkeys, int64_t nf, int b,
                               const uint64_t *__restrict__ keys, int64_t n, int32_t *__restrict__ pro) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nf) return;
  int64_t x, y, z;
  mgl_unkey(fkeys[t], b + 1, x, y, z);
  const int64_t X = x >> 1, Y = y >> 1, Z = z >> 1, m = (int64_t(1) << b) - 1;
  const int64_t sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
  for (int a = 0; a < 2; ++a)
    for (int bb = 0; bb < 2; ++bb)
      for (int d = 0; d < 2; ++d)
        pro[(4 * a + 2 * bb + d) * nf + t] =
            mgl_find(keys, n, mgl_key((X + a * sx) & m, (Y + bb * sy) & m, (Z + d * sz) & m, b));
}

// global index of the level-(L-1) cell (X, Y, Z), or -1 (no such oct)
__device__ __forceinline__ int32_t mgl_coarse_cell(HashView hv, int member, int Lc, int64_t X, int64_t Y,
                                                   int64_t Z, int N) {
  const int32_t v = hash_probe1(hv, ikey(member, Lc, uint32_t(X >> 1), uint32_t(Y >> 1), uint32_t(Z >> 1)));
  if (v < 1 || v > N) return -1;
  return 8 * (v - 1) + int32_t((X & 1) | ((Y & 1) << 1) | ((Z & 1) << 2));
}

// MG level 0: the father cell of every cell and the level-(L-1) cell across
// every face that leaves the level (-1 for the others)
__global__ void k_mgl_coarse(HashView hv, int member, int L, int N, const uint64_t *__restrict__ keys, int64_t n,
                             const int32_t *__restrict__ nb, int32_t *__restrict__ fatherg,
                             int32_t *__restrict__ acrossg, int *err) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  int64_t x, y, z;
  mgl_unkey(keys[t], L, x, y, z);
  const int64_t m = (int64_t(1) << L) - 1, mc = (int64_t(1) << (L - 1)) - 1;
  const int32_t f = mgl_coarse_cell(hv, member, L - 1, x >> 1, y >> 1, z >> 1, N);
  if (f < 0) atomicOr(err, kErrGrading);
  fatherg[t] = f < 0 ? 0 : f;
  for (int d = 0; d < 3; ++d)
    for (int sg = 0; sg < 2; ++sg) {
      const int k6 = 2 * d + sg;
      int32_t q = -1;
      if (nb[k6 * n + t] < 0) {
        const int64_t dd = sg ? 1 : -1;
        const int64_t X = (x + (d == 0) * dd) & m, Y = (y + (d == 1) * dd) & m, Z = (z + (d == 2) * dd) & m;
        q = mgl_coarse_cell(hv, member, L - 1, (X >> 1) & mc, (Y >> 1) & mc, (Z >> 1) & mc, N);
        if (q < 0) {
          atomicOr(err, kErrGrading);
          q = 0;
        }
      }
      acrossg[k6 * n + t] = q;
    }
}

}  // namespace amr
