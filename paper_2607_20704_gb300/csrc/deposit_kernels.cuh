// deposit_kernels.cuh -- Cloud-in-Cell mass deposition onto the levels of a
// mesh (paper Sec. 4, "Mass Deposition": at level l the particles of level l
// and of every finer level deposit, then the particle list is split for
// level l+1 by a prefix sum over "host cell refined").
//
// A list holds particle indices; its length lives on the device, so the
// levels run back to back without a host round trip.  One thread per
// particle of the list: the CIC weights at cell size 2^-l with the
// half-cell-shifted stencil (s = x 2^l - 1/2, i0 = floor(s), f = s - i0),
// and m (wx wy) wz 2^(3l) added with one atomic per stencil cell that exists
// at level l (a cell of a real level-l oct, found in the hash table).  Then
// a flag per particle whose host cell (the cell containing it) exists and is
// split, an exclusive prefix sum, and the compaction into the next list.
#pragma once
#include "amr_internal.cuh"

namespace amr {

template <class T>
__global__ void k_deposit_level(HashView hv, int member, int l, int N, const T *__restrict__ px,
                                const T *__restrict__ py, const T *__restrict__ pz,
                                const T *__restrict__ pm, const uint32_t *__restrict__ list,
                                const int64_t *__restrict__ count, T *rho) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= count[l]) return;
  const uint32_t p = list[t];
  const T n = T(int64_t(1) << l);
  const uint32_t mask = uint32_t((int64_t(1) << l) - 1);
  int64_t i0[3];
  T w[3][2];
  const T pos[3] = {px[p], py[p], pz[p]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T s = pos[d] * n - T(0.5);
    const T fl = floor(s);
    const T f = s - fl;
    i0[d] = int64_t(fl);
    w[d][0] = T(1) - f;
    w[d][1] = f;
  }
  const T mm = pm[p];
  const T scale = T(ldexp(1.0, 3 * l));  // 1 / dx^3, exact
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const uint32_t X = uint32_t(i0[0] + cx) & mask, Y = uint32_t(i0[1] + cy) & mask,
                   Z = uint32_t(i0[2] + cz) & mask;
    const int32_t v = hash_probe1(hv, ikey(member, l, X >> 1, Y >> 1, Z >> 1));
    if (v < 1 || v > N) continue;  // no real oct there: the cell does not exist at level l
    const int cc = int((X & 1) + 2 * (Y & 1) + 4 * (Z & 1));
    atomicAdd(rho + 8 * int64_t(v - 1) + cc, (mm * ((w[0][cx] * w[1][cy]) * w[2][cz])) * scale);
  }
}

// the base level is complete: a table from oct coordinates to oct index
// replaces the hash probes there
__global__ void k_base_table(const uint64_t *__restrict__ key, int lo, int64_t nb, int lmin, int32_t *btab) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nb) return;
  const int o = lo + int(t);
  const uint64_t k = key[o];
  const int64_t side = int64_t(1) << (lmin - 1);
  btab[(int64_t(ikey_x(k)) * side + ikey_y(k)) * side + ikey_z(k)] = o;
}

// deposit of every particle at the base level l (the list of the base level
// holds all particles; every stencil cell exists): the arithmetic of
// k_deposit_level, the oct found in the base table
template <class T>
__global__ void k_deposit_base(const int32_t *__restrict__ btab, int l, int64_t np, const T *__restrict__ px,
                               const T *__restrict__ py, const T *__restrict__ pz, const T *__restrict__ pm,
                               T *rho) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= np) return;
  const T n = T(int64_t(1) << l);
  const uint32_t mask = uint32_t((int64_t(1) << l) - 1);
  const int64_t side = int64_t(1) << (l - 1);
  int64_t i0[3];
  T w[3][2];
  const T pos[3] = {px[p], py[p], pz[p]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T s = pos[d] * n - T(0.5);
    const T fl = floor(s);
    const T f = s - fl;
    i0[d] = int64_t(fl);
    w[d][0] = T(1) - f;
    w[d][1] = f;
  }
  const T mm = pm[p];
  const T scale = T(ldexp(1.0, 3 * l));  // 1 / dx^3, exact
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const uint32_t X = uint32_t(i0[0] + cx) & mask, Y = uint32_t(i0[1] + cy) & mask,
                   Z = uint32_t(i0[2] + cz) & mask;
    const int32_t o = __ldg(btab + (int64_t(X >> 1) * side + (Y >> 1)) * side + (Z >> 1));
    const int cc = int((X & 1) + 2 * (Y & 1) + 4 * (Z & 1));
    atomicAdd(rho + 8 * int64_t(o) + cc, (mm * ((w[0][cx] * w[1][cy]) * w[2][cz])) * scale);
  }
}

// flag[p] = 1 if particle p's host cell at the base level is split
template <class T>
__global__ void k_split_base(const int32_t *__restrict__ btab, int l, const uint32_t *__restrict__ son,
                             const T *__restrict__ px, const T *__restrict__ py, const T *__restrict__ pz,
                             int64_t np, uint32_t *flag) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= np) return;
  const T n = T(int64_t(1) << l);
  const uint32_t mask = uint32_t((int64_t(1) << l) - 1);
  const int64_t side = int64_t(1) << (l - 1);
  const uint32_t X = uint32_t(int64_t(floor(px[p] * n))) & mask, Y = uint32_t(int64_t(floor(py[p] * n))) & mask,
                 Z = uint32_t(int64_t(floor(pz[p] * n))) & mask;
  const int32_t o = __ldg(btab + (int64_t(X >> 1) * side + (Y >> 1)) * side + (Z >> 1));
  flag[p] = (__ldg(son + o) >> ((X & 1) + 2 * (Y & 1) + 4 * (Z & 1))) & 1u;
}

// flag[t] = 1 if particle list[t]'s host cell at level l exists and is split;
// 0 past the end of the list (the prefix sum runs over the list's capacity)
template <class T>
__global__ void k_split_level(HashView hv, int member, int l, int N, const uint32_t *__restrict__ son,
                              const T *__restrict__ px, const T *__restrict__ py,
                              const T *__restrict__ pz, const uint32_t *__restrict__ list,
                              const int64_t *__restrict__ count, int64_t cap, uint32_t *flag) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= cap) return;
  uint32_t f = 0;
  if (t < count[l]) {
    const uint32_t p = list[t];
    const T n = T(int64_t(1) << l);
    const uint32_t mask = uint32_t((int64_t(1) << l) - 1);
    const uint32_t X = uint32_t(int64_t(floor(px[p] * n))) & mask,
                   Y = uint32_t(int64_t(floor(py[p] * n))) & mask,
                   Z = uint32_t(int64_t(floor(pz[p] * n))) & mask;
    const int32_t v = hash_probe1(hv, ikey(member, l, X >> 1, Y >> 1, Z >> 1));
    if (v >= 1 && v <= N) f = (__ldg(son + (v - 1)) >> ((X & 1) + 2 * (Y & 1) + 4 * (Z & 1))) & 1u;
  }
  flag[t] = f;
}

// the next list: the flagged particles in order (pos = exclusive prefix sum of
// flag), and its length
__global__ void k_compact_level(const uint32_t *__restrict__ list, const uint32_t *__restrict__ flag,
                                const uint32_t *__restrict__ pos, int64_t cap, int l,
                                uint32_t *__restrict__ next, int64_t *count) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= cap) return;
  if (flag[t]) next[pos[t]] = list[t];
  if (t == cap - 1) count[l + 1] = int64_t(pos[t] + flag[t]);
}

}  // namespace amr
