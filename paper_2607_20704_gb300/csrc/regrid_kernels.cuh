// regrid_kernels.cuh -- flag, grade, count, emit and prolong kernels of one
// regrid (paper Sec. 2.2: refinement of flagged cells by new child octs,
// de-refinement of split cells no longer flagged, then the level bucket and
// Hilbert sorts and the ghost cache of Sec. 2.3, which the mesh build
// shared with creation performs).
//
// Flags live in a per-oct bit mask (bit c = cell c), like the split mask.
//   flag    a cell of level l < levelmax refines when, to one of its six
//           face neighbours (the same-level cell, else the coarser cell that
//           covers it), the relative jump of rho, 2|a-b| > grad_rho (|a|+|b|),
//           or that of p exceeds its threshold, or when rho dx^3 exceeds
//           mass.  The decision is taken in FP64 with each operation rounded
//           as written (no contraction), so it is the same on every build;
//           density and pressure are computed once per cell first.
//   expand  with expand = 1 a flag also flags the 26 same-level cells around
//   grade   finest level first, a flagged cell X of level l flags the level
//           l-1 cells covering the 27 level-l cells around X (2:1 rule)
//   count   an oct above levelmin stays when its father cell is flagged; a
//           flagged leaf gets a new child oct
//   emit    the new oct list (kept octs with their state, then new octs)
//   prolong the new octs of each level, coarsest first, from their father
//           and its six face neighbours (the ghost-oct minmod formula)
#pragma once
#include "hydro_kernels.cuh"

namespace amr {

struct RegridArgs {
  int N, NE, NC;
  int64_t S;
  const uint64_t *key;    // [N] internal keys
  const uint32_t *son;    // [N] split masks
  const int32_t *father;  // [N] father oct, -1 at levelmin
  const int32_t *nbr27;   // [27][N]
  const int32_t *fnb;     // [6][NE]
  const int32_t *csrc;    // [7][NC] (entry 0: the ghost's father cell)
  const int *mlmin, *mlmax;
  const double *mgamma, *msmallr, *msmallp;
  double grad_rho, grad_p, mass;
  int expand;
  // the criteria's switches and FP32 thresholds, decided on the host
  // (conversions and FP64 compares run on GB300's slow FP64 pipe)
  int test_r, test_p, test_mass, use32;
  float thr_r32, thr_p32;
  const float *mflag32;  // [3 M]: gamma - 1, smallr, smallp in FP32
  // the mass criterion rho 2^(-3 l) > mass as rho > mass 2^(3 l): per level
  // the bits of mass 2^(3 l) (FP64, +inf past the range) and of its FP32
  // image rounded down, so that both states compare as integers
  int64_t mass_bits64[16];
  int32_t mass_bits32[16];
  uint32_t *raw;   // [N] criterion masks
  uint32_t *flag;  // [N] final masks
  int *err;
};

// density and pressure of the criterion, with the floors, every operation
// rounded as written: p = (gamma-1)(E - (m.m/2)/rho), one division per cell
__device__ __forceinline__ void flag_rho_p(const double (&u)[5], double g, double smallr,
                                           double smallp, double &rho, double &p) {
  const double r = u[0] > smallr ? u[0] : smallr;
  const double m2 = __dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])),
                              __dmul_rn(u[3], u[3]));
  const double ek = __ddiv_rn(__dmul_rn(0.5, m2), r);
  const double pr = __dmul_rn(__dsub_rn(g, 1.0), __dsub_rn(u[4], ek));
  const double pf = __dmul_rn(r, smallp);
  rho = r;
  p = pr < pf ? pf : pr;
}

// the relative jump of a and b exceeds thr > 0: 2|a-b| > thr (|a|+|b|); both
// sides are non-negative, so they compare as the integers of their bits
__device__ __forceinline__ bool jump_exceeds(double a, double b, double thr) {
  const double lhs = __dmul_rn(2.0, fabs(__dsub_rn(a, b)));
  const double rhs = __dmul_rn(thr, __dadd_rn(fabs(a), fabs(b)));
  return __double_as_longlong(lhs) > __double_as_longlong(rhs);
}

template <class T>
__device__ __forceinline__ void load_cell(const T *U, int64_t S, int64_t g, double (&u)[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) u[v] = double(U[v * S + g]);
}

// The jump tests are decided in FP32 wherever FP32 settles them, and in FP64
// (the decision above, bit for bit) everywhere else.  Each cell gets FP32
// images of its density and pressure and a bound on how far the FP32
// pressure can lie from the FP64 one; a test whose FP32 value clears the
// accumulated error bound by a factor 2 has the FP64 test's outcome, and a
// test that does not is recomputed in FP64.  The result is the FP64
// decision for every cell; GB300's FP64 rate (1/64 of FP32) made the plain
// FP64 tests the regrid's largest kernel.
//
// Error model of the FP32 images (u = 2^-24): every state component
// converts with relative error below 2u (truncation; exact for an FP32
// state), the parameters with u; rho = max(rho, smallr) is 1-Lipschitz, so
// it keeps error 2u rho (the tests allow 8u); m.m/2/rho carries at most
// about 10u of itself (conversions, squares, sum, approximate division); p =
// (gamma-1)(E - ek) then errs by at most (gamma-1)(3u |E| + 11u ek) plus its
// own roundings.  The bound stored is (gamma-1) 2^-17 (|E| + ek) (128u:
// about ten times that), and 2^-21 p for the floor rho smallp (max is
// 1-Lipschitz).  A cell whose values leave [2^-60, 2^60] gets the bound
// +inf: its tests always run in FP64.
// FP32 image of a state component: exact for an FP32 state; for FP64 the
// bits are truncated on the integer pipes (relative error below 2^-23, no
// conversion instruction: those run on the FP64 pipe), magnitudes below
// 2^-126 give 0 and above 2^128 infinity
template <class T>
__device__ __forceinline__ float to_f32(T x) {
  return float(x);
}
template <>
__device__ __forceinline__ float to_f32<double>(double x) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const uint32_t sign = uint32_t(b >> 32) & 0x80000000u;
  const int e = int((b >> 52) & 0x7FF);
  if (e < 1023 - 126) return __uint_as_float(sign);
  if (e > 1023 + 127) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | (uint32_t(e - 896) << 23) | uint32_t((b >> 29) & 0x7FFFFFu));
}

__device__ __forceinline__ bool in_range32(float x) { return x >= 0x1p-60f && x <= 0x1p60f; }

template <class T>
__global__ void k_flag_rp(RegridArgs a, const T *__restrict__ U, float *__restrict__ rp) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t N8 = 8 * int64_t(a.N);
  if (g >= N8) return;
  const int m = ikey_member(a.key[g >> 3]);
  float u[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) u[v] = to_f32(U[v * a.S + g]);
  const float gm1 = a.mflag32[3 * m], smallr = a.mflag32[3 * m + 1], smallp = a.mflag32[3 * m + 2];
  const float r = fmaxf(u[0], smallr);
  const float m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const float ek = __fdividef(0.5f * m2, r);
  const float pr = gm1 * (u[4] - ek);
  const float pf = r * smallp;
  const float p = fmaxf(pr, pf);
  float e = fmaxf(gm1 * 0x1p-17f * (fabsf(u[4]) + ek), 0x1p-21f * pf);
  const bool ok = in_range32(r) && in_range32(p) && in_range32(fabsf(u[4])) && ek <= 0x1p60f &&
                  fabsf(u[1]) <= 0x1p60f && fabsf(u[2]) <= 0x1p60f && fabsf(u[3]) <= 0x1p60f &&
                  gm1 >= 0x1p-30f && gm1 <= 0x1p30f;
  if (!ok) e = INFINITY;
  rp[g] = r;
  rp[N8 + g] = p;
  rp[2 * N8 + g] = e;
}

// 1: the FP64 jump test 2|a-b| > thr (|a|+|b|) holds, 0: it does not, -1:
// FP32 cannot tell.  a, b are FP32 images of positive values within ea, eb
// of them; thr is the FP32 image of the threshold.  The FP32 evaluation errs
// by at most (2 + thr)(ea + eb) + 2^-21 (1 + thr)(a + b) (conversions of the
// threshold, the difference, the sum and the product, each within u of its
// value); the FP64 test's own roundings are below 2^-50 of the sum.
__device__ __forceinline__ int jump_exceeds32(float a, float b, float ea, float eb, float thr) {
  const float s = a + b;
  const float gt = 2.0f * fabsf(a - b) - thr * s;
  const float bound = (2.0f + thr) * (ea + eb) + 0x1p-20f * (1.0f + thr) * s;
  if (!(bound < INFINITY)) return -1;
  if (gt > 2.0f * bound) return 1;
  if (gt < -2.0f * bound) return 0;
  return -1;
}

// the six face neighbours of cell c of oct o (same oct, a real oct, or the
// covering coarser cell of a ghost oct), as cell indices; -1 where there is
// none
__device__ __forceinline__ void flag_neighbours(const RegridArgs &a, int o, int c, int32_t (&gnb)[6]) {
  const int64_t N8 = 8 * int64_t(a.N);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int d = k >> 1, plus = k & 1, bit = 1 << d;
    if (((c >> d) & 1) != plus) {
      gnb[k] = 8 * o + (c ^ bit);
    } else {
      const int32_t ne = a.fnb[k * int64_t(a.NE) + o];
      gnb[k] = ne < 0 ? -1
                      : (ne < a.N ? 8 * ne + (c ^ bit)
                                  : int32_t(checked(a.csrc[checked(ne - a.N, 0, a.NC, a.err)], 0, N8, a.err)));
    }
  }
}

// rho 2^(-3 l) > mass, exactly (the scaling is exact wherever the product is
// a normal number; where it is not, both forms are false), compared as the
// integers of the bits: positive values order as their bits, a negative one
// is below every threshold, and a NaN is excluded
__device__ __forceinline__ bool mass_exceeds(double rho, const RegridArgs &a, int l) {
  const int64_t b = __double_as_longlong(rho);
  return b > a.mass_bits64[l] && b <= 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool mass_exceeds(float rho, const RegridArgs &a, int l) {
  const int32_t b = __float_as_int(rho);
  return b > a.mass_bits32[l] && b <= 0x7F800000;
}

// the FP32 screen of one neighbour pair (k_flag_rp's images): dr, dp = 1 the
// jump of rho (p) exceeds its threshold, 0 it does not, -1 FP32 cannot tell
// (0 also for a test that is off)
__device__ __forceinline__ void flag_screen(const RegridArgs &a, float rn, float pn, float en, float rc,
                                            float pc, float ec, int &dr, int &dp) {
  dr = a.test_r ? -1 : 0;
  dp = a.test_p ? -1 : 0;
  if (a.use32) {
    if (dr) dr = jump_exceeds32(rn, rc, 0x1p-21f * rn, 0x1p-21f * rc, a.thr_r32);
    if (dp && dr != 1) dp = jump_exceeds32(pn, pc, en, ec, a.thr_p32);
  }
}

// criterion masks, FP32 pass: one thread per real cell, the 8 cells of an
// oct in consecutive lanes; a ballot assembles the oct's mask.  A cell whose
// neighbours FP32 flags none of but leaves a test undecided goes on the list
// `undecided` (count at n_undecided) for k_flag_exact.
template <class T>
__global__ void __launch_bounds__(256) k_flag_raw(RegridArgs a, const T *__restrict__ U,
                                                  const float *__restrict__ rp,
                                                  uint32_t *__restrict__ undecided,
                                                  uint32_t *__restrict__ n_undecided) {
  const int64_t gc = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t N8 = 8 * int64_t(a.N);
  const bool in = gc < N8;
  const int o = int(gc >> 3), c = int(gc & 7);
  bool f = false, undec = false;
  if (in) {
    const uint64_t key = a.key[o];
    const int m = ikey_member(key), l = ikey_lev(key);
    if (l < a.mlmax[m]) {
      if (a.test_mass) f = mass_exceeds(U[gc], a, l);
      const float rc = rp[gc], pc = rp[N8 + gc], ec = rp[2 * N8 + gc];
      int32_t gnb[6];
      flag_neighbours(a, o, c, gnb);
      // all loads issued before the tests
      float rn[6], pn[6], en[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int64_t q = gnb[k] < 0 ? gc : gnb[k];
        rn[k] = rp[q];
        pn[k] = rp[N8 + q];
        en[k] = rp[2 * N8 + q];
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (gnb[k] < 0) continue;
        int dr, dp;
        flag_screen(a, rn[k], pn[k], en[k], rc, pc, ec, dr, dp);
        if (dr == 1 || dp == 1) f = true;
        else if (dr || dp) undec = true;
      }
    }
  }
  const unsigned b = __ballot_sync(0xFFFFFFFFu, f);
  if (in && c == 0) a.raw[o] = (b >> (threadIdx.x & 24)) & 0xFFu;
  // the list, one atomic per warp
  const unsigned lst = __ballot_sync(0xFFFFFFFFu, undec && !f);
  if (lst) {
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == __ffs(lst) - 1) base = atomicAdd(n_undecided, uint32_t(__popc(lst)));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(lst) - 1);
    if ((lst >> lane) & 1u) undecided[base + __popc(lst & ((1u << lane) - 1u))] = uint32_t(gc);
  }
}

// criterion masks, FP64 pass: the listed cells' undecided tests in FP64 (the
// decision as defined, bit for bit); a cell that one of them flags sets its
// bit with an atomic OR.  Grid-stride over the list.
template <class T>
__global__ void k_flag_exact(RegridArgs a, const T *__restrict__ U, const float *__restrict__ rp,
                             const uint32_t *__restrict__ undecided, const uint32_t *__restrict__ n_undecided) {
  const int64_t N8 = 8 * int64_t(a.N);
  const uint32_t n = *n_undecided;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int64_t gc = undecided[t];
    const int o = int(gc >> 3), c = int(gc & 7);
    const int m = ikey_member(a.key[o]);
    const float rc = rp[gc], pc = rp[N8 + gc], ec = rp[2 * N8 + gc];
    int32_t gnb[6];
    flag_neighbours(a, o, c, gnb);
    double u[5], rc64, pc64;
    load_cell(U, a.S, gc, u);
    flag_rho_p(u, a.mgamma[m], a.msmallr[m], a.msmallp[m], rc64, pc64);
    bool f = false;
    for (int k = 0; k < 6 && !f; ++k) {
      const int64_t gn = gnb[k];
      if (gn < 0) continue;
      int dr, dp;
      flag_screen(a, rp[gn], rp[N8 + gn], rp[2 * N8 + gn], rc, pc, ec, dr, dp);
      if (dr == 0 && dp == 0) continue;
      double rn64, pn64;
      load_cell(U, a.S, gn, u);
      const int mn = ikey_member(a.key[gn >> 3]);
      flag_rho_p(u, a.mgamma[mn], a.msmallr[mn], a.msmallp[mn], rn64, pn64);
      if (dr && jump_exceeds(rn64, rc64, a.grad_rho)) f = true;
      if (dp && jump_exceeds(pn64, pc64, a.grad_p)) f = true;
    }
    if (f) atomicOr(a.raw + o, 1u << c);
  }
}

// expansion over the 3x3x3 same-level block (or a copy when expand = 0); one
// thread per oct: the criterion masks of the 27 octs around it fill a 4^3
// cube of cells (the oct's 2^3 cells and one layer around them, bit
// (z+1)*16 + (y+1)*4 + (x+1) for cell offset x, y, z in [-1, 2]), and cell c
// is flagged when any bit of its 3^3 window is set.  A neighbour that is a
// ghost oct or missing holds no real cell of this level and adds nothing.
__global__ void k_flag_expand(RegridArgs a) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= a.N) return;
  const uint64_t key = a.key[o];
  const int m = ikey_member(key), l = ikey_lev(key);
  uint32_t out = 0;
  if (l < a.mlmax[m]) {
    if (!a.expand) {
      out = a.raw[o];
    } else {
      uint64_t cube = 0;
#pragma unroll
      for (int k = 0; k < 27; ++k) {
        const int ox = k % 3 - 1, oy = (k / 3) % 3 - 1, oz = k / 9 - 1;
        const int32_t e = a.nbr27[k * int64_t(a.N) + o];
        if (e < 0 || e >= a.N) continue;
        const uint32_t r = a.raw[e];
        if (!r) continue;
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          const int fx = 2 * ox + (cc & 1), fy = 2 * oy + ((cc >> 1) & 1), fz = 2 * oz + ((cc >> 2) & 1);
          if (fx < -1 || fx > 2 || fy < -1 || fy > 2 || fz < -1 || fz > 2) continue;
          cube |= uint64_t((r >> cc) & 1u) << ((fz + 1) * 16 + (fy + 1) * 4 + (fx + 1));
        }
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        uint64_t w = 0;
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) w |= uint64_t(1) << ((cz + dz) * 16 + (cy + dy) * 4 + (cx + dx));
        if (cube & w) out |= 1u << c;
      }
    }
  }
  a.flag[o] = out;
}

// grading closure from the octs [lo, hi) of one level l > levelmin: every
// flagged cell flags the level-(l-1) cells covering its 27 neighbours.  Per
// axis those are, for a cell with bit 0, the father cell's coordinate minus
// one and itself, for bit 1 itself and plus one, so the cells covered for
// the whole oct form a subset of the 3^3 level-(l-1) cells around the father
// cell.  Per axis, offset 0 and the offset away from the father oct's centre
// stay in the father oct, and the offset towards it lands in the
// neighbouring oct on that side (the father oct itself when the level has
// one oct per axis): the covered cells fall into at most 2^3 octs, whose
// cell masks are collected in one 64-bit word (byte = oct), then one atomic
// OR per oct instead of one per covered cell.
__global__ void k_flag_grade(RegridArgs a, int lo, int hi) {
  const int o = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= hi) return;
  const uint32_t mask = a.flag[o];
  if (!mask) return;
  const uint64_t key = a.key[o];
  const int l = ikey_lev(key);
  const int fo = a.father[o];
  if (fo < 0) return;
  uint32_t set27 = 0;  // bit (dz+1)*9 + (dy+1)*3 + (dx+1)
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (!((mask >> c) & 1u)) continue;
    const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int dx = (q & 1) - 1 + bx, dy = ((q >> 1) & 1) - 1 + by, dz = ((q >> 2) & 1) - 1 + bz;
      set27 |= 1u << ((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
    }
  }
  const int64_t cside = int64_t(1) << (l - 1);                  // cells per axis at level l-1
  const int64_t oside = int64_t(1) << (l - 2 > 0 ? l - 2 : 0);  // octs per axis at l-1
  const int64_t fc[3] = {int64_t(ikey_x(key)), int64_t(ikey_y(key)), int64_t(ikey_z(key))};  // father cell
  // per axis: the offset towards the neighbouring oct, and that oct's place
  // (-1, 0 or +1) relative to the father oct, periodic
  int toward[3], rel_t[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    toward[q] = (fc[q] & 1) ? 1 : -1;
    const int64_t p = (fc[q] + toward[q]) & (cside - 1);
    const int64_t dd = ((p >> 1) - (fc[q] >> 1)) & (oside - 1);  // oside is a power of two
    rel_t[q] = dd == 0 ? 0 : (dd == 1 ? 1 : -1);
  }
  uint64_t acc = 0;  // byte sx + 2 sy + 4 sz: the cells of the oct on the toward side of the axes s = 1
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    if (!((set27 >> k) & 1u)) continue;
    const int d[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
    int slot = 0, cc = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (d[q] == toward[q] && rel_t[q] != 0) slot |= 1 << q;
      cc |= int(((fc[q] + d[q]) & (cside - 1)) & 1) << q;
    }
    acc |= uint64_t(1) << (8 * slot + cc);
  }
#pragma unroll
  for (int slot = 0; slot < 8; ++slot) {
    const uint32_t bits = uint32_t(acc >> (8 * slot)) & 0xFFu;
    if (!bits) continue;
    const int rx = (slot & 1) ? rel_t[0] : 0, ry = (slot & 2) ? rel_t[1] : 0, rz = (slot & 4) ? rel_t[2] : 0;
    const int32_t e = a.nbr27[((rz + 1) * 9 + (ry + 1) * 3 + (rx + 1)) * int64_t(a.N) + fo];
    if (e < 0 || e >= a.N) {
      atomicOr(a.err, kErrGrading);
      continue;
    }
    atomicOr(a.flag + e, bits);
  }
}

// per oct: 1 if it stays (its father cell is flagged, or it is a base oct)
// at cnt[o], and the number of new child octs (flagged leaf cells) at
// cnt[N + o]; cnt[2 N] = 0, so that one exclusive scan of the 2 N + 1 words
// gives the kept octs' places, the new octs' places (after the kept octs)
// and, at 2 N, the size of the new list
__global__ void k_regrid_count(RegridArgs a, uint32_t *cnt) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o == 0) cnt[2 * int64_t(a.N)] = 0u;
  if (o >= a.N) return;
  const uint64_t key = a.key[o];
  const int fo = a.father[o];
  uint32_t k = 1;
  if (fo >= 0) {
    const int fc = int(ikey_x(key) & 1) | (int(ikey_y(key) & 1) << 1) | (int(ikey_z(key) & 1) << 2);
    k = (a.flag[fo] >> fc) & 1u;
  }
  cnt[o] = k;
  cnt[a.N + o] = __popc(a.flag[o] & ~a.son[o]);
}

// the new oct list from the scanned counts pos (k_regrid_count): kept octs
// at pos[o], new child octs after all K kept ones, at pos[N + o] in cell
// order; src names the old oct whose state an entry keeps (~0 for a new oct)
__global__ void k_regrid_emit(RegridArgs a, const uint32_t *pos, uint8_t *lvl, uint16_t *mem,
                              uint32_t *oi, uint32_t *oj, uint32_t *ok, uint32_t *src,
                              uint8_t *is_new) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= a.N) return;
  const uint64_t key = a.key[o];
  const int l = ikey_lev(key);
  const uint32_t x = ikey_x(key), y = ikey_y(key), z = ikey_z(key);
  if (pos[o + 1] != pos[o]) {  // kept (pos[N] is the number of kept octs)
    const int64_t t = pos[o];
    lvl[t] = uint8_t(l);
    mem[t] = uint16_t(ikey_member(key));
    oi[t] = x;
    oj[t] = y;
    ok[t] = z;
    is_new[t] = 0;
    src[t] = uint32_t(o);
  }
  const uint32_t nm = a.flag[o] & ~a.son[o];
  int64_t t = pos[a.N + o];
  for (int c = 0; c < 8; ++c) {
    if (!((nm >> c) & 1u)) continue;
    lvl[t] = uint8_t(l + 1);
    mem[t] = uint16_t(ikey_member(key));
    oi[t] = 2 * x + (c & 1);
    oj[t] = 2 * y + ((c >> 1) & 1);
    ok[t] = 2 * z + ((c >> 2) & 1);
    is_new[t] = 1;
    src[t] = ~0u;
    ++t;
  }
}

// Batch repack: every oct of a kept member goes to its place in the new oct
// list (member id remapped, state widened to FP64 exactly); octs of dropped
// members (remap -1) are left out.  dst[m] is the new list position of old
// member m's first oct, base[m] its old first mesh index.
template <class T>
__global__ void k_repack_emit(int64_t N, int64_t S, const uint64_t *__restrict__ key,
                              const T *__restrict__ U, const int *__restrict__ remap,
                              const int64_t *__restrict__ dst, const int64_t *__restrict__ base,
                              int64_t n_out, uint8_t *lvl, uint16_t *mem, uint32_t *oi, uint32_t *oj,
                              uint32_t *ok, double *Uout) {
  const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (o >= N) return;
  const uint64_t k = key[o];
  const int mb = ikey_member(k);
  const int nm = remap[mb];
  if (nm < 0) return;
  const int64_t t = dst[mb] + (o - base[mb]);
  lvl[t] = uint8_t(ikey_lev(k));
  mem[t] = uint16_t(nm);
  oi[t] = ikey_x(k);
  oj[t] = ikey_y(k);
  ok[t] = ikey_z(k);
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int c = 0; c < 8; ++c) Uout[v * 8 * n_out + 8 * t + c] = double(U[v * S + 8 * o + c]);
}

// new octs of [lo, hi) (one level) take the minmod prolongation of their
// father cell from the father's face neighbours (all real after grading);
// one thread per (oct, variable), 5 (hi - lo) threads
template <class T>
__global__ void k_prolong_new(int N, int NE, int64_t S, const uint64_t *__restrict__ key,
                              const int32_t *__restrict__ father, const int32_t *__restrict__ fnb,
                              const uint8_t *__restrict__ is_new, T *U, int lo, int hi, int *err) {
  const int64_t tid = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int o = lo + int(tid / 5), v = int(tid % 5);
  if (o >= hi || !is_new[o]) return;
  const int fo = father[o];
  const uint64_t k = key[o];
  const int fc = int(ikey_x(k) & 1) | (int(ikey_y(k) & 1) << 1) | (int(ikey_z(k) & 1) << 2);
  int64_t gm[3], gp[3];
  for (int d = 0; d < 3; ++d) {
    const int bit = 1 << d;
    for (int plus = 0; plus < 2; ++plus) {
      int64_t g;
      if (((fc >> d) & 1) != plus) {
        g = 8 * int64_t(fo) + (fc ^ bit);
      } else {
        const int32_t ne = fnb[(2 * d + plus) * int64_t(NE) + fo];
        if (ne < 0 || ne >= N) {
          atomicOr(err, kErrGrading);
          return;
        }
        g = 8 * int64_t(ne) + (fc ^ bit);
      }
      (plus ? gp : gm)[d] = g;
    }
  }
  const int64_t gc = 8 * int64_t(fo) + fc;
  const T *Uv = U + v * S;
  const T uc = Uv[gc];
  const T sx = minmod(Uv[gp[0]] - uc, uc - Uv[gm[0]]);
  const T sy = minmod(Uv[gp[1]] - uc, uc - Uv[gm[1]]);
  const T sz = minmod(Uv[gp[2]] - uc, uc - Uv[gm[2]]);
  T *dst = U + v * S + 8 * int64_t(o);
  const T h = T(0.25);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T hx = (c & 1) ? h : -h, hy = (c & 2) ? h : -h, hz = (c & 4) ? h : -h;
    dst[c] = ((uc + hx * sx) + hy * sy) + hz * sz;
  }
}

__global__ void k_gather_u8(const uint32_t *__restrict__ perm, const uint8_t *__restrict__ src,
                            int64_t n, uint8_t *__restrict__ dst) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) dst[t] = src[perm[t]];
}

}  // namespace amr
