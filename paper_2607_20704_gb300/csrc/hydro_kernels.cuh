// hydro_kernels.cuh -- one AMR level step of compressible Euler (paper Sec. 3:
// MUSCL-Hancock predictor-corrector with an HLLC Riemann solver and two
// ghost cells per side; Sec. 2.3 ghost octs; Table 1 stages godunov /
// set uold / upload), as non-redundant per-cell passes:
//
//   k_prolong   ghost octs of the level from their father cell (minmod)
//   k_prim      primitive variables of every real and ghost cell
//   k_predict   limited slopes and the Hancock half-step, once per cell
//   k_flux      one HLLC flux per face (owned by the cell on its minus side)
//   k_update    conservative update of leaf cells + pending reflux
//   k_reflux    fixed-order sum of coarse-fine fluxes for level l-1 cells
//   k_restrict  father cell = mean of its 8 children
//
// The paper's kernels gather a 6x6x6 stencil per oct and recompute the
// slopes and predictor of its ghost ring (8x work per cell at nsubgrid=1).
// On GB300 the FP64 rate is far below the memory rate, so each cell's
// predictor and each face's Riemann solve is computed exactly once and the
// intermediate states go through L2/HBM instead.
#pragma once
#include "hydro_args.cuh"

namespace amr {

// ---------------------------------------------------------------------------
// arithmetic helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double minmod(double a, double b) {
  // 0 for opposite signs or a zero argument, else the argument of smaller
  // magnitude; decided on the bit patterns (integer pipes, no FP64 issue)
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const long long ma = ia & 0x7FFFFFFFFFFFFFFFll, mb = ib & 0x7FFFFFFFFFFFFFFFll;
  if (((ia ^ ib) < 0) | (ma == 0) | (mb == 0)) return 0.0;
  return ma < mb ? a : b;
}
__device__ __forceinline__ float minmod(float a, float b) {
  const int ia = __float_as_int(a), ib = __float_as_int(b);
  const int ma = ia & 0x7FFFFFFF, mb = ib & 0x7FFFFFFF;
  if (((ia ^ ib) < 0) | (ma == 0) | (mb == 0)) return 0.0f;
  return ma < mb ? a : b;
}
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }

// 1/x by Newton-Raphson (e = 1 - x r, r += r e) from the hardware's
// approximate reciprocal: each step doubles the correct bits, two steps take
// the approximation to double precision (within an ulp or two of 1/x, checked
// against the correctly rounded quotient by the parity tests).  Operands here
// are positive, finite and normal (densities, sums of rho |u - S|, wave-speed
// gaps), so the flush-to-zero form is safe.
__device__ __forceinline__ double rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <class T>
__device__ __forceinline__ T level_dtdx(const LevelArgs<T> &a);
template <>
__device__ __forceinline__ double level_dtdx<double>(const LevelArgs<double> &a) {
  return a.dt_dev ? __ldg(a.dt_dev) * a.dtdx_scale : a.dtdx_host;
}
template <>
__device__ __forceinline__ float level_dtdx<float>(const LevelArgs<float> &a) {
  // dtdx_scale is a power of two, exact in float
  return a.dtf_dev ? __ldg(a.dtf_dev) * float(a.dtdx_scale) : a.dtdx_host;
}

// extended oct index of local oct index q, and back
template <class T>
__device__ __forceinline__ int ext_of_local(const LevelArgs<T> &a, int q) {
  return q < a.nl ? a.lo + q : a.N + a.clo + (q - a.nl);
}
template <class T>
__device__ __forceinline__ int local_of_ext(const LevelArgs<T> &a, int e) {
  return e < a.N ? e - a.lo : e - a.N - a.clo + a.nl;
}

// local index of the face neighbour of local cell t (extended oct e, cell c)
// along axis d on side `plus`; -1 when the neighbouring oct does not exist
template <class T>
__device__ __forceinline__ int nbr_local(const LevelArgs<T> &a, int t, int e, int c, int d,
                                         int plus) {
  const int bit = 1 << d;
  if (((c >> d) & 1) != plus) return t ^ bit;
  const int32_t ne = __ldg(a.fnb + (2 * d + plus) * int64_t(a.NE) + e);
  if (ne < 0) return -1;
  return 8 * local_of_ext(a, ne) + (c ^ bit);
}

template <class T>
__device__ __forceinline__ bool cell_is_split(const LevelArgs<T> &a, int t) {
  const int q = t >> 3;
  if (q >= a.nl) return false;  // ghost cells are leaves
  return (__ldg(a.son + a.lo + q) >> (t & 7)) & 1u;
}

// ---------------------------------------------------------------------------
// ghost octs: child = U_C + sum_d (+-1/4) minmod(U(C+e_d)-U(C), U(C)-U(C-e_d))
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_prolong(LevelArgs<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 5 * a.ncl) return;
  const int v = q / a.ncl;
  const int s = q - v * a.ncl;
  const int cs = a.clo + s;
  const T *Uv = a.U + v * a.S;
  T src[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) src[k] = Uv[__ldg(a.csrc + k * int64_t(a.NC) + cs)];
  const T uc = src[0];
  const T sx = minmod(src[2] - uc, uc - src[1]);
  const T sy = minmod(src[4] - uc, uc - src[3]);
  const T sz = minmod(src[6] - uc, uc - src[5]);
  T *dst = a.U + v * a.S + 8 * int64_t(a.N + cs);
  const T h = T(0.25);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T hx = (c & 1) ? h : -h, hy = (c & 2) ? h : -h, hz = (c & 4) ? h : -h;
    dst[c] = ((uc + hx * sx) + hy * sy) + hz * sz;
  }
}

// ---------------------------------------------------------------------------
// primitives of every real and ghost cell of the level
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_prim(LevelArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.LS) return;
  const int g = 8 * ext_of_local(a, t >> 3) + (t & 7);
  const T u0 = a.U[g], u1 = a.U[a.S + g], u2 = a.U[2 * a.S + g], u3 = a.U[3 * a.S + g],
          u4 = a.U[4 * a.S + g];
  const T r = vmax(u0, a.smallr);
  const T ir = rcp(r);
  const T vx = u1 * ir, vy = u2 * ir, vz = u3 * ir;
  const T ek = T(0.5) * r * ((vx * vx + vy * vy) + vz * vz);
  const T p = vmax((a.gamma - T(1)) * (u4 - ek), r * a.smallp);
  a.W[t] = r;
  a.W[a.LS + t] = vx;
  a.W[2 * a.LS + t] = vy;
  a.W[3 * a.LS + t] = vz;
  a.W[4 * a.LS + t] = p;
}

// ---------------------------------------------------------------------------
// limited slopes and Hancock predictor W* = W + dt/(2dx) S(W, dW)
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_predict(LevelArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.LS) return;
  const int e = ext_of_local(a, t >> 3);
  const int c = t & 7;
  T w[5], dw[3][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) w[v] = a.W[v * a.LS + t];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int tm = nbr_local(a, t, e, c, d, 0);
    const int tp = nbr_local(a, t, e, c, d, 1);
    if (tm < 0 || tp < 0) {  // outer ring of a ghost oct: never used
#pragma unroll
      for (int v = 0; v < 5; ++v) dw[d][v] = T(0);
      continue;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T wm = a.W[v * a.LS + tm], wp = a.W[v * a.LS + tp];
      dw[d][v] = minmod(wp - w[v], w[v] - wm);
    }
  }
  const T r = w[0], p = w[4], g = a.gamma;
  const T ir = rcp(r);
  const T gp = g * p;
  T s[5];
  s[0] = -(((w[1] * dw[0][0] + r * dw[0][1]) + (w[2] * dw[1][0] + r * dw[1][2])) +
           (w[3] * dw[2][0] + r * dw[2][3]));
#pragma unroll
  for (int k = 0; k < 3; ++k)
    s[1 + k] = -((w[1] * dw[0][1 + k] + w[2] * dw[1][1 + k]) + w[3] * dw[2][1 + k]) - dw[k][4] * ir;
  s[4] = -(((w[1] * dw[0][4] + gp * dw[0][1]) + (w[2] * dw[1][4] + gp * dw[1][2])) +
           (w[3] * dw[2][4] + gp * dw[2][3]));
  const T hdt = T(0.5) * level_dtdx(a);
#pragma unroll
  for (int v = 0; v < 5; ++v) a.Q[v * a.LS + t] = w[v] + hdt * s[v];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < 5; ++v) a.Q[(5 + 5 * d + v) * a.LS + t] = dw[d][v];
}

// ---------------------------------------------------------------------------
// HLLC flux normal to axis D from face states qL, qR (rho, u, v, w, p):
// S_L = min(u) - max(c), S_R = max(u) + max(c); star speed and pressure from
// the two-wave HLL jump conditions; physical flux of the state sampled at
// x/t = 0 (Toro's HLLC); transverse velocities from the upwind side.
// max(c) takes one square root: c^2 = gamma p / rho is compared across the
// face by cross-multiplication and only the larger is divided and rooted.
// ---------------------------------------------------------------------------
template <int D, class T>
__device__ __forceinline__ void hllc(const T (&qL)[5], const T (&qR)[5], T g, T igm1, T (&F)[5]) {
  constexpr int in = 1 + D, t1 = D == 0 ? 2 : 1, t2 = D == 2 ? 2 : 3;
  const T rl = qL[0], ul = qL[in], pl = qL[4];
  const T rr = qR[0], ur = qR[in], pr = qR[4];
  const T el = pl * igm1 + T(0.5) * rl * ((qL[1] * qL[1] + qL[2] * qL[2]) + qL[3] * qL[3]);
  const T er = pr * igm1 + T(0.5) * rr * ((qR[1] * qR[1] + qR[2] * qR[2]) + qR[3] * qR[3]);
  const T gpl = g * pl, gpr = g * pr;
  const bool lbig = gpl * rr > gpr * rl;
  const T cmax = vsqrt((lbig ? gpl : gpr) * rcp(lbig ? rl : rr));
  const T sl = vmin(ul, ur) - cmax;
  const T sr = vmax(ul, ur) + cmax;
  const T rcl = rl * (ul - sl), rcr = rr * (sr - ur);
  const T irc = rcp(rcl + rcr);
  const T us = ((rcr * ur + rcl * ul) + (pl - pr)) * irc;
  const T ps = ((rcr * pl + rcl * pr) + rcl * rcr * (ul - ur)) * irc;
  T ro, uo, po, eo, v1, v2;
  if (sl > T(0)) {
    ro = rl; uo = ul; po = pl; eo = el; v1 = qL[t1]; v2 = qL[t2];
  } else if (us > T(0)) {
    const T id = rcp(sl - us);
    ro = rl * (sl - ul) * id;
    eo = ((sl - ul) * el - pl * ul + ps * us) * id;
    uo = us; po = ps; v1 = qL[t1]; v2 = qL[t2];
  } else if (sr > T(0)) {
    const T id = rcp(sr - us);
    ro = rr * (sr - ur) * id;
    eo = ((sr - ur) * er - pr * ur + ps * us) * id;
    uo = us; po = ps; v1 = qR[t1]; v2 = qR[t2];
  } else {
    ro = rr; uo = ur; po = pr; eo = er; v1 = qR[t1]; v2 = qR[t2];
  }
  const T mf = ro * uo;
  F[0] = mf;
  F[in] = mf * uo + po;
  F[t1] = mf * v1;
  F[t2] = mf * v2;
  F[4] = (eo + po) * uo;
}

// flux across the plus face of local cell t along axis D (neighbour tn)
template <int D, class T>
__device__ __forceinline__ void face_flux(const LevelArgs<T> &a, int t, int tn, T (&F)[5]) {
  T qL[5], qR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = a.Q[v * a.LS + t] + T(0.5) * a.Q[(5 + 5 * D + v) * a.LS + t];
    qR[v] = a.Q[v * a.LS + tn] - T(0.5) * a.Q[(5 + 5 * D + v) * a.LS + tn];
  }
  qL[0] = vmax(qL[0], a.smallr);
  qR[0] = vmax(qR[0], a.smallr);
  qL[4] = vmax(qL[4], qL[0] * a.smallp);
  qR[4] = vmax(qR[4], qR[0] * a.smallp);
  hllc<D>(qL, qR, a.gamma, a.igm1, F);
}

template <int D, class T>
__device__ __forceinline__ void flux_dir(const LevelArgs<T> &a, int t, int e, int c, int q,
                                         bool real, bool split, T dtdx) {
  T F[5] = {T(0), T(0), T(0), T(0), T(0)};
  const int tn = nbr_local(a, t, e, c, D, 1);
  bool need = false, nreal = false;
  if (tn >= 0) {
    nreal = (tn >> 3) < a.nl;
    need = (real || nreal) && !split && !cell_is_split(a, tn);
  }
  if (need) {
    face_flux<D>(a, t, tn, F);
    if (a.reflux && (real != nreal)) {
      constexpr int d1 = D == 0 ? 1 : 0, d2 = D == 2 ? 1 : 2;
      const int ab = (((c >> d1) & 1) << 1) | ((c >> d2) & 1);
      int gslot;
      T sg;
      if (real) {  // ghost on the plus side: the face is the coarse cell's minus face
        gslot = (a.clo + (tn >> 3) - a.nl) * 24 + (2 * D) * 4 + ab;
        sg = T(1);
      } else {     // ghost on the minus side: the coarse cell's plus face
        gslot = (a.clo + q - a.nl) * 24 + (2 * D + 1) * 4 + ab;
        sg = T(-1);
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) a.C[v * a.CS + gslot] = (sg * dtdx) * F[v] / T(8);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) a.F[(5 * D + v) * a.LS + t] = F[v];
}

// One thread per real or ghost cell: the fluxes of its three plus faces.
// A face is needed when at least one side is a real cell and neither side
// is split; other faces carry zero.  A needed face with a ghost on one side
// is a coarse-fine face: its flux, times sigma dt/dx / 8, goes to slot
// (direction seen from the coarse cell, fine face a,b) of the ghost oct.
template <class T>
__global__ void k_flux(LevelArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.LS) return;
  const int q = t >> 3;
  const int e = ext_of_local(a, q);
  const int c = t & 7;
  const bool real = q < a.nl;
  const bool split = cell_is_split(a, t);
  const T dtdx = level_dtdx(a);
  flux_dir<0>(a, t, e, c, q, real, split, dtdx);
  flux_dir<1>(a, t, e, c, q, real, split, dtdx);
  flux_dir<2>(a, t, e, c, q, real, split, dtdx);
}

// U <- (U + dt/dx sum_d (F_d- - F_d+)) + R on leaf cells; R <- 0
template <class T>
__global__ void k_update(LevelArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * a.nl) return;
  if (cell_is_split(a, t)) return;
  const int e = a.lo + (t >> 3);
  const int c = t & 7;
  const int tm0 = nbr_local(a, t, e, c, 0, 0), tm1 = nbr_local(a, t, e, c, 1, 0),
            tm2 = nbr_local(a, t, e, c, 2, 0);
  const T dtdx = level_dtdx(a);
  const int g = 8 * e + c;
  const int rs = __ldg(a.rslot + g);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const T dx = a.F[(0 + v) * a.LS + tm0] - a.F[(0 + v) * a.LS + t];
    const T dy = a.F[(5 + v) * a.LS + tm1] - a.F[(5 + v) * a.LS + t];
    const T dz = a.F[(10 + v) * a.LS + tm2] - a.F[(10 + v) * a.LS + t];
    const T du = (dx + dy) + dz;
    T *Ug = a.U + v * a.S + g;
    T u = *Ug + dtdx * du;
    if (rs >= 0) {
      T *Rv = a.Rc + v * int64_t(a.NC) + rs;
      u = u + *Rv;
      *Rv = T(0);
    }
    *Ug = u;
  }
}

// R(X) += sum of the 24 slots of the ghost oct whose father is X, in slot
// order (direction -x,+x,-y,+y,-z,+z seen from X, then fine face)
template <class T>
__global__ void k_reflux(LevelArgs<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 5 * a.ncl) return;
  const int v = q / a.ncl;
  const int s = a.clo + (q - v * a.ncl);
  const T *cv = a.C + v * a.CS + 24 * int64_t(s);
  T *Rv = a.Rc + v * int64_t(a.NC) + s;
  T acc = *Rv;
#pragma unroll
  for (int k = 0; k < 24; ++k) acc += cv[k];
  *Rv = acc;
}

// father cell = (sum of the 8 children in child order) / 8
template <class T>
__global__ void k_restrict(LevelArgs<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 5 * a.nl) return;
  const int v = q / a.nl;
  const int o = a.lo + (q - v * a.nl);
  const uint64_t k = __ldg(a.key + o);
  const int fc = int((key_x(k) & 1) | ((key_y(k) & 1) << 1) | ((key_z(k) & 1) << 2));
  const int f = __ldg(a.father + o);
  const T *src = a.U + v * a.S + 8 * o;
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) s += src[c];
  a.U[v * a.S + 8 * f + fc] = s * T(0.125);
}

// ---------------------------------------------------------------------------
// FP32 level step in fewer launches.  FP32 arithmetic is cheap on GB300, so
// these kernels trade recomputation for memory round trips and launches:
// k_predict_u derives the primitives of a cell and its six face neighbours
// from U directly (no W array); k_flux_update solves all six faces of a
// real leaf cell and updates it in place (each interior face is solved by
// both of its cells, bit-identically, so the update matches the split
// kernels); coarse-fine faces are owned by the real cell.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void prim_at(const LevelArgs<T> &a, int t, T (&w)[5]) {
  const int g = 8 * ext_of_local(a, t >> 3) + (t & 7);
  const T r = vmax(a.U[g], a.smallr);
  const T ir = rcp(r);
  const T vx = a.U[a.S + g] * ir, vy = a.U[2 * a.S + g] * ir, vz = a.U[3 * a.S + g] * ir;
  const T ek = T(0.5) * r * ((vx * vx + vy * vy) + vz * vz);
  w[0] = r;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = vmax((a.gamma - T(1)) * (a.U[4 * a.S + g] - ek), r * a.smallp);
}

template <class T>
__global__ void k_predict_u(LevelArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.LS) return;
  const int e = ext_of_local(a, t >> 3);
  const int c = t & 7;
  T w[5], dw[3][5];
  prim_at(a, t, w);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int tm = nbr_local(a, t, e, c, d, 0);
    const int tp = nbr_local(a, t, e, c, d, 1);
    if (tm < 0 || tp < 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) dw[d][v] = T(0);
      continue;
    }
    T wm[5], wp[5];
    prim_at(a, tm, wm);
    prim_at(a, tp, wp);
#pragma unroll
    for (int v = 0; v < 5; ++v) dw[d][v] = minmod(wp[v] - w[v], w[v] - wm[v]);
  }
  const T r = w[0], p = w[4], g = a.gamma;
  const T ir = rcp(r);
  const T gp = g * p;
  T s[5];
  s[0] = -(((w[1] * dw[0][0] + r * dw[0][1]) + (w[2] * dw[1][0] + r * dw[1][2])) +
           (w[3] * dw[2][0] + r * dw[2][3]));
#pragma unroll
  for (int k = 0; k < 3; ++k)
    s[1 + k] = -((w[1] * dw[0][1 + k] + w[2] * dw[1][1 + k]) + w[3] * dw[2][1 + k]) - dw[k][4] * ir;
  s[4] = -(((w[1] * dw[0][4] + gp * dw[0][1]) + (w[2] * dw[1][4] + gp * dw[1][2])) +
           (w[3] * dw[2][4] + gp * dw[2][3]));
  const T hdt = T(0.5) * level_dtdx(a);
#pragma unroll
  for (int v = 0; v < 5; ++v) a.Q[v * a.LS + t] = w[v] + hdt * s[v];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < 5; ++v) a.Q[(5 + 5 * d + v) * a.LS + t] = dw[d][v];
}

// the two faces of local cell t along axis D; du += F(minus) - F(plus)
template <int D, class T>
__device__ __forceinline__ void faces_dir(const LevelArgs<T> &a, int t, int e, int c, T dtdx,
                                          T (&du)[5]) {
  constexpr int d1 = D == 0 ? 1 : 0, d2 = D == 2 ? 1 : 2;
  const int ab = (((c >> d1) & 1) << 1) | ((c >> d2) & 1);
  T Fm[5] = {T(0), T(0), T(0), T(0), T(0)}, Fp[5] = {T(0), T(0), T(0), T(0), T(0)};
  const int tm = nbr_local(a, t, e, c, D, 0);
  if (!cell_is_split(a, tm)) {
    face_flux<D>(a, tm, t, Fm);
    if (a.reflux && (tm >> 3) >= a.nl) {  // ghost on the minus side
      const int gslot = (a.clo + (tm >> 3) - a.nl) * 24 + (2 * D + 1) * 4 + ab;
#pragma unroll
      for (int v = 0; v < 5; ++v) a.C[v * a.CS + gslot] = (T(-1) * dtdx) * Fm[v] / T(8);
    }
  }
  const int tp = nbr_local(a, t, e, c, D, 1);
  if (!cell_is_split(a, tp)) {
    face_flux<D>(a, t, tp, Fp);
    if (a.reflux && (tp >> 3) >= a.nl) {  // ghost on the plus side
      const int gslot = (a.clo + (tp >> 3) - a.nl) * 24 + (2 * D) * 4 + ab;
#pragma unroll
      for (int v = 0; v < 5; ++v) a.C[v * a.CS + gslot] = (T(1) * dtdx) * Fp[v] / T(8);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) du[v] = Fm[v] - Fp[v];
}

template <class T>
__global__ void k_flux_update(LevelArgs<T> a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * a.nl) return;
  if (cell_is_split(a, t)) return;
  const int e = a.lo + (t >> 3);
  const int c = t & 7;
  const T dtdx = level_dtdx(a);
  T dx[5], dy[5], dz[5];
  faces_dir<0>(a, t, e, c, dtdx, dx);
  faces_dir<1>(a, t, e, c, dtdx, dy);
  faces_dir<2>(a, t, e, c, dtdx, dz);
  const int g = 8 * e + c;
  const int rs = __ldg(a.rslot + g);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T *Ug = a.U + v * a.S + g;
    T u = *Ug + dtdx * ((dx[v] + dy[v]) + dz[v]);
    if (rs >= 0) {
      T *Rv = a.Rc + v * int64_t(a.NC) + rs;
      u = u + *Rv;
      *Rv = T(0);
    }
    *Ug = u;
  }
}

// k_reflux and k_restrict in one launch: they touch disjoint data (reflux
// sums go to the pending reflux of leaf cells of level l-1, restriction
// writes split cells of level l-1)
template <class T>
__global__ void k_reflux_restrict(LevelArgs<T> a, int do_restrict) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int nref = a.reflux ? 5 * a.ncl : 0;
  if (q < nref) {
    const int v = q / a.ncl;
    const int s = a.clo + (q - v * a.ncl);
    const T *cv = a.C + v * a.CS + 24 * int64_t(s);
    T *Rv = a.Rc + v * int64_t(a.NC) + s;
    T acc = *Rv;
#pragma unroll
    for (int k = 0; k < 24; ++k) acc += cv[k];
    *Rv = acc;
    return;
  }
  const int r = q - nref;
  if (!do_restrict || r >= 5 * a.nl) return;
  const int v = r / a.nl;
  const int o = a.lo + (r - v * a.nl);
  const uint64_t k = __ldg(a.key + o);
  const int fc = int((key_x(k) & 1) | ((key_y(k) & 1) << 1) | ((key_z(k) & 1) << 2));
  const int f = __ldg(a.father + o);
  const T *src = a.U + v * a.S + 8 * o;
  T sum = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) sum += src[c];
  a.U[v * a.S + 8 * f + fc] = sum * T(0.125);
}

// ---------------------------------------------------------------------------
// CFL time step: per-level max of sum_d (|u_d| + c) over leaf cells (cell
// speeds in the state's precision, the maximum and dt in FP64), warp-shuffle
// then block reduction, one integer atomicMax per block on the bit pattern
// (non-negative doubles order like their bits), then dt on one thread.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_cfl(CflArgs a, const T *U) {
  const int l = a.lmin + blockIdx.y;
  const int64_t lo = a.lo[l], n8 = 8 * (a.lo[l + 1] - lo);
  const T g = T(a.gamma), smallr = T(a.smallr), smallp = T(a.smallp);
  double s = 0.0;
  bool bad = false;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n8;
       t += int64_t(gridDim.x) * blockDim.x) {
    if ((__ldg(a.son + lo + (t >> 3)) >> (t & 7)) & 1u) continue;
    const int64_t gi = 8 * lo + t;
    const T u0 = U[gi], u1 = U[a.S + gi], u2 = U[2 * a.S + gi], u3 = U[3 * a.S + gi],
            u4 = U[4 * a.S + gi];
    const T r = vmax(u0, smallr);
    const T ir = rcp(r);
    const T vx = u1 * ir, vy = u2 * ir, vz = u3 * ir;
    const T ek = T(0.5) * r * ((vx * vx + vy * vy) + vz * vz);
    const T p = vmax((g - T(1)) * (u4 - ek), r * smallp);
    const T cs = vsqrt(g * p * ir);
    const T st = ((fabs(vx) + cs) + (fabs(vy) + cs)) + (fabs(vz) + cs);
    if (!isfinite(st) || !isfinite(u0 + u1 + u2 + u3 + u4))
      bad = true;
    else
      s = fmax(s, double(st));
  }
  if (bad) atomicOr(a.err, kErrNaN);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
  __shared__ double wmax[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) wmax[warp] = s;
  __syncthreads();
  if (warp == 0) {
    s = lane < int(blockDim.x >> 5) ? wmax[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
    if (lane == 0 && s > 0.0) atomicMax(a.smax + l, (unsigned long long)__double_as_longlong(s));
  }
}

__global__ void k_dt(CflArgs a) {
  double dt = __longlong_as_double(0x7FF0000000000000ll);  // +inf
  for (int l = a.lmin; l <= a.lmax; ++l) {
    const unsigned long long b = a.smax[l];
    a.smax[l] = 0ull;
    if (b == 0ull) continue;
    const double smax = __longlong_as_double((long long)b);
    const double dtl = a.cfl * ldexp(1.0, -l) / smax;
    const double dtc = dtl * ldexp(1.0, l - a.lmin);
    dt = fmin(dt, dtc);
  }
  *a.dt_dev = dt;
  *a.dtf_dev = float(dt);
}

template <class T>
__global__ void k_to_double(const T *src, int64_t src_stride, int64_t count, double *dst) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 5 * count) return;
  const int v = int(q / count);
  dst[q] = double(src[v * src_stride + q % count]);
}
template <class T>
__global__ void k_from_double(const double *src, int64_t count, T *dst, int64_t dst_stride) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 5 * count) return;
  const int v = int(q / count);
  dst[v * dst_stride + q % count] = T(src[q]);
}

}  // namespace amr
