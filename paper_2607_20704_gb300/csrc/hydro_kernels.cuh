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
//   k_reflux_restrict  fixed-order sum of coarse-fine fluxes for the coarse
//               cells, and father cell = mean of its 8 children
//
// (FP32 fuses k_prim into k_predict_u and k_flux with k_update.)
//
// The paper's kernels gather a 6x6x6 stencil per oct and recompute the
// slopes and predictor of its ghost ring (8x work per cell at nsubgrid=1).
// On GB300 the FP64 rate is far below the memory rate, so each cell's
// predictor and each face's Riemann solve is computed exactly once and the
// intermediate states go through L2/HBM instead.
//
// Every kernel is persistent over a flattened work list of tiles, each tile
// one block's worth of items of one (member mesh, level) segment, so one
// launch advances a level of many meshes at once.
#pragma once
#include "hydro_args.cuh"

namespace amr {

// ---------------------------------------------------------------------------
// arithmetic helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double minmod(double a, double b) {
  // 0 for opposite signs or a zero argument, else the argument of smaller
  // magnitude; decided on the bit patterns (integer pipes, no FP64 issue):
  // the bits shifted left by one drop the sign and order the magnitudes
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const unsigned long long ma = (unsigned long long)ia << 1, mb = (unsigned long long)ib << 1;
  if (((ia ^ ib) < 0) | (ma == 0) | (mb == 0)) return 0.0;
  return ma < mb ? a : b;
}
// FP32: the definition as written, 0 when a b <= 0 (the FP32 pipes have room)
__device__ __forceinline__ float minmod(float a, float b) {
  const float m = fabsf(a) < fabsf(b) ? a : b;
  return a * b > 0.0f ? m : 0.0f;
}
// FP64 compares, min and max decided on the bit patterns: GB300's FP64 pipe
// is 1/64 of its FP32 rate and these kernels are bound by it, while the
// integer pipes have room.  ord() maps a non-NaN double to a signed integer
// of the same order (-0 just below +0); a NaN argument propagates instead of
// being dropped (the time-step reduction reports it).
__device__ __forceinline__ long long ord(double x) {
  const long long i = __double_as_longlong(x);
  return i ^ ((i >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double vmax(double a, double b) { return ord(a) < ord(b) ? b : a; }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return ord(b) < ord(a) ? b : a; }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
// x > 0
__device__ __forceinline__ bool pos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool pos(float x) { return x > 0.0f; }
// x is neither infinite nor NaN (exponent field not all ones)
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
}
__device__ __forceinline__ bool finite_bits(float x) {
  return ((__float_as_int(x) >> 23) & 0xFF) != 0xFF;
}
// a > b for a, b >= 0
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool gt_nonneg(float a, float b) { return __float_as_int(a) > __float_as_int(b); }
__device__ __forceinline__ double vsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }

// 1/x from the hardware's approximate reciprocal r (relative error near
// 2^-20 on GB300, measured) by one third-order step of the series
// 1/x = r / (1 - e) = r (1 + e + e^2 + ...), e = 1 - x r: the error drops to
// about e^3 (2^-60), so the result is within an ulp or two of 1/x, as two
// Newton steps would give, with three FMAs instead of four (checked against
// the correctly rounded quotient by the parity tests).  Operands here are
// positive, finite and normal (densities, sums of rho |u - S|, wave-speed
// gaps), so the flush-to-zero form is safe.
__device__ __forceinline__ double rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 1/sqrt(x) from the hardware approximation y (x y^2 within about 2^-19 of
// 1, measured) by one third-order step of the binomial series
// (1 - h)^(-1/2) = 1 + h/2 + 3h^2/8 + ..., h = 1 - x y^2: the error drops to
// about h^3, double precision in five operations (two Newton steps take
// seven).  x is a positive normal number here (gamma p rho).
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = fma(-x, y * y, 1.0);
  return fma(y, h * fma(0.375, h, 0.5), y);
}
__device__ __forceinline__ float rsqrt_nr(float x) { return rsqrtf(x); }

// sqrt(c2) of the time-step reduction: c2 rsqrt(c2) in FP64 (within an ulp
// or two of the correctly rounded root; 0 for c2 = 0; NaN propagates), the
// library's sqrtf in FP32
__device__ __forceinline__ double sound_speed(double c2) { return c2 > 0.0 ? c2 * rsqrt_nr(c2) : sqrt(c2); }
__device__ __forceinline__ float sound_speed(float c2) { return sqrtf(c2); }

// ---------------------------------------------------------------------------
// segment context: what a thread needs to know about its (member, level)
// ---------------------------------------------------------------------------
template <class T>
struct SegCtx {
  int lo, nl, clo, ncl, base, flags;
  T gamma, igm1, smallr, smallp, dtdx;
};

__device__ __forceinline__ double seg_dtdx(const StepArgs<double> &a, const Seg &s) {
  return a.dtdx_dev ? __ldg(a.dtdx_dev + s.member) : ldexp(a.dt_host, s.level);
}
__device__ __forceinline__ float seg_dtdx(const StepArgs<float> &a, const Seg &s) {
  // scaling by a power of two is exact, so this is float(dt 2^l)
  return a.dtdxf_dev ? __ldg(a.dtdxf_dev + s.member) : ldexpf(float(a.dt_host), s.level);
}

template <class T>
__device__ __forceinline__ SegCtx<T> seg_ctx(const StepArgs<T> &a, int seg) {
  const Seg s = a.segs[seg];
  SegCtx<T> c;
  c.lo = s.lo;
  c.nl = s.nl;
  c.clo = s.clo;
  c.ncl = s.ncl;
  c.base = s.base;
  c.flags = s.flags;
  c.gamma = __ldg(a.mgamma + s.member);
  c.igm1 = __ldg(a.migm1 + s.member);
  c.smallr = __ldg(a.msmallr + s.member);
  c.smallp = __ldg(a.msmallp + s.member);
  c.dtdx = seg_dtdx(a, s);
  return c;
}

// persistent loop over the launch's tiles: body(ctx, item) for every item of
// the tile that lies inside the segment's domain of `size(ctx)` items
template <class T, class Size, class Body>
__device__ __forceinline__ void tile_loop(const StepArgs<T> &a, Size size, Body body) {
  for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
    const Tile td = tile_at(a.tpre, a.tseg0, a.tnseg, a.tstep, ti);
    if (a.mact && !__ldg(a.mact + a.segs[td.seg].member)) continue;  // finished member
    const SegCtx<T> sc = seg_ctx(a, td.seg);
#ifdef AMR_CHECKED
    // the segment's local cells must fit the scratch arrays
    if (sc.base < 0 || sc.base + 8 * (sc.nl + sc.ncl) > a.LS) {
      atomicOr(a.err, kErrIndex);
      continue;
    }
#endif
    const int item = td.start + threadIdx.x;
    if (item < size(sc)) body(sc, item);
  }
}

// extended oct index of local oct index q, and back
template <class T>
__device__ __forceinline__ int ext_of_local(const StepArgs<T> &a, const SegCtx<T> &s, int q) {
  return q < s.nl ? s.lo + q : a.N + s.clo + (q - s.nl);
}
template <class T>
__device__ __forceinline__ int local_of_ext(const StepArgs<T> &a, const SegCtx<T> &s, int e) {
  return e < a.N ? e - s.lo : e - a.N - s.clo + s.nl;
}

// local index of the face neighbour of local cell t (extended oct e, cell c)
// along axis d on side `plus`; -1 when the neighbouring oct does not exist
template <class T>
__device__ __forceinline__ int nbr_local(const StepArgs<T> &a, const SegCtx<T> &s, int t, int e,
                                         int c, int d, int plus) {
  const int bit = 1 << d;
  if (((c >> d) & 1) != plus) return t ^ bit;
  const int32_t ne = __ldg(a.fnb + (2 * d + plus) * int64_t(a.NE) + e);
  if (ne < 0) return -1;
  // a face neighbour is in the same (member, level) segment: else "none"
  const int q = int(checked(local_of_ext(a, s, ne), 0, s.nl + s.ncl, a.err, -1));
  return q < 0 ? -1 : 8 * q + (c ^ bit);
}

template <class T>
__device__ __forceinline__ bool cell_is_split(const StepArgs<T> &a, const SegCtx<T> &s, int t) {
  const int q = t >> 3;
  if (q >= s.nl) return false;  // ghost cells are leaves
  return (__ldg(a.son + s.lo + q) >> (t & 7)) & 1u;
}

// ---------------------------------------------------------------------------
// ghost octs: child = U_C + sum_d (+-1/4) minmod(U(C+e_d)-U(C), U(C)-U(C-e_d))
// domain: 5 * ncl (variable, ghost oct)
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_prolong(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 5 * s.ncl; }, [&](const SegCtx<T> &s, int q) {
    const int v = q / s.ncl;
    const int cs = s.clo + (q - v * s.ncl);
    const T *Uv = a.U + v * a.S;
    T src[7];
#pragma unroll
    for (int k = 0; k < 7; ++k)
      src[k] = Uv[checked(__ldg(a.csrc + k * int64_t(a.NC) + cs), 0, 8 * int64_t(a.NE), a.err)];
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
  });
}

// ---------------------------------------------------------------------------
// primitives of every real and ghost cell; domain: 8 (nl + ncl)
// ---------------------------------------------------------------------------
// primitives (rho, u, v, w, p) of the conservative state (u0..u4), with the
// density and pressure floors
template <class T>
__device__ __forceinline__ void prim_of(const SegCtx<T> &s, T u0, T u1, T u2, T u3, T u4, T (&w)[5]) {
  const T r = vmax(u0, s.smallr);
  const T ir = rcp(r);
  const T vx = u1 * ir, vy = u2 * ir, vz = u3 * ir;
  const T ek = T(0.5) * r * ((vx * vx + vy * vy) + vz * vz);
  w[0] = r;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = vmax((s.gamma - T(1)) * (u4 - ek), r * s.smallp);
}

template <class T>
__device__ __forceinline__ void prim_at(const StepArgs<T> &a, const SegCtx<T> &s, int t,
                                        T (&w)[5]) {
  const int g = 8 * ext_of_local(a, s, t >> 3) + (t & 7);
  prim_of(s, a.U[g], a.U[a.S + g], a.U[2 * a.S + g], a.U[3 * a.S + g], a.U[4 * a.S + g], w);
}

template <class T>
__global__ void k_prim(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 8 * (s.nl + s.ncl); },
            [&](const SegCtx<T> &s, int t) {
              T w[5];
              prim_at(a, s, t, w);
              const int o = s.base + t;
#pragma unroll
              for (int v = 0; v < 5; ++v) a.W[v * a.LS + o] = w[v];
            });
}

// ---------------------------------------------------------------------------
// limited slopes and Hancock predictor W* = W + dt/(2dx) S(W, dW)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void predictor(const SegCtx<T> &s, const T (&w)[5],
                                          const T (&dw)[3][5], T (&ws)[5]) {
  const T r = w[0], p = w[4], g = s.gamma;
  const T ir = rcp(r);
  const T gp = g * p;
  T src[5];
  src[0] = -(((w[1] * dw[0][0] + r * dw[0][1]) + (w[2] * dw[1][0] + r * dw[1][2])) +
             (w[3] * dw[2][0] + r * dw[2][3]));
#pragma unroll
  for (int k = 0; k < 3; ++k)
    src[1 + k] =
        -((w[1] * dw[0][1 + k] + w[2] * dw[1][1 + k]) + w[3] * dw[2][1 + k]) - dw[k][4] * ir;
  src[4] = -(((w[1] * dw[0][4] + gp * dw[0][1]) + (w[2] * dw[1][4] + gp * dw[1][2])) +
             (w[3] * dw[2][4] + gp * dw[2][3]));
  const T hdt = T(0.5) * s.dtdx;
#pragma unroll
  for (int v = 0; v < 5; ++v) ws[v] = w[v] + hdt * src[v];
}

template <class T>
__device__ __forceinline__ void store_q(const StepArgs<T> &a, int o, const T (&ws)[5],
                                        const T (&dw)[3][5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) a.Q[v * a.LS + o] = ws[v];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < 5; ++v) a.Q[(5 + 5 * d + v) * a.LS + o] = dw[d][v];
}

template <class T>
__global__ void k_predict(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 8 * (s.nl + s.ncl); },
            [&](const SegCtx<T> &s, int t) {
              const int e = ext_of_local(a, s, t >> 3);
              const int c = t & 7;
              const int o = s.base + t;
              T w[5], dw[3][5], ws[5];
#pragma unroll
              for (int v = 0; v < 5; ++v) w[v] = a.W[v * a.LS + o];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                const int tm = nbr_local(a, s, t, e, c, d, 0);
                const int tp = nbr_local(a, s, t, e, c, d, 1);
                if (tm < 0 || tp < 0) {  // outer ring of a ghost oct: never used
#pragma unroll
                  for (int v = 0; v < 5; ++v) dw[d][v] = T(0);
                  continue;
                }
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                  const T wm = a.W[v * a.LS + s.base + tm], wp = a.W[v * a.LS + s.base + tp];
                  dw[d][v] = minmod(wp - w[v], w[v] - wm);
                }
              }
              predictor(s, w, dw, ws);
              store_q(a, o, ws, dw);
            });
}

// FP32: primitives of the cell and its six face neighbours derived from U
// directly (no W array)
template <class T>
__global__ void __launch_bounds__(512, 3) k_predict_u(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 8 * (s.nl + s.ncl); },
            [&](const SegCtx<T> &s, int t) {
              const int e = ext_of_local(a, s, t >> 3);
              const int c = t & 7;
              T w[5], dw[3][5], ws[5];
              prim_at(a, s, t, w);
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                const int tm = nbr_local(a, s, t, e, c, d, 0);
                const int tp = nbr_local(a, s, t, e, c, d, 1);
                if (tm < 0 || tp < 0) {
#pragma unroll
                  for (int v = 0; v < 5; ++v) dw[d][v] = T(0);
                  continue;
                }
                T wm[5], wp[5];
                prim_at(a, s, tm, wm);
                prim_at(a, s, tp, wp);
#pragma unroll
                for (int v = 0; v < 5; ++v) dw[d][v] = minmod(wp[v] - w[v], w[v] - wm[v]);
              }
              predictor(s, w, dw, ws);
              store_q(a, s.base + t, ws, dw);
            });
}

// max(c_L, c_R) with c^2 = gamma p / rho, from a = gamma p and rho per side.
// FP64: c^2 compared by cross-multiplication, then for the larger side
// c = a / sqrt(a rho) -- one reciprocal square root instead of a reciprocal
// and a square root.  FP32 keeps the quotient form: a rho can leave float's
// range at the density and pressure floors (about 1e-41), a / rho cannot.
__device__ __forceinline__ double max_sound_speed(double al, double rl, double ar, double rr) {
  const bool lbig = gt_nonneg(al * rr, ar * rl);
  const double a = lbig ? al : ar;
  return a * rsqrt_nr(a * (lbig ? rl : rr));
}
__device__ __forceinline__ float max_sound_speed(float al, float rl, float ar, float rr) {
  return sqrtf(fmaxf(al * rcp(rl), ar * rcp(rr)));
}

// ---------------------------------------------------------------------------
// HLLC flux normal to axis D from face states qL, qR (rho, u, v, w, p):
// S_L = min(u) - max(c), S_R = max(u) + max(c); star speed and pressure from
// the two-wave HLL jump conditions; physical flux of the state sampled at
// x/t = 0 (Toro's HLLC); transverse velocities from the upwind side.
// max(c) of the two sides, c^2 = gamma p / rho (see max_sound_speed).
// ---------------------------------------------------------------------------
template <int D, class T>
__device__ __forceinline__ void hllc(const T (&qL)[5], const T (&qR)[5], T g, T igm1, T (&F)[5]) {
  constexpr int in = 1 + D, t1 = D == 0 ? 2 : 1, t2 = D == 2 ? 2 : 3;
  const T rl = qL[0], ul = qL[in], pl = qL[4];
  const T rr = qR[0], ur = qR[in], pr = qR[4];
  // total energy of a side (computed for the sampled side only)
  auto energy = [igm1](const T(&q)[5]) {
    return q[4] * igm1 + T(0.5) * q[0] * ((q[1] * q[1] + q[2] * q[2]) + q[3] * q[3]);
  };
  const T cmax = max_sound_speed(g * pl, rl, g * pr, rr);
  const T sl = vmin(ul, ur) - cmax;
  const T sr = vmax(ul, ur) + cmax;
  const T rcl = rl * (ul - sl), rcr = rr * (sr - ur);
  const T irc = rcp(rcl + rcr);
  const T us = ((rcr * ur + rcl * ul) + (pl - pr)) * irc;
  const T ps = ((rcr * pl + rcl * pr) + rcl * rcr * (ul - ur)) * irc;
  // The sampled side K is the left one when S_L > 0 or u* > 0; its star
  // state is taken when S_L <= 0 (left) or S_R > 0 (right).  Selected
  // without divergent branches: the side's state and energy, then one star
  // state (unused in the supersonic cases) with the arithmetic of Toro's
  // four cases.
  T ro, uo, po, eo, v1, v2;
  {
    const bool left = pos(sl) || pos(us);
    const bool star = left ? !pos(sl) : pos(sr);
    T qk[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qk[v] = left ? qL[v] : qR[v];
    const T rk = qk[0], uk = qk[in], pk = qk[4], ek = energy(qk);
    const T sk = left ? sl : sr;
    v1 = qk[t1];
    v2 = qk[t2];
    const T id = rcp(sk - us);
    const T rs = rk * (sk - uk) * id;
    const T es = ((sk - uk) * ek - pk * uk + ps * us) * id;
    ro = star ? rs : rk;
    eo = star ? es : ek;
    uo = star ? us : uk;
    po = star ? ps : pk;
  }
  const T mf = ro * uo;
  F[0] = mf;
  F[in] = mf * uo + po;
  F[t1] = mf * v1;
  F[t2] = mf * v2;
  F[4] = (eo + po) * uo;
}

// face states W* +- dW/2 of the two cells of a face (with the floors) and
// their HLLC flux
template <int D, class T>
__device__ __forceinline__ void face_flux_states(const SegCtx<T> &s, T (&qL)[5], T (&qR)[5], T (&F)[5]) {
  qL[0] = vmax(qL[0], s.smallr);
  qR[0] = vmax(qR[0], s.smallr);
  qL[4] = vmax(qL[4], qL[0] * s.smallp);
  qR[4] = vmax(qR[4], qR[0] * s.smallp);
  hllc<D>(qL, qR, s.gamma, s.igm1, F);
}

// flux across the face between local cells tl (minus side) and tr (plus side)
template <int D, class T>
__device__ __forceinline__ void face_flux(const StepArgs<T> &a, const SegCtx<T> &s, int tl, int tr,
                                          T (&F)[5]) {
  T qL[5], qR[5];
  const int ol = s.base + tl, orr = s.base + tr;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    // Q is read-only while faces are solved (the read-only path lets the
    // compiler keep a cell's values across its faces)
    qL[v] = __ldg(a.Q + v * a.LS + ol) + T(0.5) * __ldg(a.Q + (5 + 5 * D + v) * a.LS + ol);
    qR[v] = __ldg(a.Q + v * a.LS + orr) - T(0.5) * __ldg(a.Q + (5 + 5 * D + v) * a.LS + orr);
  }
  face_flux_states<D>(s, qL, qR, F);
}

// reflux slot of a coarse-fine face: ghost oct g (local oct index), the
// direction of the face seen from the ghost's father cell X, fine face (a,b)
template <int D>
__device__ __forceinline__ int64_t reflux_slot(int clo, int nl, int gq, int dirX, int c) {
  constexpr int d1 = D == 0 ? 1 : 0, d2 = D == 2 ? 1 : 2;
  const int ab = (((c >> d1) & 1) << 1) | ((c >> d2) & 1);
  return int64_t(clo + gq - nl) * 24 + dirX * 4 + ab;
}

template <int D, class T>
__device__ __forceinline__ void flux_dir(const StepArgs<T> &a, const SegCtx<T> &s, int t, int e,
                                         int c, bool real, bool split) {
  T F[5] = {T(0), T(0), T(0), T(0), T(0)};
  const int tn = nbr_local(a, s, t, e, c, D, 1);
  bool need = false, nreal = false;
  if (tn >= 0) {
    nreal = (tn >> 3) < s.nl;
    need = (real || nreal) && !split && !cell_is_split(a, s, tn);
  }
  if (need) {
    face_flux<D>(a, s, t, tn, F);
    if (a.reflux && (real != nreal)) {
      // ghost on the plus side: the coarse cell's minus face (sigma +1);
      // ghost on the minus side: its plus face (sigma -1)
      const int64_t gslot = real ? reflux_slot<D>(s.clo, s.nl, tn >> 3, 2 * D, c)
                             : reflux_slot<D>(s.clo, s.nl, t >> 3, 2 * D + 1, c);
      const T sg = real ? T(1) : T(-1);
#pragma unroll
      for (int v = 0; v < 5; ++v)
        a.C[v * a.CS + checked(gslot, 0, a.CS, a.err)] = (sg * s.dtdx) * F[v] / T(8);
    }
  }
  const int o = s.base + t;
#pragma unroll
  for (int v = 0; v < 5; ++v) a.F[(5 * D + v) * a.LS + o] = F[v];
}

// One thread per real or ghost cell: the fluxes of its three plus faces.
// A face is needed when at least one side is a real cell and neither side
// is split; other faces carry zero.  A needed face with a ghost on one side
// is a coarse-fine face: its flux, times sigma dt/dx / 8, goes to slot
// (direction seen from the coarse cell, fine face a,b) of the ghost oct.
template <class T>
__global__ void k_flux(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 8 * (s.nl + s.ncl); },
            [&](const SegCtx<T> &s, int t) {
              const int q = t >> 3;
              const int e = ext_of_local(a, s, q);
              const int c = t & 7;
              const bool real = q < s.nl;
              const bool split = cell_is_split(a, s, t);
              flux_dir<0>(a, s, t, e, c, real, split);
              flux_dir<1>(a, s, t, e, c, real, split);
              flux_dir<2>(a, s, t, e, c, real, split);
            });
}

// U <- (U + dt/dx sum_d (F_d- - F_d+)) + R on leaf cells; R <- 0.  The new
// state goes to `out` (stride `ostride`): U itself, or a buffer when other
// blocks may still read the old state.
template <class T>
__device__ __forceinline__ void update_cell_to(const StepArgs<T> &a, const SegCtx<T> &s, int g,
                                               const T (&dx)[5], const T (&dy)[5], const T (&dz)[5],
                                               T *out, int64_t ostride) {
  const int rs = int(checked(__ldg(a.rslot + g), -1, a.NC, a.err, -1));
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T u = a.U[v * a.S + g] + s.dtdx * ((dx[v] + dy[v]) + dz[v]);
    if (rs >= 0) {
      T *Rv = a.Rc + v * int64_t(a.NC) + rs;
      u = u + *Rv;
      *Rv = T(0);
    }
    out[v * ostride] = u;
  }
}

template <class T>
__device__ __forceinline__ void update_cell(const StepArgs<T> &a, const SegCtx<T> &s, int g,
                                            const T (&dx)[5], const T (&dy)[5], const T (&dz)[5]) {
  update_cell_to(a, s, g, dx, dy, dz, a.U + g, a.S);
}

template <class T>
__global__ void k_update(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 8 * s.nl; }, [&](const SegCtx<T> &s, int t) {
    if (cell_is_split(a, s, t)) return;
    const int e = s.lo + (t >> 3);
    const int c = t & 7;
    const int o = s.base + t;
    const int om[3] = {s.base + nbr_local(a, s, t, e, c, 0, 0), s.base + nbr_local(a, s, t, e, c, 1, 0),
                       s.base + nbr_local(a, s, t, e, c, 2, 0)};
    T dx[5], dy[5], dz[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      dx[v] = a.F[(0 + v) * a.LS + om[0]] - a.F[(0 + v) * a.LS + o];
      dy[v] = a.F[(5 + v) * a.LS + om[1]] - a.F[(5 + v) * a.LS + o];
      dz[v] = a.F[(10 + v) * a.LS + om[2]] - a.F[(10 + v) * a.LS + o];
    }
    update_cell(a, s, 8 * e + c, dx, dy, dz);
  });
}

// FP32: the two faces of local cell t along axis D, du = F(minus) - F(plus);
// each interior face is solved by both of its cells (bit-identically), and a
// coarse-fine face by its real cell, which also fills the reflux slot
template <int D, class T>
__device__ __forceinline__ void faces_dir(const StepArgs<T> &a, const SegCtx<T> &s, int t, int e,
                                          int c, T (&du)[5]) {
  T Fm[5] = {T(0), T(0), T(0), T(0), T(0)}, Fp[5] = {T(0), T(0), T(0), T(0), T(0)};
  const int tm = nbr_local(a, s, t, e, c, D, 0);
  if (!cell_is_split(a, s, tm)) {
    face_flux<D>(a, s, tm, t, Fm);
    if (a.reflux && (tm >> 3) >= s.nl) {
      const int64_t gslot = reflux_slot<D>(s.clo, s.nl, tm >> 3, 2 * D + 1, c);
#pragma unroll
      for (int v = 0; v < 5; ++v)
        a.C[v * a.CS + checked(gslot, 0, a.CS, a.err)] = (T(-1) * s.dtdx) * Fm[v] / T(8);
    }
  }
  const int tp = nbr_local(a, s, t, e, c, D, 1);
  if (!cell_is_split(a, s, tp)) {
    face_flux<D>(a, s, t, tp, Fp);
    if (a.reflux && (tp >> 3) >= s.nl) {
      const int64_t gslot = reflux_slot<D>(s.clo, s.nl, tp >> 3, 2 * D, c);
#pragma unroll
      for (int v = 0; v < 5; ++v)
        a.C[v * a.CS + checked(gslot, 0, a.CS, a.err)] = (T(1) * s.dtdx) * Fp[v] / T(8);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) du[v] = Fm[v] - Fp[v];
}

template <class T>
__global__ void __launch_bounds__(512, 3) k_flux_update(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 8 * s.nl; }, [&](const SegCtx<T> &s, int t) {
    if (cell_is_split(a, s, t)) return;
    const int e = s.lo + (t >> 3);
    const int c = t & 7;
    T dx[5], dy[5], dz[5];
    faces_dir<0>(a, s, t, e, c, dx);
    faces_dir<1>(a, s, t, e, c, dy);
    faces_dir<2>(a, s, t, e, c, dz);
    update_cell(a, s, 8 * e + c, dx, dy, dz);
  });
}

// Reflux: R(X) += sum of the 24 slots of the ghost oct whose father is X, in
// slot order (direction -x,+x,-y,+y,-z,+z seen from X, then fine face).
// Restriction: father cell = (sum of the 8 children in child order) / 8.
// They touch disjoint data (leaf cells' pending reflux, split cells).
// domain: 5 ncl (if kSegReflux) + 5 nl (if kSegRestrict)
template <class T>
__global__ void k_reflux_restrict(StepArgs<T> a) {
  tile_loop(a,
            [](const SegCtx<T> &s) {
              return ((s.flags & kSegReflux) ? 5 * s.ncl : 0) + ((s.flags & kSegRestrict) ? 5 * s.nl : 0);
            },
            [&](const SegCtx<T> &s, int q) {
              const int nref = (s.flags & kSegReflux) ? 5 * s.ncl : 0;
              if (q < nref) {
                const int v = q / s.ncl;
                const int g = s.clo + (q - v * s.ncl);
                const T *cv = a.C + v * a.CS + 24 * int64_t(g);
                T *Rv = a.Rc + v * int64_t(a.NC) + g;
                T acc = *Rv;
#pragma unroll
                for (int k = 0; k < 24; ++k) acc += cv[k];
                *Rv = acc;
                return;
              }
              const int r = q - nref;
              const int v = r / s.nl;
              const int o = s.lo + (r - v * s.nl);
              const uint64_t k = __ldg(a.key + o);
              const int fc = int((ikey_x(k) & 1) | ((ikey_y(k) & 1) << 1) | ((ikey_z(k) & 1) << 2));
              const int f = int(checked(__ldg(a.father + o), 0, a.N, a.err));
              const T *src = a.U + v * a.S + 8 * int64_t(o);
              T sum = T(0);
#pragma unroll
              for (int c = 0; c < 8; ++c) sum += src[c];
              a.U[v * a.S + 8 * int64_t(f) + fc] = sum * T(0.125);
            });
}

// ---------------------------------------------------------------------------
// CFL time step: per (member, level) max of sum_d (|u_d| + c) over leaf cells
// (cell speeds in the state's precision, the maximum and dt in FP64): block
// reduction of each tile (warp shuffles, then shared memory), one integer
// atomicMax per tile on the bit pattern (non-negative doubles order like their
// bits); then one thread per member computes its dt.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void cfl_flush(const CflArgs &a, double s, int seg, double *wmax) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
  if (lane == 0) wmax[warp] = s;
  __syncthreads();
  if (warp == 0) {
    s = lane < int(blockDim.x >> 5) ? wmax[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
    if (lane == 0 && s > 0.0) {
      const Seg sg = a.segs[seg];
      atomicMax(a.smax + 16 * sg.member + sg.level, (unsigned long long)__double_as_longlong(s));
    }
  }
  __syncthreads();
}

// Each block keeps a running maximum per thread while its tiles stay in one
// segment and reduces it (one atomicMax) when the segment changes.
// The running maximum is kept in the state's type (float to double is exact
// and monotonic, so converting once per flush gives the same maximum) and
// the parameters are read in that type: no conversions per cell, which would
// run on the FP64 pipe.
template <class T>
__global__ void k_cfl(CflArgs a, const T *U) {
  __shared__ double wmax[32];
  T s = T(0);
  int cur = -1;
  const T *mgamma = static_cast<const T *>(a.mgamma_t), *msmallr = static_cast<const T *>(a.msmallr_t),
          *msmallp = static_cast<const T *>(a.msmallp_t);
  for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
    const Tile td = tile_at(a.tpre, a.tseg0, a.tnseg, a.tstep, ti);
    if (td.seg != cur) {
      if (cur >= 0) cfl_flush<T>(a, double(s), cur, wmax);
      s = T(0);
      cur = td.seg;
    }
    const Seg sg = a.segs[td.seg];
    const int t = td.start + threadIdx.x;
    if (t < 8 * sg.nl && a.mrem[sg.member] != 0 &&
        !((__ldg(a.son + sg.lo + (t >> 3)) >> (t & 7)) & 1u)) {
      const T g = mgamma[sg.member], smallr = msmallr[sg.member], smallp = msmallp[sg.member];
      const int64_t gi = 8 * int64_t(sg.lo) + t;
      const T u0 = U[gi], u1 = U[a.S + gi], u2 = U[2 * a.S + gi], u3 = U[3 * a.S + gi],
              u4 = U[4 * a.S + gi];
      const T r = vmax(u0, smallr);
      const T ir = rcp(r);
      const T vx = u1 * ir, vy = u2 * ir, vz = u3 * ir;
      const T ek = T(0.5) * r * ((vx * vx + vy * vy) + vz * vz);
      const T p = vmax((g - T(1)) * (u4 - ek), r * smallp);
      const T cs = sound_speed(g * p * ir);
      const T st = ((fabs(vx) + cs) + (fabs(vy) + cs)) + (fabs(vz) + cs);
      if (!finite_bits(st) || !(finite_bits(u0) && finite_bits(u1) && finite_bits(u2) &&
                                finite_bits(u3) && finite_bits(u4))) {
        atomicOr(a.err, kErrNaN);
        atomicOr(a.merr + sg.member, kErrNaN);
      } else if (gt_nonneg(st, s)) {
        s = st;
      }
    }
  }
  if (cur >= 0) cfl_flush<T>(a, double(s), cur, wmax);
}

__global__ void k_dt(CflArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.nmembers) return;
  const int lmin = a.mlmin[m];
  double dt = __longlong_as_double(0x7FF0000000000000ll);  // +inf
  for (int l = lmin; l <= kMaxLev; ++l) {
    const unsigned long long b = a.smax[16 * m + l];
    a.smax[16 * m + l] = 0ull;
    if (b == 0ull) continue;
    const double smax = __longlong_as_double((long long)b);
    const double dtl = a.mcfl[m] * ldexp(1.0, -l) / smax;
    const double dtc = dtl * ldexp(1.0, l - lmin);
    dt = fmin(dt, dtc);
  }
  // a member with no coarse steps left keeps its state and its last dt
  const int rem = a.mrem[m];
  if (a.consume) {
    a.mact[m] = rem != 0;
    if (rem > 0) a.mrem[m] = rem - 1;
  }
  if (rem == 0) return;
  a.dt_dev[m] = dt;
  a.dtdx_dev[m] = ldexp(dt, lmin);
  a.dtdxf_dev[m] = ldexpf(float(dt), lmin);
}

// ---------------------------------------------------------------------------
// Conservation totals of one level (FP64 in both precisions, fixed order, no
// atomics): block b sums the leaf cells of [b chunk, (b+1) chunk) of the
// level's cells, thread t the cells b chunk + t + 256 k in increasing k, then
// a fixed butterfly over each warp and the 8 warp sums in warp order;
// partial[v G + b].  k_totals_sum adds a level's G partials in block order,
// scales by dx^3 (exact: a power of two) into lev[5 l + v], and with
// all_levels adds the levels' totals in ascending level order into out.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_totals(const T *__restrict__ U, int64_t S,
                                                const uint32_t *__restrict__ son, int64_t c0,
                                                int64_t n, int64_t chunk, double *partial, int G) {
  __shared__ double ws[5][8];
  const int64_t b0 = blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t t = b0 + threadIdx.x; t < b1; t += 256) {
    const int64_t g = c0 + t;
    if ((__ldg(son + (g >> 3)) >> (g & 7)) & 1u) continue;  // split: not a leaf
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += double(U[v * S + g]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[v] += __shfl_xor_sync(0xFFFFFFFFu, acc[v], off);
    if (lane == 0) ws[v][warp] = acc[v];
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += ws[threadIdx.x][w];
    partial[threadIdx.x * int64_t(G) + blockIdx.x] = sum;
  }
}

__global__ void k_totals_sum(const double *partial, int G, int level, double *lev, int all_levels,
                             int lmin, int lmax, double *out) {
  const int v = threadIdx.x;
  if (v >= 5) return;
  double sum = 0.0;
  for (int b = 0; b < G; ++b) sum += partial[v * int64_t(G) + b];
  lev[5 * level + v] = ldexp(sum, -3 * level);
  if (all_levels) {
    double t = 0.0;
    for (int l = lmin; l <= lmax; ++l) t += lev[5 * l + v];
    out[v] = t;
  } else {
    out[v] = lev[5 * level + v];
  }
}

template <class T>
__global__ void k_to_double(const T *src, int64_t src_stride, int64_t count, double *dst) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 5 * count) return;
  const int v = int(q / count);
  dst[q] = double(src[v * src_stride + q % count]);
}
// five rows of `count` doubles from src (row stride src_stride) to dst (row
// stride dst_stride), 16 bytes per thread; count and both strides even, both
// bases 16-byte aligned (the state's rows start at multiples of 8 cells)
__global__ void k_rows_copy(const double2 *__restrict__ src, int64_t src_stride2, int64_t count2,
                            double2 *__restrict__ dst, int64_t dst_stride2) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 5 * count2) return;
  const int64_t v = q / count2, j = q - v * count2;
  dst[v * dst_stride2 + j] = __ldg(src + v * src_stride2 + j);
}

template <class T>
__global__ void k_from_double(const double *src, int64_t count, T *dst, int64_t dst_stride) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 5 * count) return;
  const int v = int(q / count);
  dst[v * dst_stride + q % count] = T(src[q]);
}

}  // namespace amr
