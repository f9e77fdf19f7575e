// rock_kernels.cuh -- the level step as one fused shared-memory kernel per
// block of octs (the paper's "rock" kernel, Sec. 3, with `nsubgrid` NS octs
// per axis in the inner block), and the planar sweep (the paper's "paper"
// kernel) further down.
//
// A CTA takes one block: the real octs of one (member, level) segment that
// share an aligned NS^3 group of oct positions (consecutive in the level's
// Hilbert order).  Its cube is the block and one ring of octs around it, an
// E^3 cube of cells (E = 2 NS + 4), real or ghost octs found through the
// 27-neighbour table; the eight corner octs of the ring feed no face of the
// block and are not staged.  Phases, separated by block barriers:
//
//   A  each thread holds one cell of the block's own octs in registers (a
//      coalesced load in mesh order); every other oct of the cube is loaded
//      with 16-byte vector loads, 8 cells per (oct, variable)
//   B  primitives of every staged cell, in place
//   C  limited slopes and the Hancock predictor of the inner IN^3 cells
//      (IN = 2 NS; W* and three slopes kept) and of the six face rings
//      around them, which keep only the face state they feed (W* +- dW/2
//      towards the block)
//   D  HLLC flux of every face of the inner cells, into the primitives'
//      storage (no longer read); coarse-fine faces fill their reflux slots
//   E  each thread updates its own leaf cell into the level scratch W
//
// Shared memory (FP32): 5 E^3 + 20 IN^3 + 30 IN^2 words, 84 KB at NS = 4 (two
// blocks per SM), 17 KB at NS = 2.  Per inner cell at NS = 4 the block
// computes 3.4 primitives, 1.75 predictors and 3.4 face solves, against
// 1, 1 and 3 when each is computed once.  Ring cells are staged by every
// block that touches them and a face between two blocks is solved by both,
// with the same arithmetic, so both see the same flux.  Every value comes
// from the device functions of the per-cell passes (primitives, slopes,
// predictor, face states, HLLC, update) in the same order, so the two paths
// agree bit for bit.
//
// Other blocks still read the old states of a block's cells while it runs,
// so new states go to the level scratch W; k_commit_post copies them into U
// together with the level's reflux sums and restriction.
#pragma once
#include "hydro_kernels.cuh"

namespace amr {

template <int NS>
struct Rock {
  static constexpr int E = 2 * NS + 4;      // cells per axis of the cube
  static constexpr int C = E * E * E;
  static constexpr int NO = NS + 2;         // octs per axis of the cube
  static constexpr int NOC = NO * NO * NO;
  static constexpr int NB = NS * NS * NS;   // oct positions of the block
  static constexpr int IN = 2 * NS;         // inner cells per axis, cube cells [2, 2 + IN)
  static constexpr int IC = IN * IN * IN;
  static constexpr int RC = IN * IN;        // cells of one face ring
  static constexpr int FS = IC + RC;        // faces per axis: inner cells' minus faces + last layer
  static constexpr int THREADS = NS == 4 ? 512 : NS == 2 ? 128 : 32;
  static_assert(15 * FS <= 5 * C, "fluxes reuse the primitives' storage");
  static_assert(THREADS >= 8 * NB, "one thread per cell of the block");
  template <class T>
  static constexpr size_t smem() {
    return sizeof(T) * (5 * C + 20 * IC + 30 * RC) + 4 * (NOC + NB) + C;
  }
  // blocks per SM the register budget is sized for
  template <class T>
  static constexpr int min_blocks() {
    return NS == 4 ? (sizeof(T) == 4 ? 2 : 1) : NS == 2 ? (sizeof(T) == 4 ? 8 : 4) : 16;
  }
};

enum : uint8_t { kCellNone = 0, kCellGhost = 1, kCellLeaf = 2, kCellSplit = 3, kCellOwn = 16 };

// The face between cube cells a (minus side) and b (plus side) along axis D,
// from the cells' W* and slopes along D (qa, qb: 20 values at stride qs).  It
// is solved when neither side is missing or split and one side is a leaf cell
// of the block's own octs; returns 0 if not solved, +1 for a coarse-fine face
// with the ghost on the plus side, -1 with the ghost on the minus side, 2
// otherwise.
template <class T>
__device__ __forceinline__ int solve_face(const SegCtx<T> &s, int D, const T *qa, const T *qb, int qs,
                                          uint8_t ta_full, uint8_t tb_full, T (&F)[5]) {
  const uint8_t ta = ta_full & 15, tb = tb_full & 15;
  const bool own_leaf = ta_full == (kCellLeaf | kCellOwn) || tb_full == (kCellLeaf | kCellOwn);
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = T(0);
  if (!(ta != kCellNone && tb != kCellNone && ta != kCellSplit && tb != kCellSplit && own_leaf)) return 0;
  T qL[5], qR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = qa[v * qs] + T(0.5) * qa[(5 + 5 * D + v) * qs];
    qR[v] = qb[v * qs] - T(0.5) * qb[(5 + 5 * D + v) * qs];
  }
  if (D == 0)
    face_flux_states<0>(s, qL, qR, F);
  else if (D == 1)
    face_flux_states<1>(s, qL, qR, F);
  else
    face_flux_states<2>(s, qL, qR, F);
  if ((ta == kCellGhost) == (tb == kCellGhost)) return 2;
  return tb == kCellGhost ? 1 : -1;
}

// reflux slot of a solved coarse-fine face: ghost oct eg (extended index),
// minus cell's index cmin in its oct, ghost side `side` (+1 plus, -1 minus)
template <class T>
__device__ __forceinline__ void reflux_write(const StepArgs<T> &a, const SegCtx<T> &s, int D, int eg, int cmin,
                                             int side, const T (&F)[5]) {
  const int d1 = D == 0 ? 1 : 0, d2 = D == 2 ? 1 : 2;
  const int ab = (((cmin >> d1) & 1) << 1) | ((cmin >> d2) & 1);
  const int64_t gslot = int64_t(eg - a.N) * 24 + (side > 0 ? 2 * D : 2 * D + 1) * 4 + ab;
  const T sgn = side > 0 ? T(1) : T(-1);
#pragma unroll
  for (int v = 0; v < 5; ++v) a.C[v * a.CS + checked(gslot, 0, a.CS, a.err)] = (sgn * s.dtdx) * F[v] / T(8);
}

// the extended index of every oct of the cube around a block (positions -1..NS
// per axis): the 27-neighbour entry of a real oct of the block within one
// position (every position a leaf cell's stencil reaches has one); -1
// elsewhere.  Ends with a barrier.
template <class T, int NS, int THREADS>
__device__ __forceinline__ void cube_octs(const StepArgs<T> &a, int o0, int o1, int32_t *opos, int32_t *octs) {
  constexpr int NO = NS + 2;
  const int nb = o1 - o0;
  if (threadIdx.x < nb) {
    const uint64_t k = __ldg(a.key + o0 + threadIdx.x);
    opos[threadIdx.x] = int(ikey_x(k) & (NS - 1)) | (int(ikey_y(k) & (NS - 1)) << 4) |
                        (int(ikey_z(k) & (NS - 1)) << 8);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NO * NO * NO; p += THREADS) {
    const int px = p % NO - 1, py = (p / NO) % NO - 1, pz = p / (NO * NO) - 1;
    int found = -1;
    for (int b = 0; b < nb && found < 0; ++b) {
      const int op = opos[b];
      const int dx = px - (op & 15), dy = py - ((op >> 4) & 15), dz = pz - (op >> 8);
      if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;
      const int dir = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
      found = int(checked(__ldg(a.nbr27 + dir * int64_t(a.N) + o0 + b), -1, a.NE, a.err, -1));
    }
    octs[p] = found;
  }
  __syncthreads();
}

// kind of cube cell (x, y, z) and its extended oct e / index c in its oct
template <class T, int NS>
__device__ __forceinline__ uint8_t cube_cell(const StepArgs<T> &a, const int32_t *octs, int x, int y, int z,
                                             int o0, int o1, int &e, int &c) {
  constexpr int NO = NS + 2;
  e = octs[(x >> 1) + NO * ((y >> 1) + NO * (z >> 1))];
  c = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
  if (e < 0) return kCellNone;
  uint8_t ty = e >= a.N ? kCellGhost : (((__ldg(a.son + e) >> c) & 1u) ? kCellSplit : kCellLeaf);
  if (e >= o0 && e < o1) ty |= kCellOwn;  // a cell of the block's own octs
  return ty;
}


// 8 consecutive values (the cells of one oct, one variable) with 16-byte
// loads and stores
__device__ __forceinline__ void load_oct8(const float *p, float (&o)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
  const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load_oct8(const double *p, double (&o)[8]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + h);
    o[2 * h] = a.x;
    o[2 * h + 1] = a.y;
  }
}
// 4 consecutive values (16-byte aligned)
__device__ __forceinline__ void load_oct4(const float *p, float (&o)[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void load_oct4(const double *p, double (&o)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void store_oct8(float *p, const float (&o)[8]) {
  reinterpret_cast<float4 *>(p)[0] = make_float4(o[0], o[1], o[2], o[3]);
  reinterpret_cast<float4 *>(p)[1] = make_float4(o[4], o[5], o[6], o[7]);
}
__device__ __forceinline__ void store_oct8(double *p, const double (&o)[8]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) reinterpret_cast<double2 *>(p)[h] = make_double2(o[2 * h], o[2 * h + 1]);
}

// the face between cube cells of kinds ta (minus side) and tb (plus side) is
// solved when neither side is missing or split and one side is a leaf cell
// of the block's own octs: 0 not solved, +1 / -1 a coarse-fine face with the
// ghost on the plus / minus side, 2 otherwise
__device__ __forceinline__ int face_kind(uint8_t ta_full, uint8_t tb_full) {
  const uint8_t ta = ta_full & 15, tb = tb_full & 15;
  const bool own_leaf = ta_full == (kCellLeaf | kCellOwn) || tb_full == (kCellLeaf | kCellOwn);
  if (!(ta != kCellNone && tb != kCellNone && ta != kCellSplit && tb != kCellSplit && own_leaf)) return 0;
  if ((ta == kCellGhost) == (tb == kCellGhost)) return 2;
  return tb == kCellGhost ? 1 : -1;
}

template <class T>
__device__ __forceinline__ void face_flux_dir(const SegCtx<T> &s, int D, T (&qL)[5], T (&qR)[5], T (&F)[5]) {
  if (D == 0)
    face_flux_states<0>(s, qL, qR, F);
  else if (D == 1)
    face_flux_states<1>(s, qL, qR, F);
  else
    face_flux_states<2>(s, qL, qR, F);
}

template <class T, int NS>
__global__ void __launch_bounds__(Rock<NS>::THREADS, Rock<NS>::template min_blocks<T>())
    k_rock(StepArgs<T> a, const int32_t *__restrict__ blk) {
  using R = Rock<NS>;
  constexpr int E = R::E, C = R::C, NO = R::NO, NOC = R::NOC, NB = R::NB, IN = R::IN, IC = R::IC,
                RC = R::RC, FS = R::FS, TH = R::THREADS;
  constexpr int LIN = NS == 4 ? 3 : NS == 2 ? 2 : 1;  // log2(IN)
  extern __shared__ __align__(16) unsigned char rock_smem[];
  T *sP = reinterpret_cast<T *>(rock_smem);  // [5][C]: primitives of the cube
  T *sF = sP;                                // [3][5][FS]: fluxes (phase D on)
  T *sQ = sP + 5 * C;                        // [20][IC]: W*, dW_x, dW_y, dW_z of inner cells
  T *sR = sQ + 20 * IC;                      // [6][5][RC]: face states of the six rings
  int32_t *octs = reinterpret_cast<int32_t *>(sR + 30 * RC);  // [NOC] extended oct index or -1
  int32_t *pos_oct = octs + NOC;                               // [NB] own oct at each position
  uint8_t *ctype = reinterpret_cast<uint8_t *>(pos_oct + NB);  // [C] kind of each cube cell
  const int t = threadIdx.x;

  for (int q = t; q < NB; q += TH) pos_oct[q] = -1;
  __syncthreads();
  for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
    const Tile td = tile_at(a.tpre, a.tseg0, a.tnseg, a.tstep, ti);
    const Seg sg = a.segs[td.seg];
    if (a.mact && !__ldg(a.mact + sg.member)) continue;  // finished member (block-uniform)
    const SegCtx<T> s = seg_ctx(a, td.seg);
    const int gb = sg.blk0 + td.start;
    const int o0 = int(checked(__ldg(blk + gb), s.lo, s.lo + s.nl, a.err, s.lo));
    const int o1 = int(checked(__ldg(blk + gb + 1), o0 + 1, s.lo + s.nl + 1, a.err, o0 + 1));
    const int nb = o1 - o0;

    // A1. the own octs' positions in the block
    for (int b = t; b < nb; b += TH) {
      const uint64_t k = __ldg(a.key + o0 + b);
      pos_oct[int(ikey_x(k) & (NS - 1)) + NS * (int(ikey_y(k) & (NS - 1)) + NS * int(ikey_z(k) & (NS - 1)))] =
          o0 + b;
    }
    __syncthreads();

    // A2. two threads per cube oct (cells 4 h .. 4 h + 3, one 16-byte load
    // per variable in FP32): the oct's extended index (own octs from the
    // position table; every other oct through the 27-neighbour entry of an
    // own oct within one position; the eight corners feed no face), the kind
    // of its cells and their primitives
    for (int it = t; it < 2 * NOC; it += TH) {
      const int p = it >> 1, h = it & 1;
      const int px = p % NO - 1, py = (p / NO) % NO - 1, pz = p / (NO * NO) - 1;
      const int out = (px < 0 || px >= NS) + (py < 0 || py >= NS) + (pz < 0 || pz >= NS);
      int e = -1;
      bool home = false;
      if (out < 3) {
        int rx = px < 0 ? 0 : px >= NS ? NS - 1 : px;
        int ry = py < 0 ? 0 : py >= NS ? NS - 1 : py;
        int rz = pz < 0 ? 0 : pz >= NS ? NS - 1 : pz;
        int ob = pos_oct[rx + NS * (ry + NS * rz)];
        if (ob < 0) {  // a partial block: any own oct within one position
          for (int d = 0; d < 27 && ob < 0; ++d) {
            const int qx = px + d % 3 - 1, qy = py + (d / 3) % 3 - 1, qz = pz + d / 9 - 1;
            if (qx < 0 || qx >= NS || qy < 0 || qy >= NS || qz < 0 || qz >= NS) continue;
            const int c = pos_oct[qx + NS * (qy + NS * qz)];
            if (c >= 0) {
              ob = c;
              rx = qx;
              ry = qy;
              rz = qz;
            }
          }
        }
        if (ob >= 0) {
          if (rx == px && ry == py && rz == pz) {
            e = ob;
            home = true;
          } else {
            const int dir = (pz - rz + 1) * 9 + (py - ry + 1) * 3 + (px - rx + 1);
            e = int(checked(__ldg(a.nbr27 + dir * int64_t(a.N) + ob), -1, a.NE, a.err, -1));
          }
        }
      }
      if (h == 0) octs[p] = e;
      // cells 4 h .. 4 h + 3 of the oct: the plane cz = h
      const int q0 = 2 * (px + 1) + E * (2 * (py + 1) + E * (2 * (pz + 1) + h));
      const uint32_t sm = (e >= 0 && e < a.N) ? __ldg(a.son + e) : 0u;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint8_t ty = kCellNone;
        if (e >= a.N)
          ty = kCellGhost;
        else if (e >= 0)
          ty = uint8_t(((sm >> (4 * h + c)) & 1u) ? kCellSplit : kCellLeaf) |
               (home ? uint8_t(kCellOwn) : uint8_t(0));
        ctype[q0 + (c & 1) + E * (c >> 1)] = ty;
      }
      if (e < 0) continue;
      T uv[5][4];
#pragma unroll
      for (int v = 0; v < 5; ++v) load_oct4(a.U + v * a.S + 8 * int64_t(e) + 4 * h, uv[v]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        T w[5];
        prim_of(s, uv[0][c], uv[1][c], uv[2][c], uv[3][c], uv[4][c], w);
        const int q = q0 + (c & 1) + E * (c >> 1);
#pragma unroll
        for (int v = 0; v < 5; ++v) sP[v * C + q] = w[v];
      }
    }
    __syncthreads();

    // C. slopes and predictor: inner cells g < IC (cube order, x fastest),
    // then the six face rings (side = 2 D + plus; transverse cells
    // rr = j + IN k, the lower axis j).  Every cell a solved face needs has
    // all six neighbours staged (they lie within the own octs' 26-oct
    // neighbourhoods); the slopes of other cells are not used.
    for (int g = t; g < IC + 6 * RC; g += TH) {
      int x, y, z, side = -1, rr = 0;
      if (g < IC) {
        x = 2 + (g & (IN - 1));
        y = 2 + ((g >> LIN) & (IN - 1));
        z = 2 + (g >> (2 * LIN));
      } else {
        side = (g - IC) >> (2 * LIN);
        rr = (g - IC) & (RC - 1);
        const int D = side >> 1, along = (side & 1) ? 2 + IN : 1;
        const int j = 2 + (rr & (IN - 1)), k = 2 + (rr >> LIN);
        x = D == 0 ? along : j;
        y = D == 1 ? along : (D == 0 ? j : k);
        z = D == 2 ? along : k;
      }
      const int cq = x + E * (y + E * z);
      const uint8_t ty = ctype[cq] & 15;
      if (ty == kCellNone || ty == kCellSplit) continue;  // feeds no solved face
      T w[5], dw[3][5], ws[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) w[v] = sP[v * C + cq];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int st = d == 0 ? 1 : d == 1 ? E : E * E;
#pragma unroll
        for (int v = 0; v < 5; ++v) dw[d][v] = minmod(sP[v * C + cq + st] - w[v], w[v] - sP[v * C + cq - st]);
      }
      predictor(s, w, dw, ws);
      if (side < 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) sQ[v * IC + g] = ws[v];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) sQ[(5 + 5 * d + v) * IC + g] = dw[d][v];
      } else {
        const int D = side >> 1;
        // the minus ring feeds the left state of the first face, the plus
        // ring the right state of the last
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const T dd = D == 0 ? dw[0][v] : D == 1 ? dw[1][v] : dw[2][v];
          sR[(5 * side + v) * RC + rr] = (side & 1) ? ws[v] - T(0.5) * dd : ws[v] + T(0.5) * dd;
        }
      }
    }
    __syncthreads();

    // D. fluxes.  Items w < 3 IC: the minus face along D = w / IC of inner
    // cell w % IC, stored at [D][cell]; items beyond: the plus face of the
    // last inner layer along D at transverse cell rr, stored at [D][IC + rr].
    for (int wi = t; wi < 3 * (IC + RC); wi += TH) {
      int D, gm, gp, rr;  // inner index of the minus / plus cell (-1: ring)
      if (wi < 3 * IC) {
        D = wi >> (3 * LIN);
        gp = wi & (IC - 1);
        const int xi = gp & (IN - 1), yi = (gp >> LIN) & (IN - 1), zi = gp >> (2 * LIN);
        const int cd = D == 0 ? xi : D == 1 ? yi : zi;
        rr = D == 0 ? yi + IN * zi : D == 1 ? xi + IN * zi : xi + IN * yi;
        gm = cd > 0 ? gp - (D == 0 ? 1 : D == 1 ? IN : IN * IN) : -1;
      } else {
        D = (wi - 3 * IC) >> (2 * LIN);
        rr = (wi - 3 * IC) & (RC - 1);
        const int j = rr & (IN - 1), k = rr >> LIN;
        gm = D == 0 ? (IN - 1) + IN * (j + IN * k) : D == 1 ? j + IN * ((IN - 1) + IN * k)
                                                            : j + IN * (k + IN * (IN - 1));
        gp = -1;
      }
      // cube cells of the two sides
      const int st = D == 0 ? 1 : D == 1 ? E : E * E;
      int cb;
      if (gp >= 0) {
        cb = (2 + (gp & (IN - 1))) + E * ((2 + ((gp >> LIN) & (IN - 1))) + E * (2 + (gp >> (2 * LIN))));
      } else {
        cb = (2 + (gm & (IN - 1))) + E * ((2 + ((gm >> LIN) & (IN - 1))) + E * (2 + (gm >> (2 * LIN)))) + st;
      }
      const int ca = cb - st;
      T F[5] = {T(0), T(0), T(0), T(0), T(0)};
      const int kind = face_kind(ctype[ca], ctype[cb]);
      if (kind) {
        T qL[5], qR[5];
        if (gm < 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v) qL[v] = sR[(5 * (2 * D) + v) * RC + rr];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) qL[v] = sQ[v * IC + gm] + T(0.5) * sQ[(5 + 5 * D + v) * IC + gm];
        }
        if (gp < 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v) qR[v] = sR[(5 * (2 * D + 1) + v) * RC + rr];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) qR[v] = sQ[v * IC + gp] - T(0.5) * sQ[(5 + 5 * D + v) * IC + gp];
        }
        face_flux_dir(s, D, qL, qR, F);
        if (a.reflux && (kind == 1 || kind == -1)) {
          const int cg = kind > 0 ? cb : ca;
          const int gx = cg % E, gy = (cg / E) % E, gz = cg / (E * E);
          const int eg = octs[(gx >> 1) + NO * ((gy >> 1) + NO * (gz >> 1))];
          const int mx = ca % E, my = (ca / E) % E, mz = ca / (E * E);
          reflux_write(a, s, D, eg, (mx & 1) | ((my & 1) << 1) | ((mz & 1) << 2), kind, F);
        }
      }
      // sF aliases sP, whose last reads (phase C) ended at the barrier above
      const int fi = gp >= 0 ? gp : IC + rr;
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[(5 * D + v) * FS + fi] = F[v];
    }
    __syncthreads();

    // E. update, one thread per inner cell (cube order): a leaf cell of the
    // block's own octs takes its new state into W
    for (int q = t; q < NB; q += TH) pos_oct[q] = -1;  // for the next block
    for (int gi = t; gi < IC; gi += TH) {
      const int xi = gi & (IN - 1), yi = (gi >> LIN) & (IN - 1), zi = gi >> (2 * LIN);
      const int cq = (2 + xi) + E * ((2 + yi) + E * (2 + zi));
      if (ctype[cq] != (kCellLeaf | kCellOwn)) continue;
      const int e = octs[(1 + (xi >> 1)) + NO * ((1 + (yi >> 1)) + NO * (1 + (zi >> 1)))];
      const int c = (xi & 1) | ((yi & 1) << 1) | ((zi & 1) << 2);
      // minus face: [D][gi]; plus face: the next cell's minus face, or the
      // last layer's plus face
      const int pf[3] = {xi < IN - 1 ? gi + 1 : IC + yi + IN * zi,
                         yi < IN - 1 ? gi + IN : IC + xi + IN * zi,
                         zi < IN - 1 ? gi + IN * IN : IC + xi + IN * yi};
      T du[3][5];
#pragma unroll
      for (int D = 0; D < 3; ++D)
#pragma unroll
        for (int v = 0; v < 5; ++v) du[D][v] = sF[(5 * D + v) * FS + gi] - sF[(5 * D + v) * FS + pf[D]];
      const int64_t g = 8 * int64_t(e) + c;
      const int rs = int(checked(__ldg(a.rslot + g), -1, a.NC, a.err, -1));
      T *out = a.W + s.base + 8 * (e - s.lo) + c;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        T u = __ldg(a.U + v * a.S + g) + s.dtdx * ((du[0][v] + du[1][v]) + du[2][v]);
        if (rs >= 0) {
          T *Rv = a.Rc + v * int64_t(a.NC) + rs;
          u = u + *Rv;
          *Rv = T(0);
        }
        out[v * a.LS] = u;
      }
    }
    __syncthreads();
  }
}

// After a fused kernel: the new states of the level's leaf cells from the
// scratch W into U, the reflux sums of the level's ghost octs and the
// restriction onto the father cells (what k_reflux_restrict does after the
// per-cell passes, with the commit folded in).  Thread per (oct, variable):
// 8 values in, 8 out, the restriction from the same 8 values.
// domain: 5 ncl (if kSegReflux) + 5 nl
template <class T>
__global__ void k_commit_post(StepArgs<T> a) {
  tile_loop(a,
            [](const SegCtx<T> &s) { return ((s.flags & kSegReflux) ? 5 * s.ncl : 0) + 5 * s.nl; },
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
              const int ol = r - v * s.nl;
              const int o = s.lo + ol;
              const uint32_t sm = __ldg(a.son + o);
              T *u = a.U + v * a.S + 8 * int64_t(o);
              T val[8];
              load_oct8(a.W + v * a.LS + s.base + 8 * ol, val);  // leaf cells: new states
              if (sm) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                  if ((sm >> c) & 1u) val[c] = u[c];  // split cells keep their restricted value
              }
              store_oct8(u, val);
              if (s.flags & kSegRestrict) {
                const uint64_t k = __ldg(a.key + o);
                const int fc = int((ikey_x(k) & 1) | ((ikey_y(k) & 1) << 1) | ((ikey_z(k) & 1) << 2));
                const int f = int(checked(__ldg(a.father + o), 0, a.N, a.err));
                T sum = T(0);
#pragma unroll
                for (int c = 0; c < 8; ++c) sum += val[c];
                a.U[v * a.S + 8 * int64_t(f) + fc] = sum * T(0.125);
              }
            });
}

}  // namespace amr

namespace amr {

// ---------------------------------------------------------------------------
// The paper's planar kernel (Sec. 3, the "paper" kernel): the same block of
// nsubgrid^3 octs and the same cube of cells as the rock kernel, but only a
// window of it is staged: the cube is swept along z, plane by plane, keeping
// the primitives of three planes, the predicted states and slopes of two, the
// z-face fluxes of two face planes and the in-plane fluxes of the plane being
// updated.  At plane zc of the sweep: primitives of plane zc; predictor of
// plane zc - 1; fluxes of the z faces between planes zc - 2 and zc - 1 and, if
// zc - 2 is an inner plane, its in-plane fluxes and the update of its leaf
// cells.  The arithmetic is that of the rock kernel and the per-cell passes.
// ---------------------------------------------------------------------------
template <int NS>
struct Sweep {
  static constexpr int E = 2 * NS + 4, P = E * E;  // cube side, cells of a plane
  static constexpr int NO = NS + 2, NOC = NO * NO * NO;
  static constexpr int QE = E - 2, QP = QE * QE;   // predictor region of a plane
  static constexpr int IN = 2 * NS, FP = IN + 1;   // inner cells per axis, face positions
  static constexpr int ZF = IN * IN;               // z faces of a face plane
  static constexpr int FNP = FP * IN;              // x (or y) faces of a plane
  static constexpr int THREADS = NS == 4 ? 128 : NS == 2 ? 64 : 32;
  template <class T>
  static constexpr size_t smem() {
    return sizeof(T) * (3 * 5 * P + 2 * 20 * QP + 2 * 5 * ZF + 2 * 5 * FNP) + 4 * NOC + 4 * NS * NS * NS +
           E * E * E;
  }
};

template <class T, int NS>
__global__ void __launch_bounds__(Sweep<NS>::THREADS) k_sweep(StepArgs<T> a, const int32_t *__restrict__ blk) {
  using R = Sweep<NS>;
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  T *sW = reinterpret_cast<T *>(sweep_smem);  // [3][5][P]: primitives, plane z at slot z % 3
  T *sQ = sW + 3 * 5 * R::P;                  // [2][20][QP]: W* and slopes, plane z at slot z % 2
  T *sFz = sQ + 2 * 20 * R::QP;               // [2][5][ZF]: z faces above plane z at slot z % 2
  T *sFx = sFz + 2 * 5 * R::ZF;               // [5][FNP]: x faces of the plane being updated
  T *sFy = sFx + 5 * R::FNP;                  // [5][FNP]: y faces
  int32_t *octs = reinterpret_cast<int32_t *>(sFy + 5 * R::FNP);  // [NOC]
  int32_t *opos = octs + R::NOC;                                  // [NS^3]
  uint8_t *ctype = reinterpret_cast<uint8_t *>(opos + NS * NS * NS);  // [E^3]
  constexpr int E = R::E, P = R::P, NO = R::NO, QE = R::QE, QP = R::QP, IN = R::IN, FP = R::FP,
                ZF = R::ZF, FNP = R::FNP, TH = R::THREADS;

  for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
    const Tile td = tile_at(a.tpre, a.tseg0, a.tnseg, a.tstep, ti);
    const Seg sg = a.segs[td.seg];
    if (a.mact && !__ldg(a.mact + sg.member)) continue;  // finished member (block-uniform)
    const SegCtx<T> s = seg_ctx(a, td.seg);
    const int gb = sg.blk0 + td.start;
    const int o0 = int(checked(__ldg(blk + gb), s.lo, s.lo + s.nl, a.err, s.lo));
    const int o1 = int(checked(__ldg(blk + gb + 1), o0 + 1, s.lo + s.nl + 1, a.err, o0 + 1));
    cube_octs<T, NS, TH>(a, o0, o1, opos, octs);
    for (int q = threadIdx.x; q < E * E * E; q += TH) {
      int e, c;
      ctype[q] = cube_cell<T, NS>(a, octs, q % E, (q / E) % E, q / (E * E), o0, o1, e, c);
    }
    __syncthreads();

    for (int zc = 0; zc < E; ++zc) {
      // primitives of plane zc
      T *Wc = sW + (zc % 3) * 5 * P;
      for (int q = threadIdx.x; q < P; q += TH) {
        const int x = q % E, y = q / E;
        int e, c;
        if (cube_cell<T, NS>(a, octs, x, y, zc, o0, o1, e, c) == kCellNone) continue;
        const int64_t g = 8 * int64_t(e) + c;
        T w[5];
        prim_of(s, a.U[g], a.U[a.S + g], a.U[2 * a.S + g], a.U[3 * a.S + g], a.U[4 * a.S + g], w);
#pragma unroll
        for (int v = 0; v < 5; ++v) Wc[v * P + q] = w[v];
      }
      __syncthreads();

      // slopes and predictor of plane zq = zc - 1 (region [1, E-1) in x, y)
      const int zq = zc - 1;
      if (zq >= 1 && zq <= E - 2) {
        const T *Wm = sW + ((zq + 2) % 3) * 5 * P, *W0 = sW + (zq % 3) * 5 * P, *Wp = Wc;
        T *Q = sQ + (zq % 2) * 20 * QP;
        for (int q = threadIdx.x; q < QP; q += TH) {
          const int x = 1 + q % QE, y = 1 + q / QE;
          const int pq = x + E * y, cq = pq + P * zq;
          if (ctype[cq] == kCellNone) continue;
          T w[5], dw[3][5], ws[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) w[v] = W0[v * P + pq];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const int st = d == 0 ? 1 : d == 1 ? E : P;
            if (ctype[cq - st] == kCellNone || ctype[cq + st] == kCellNone) {
#pragma unroll
              for (int v = 0; v < 5; ++v) dw[d][v] = T(0);
              continue;
            }
            const T *Wlo = d == 2 ? Wm + pq : W0 + pq - st;
            const T *Whi = d == 2 ? Wp + pq : W0 + pq + st;
#pragma unroll
            for (int v = 0; v < 5; ++v) dw[d][v] = minmod(Whi[v * P] - w[v], w[v] - Wlo[v * P]);
          }
          predictor(s, w, dw, ws);
#pragma unroll
          for (int v = 0; v < 5; ++v) Q[v * QP + q] = ws[v];
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v) Q[(5 + 5 * d + v) * QP + q] = dw[d][v];
        }
      }
      __syncthreads();

      // plane zu = zc - 2: its upper z faces; if it is an inner plane, its
      // in-plane faces and the update of the block's leaf cells in it
      const int zu = zq - 1;
      if (zu >= 1 && zu <= IN + 1) {
        const T *Qu = sQ + (zu % 2) * 20 * QP, *Qq = sQ + (zq % 2) * 20 * QP;
        T *Fzc = sFz + (zu % 2) * 5 * ZF;
        const bool inner = zu >= 2 && zu < 2 + IN;
        const int nf = ZF + (inner ? 2 * FNP : 0);
        for (int f = threadIdx.x; f < nf; f += TH) {
          int D, m[3], p[3], fi;
          T *Fd;
          if (f < ZF) {
            D = 2;
            m[0] = p[0] = 2 + f % IN;
            m[1] = p[1] = 2 + f / IN;
            m[2] = zu;
            p[2] = zq;
            Fd = Fzc;
            fi = f;
          } else if (f < ZF + FNP) {
            D = 0;
            fi = f - ZF;
            m[0] = 1 + fi % FP;
            p[0] = m[0] + 1;
            m[1] = p[1] = 2 + fi / FP;
            m[2] = p[2] = zu;
            Fd = sFx;
          } else {
            D = 1;
            fi = f - ZF - FNP;
            m[1] = 1 + fi % FP;
            p[1] = m[1] + 1;
            m[0] = p[0] = 2 + fi / FP;
            m[2] = p[2] = zu;
            Fd = sFy;
          }
          const int ca = m[0] + E * (m[1] + E * m[2]), cb = p[0] + E * (p[1] + E * p[2]);
          const T *qa = (m[2] == zu ? Qu : Qq) + (m[0] - 1) + QE * (m[1] - 1);
          const T *qb = (p[2] == zu ? Qu : Qq) + (p[0] - 1) + QE * (p[1] - 1);
          T F[5];
          const int kind = solve_face(s, D, qa, qb, QP, ctype[ca], ctype[cb], F);
          if (a.reflux && (kind == 1 || kind == -1)) {
            const int cg = kind > 0 ? cb : ca;
            const int gx = cg % E, gy = (cg / E) % E, gz = cg / (E * E);
            const int eg = octs[(gx >> 1) + NO * ((gy >> 1) + NO * (gz >> 1))];
            reflux_write(a, s, D, eg, (m[0] & 1) | ((m[1] & 1) << 1) | ((m[2] & 1) << 2), kind, F);
          }
          const int fs = D == 2 ? ZF : FNP;
#pragma unroll
          for (int v = 0; v < 5; ++v) Fd[v * fs + fi] = F[v];
        }
        __syncthreads();
        if (inner) {
          const T *Fzl = sFz + ((zu + 1) % 2) * 5 * ZF;  // the z faces below plane zu
          for (int q = threadIdx.x; q < IN * IN; q += TH) {
            const int x = 2 + q % IN, y = 2 + q / IN;
            if (ctype[x + E * (y + E * zu)] != (kCellLeaf | kCellOwn)) continue;
            int e, c;
            cube_cell<T, NS>(a, octs, x, y, zu, o0, o1, e, c);
            T du[3][5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              du[0][v] = sFx[v * FNP + (x - 2) + FP * (y - 2)] - sFx[v * FNP + (x - 1) + FP * (y - 2)];
              du[1][v] = sFy[v * FNP + (y - 2) + FP * (x - 2)] - sFy[v * FNP + (y - 1) + FP * (x - 2)];
              du[2][v] = Fzl[v * ZF + (x - 2) + IN * (y - 2)] - Fzc[v * ZF + (x - 2) + IN * (y - 2)];
            }
            const int t = 8 * (e - s.lo) + c;
            update_cell_to(a, s, 8 * e + c, du[0], du[1], du[2], a.W + s.base + t, int64_t(a.LS));
          }
        }
        __syncthreads();
      }
    }
  }
}

}  // namespace amr
