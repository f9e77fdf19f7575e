// rock_kernels.cuh -- the level step as one fused shared-memory kernel per
// block of octs (the paper's "rock" kernel, Sec. 3, with `nsubgrid` NS octs
// per axis in the inner block).
//
// nsubgrid 4 (a 12^3 cube, 150 KB of shared memory) exists for FP32 only:
// in FP64 it would need 300 KB, more than an SM has.
//
// A CTA takes one block: the real octs of one (member, level) segment that
// share an aligned NS^3 group of oct positions (consecutive in the level's
// Hilbert order).  It stages the conservative state of the block and of one
// ring of octs around it -- an E^3 cube of cells, E = 2 NS + 4, real or ghost
// octs found through the 27-neighbour table -- in shared memory and does
// the whole step there: primitives of the cube, limited slopes and the
// Hancock predictor on the cube less its outer layer, the HLLC fluxes of
// every face of the inner cells, and the update of the block's leaf cells
// (with the pending reflux of coarse cells).  Coarse-fine faces fill their
// reflux slots as in the per-cell passes.  Ring cells are staged by every
// block that touches them and their faces are solved by both blocks, with
// the same arithmetic, so the two sides of a face see the same flux.
//
// The new states go to the level scratch W (other blocks still read the old
// ones), and a second kernel copies them into U.  Every value is computed by
// the same device functions as the per-cell passes (primitives, slopes,
// predictor, face states, HLLC, update), so the two paths agree bit for bit.
#pragma once
#include "hydro_kernels.cuh"

namespace amr {

template <int NS>
struct Rock {
  static constexpr int E = 2 * NS + 4;          // cells per axis of the staged cube
  static constexpr int C = E * E * E;
  static constexpr int NO = NS + 2;             // octs per axis of the cube
  static constexpr int NOC = NO * NO * NO;
  static constexpr int QE = E - 2;              // predictor region [1, E-1)
  static constexpr int QC = QE * QE * QE;
  static constexpr int IN = 2 * NS;             // inner cells per axis, [2, 2 + IN)
  static constexpr int IC = IN * IN * IN;
  static constexpr int FP = IN + 1;             // face positions along an axis
  static constexpr int FN = FP * IN * IN;       // faces per axis
  static constexpr int THREADS = NS == 4 ? 512 : 256;
  template <class T>
  static constexpr size_t smem() {
    return sizeof(T) * (5 * C + 20 * QC + 15 * FN) + 4 * NOC + 4 * NS * NS * NS + C;
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

template <class T, int NS>
__global__ void __launch_bounds__(Rock<NS>::THREADS) k_rock(StepArgs<T> a, const int32_t *__restrict__ blk) {
  using R = Rock<NS>;
  extern __shared__ __align__(16) unsigned char rock_smem[];
  T *sW = reinterpret_cast<T *>(rock_smem);   // [5][C]: U, then W
  T *sQ = sW + 5 * R::C;                      // [20][QC]: W*, dW_x, dW_y, dW_z
  T *sF = sQ + 20 * R::QC;                    // [3][5][FN]
  int32_t *octs = reinterpret_cast<int32_t *>(sF + 15 * R::FN);  // [NOC]
  int32_t *opos = octs + R::NOC;                                  // [NS^3] block octs' positions
  uint8_t *ctype = reinterpret_cast<uint8_t *>(opos + NS * NS * NS);  // [C]
  constexpr int E = R::E, NO = R::NO, QE = R::QE, IN = R::IN, FP = R::FP, FN = R::FN;

  for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
    const Tile td = a.tiles[ti];
    const Seg sg = a.segs[td.seg];
    if (a.mact && !__ldg(a.mact + sg.member)) continue;  // finished member (block-uniform)
    const SegCtx<T> s = seg_ctx(a, td.seg);
    const int gb = sg.blk0 + td.start;
    const int o0 = int(checked(__ldg(blk + gb), s.lo, s.lo + s.nl, a.err, s.lo));
    const int o1 = int(checked(__ldg(blk + gb + 1), o0 + 1, s.lo + s.nl + 1, a.err, o0 + 1));

    // 1. extended index of every oct of the cube
    cube_octs<T, NS, R::THREADS>(a, o0, o1, opos, octs);

    // 2. conservative state and kind of every cell of the cube
    for (int q = threadIdx.x; q < R::C; q += R::THREADS) {
      int e, c;
      const uint8_t ty = cube_cell<T, NS>(a, octs, q % E, (q / E) % E, q / (E * E), o0, o1, e, c);
      if (ty != kCellNone) {
        const int64_t g = 8 * int64_t(e) + c;
#pragma unroll
        for (int v = 0; v < 5; ++v) sW[v * R::C + q] = a.U[v * a.S + g];
      }
      ctype[q] = ty;
    }
    __syncthreads();

    // 3. primitives, in place
    for (int q = threadIdx.x; q < R::C; q += R::THREADS) {
      if (ctype[q] == kCellNone) continue;
      T w[5];
      prim_of(s, sW[q], sW[R::C + q], sW[2 * R::C + q], sW[3 * R::C + q], sW[4 * R::C + q], w);
#pragma unroll
      for (int v = 0; v < 5; ++v) sW[v * R::C + q] = w[v];
    }
    __syncthreads();

    // 4. slopes and predictor on [1, E-1)^3; a slope along an axis with a
    // missing neighbour is zero (such cells feed no face of the block)
    for (int q = threadIdx.x; q < R::QC; q += R::THREADS) {
      const int x = 1 + q % QE, y = 1 + (q / QE) % QE, z = 1 + q / (QE * QE);
      const int cq = x + E * (y + E * z);
      if (ctype[cq] == kCellNone) continue;
      T w[5], dw[3][5], ws[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) w[v] = sW[v * R::C + cq];
      const int st[3] = {1, E, E * E};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int cm = cq - st[d], cp = cq + st[d];
        if (ctype[cm] == kCellNone || ctype[cp] == kCellNone) {
#pragma unroll
          for (int v = 0; v < 5; ++v) dw[d][v] = T(0);
          continue;
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) dw[d][v] = minmod(sW[v * R::C + cp] - w[v], w[v] - sW[v * R::C + cm]);
      }
      predictor(s, w, dw, ws);
#pragma unroll
      for (int v = 0; v < 5; ++v) sQ[v * R::QC + q] = ws[v];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) sQ[(5 + 5 * d + v) * R::QC + q] = dw[d][v];
    }
    __syncthreads();

    // 5. fluxes of the faces of the inner cells: along axis D, face i lies
    // between cube cells 1 + i and 2 + i; a face is solved when one side is
    // a leaf cell of the block's own octs and neither side is split
    for (int f = threadIdx.x; f < 3 * FN; f += R::THREADS) {
      const int D = f / FN, r = f - D * FN;
      const int i = r % FP, j = 2 + (r / FP) % IN, k = 2 + r / (FP * IN);
      int am[3], bm[3];
      am[D] = 1 + i;
      bm[D] = 2 + i;
      am[D == 0 ? 1 : 0] = bm[D == 0 ? 1 : 0] = j;
      am[D == 2 ? 1 : 2] = bm[D == 2 ? 1 : 2] = k;
      const int ca = am[0] + E * (am[1] + E * am[2]), cb = bm[0] + E * (bm[1] + E * bm[2]);
      const int qa = (am[0] - 1) + QE * ((am[1] - 1) + QE * (am[2] - 1));
      const int qb = (bm[0] - 1) + QE * ((bm[1] - 1) + QE * (bm[2] - 1));
      T F[5];
      const int kind = solve_face(s, D, sQ + qa, sQ + qb, R::QC, ctype[ca], ctype[cb], F);
      if (a.reflux && (kind == 1 || kind == -1)) {
        const int cg = kind > 0 ? cb : ca;
        const int gx = cg % E, gy = (cg / E) % E, gz = cg / (E * E);
        const int eg = octs[(gx >> 1) + NO * ((gy >> 1) + NO * (gz >> 1))];
        reflux_write(a, s, D, eg, (am[0] & 1) | ((am[1] & 1) << 1) | ((am[2] & 1) << 2), kind, F);
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[(5 * D + v) * FN + r] = F[v];
    }
    __syncthreads();

    // 6. the block's leaf cells: new state into the level scratch W
    for (int q = threadIdx.x; q < R::IC; q += R::THREADS) {
      const int x = 2 + q % IN, y = 2 + (q / IN) % IN, z = 2 + q / (IN * IN);
      const int cq = x + E * (y + E * z);
      if (ctype[cq] != (kCellLeaf | kCellOwn)) continue;
      const int e = octs[(x >> 1) + NO * ((y >> 1) + NO * (z >> 1))];
      const int c = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
      const int m[3] = {x, y, z};
      T du[3][5];
#pragma unroll
      for (int D = 0; D < 3; ++D) {
        // faces of the cell along D: minus face i = m - 2, plus face i = m - 1
        const int t1 = D == 0 ? y : x, t2 = D == 2 ? y : z;
        const int rm = (m[D] - 2) + FP * ((t1 - 2) + IN * (t2 - 2));
#pragma unroll
        for (int v = 0; v < 5; ++v) du[D][v] = sF[(5 * D + v) * FN + rm] - sF[(5 * D + v) * FN + rm + 1];
      }
      const int t = 8 * (e - s.lo) + c;
      update_cell_to(a, s, 8 * e + c, du[0], du[1], du[2], a.W + s.base + t, int64_t(a.LS));
    }
    __syncthreads();
  }
}

// the new states of the leaf cells, from the level scratch into U
// domain: 8 nl (real cells)
template <class T>
__global__ void k_rock_commit(StepArgs<T> a) {
  tile_loop(a, [](const SegCtx<T> &s) { return 8 * s.nl; }, [&](const SegCtx<T> &s, int t) {
    if (cell_is_split(a, s, t)) return;
    const int64_t g = 8 * int64_t(s.lo + (t >> 3)) + (t & 7);
#pragma unroll
    for (int v = 0; v < 5; ++v) a.U[v * a.S + g] = a.W[v * a.LS + s.base + t];
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
    const Tile td = a.tiles[ti];
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
