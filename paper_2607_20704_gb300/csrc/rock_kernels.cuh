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

    // 1. extended index of every oct of the cube (positions -1..NS per axis
    // around the block): the 27-neighbour entry of a real oct of the block
    // within one position (every position a leaf cell's stencil reaches has
    // one); -1 elsewhere
    const int nb = o1 - o0;
    if (threadIdx.x < nb) {
      const uint64_t k = __ldg(a.key + o0 + threadIdx.x);
      opos[threadIdx.x] = int(ikey_x(k) & (NS - 1)) | (int(ikey_y(k) & (NS - 1)) << 4) |
                          (int(ikey_z(k) & (NS - 1)) << 8);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < R::NOC; p += R::THREADS) {
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

    // 2. conservative state and kind of every cell of the cube
    for (int q = threadIdx.x; q < R::C; q += R::THREADS) {
      const int x = q % E, y = (q / E) % E, z = q / (E * E);
      const int e = octs[(x >> 1) + NO * ((y >> 1) + NO * (z >> 1))];
      const int c = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
      uint8_t ty = kCellNone;
      if (e >= 0) {
        const int64_t g = 8 * int64_t(e) + c;
#pragma unroll
        for (int v = 0; v < 5; ++v) sW[v * R::C + q] = a.U[v * a.S + g];
        ty = e >= a.N ? kCellGhost : (((__ldg(a.son + e) >> c) & 1u) ? kCellSplit : kCellLeaf);
        if (e >= o0 && e < o1) ty |= kCellOwn;  // a cell of the block's own octs
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
      const uint8_t ta = ctype[ca] & 15, tb = ctype[cb] & 15;
      const bool own_leaf = (ctype[ca] == (kCellLeaf | kCellOwn)) || (ctype[cb] == (kCellLeaf | kCellOwn));
      const bool solve = ta != kCellNone && tb != kCellNone && ta != kCellSplit && tb != kCellSplit && own_leaf;
      T F[5] = {T(0), T(0), T(0), T(0), T(0)};
      if (solve) {
        const int qa = (am[0] - 1) + QE * ((am[1] - 1) + QE * (am[2] - 1));
        const int qb = (bm[0] - 1) + QE * ((bm[1] - 1) + QE * (bm[2] - 1));
        T qL[5], qR[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          qL[v] = sQ[v * R::QC + qa] + T(0.5) * sQ[(5 + 5 * D + v) * R::QC + qa];
          qR[v] = sQ[v * R::QC + qb] - T(0.5) * sQ[(5 + 5 * D + v) * R::QC + qb];
        }
        if (D == 0)
          face_flux_states<0>(s, qL, qR, F);
        else if (D == 1)
          face_flux_states<1>(s, qL, qR, F);
        else
          face_flux_states<2>(s, qL, qR, F);
        // coarse-fine face: the block's leaf on one side, a ghost on the other
        if (a.reflux && (ta == kCellGhost) != (tb == kCellGhost)) {
          const bool ghost_plus = tb == kCellGhost;
          const int cg = ghost_plus ? cb : ca;
          const int gx = cg % E, gy = (cg / E) % E, gz = cg / (E * E);
          const int eg = octs[(gx >> 1) + NO * ((gy >> 1) + NO * (gz >> 1))];
          const int cmin = (am[0] & 1) | ((am[1] & 1) << 1) | ((am[2] & 1) << 2);
          const int d1 = D == 0 ? 1 : 0, d2 = D == 2 ? 1 : 2;
          const int ab = (((cmin >> d1) & 1) << 1) | ((cmin >> d2) & 1);
          const int gslot = (eg - a.N) * 24 + (ghost_plus ? 2 * D : 2 * D + 1) * 4 + ab;
          const T sgn = ghost_plus ? T(1) : T(-1);
#pragma unroll
          for (int v = 0; v < 5; ++v) a.C[v * a.CS + checked(gslot, 0, a.CS, a.err)] = (sgn * s.dtdx) * F[v] / T(8);
        }
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
