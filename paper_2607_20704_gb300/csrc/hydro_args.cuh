// hydro_args.cuh -- arguments of the level-step and time-step kernels.
#pragma once
#include "amr_internal.cuh"

namespace amr {

// One (member mesh, level) piece of a level-step launch.  Real octs of the
// segment are mesh indices [lo, lo+nl), its ghost octs cache slots
// [clo, clo+ncl).  "Local" cell indices t in [0, 8(nl+ncl)) number the real
// cells first, then the ghost cells; the scratch arrays hold the segment at
// [base, base + 8(nl+ncl)).
struct Seg {
  int member, level;
  int lo, nl;
  int clo, ncl;
  int base;
  int flags;  // kSegReflux: sum coarse-fine fluxes; kSegRestrict: restrict
  int blk0;   // fused kernel: the segment's first block of octs (global index)
  int nblk;   // and its number of blocks
};
enum : int { kSegReflux = 1, kSegRestrict = 2 };

// A launch covers a flattened list of tiles; tile (seg, start) is the block
// of domain items [start, start + step) of segment seg.  A list stores only
// its segments' cumulative tile counts (tpre[q] = first tile of its q-th
// segment, tpre[nseg] = all tiles); a kernel finds the segment of tile ti by
// binary search.
struct Tile {
  int seg, start;
};

// the last segment of the list whose first tile is <= ti (segments without
// tiles share their successor's first tile and are passed over)
__device__ __forceinline__ Tile tile_at(const int *__restrict__ tpre, int seg0, int nseg, int step, int ti) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(tpre + mid) <= ti)
      lo = mid;
    else
      hi = mid - 1;
  }
  return Tile{seg0 + lo, (ti - __ldg(tpre + lo)) * step};
}

// Everything a level-step launch needs, passed by value.  Oct counts and cell
// indices fit in 32 bits (at most 2^26 real octs, and 8 (real + ghost octs)
// <= 2^31 - 1, both checked by the host before any state is allocated), so
// kernels index cells with int; every product with a stride (S, LS, CS) is
// formed in 64 bits, since 20 LS exceeds 2^31 from about 107 M local cells on.
template <class T>
struct StepArgs {
  int N, NE, NC;      // real octs; real + ghost octs; ghost octs (all members)
  int64_t LS;         // stride of the scratch arrays
  int64_t S;          // stride of U (8*NE)
  int64_t CS;         // stride of the reflux slots (24*NC)
  T *U;
  T *Rc;                  // [5][NC] pending reflux of the father of ghost oct s
  const int32_t *rslot;   // [8N] ghost slot whose father is this cell, or -1
  const int32_t *fnb;     // [6][NE] face neighbours (extended index, -1 none)
  const int32_t *nbr27;   // [27][N] same-level octs around each real oct, (dz,dy,dx) order
  const uint32_t *son;    // [N] split mask
  const int32_t *father;  // [N] father oct (mesh index), -1 at a member's levelmin
  const uint64_t *key;    // [N] internal keys
  const int32_t *csrc;    // [7][NC] prolongation sources (global cell indices)
  T *W, *Q, *F, *C;       // scratch W[5][LS], Q[20][LS], F[15][LS]; slots C[5][CS]
  const Seg *segs;
  const int *tpre;                  // the list's tile prefix (see Tile)
  int tseg0, tnseg, tstep, ntiles;  // first segment, segments, items per tile, tiles
  // per member: gamma, 1/(gamma-1), floors
  const T *mgamma, *migm1, *msmallr, *msmallp;
  // dt/dx: from the device time step of each member's coarse step
  // (dt_m 2^levelmin_m, the same for every level of the member), or, when
  // both pointers are NULL, dt_host 2^level for every segment
  const double *dtdx_dev;
  const float *dtdxf_dev;
  double dt_host;
  // members taking part in this coarse step (1) or finished (0); NULL: all
  const int *mact;
  int reflux;
  int *err;  // device error word (range errors of bounds-checked builds)
};

struct CflArgs {
  const Seg *segs;
  const int *tpre;
  int tseg0, tnseg, tstep, ntiles;
  int64_t S;
  const uint32_t *son;
  const double *mgamma, *msmallr, *msmallp, *mcfl;
  const void *mgamma_t, *msmallr_t, *msmallp_t;  // the same in the state's type
  const int *mlmin;
  int nmembers;
  unsigned long long *smax;  // [16 * members] bit patterns of per-level maxima
  int *mrem;                 // [members] coarse steps left (-1: unlimited)
  int *mact;                 // [members] 1 if the member steps in this coarse step
  int consume;               // 1: this reduction starts a coarse step (counts down)
  double *dt_dev;            // [members] coarse dt
  double *dtdx_dev;          // [members] dt_m 2^levelmin_m
  float *dtdxf_dev;          // float copy for the FP32 kernels
  int *err;
  int *merr;                 // [members] error bits of each member
};

}  // namespace amr
