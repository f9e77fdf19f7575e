// hydro_args.cuh -- arguments of the level-step and time-step kernels.
#pragma once
#include "amr_internal.cuh"

namespace amr {

// Everything one level step needs, passed by value.  "Local" cell indices
// t in [0, LS) number the level's real cells first (8*nl) and then the
// cells of its ghost octs (8*ncl); scratch arrays are indexed by t.
template <class T>
struct LevelArgs {
  int l, lmin;
  int64_t lo, nl;    // real octs of the level: mesh indices [lo, lo+nl)
  int64_t clo, ncl;  // ghost octs of the level: cache slots [clo, clo+ncl)
  int64_t N, NE;     // real octs; real + ghost octs (extended index range)
  int64_t S;         // stride of U (8*NE)
  int64_t RS;        // stride of R (8*N)
  int64_t LS;        // stride of the scratch arrays (8*(nl+ncl))
  int64_t CS;        // stride of the reflux contribution slots (24*NC): every
                     // ghost oct owns 24 slots, written only by its own level
  T *U, *R;
  const int32_t *fnb;     // [6][NE] face neighbours (extended index, -1 none)
  const uint32_t *son;    // [N] split mask
  const int32_t *father;  // [N] father oct (mesh index), -1 at levelmin
  const uint64_t *key;    // [N]
  const int32_t *csrc;    // [7][NC] prolongation sources (global cell indices)
  int64_t NC;
  T *W, *Q, *F, *C;       // scratch: W[5][LS], Q[20][LS], F[15][LS]; C[5][CS]
  const double *dt_dev;   // if not NULL: dt = *dt_dev * dt_scale
  double dt_scale, dt_host;
  double inv_dx;          // 2^l
  T gamma, smallr, smallp;
  int reflux;
};


struct CflArgs {
  int lmin, lmax;
  int64_t lo[kMaxLev + 2];  // level offsets of the real octs
  int64_t S;
  const uint32_t *son;
  double gamma, smallr, smallp, cfl;
  unsigned long long *smax;  // [16] bit patterns of per-level maxima
  double *dt_dev;
  int *err;
};



}  // namespace amr
