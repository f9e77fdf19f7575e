// hydro_args.cuh -- arguments of the level-step and time-step kernels.
#pragma once
#include "amr_internal.cuh"

namespace amr {

// Everything one level step needs, passed by value.  "Local" cell indices
// t in [0, LS) number the level's real cells first (8*nl) and then the
// cells of its ghost octs (8*ncl); scratch arrays are indexed by t.  Every
// count fits in 32 bits (at most 2^26 real octs), so kernels index with int.
template <class T>
struct LevelArgs {
  int l, lmin;
  int lo, nl;     // real octs of the level: mesh indices [lo, lo+nl)
  int clo, ncl;   // ghost octs of the level: cache slots [clo, clo+ncl)
  int N, NE, NC;  // real octs; real + ghost octs; ghost octs
  int LS;         // stride of the scratch arrays (8*(nl+ncl))
  int64_t S;      // stride of U (8*NE)
  int64_t CS;     // stride of the reflux contribution slots (24*NC): every
                  // ghost oct owns 24 slots, written only by its own level
  T *U;
  T *Rc;                  // [5][NC] pending reflux of the father of ghost oct s
  const int32_t *rslot;   // [8N] ghost slot whose father is this cell, or -1
  const int32_t *fnb;     // [6][NE] face neighbours (extended index, -1 none)
  const uint32_t *son;    // [N] split mask
  const int32_t *father;  // [N] father oct (mesh index), -1 at levelmin
  const uint64_t *key;    // [N]
  const int32_t *csrc;    // [7][NC] prolongation sources (global cell indices)
  T *W, *Q, *F, *C;       // scratch: W[5][LS], Q[20][LS], F[15][LS]; C[5][CS]
  // dt/dx of this level step: from the device dt of the coarse step
  // (dt_dev, or its float copy dtf_dev) times dtdx_scale = 2^(l - k) for the
  // k-th halving, or the host value dtdx_host when both pointers are NULL
  const double *dt_dev;
  const float *dtf_dev;
  double dtdx_scale;
  T dtdx_host;
  T gamma, igm1, smallr, smallp;  // igm1 = 1/(gamma - 1)
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
  float *dtf_dev;            // float copy of dt for the FP32 kernels
  int *err;
};

}  // namespace amr
