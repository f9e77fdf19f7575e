// amr_api.cu -- C ABI of the GB300 level-advance library (see include/amr.h).
// Host orchestration only: every step of the mesh build, index and level
// step runs in the kernels of index_kernels.cuh and hydro_kernels.cuh,
// compiled here as one translation unit.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "hydro_kernels.cuh"
#include "index_kernels.cuh"

using namespace amr;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static amr_status fail(amr_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess)                                                              \
      return fail(AMR_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),    \
                  __FILE__, __LINE__);                                                  \
  } while (0)

#define AMR_TRY(expr)              \
  do {                             \
    amr_status _s = (expr);        \
    if (_s != AMR_OK) return _s;   \
  } while (0)

extern "C" const char *amr_last_error(void) { return g_last_error.c_str(); }

// lets other translation units of the library set the calling thread's text
void amr_set_error_text(const char *text) { g_last_error = text ? text : ""; }

extern "C" const char *amr_status_string(amr_status s) {
  switch (s) {
    case AMR_OK: return "AMR_OK";
    case AMR_EINVAL: return "AMR_EINVAL";
    case AMR_ENOMEM: return "AMR_ENOMEM";
    case AMR_EGRADING: return "AMR_EGRADING";
    case AMR_EDUP: return "AMR_EDUP";
    case AMR_ECUDA: return "AMR_ECUDA";
    case AMR_ETIMEOUT: return "AMR_ETIMEOUT";
    case AMR_ENAN: return "AMR_ENAN";
  }
  return "AMR_?";
}

// ---------------------------------------------------------------------------
// kernel registry (names, per-kernel timing)
// ---------------------------------------------------------------------------
enum Kid {
  K_SORT_KEYS, K_RADIX_HIST, K_RADIX_SCATTER, K_SCAN, K_GATHER, K_HASH_INSERT, K_FATHER_SON,
  K_GRADING, K_NEIGHBOURS, K_CLAIM, K_CACHE_FINALIZE, K_NBR_FIX, K_FACES, K_CACHE_SOURCES,
  K_LOOKUP, K_PROLONG, K_PRIM, K_PREDICT, K_FLUX, K_UPDATE, K_REFLUX, K_RESTRICT, K_CFL, K_DT,
  K_CONVERT, K_COUNT
};
static const char *kKernelNames[K_COUNT] = {
    "sort_keys", "radix_hist", "radix_scatter", "scan", "gather_octs", "hash_insert",
    "father_son", "grading", "neighbours", "claim_comp", "cache_finalize", "neighbours_fix",
    "faces", "cache_sources", "lookup", "prolong", "prim", "predict", "flux", "update",
    "reflux", "restrict", "cfl", "dt", "convert"};

extern "C" const char *amr_kernel_name(int t) {
  return (t >= 0 && t < K_COUNT) ? kKernelNames[t] : nullptr;
}

struct TimedLaunch {
  int kid;
  cudaEvent_t e0, e1;
};

struct DevBuf {
  void *p;
  size_t bytes;
};

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------
struct amr_mesh {
  amr_params p{};
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int device = 0;
  size_t bytes = 0;
  std::vector<DevBuf> bufs;

  int64_t N = 0, NC = 0, NE = 0, S = 0;
  int64_t lo[kMaxLev + 2] = {0};   // real octs of level l: [lo[l], lo[l+1])
  int64_t clo[kMaxLev + 2] = {0};  // ghost octs of level l: [clo[l], clo[l+1])
  int64_t leaf[kMaxLev + 1] = {0};
  int B = 1;                       // bits per coordinate in ghost sort keys

  // index
  uint64_t *key = nullptr;
  int32_t *nbr27 = nullptr, *fnb = nullptr, *father = nullptr, *csrc = nullptr;
  uint32_t *son = nullptr;
  uint64_t *ckey = nullptr;
  HashView hash{};
  uint64_t hcap = 0;
  uint64_t *claim = nullptr, *comp0 = nullptr, *comp1 = nullptr;
  uint32_t *val0 = nullptr, *val1 = nullptr;
  int64_t claim_cap = 0;
  uint32_t *counters = nullptr;  // [0] claim count, [1..16] ghost level counts
  uint32_t *table = nullptr, *scan_tmp = nullptr;
  int64_t table_cap = 0, scan_cap = 0;

  // state and scratch
  void *U = nullptr, *Rc = nullptr;  // Rc: pending reflux per ghost oct [5][NC]
  int32_t *rslot = nullptr;          // [8N] ghost slot whose father is the cell
  void *W = nullptr, *Q = nullptr, *F = nullptr, *C = nullptr;
  int64_t max_ls = 0, max_cs = 0;
  double *dt_dev = nullptr;
  float *dtf_dev = nullptr;
  unsigned long long *smax = nullptr;
  int *err = nullptr;

  // work accounting
  int64_t launches = 0, graph_launches = 0;
  bool capturing = false;
  int64_t capture_kernels = 0;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_kernels = 0;
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
  double kernel_ms[K_COUNT] = {0};
  int64_t kernel_n[K_COUNT] = {0};
  cudaError_t launch_err = cudaSuccess;  // first failed launch
  int launch_err_kid = -1;

  size_t elem() const { return p.precision == 4 ? 4 : 8; }
};

static amr_status dev_alloc(amr_mesh *h, void **out, size_t bytes) {
  *out = nullptr;
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  if (h->p.hbm_budget_bytes && h->bytes + bytes > h->p.hbm_budget_bytes)
    return fail(AMR_ENOMEM, "device allocation of %zu bytes exceeds the budget (%zu of %zu held)",
                bytes, h->bytes, h->p.hbm_budget_bytes);
  void *ptr = nullptr;
  if (h->p.alloc) {
    ptr = h->p.alloc(bytes, (void *)h->s, h->p.alloc_user);
    if (!ptr) return fail(AMR_ENOMEM, "caller allocator refused %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMallocAsync(&ptr, bytes, h->s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(AMR_ENOMEM, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  h->bufs.push_back({ptr, bytes});
  h->bytes += bytes;
  *out = ptr;
  return AMR_OK;
}

static void dev_free(amr_mesh *h, void *ptr) {
  if (!ptr) return;
  for (size_t t = 0; t < h->bufs.size(); ++t) {
    if (h->bufs[t].p == ptr) {
      if (h->p.free)
        h->p.free(ptr, h->bufs[t].bytes, (void *)h->s, h->p.alloc_user);
      else
        cudaFreeAsync(ptr, h->s);
      h->bytes -= h->bufs[t].bytes;
      h->bufs.erase(h->bufs.begin() + t);
      return;
    }
  }
}

template <class P>
static amr_status alloc_n(amr_mesh *h, P **out, int64_t n) {
  void *p = nullptr;
  AMR_TRY(dev_alloc(h, &p, sizeof(P) * size_t(n > 0 ? n : 1)));
  *out = static_cast<P *>(p);
  return AMR_OK;
}

static cudaEvent_t take_event(amr_mesh *h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

template <typename... KArgs, typename... Args>
static void launch(amr_mesh *h, int kid, void (*kern)(KArgs...), dim3 grid, dim3 block,
                   Args &&...args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
  const bool timed = h->timing && !h->capturing;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    e0 = take_event(h);
    cudaEventRecord(e0, h->s);
  }
  kern<<<grid, block, 0, h->s>>>(std::forward<Args>(args)...);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess && h->launch_err == cudaSuccess) {
    h->launch_err = le;
    h->launch_err_kid = kid;
  }
  if (timed) {
    e1 = take_event(h);
    cudaEventRecord(e1, h->s);
    h->pending.push_back({kid, e0, e1});
  }
  if (h->capturing)
    ++h->capture_kernels;
  else
    ++h->launches;
}

static inline unsigned nblocks(int64_t n, int b = 256) { return unsigned((n + b - 1) / b); }

// device error word -> status
static amr_status check_device(amr_mesh *h, const char *where) {
  if (h->launch_err != cudaSuccess) {
    const cudaError_t le = h->launch_err;
    h->launch_err = cudaSuccess;
    return fail(AMR_ECUDA, "%s: launch of kernel %s failed: %s", where,
                h->launch_err_kid >= 0 ? kKernelNames[h->launch_err_kid] : "?", cudaGetErrorString(le));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AMR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  if (!err) return AMR_OK;
  CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));
  if (err & kErrRange) return fail(AMR_EINVAL, "%s: level or coordinate out of range", where);
  if (err & kErrDup) return fail(AMR_EDUP, "%s: an oct is listed twice", where);
  if (err & kErrGrading)
    return fail(AMR_EGRADING, "%s: the octree is not graded (a father-cell neighbourhood is missing)", where);
  if (err & kErrNaN) return fail(AMR_ENAN, "%s: non-finite leaf state", where);
  if (err & kErrTimeout) return fail(AMR_ETIMEOUT, "%s: a device wait gave up", where);
  return fail(AMR_ECUDA, "%s: internal index error (bits 0x%x)", where, err);
}

// ---------------------------------------------------------------------------
// scans and radix sort (host drivers of the index kernels)
// ---------------------------------------------------------------------------
static void scan_exclusive(amr_mesh *h, uint32_t *data, int64_t n, uint32_t *tmp) {
  const int64_t nb = (n + kScanItems - 1) / kScanItems;
  launch(h, K_SCAN, k_scan_block, dim3(unsigned(nb)), dim3(256), data, n, tmp);
  if (nb > 1) {
    scan_exclusive(h, tmp, nb, tmp + ((nb + 255) & ~int64_t(255)));
    launch(h, K_SCAN, k_scan_add, dim3(nblocks(n)), dim3(256), data, n, (const uint32_t *)tmp);
  }
}

static int64_t scan_tmp_size(int64_t n) {
  int64_t tot = 0;
  while (n > 1) {
    n = (n + kScanItems - 1) / kScanItems;
    tot += (n + 255) & ~int64_t(255);
  }
  return tot + 256;
}

// Stable LSD sort of (keys, vals) by the given digits; returns the buffers
// that hold the result in (*k, *v).
static void radix_sort(amr_mesh *h, uint64_t **k, uint32_t **v, uint64_t *k_alt, uint32_t *v_alt,
                       int64_t n, const std::vector<std::pair<int, int>> &digits) {
  if (n <= 0) return;
  const int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
  uint64_t *ka = *k, *kb = k_alt;
  uint32_t *va = *v, *vb = v_alt;
  for (auto &dg : digits) {
    const int shift = dg.first, nbits = dg.second;
    launch(h, K_RADIX_HIST, k_radix_hist, dim3(unsigned(ntiles)), dim3(kRadixTile),
           (const uint64_t *)ka, n, shift, nbits, h->table, ntiles);
    scan_exclusive(h, h->table, (int64_t(1) << nbits) * ntiles, h->scan_tmp);
    launch(h, K_RADIX_SCATTER, k_radix_scatter, dim3(unsigned(ntiles)), dim3(kRadixTile),
           (const uint64_t *)ka, (const uint32_t *)va, kb, vb, n, shift, nbits,
           (const uint32_t *)h->table, ntiles);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  *k = ka;
  *v = va;
}

static std::vector<std::pair<int, int>> digits_for(int shift0, int bits) {
  std::vector<std::pair<int, int>> d;
  for (int s = 0; s < bits; s += 8) d.push_back({shift0 + s, bits - s < 8 ? bits - s : 8});
  return d;
}

// ---------------------------------------------------------------------------
// level-step arguments
// ---------------------------------------------------------------------------
template <class T>
static LevelArgs<T> level_args(amr_mesh *h, int l, const double *dt_dev, double scale, double dt) {
  LevelArgs<T> a{};
  a.l = l;
  a.lmin = h->p.levelmin;
  a.lo = int(h->lo[l]);
  a.nl = int(h->lo[l + 1] - h->lo[l]);
  a.clo = int(h->clo[l]);
  a.ncl = int(h->clo[l + 1] - h->clo[l]);
  a.N = int(h->N);
  a.NE = int(h->NE);
  a.NC = int(h->NC);
  a.S = h->S;
  a.LS = 8 * (a.nl + a.ncl);
  a.CS = 24 * h->NC;
  a.U = static_cast<T *>(h->U);
  a.Rc = static_cast<T *>(h->Rc);
  a.rslot = h->rslot;
  a.fnb = h->fnb;
  a.son = h->son;
  a.father = h->father;
  a.key = h->key;
  a.csrc = h->csrc;
  a.W = static_cast<T *>(h->W);
  a.Q = static_cast<T *>(h->Q);
  a.F = static_cast<T *>(h->F);
  a.C = static_cast<T *>(h->C);
  a.dt_dev = dt_dev;
  a.dtf_dev = dt_dev ? h->dtf_dev : nullptr;
  a.dtdx_scale = scale * ldexp(1.0, l);
  a.dtdx_host = T(dt * ldexp(1.0, l));
  a.gamma = T(h->p.gamma);
  a.igm1 = T(1.0 / (h->p.gamma - 1.0));
  a.smallr = T(h->p.smallr);
  a.smallp = T(h->p.smallc * h->p.smallc / h->p.gamma);
  a.reflux = h->p.reflux;
  return a;
}

template <class T>
static void run_level_step(amr_mesh *h, int l, const double *dt_dev, double scale, double dt) {
  LevelArgs<T> a = level_args<T>(h, l, dt_dev, scale, dt);
  if (a.nl == 0) return;
  if (a.ncl) launch(h, K_PROLONG, k_prolong<T>, dim3(nblocks(5 * a.ncl)), dim3(256), a);
  if (sizeof(T) == 4) {
    // FP32: primitives recomputed inside the predictor; each leaf cell solves
    // its six faces and updates itself
    launch(h, K_PREDICT, k_predict_u<T>, dim3(nblocks(a.LS)), dim3(256), a);
    launch(h, K_FLUX, k_flux_update<T>, dim3(nblocks(8 * a.nl)), dim3(256), a);
  } else {
    // FP64: every predictor and every face solve exactly once
    launch(h, K_PRIM, k_prim<T>, dim3(nblocks(a.LS)), dim3(256), a);
    launch(h, K_PREDICT, k_predict<T>, dim3(nblocks(a.LS)), dim3(256), a);
    launch(h, K_FLUX, k_flux<T>, dim3(nblocks(a.LS)), dim3(256), a);
    launch(h, K_UPDATE, k_update<T>, dim3(nblocks(8 * a.nl)), dim3(256), a);
  }
  const int do_restrict = l > h->p.levelmin;
  const int64_t nq = (h->p.reflux ? 5 * int64_t(a.ncl) : 0) + (do_restrict ? 5 * int64_t(a.nl) : 0);
  if (nq) launch(h, K_RESTRICT, k_reflux_restrict<T>, dim3(nblocks(nq)), dim3(256), a, do_restrict);
}

static void level_step(amr_mesh *h, int l, const double *dt_dev, double scale, double dt) {
  if (h->p.precision == 4)
    run_level_step<float>(h, l, dt_dev, scale, dt);
  else
    run_level_step<double>(h, l, dt_dev, scale, dt);
}

static CflArgs cfl_args(amr_mesh *h) {
  CflArgs a{};
  a.lmin = h->p.levelmin;
  a.lmax = h->p.levelmax;
  for (int l = 0; l <= kMaxLev + 1; ++l) a.lo[l] = h->lo[l];
  a.S = h->S;
  a.son = h->son;
  a.gamma = h->p.gamma;
  a.smallr = h->p.smallr;
  a.smallp = h->p.smallc * h->p.smallc / h->p.gamma;
  a.cfl = h->p.cfl;
  a.smax = h->smax;
  a.dt_dev = h->dt_dev;
  a.dtf_dev = h->dtf_dev;
  a.err = h->err;
  return a;
}

static void cfl_device(amr_mesh *h) {
  CflArgs a = cfl_args(h);
  int64_t maxcells = 0;
  for (int l = h->p.levelmin; l <= h->p.levelmax; ++l)
    maxcells = std::max<int64_t>(maxcells, 8 * (h->lo[l + 1] - h->lo[l]));
  // a few waves of 256-thread blocks per level, grid-stride inside
  dim3 grid(std::min<unsigned>(nblocks(maxcells), 152 * 4), unsigned(h->p.levelmax - h->p.levelmin + 1));
  if (h->p.precision == 4)
    launch(h, K_CFL, k_cfl<float>, grid, dim3(256), a, (const float *)h->U);
  else
    launch(h, K_CFL, k_cfl<double>, grid, dim3(256), a, (const double *)h->U);
  launch(h, K_DT, k_dt, dim3(1), dim3(1), a);
}

static void advance_level(amr_mesh *h, int l, double scale) {
  if (l + 1 <= h->p.levelmax && h->lo[l + 2] > h->lo[l + 1]) {
    advance_level(h, l + 1, 0.5 * scale);
    advance_level(h, l + 1, 0.5 * scale);
  }
  level_step(h, l, h->dt_dev, scale, 0.0);
}

// ---------------------------------------------------------------------------
// index build (create and re-index)
// ---------------------------------------------------------------------------
static amr_status build_index(amr_mesh *h, bool first) {
  const int64_t N = h->N;
  cudaMemsetAsync(h->hash.key, 0xFF, sizeof(uint64_t) * h->hcap, h->s);
  cudaMemsetAsync(h->hash.val, 0, sizeof(int32_t) * h->hcap, h->s);
  cudaMemsetAsync(h->son, 0, sizeof(uint32_t) * N, h->s);
  cudaMemsetAsync(h->counters, 0, sizeof(uint32_t) * 32, h->s);
  launch(h, K_HASH_INSERT, k_hash_insert, dim3(nblocks(N)), dim3(256), h->hash,
         (const uint64_t *)h->key, N, h->err);
  const int64_t first_fine = h->lo[h->p.levelmin + 1];
  cudaMemsetAsync(h->father, 0xFF, sizeof(int32_t) * N, h->s);
  launch(h, K_FATHER_SON, k_father_son, dim3(nblocks(N - first_fine)), dim3(256), h->hash,
         (const uint64_t *)h->key, first_fine, N, h->father, h->son, h->err);
  if (first)
    launch(h, K_GRADING, k_grading, dim3(nblocks(8 * 27 * (N - first_fine))), dim3(256), h->hash,
           (const uint64_t *)h->key, first_fine, N, h->err);
  launch(h, K_NEIGHBOURS, k_neighbours, dim3(nblocks(27 * N)), dim3(256), h->hash,
         (const uint64_t *)h->key, N, h->nbr27, h->claim, h->counters, h->claim_cap, h->err);
  if (first) {  // create: stop after the claims; the caller sizes the ghost buffers
    AMR_TRY(check_device(h, "amr_create"));
    uint32_t nc = 0;
    CUDA_TRY(cudaMemcpyAsync(&nc, h->counters, sizeof nc, cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    h->NC = nc;
    return AMR_OK;
  }
  const int64_t NC = h->NC;
  if (NC > 0) {
    launch(h, K_CLAIM, k_claim_to_comp, dim3(nblocks(NC)), dim3(256), (const uint64_t *)h->claim,
           NC, h->B, h->comp0, h->val0);
    uint64_t *k = h->comp0;
    uint32_t *v = h->val0;
    radix_sort(h, &k, &v, h->comp1, h->val1, NC, digits_for(0, 4 + 3 * h->B));
    launch(h, K_CACHE_FINALIZE, k_cache_finalize, dim3(nblocks(NC)), dim3(256), h->hash,
           (const uint64_t *)k, NC, h->B, N, h->ckey, h->counters + 1, h->err);
    launch(h, K_NBR_FIX, k_neighbours_fix, dim3(nblocks(27 * N)), dim3(256), h->hash,
           (const uint64_t *)h->key, N, h->nbr27, h->err);
  }
  return AMR_OK;
}

static amr_status build_faces_and_sources(amr_mesh *h) {
  launch(h, K_FACES, k_faces_real, dim3(nblocks(6 * h->N)), dim3(256), (const int32_t *)h->nbr27,
         h->N, h->NE, h->fnb);
  if (h->NC) {
    launch(h, K_FACES, k_faces_cache, dim3(nblocks(6 * h->NC)), dim3(256), h->hash,
           (const uint64_t *)h->ckey, h->NC, h->N, h->NE, h->fnb);
    cudaMemsetAsync(h->rslot, 0xFF, sizeof(int32_t) * 8 * h->N, h->s);
    launch(h, K_CACHE_SOURCES, k_cache_sources, dim3(nblocks(h->NC)), dim3(256), h->hash,
           (const uint64_t *)h->ckey, h->NC, h->N, h->p.levelmin, h->csrc, h->rslot, h->err);
  }
  return AMR_OK;
}

static amr_status reindex(amr_mesh *h) {
  AMR_TRY(build_index(h, false));
  AMR_TRY(build_faces_and_sources(h));
  if (h->max_cs) cudaMemsetAsync(h->C, 0, h->elem() * 5 * size_t(h->max_cs), h->s);
  return AMR_OK;
}

// ---------------------------------------------------------------------------
// create / destroy
// ---------------------------------------------------------------------------
extern "C" void amr_params_default(amr_params *p) {
  std::memset(p, 0, sizeof *p);
  p->levelmin = 1;
  p->levelmax = 1;
  p->gamma = 1.4;
  p->cfl = 0.8;
  p->smallr = 1e-10;
  p->smallc = 1e-10;
  p->precision = 8;
  p->reflux = 1;
  p->reindex_every_step = 1;
  p->use_graphs = 1;
}

static void destroy_all(amr_mesh *h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (auto &t : h->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  while (!h->bufs.empty()) dev_free(h, h->bufs.back().p);
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->own_stream && h->s) cudaStreamDestroy(h->s);
  delete h;
}

template <class T>
static void initial_restriction(amr_mesh *h) {
  for (int l = h->p.levelmax; l > h->p.levelmin; --l) {
    LevelArgs<T> a = level_args<T>(h, l, nullptr, 1.0, 0.0);
    if (a.nl) launch(h, K_RESTRICT, k_restrict<T>, dim3(nblocks(5 * a.nl)), dim3(256), a);
  }
}

static amr_status create_impl(amr_mesh *h, int64_t n, const uint8_t *level, const uint32_t *i,
                              const uint32_t *j, const uint32_t *k, const uint64_t *hk,
                              const double *U) {
  const amr_params &p = h->p;
  // inputs to the device
  uint8_t *d_lvl;
  uint32_t *d_i, *d_j, *d_k, *perm, *perm_alt;
  uint64_t *d_hk = nullptr, *comp, *comp_alt;
  double *d_U;
  AMR_TRY(alloc_n(h, &d_lvl, n));
  AMR_TRY(alloc_n(h, &d_i, n));
  AMR_TRY(alloc_n(h, &d_j, n));
  AMR_TRY(alloc_n(h, &d_k, n));
  AMR_TRY(alloc_n(h, &d_U, 40 * n));
  if (hk) AMR_TRY(alloc_n(h, &d_hk, n));
  AMR_TRY(alloc_n(h, &perm, n));
  AMR_TRY(alloc_n(h, &perm_alt, n));
  AMR_TRY(alloc_n(h, &comp, n));
  AMR_TRY(alloc_n(h, &comp_alt, n));
  AMR_TRY(alloc_n(h, &h->err, 1));
  CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));
  CUDA_TRY(cudaMemcpyAsync(d_lvl, level, n, cudaMemcpyHostToDevice, h->s));
  CUDA_TRY(cudaMemcpyAsync(d_i, i, 4 * n, cudaMemcpyHostToDevice, h->s));
  CUDA_TRY(cudaMemcpyAsync(d_j, j, 4 * n, cudaMemcpyHostToDevice, h->s));
  CUDA_TRY(cudaMemcpyAsync(d_k, k, 4 * n, cudaMemcpyHostToDevice, h->s));
  CUDA_TRY(cudaMemcpyAsync(d_U, U, sizeof(double) * 40 * n, cudaMemcpyHostToDevice, h->s));
  if (hk) CUDA_TRY(cudaMemcpyAsync(d_hk, hk, 8 * n, cudaMemcpyHostToDevice, h->s));

  // sort: Hilbert digits (LSD), then the level bucket pass with prefix sums
  h->table_cap = 256 * ((n + kRadixTile - 1) / kRadixTile) + 256;
  h->scan_cap = scan_tmp_size(h->table_cap);
  AMR_TRY(alloc_n(h, &h->table, h->table_cap));
  AMR_TRY(alloc_n(h, &h->scan_tmp, h->scan_cap));
  launch(h, K_SORT_KEYS, k_make_sort_keys, dim3(nblocks(n)), dim3(256), (const uint8_t *)d_lvl,
         (const uint32_t *)d_i, (const uint32_t *)d_j, (const uint32_t *)d_k,
         (const uint64_t *)d_hk, n, p.levelmin, p.levelmax, comp, perm, h->err);
  AMR_TRY(check_device(h, "amr_create"));
  int hbits = hk ? 58 : 3 * (p.levelmax - 1);
  std::vector<std::pair<int, int>> digits = digits_for(0, hbits);
  digits.push_back({58, 4});  // level bucket sort
  uint64_t *kk = comp;
  uint32_t *vv = perm;
  radix_sort(h, &kk, &vv, comp_alt, perm_alt, n, digits);

  // keys in mesh order, level offsets
  h->N = n;
  AMR_TRY(alloc_n(h, &h->key, n));
  AMR_TRY(alloc_n(h, &h->counters, 32));
  CUDA_TRY(cudaMemsetAsync(h->counters, 0, sizeof(uint32_t) * 32, h->s));
  launch(h, K_GATHER, k_gather_octs<double>, dim3(nblocks(n)), dim3(256), (const uint32_t *)vv,
         (const uint8_t *)d_lvl, (const uint32_t *)d_i, (const uint32_t *)d_j,
         (const uint32_t *)d_k, (const double *)nullptr, n, h->key, (double *)nullptr, int64_t(0),
         h->counters);
  uint32_t counts[16];
  CUDA_TRY(cudaMemcpyAsync(counts, h->counters, sizeof counts, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  int64_t acc = 0;
  for (int l = 0; l <= kMaxLev; ++l) {
    h->lo[l] = acc;
    acc += counts[l];
  }
  h->lo[kMaxLev + 1] = acc;
  const int64_t side = int64_t(1) << (p.levelmin - 1);
  if (int64_t(counts[p.levelmin]) != side * side * side)
    return fail(AMR_EGRADING, "amr_create: level %d holds %u octs, a complete base needs %lld",
                p.levelmin, counts[p.levelmin], (long long)(side * side * side));

  // hash table, father/son, grading, neighbours, ghost cache
  h->B = p.levelmax - 1 > 0 ? p.levelmax - 1 : 1;
  h->claim_cap = 4 * n + 1024;
  uint64_t cap = 1024;
  while (cap < uint64_t(4 * n)) cap <<= 1;
  for (int attempt = 0; attempt < 3; ++attempt) {
    h->hcap = cap;
    AMR_TRY(alloc_n(h, &h->hash.key, cap));
    AMR_TRY(alloc_n(h, &h->hash.val, cap));
    h->hash.mask = cap - 1;
    if (!h->son) {
      AMR_TRY(alloc_n(h, &h->son, n));
      AMR_TRY(alloc_n(h, &h->father, n));
      AMR_TRY(alloc_n(h, &h->nbr27, 27 * n));
      AMR_TRY(alloc_n(h, &h->claim, h->claim_cap));
    }
    AMR_TRY(build_index(h, true));
    if (uint64_t(2 * (n + h->NC)) <= cap && h->NC <= h->claim_cap) break;
    // too full for the ghosts: grow and rebuild
    dev_free(h, h->hash.key);
    dev_free(h, h->hash.val);
    while (cap < uint64_t(2 * (n + h->NC))) cap <<= 1;
    if (h->NC > h->claim_cap) {
      dev_free(h, h->claim);
      h->claim_cap = h->NC + 1024;
      AMR_TRY(alloc_n(h, &h->claim, h->claim_cap));
    }
    h->NC = 0;
    CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));
  }
  const int64_t NC = h->NC;
  AMR_TRY(alloc_n(h, &h->ckey, NC));
  AMR_TRY(alloc_n(h, &h->comp0, NC));
  AMR_TRY(alloc_n(h, &h->comp1, NC));
  AMR_TRY(alloc_n(h, &h->val0, NC));
  AMR_TRY(alloc_n(h, &h->val1, NC));
  if (256 * ((NC + kRadixTile - 1) / kRadixTile) + 256 > h->table_cap) {
    dev_free(h, h->table);
    dev_free(h, h->scan_tmp);
    h->table_cap = 256 * ((NC + kRadixTile - 1) / kRadixTile) + 256;
    h->scan_cap = scan_tmp_size(h->table_cap);
    AMR_TRY(alloc_n(h, &h->table, h->table_cap));
    AMR_TRY(alloc_n(h, &h->scan_tmp, h->scan_cap));
  }
  // finish the index (sorted ghosts, ghost slots in the table)
  if (NC > 0) {
    launch(h, K_CLAIM, k_claim_to_comp, dim3(nblocks(NC)), dim3(256), (const uint64_t *)h->claim,
           NC, h->B, h->comp0, h->val0);
    uint64_t *ck = h->comp0;
    uint32_t *cv = h->val0;
    radix_sort(h, &ck, &cv, h->comp1, h->val1, NC, digits_for(0, 4 + 3 * h->B));
    launch(h, K_CACHE_FINALIZE, k_cache_finalize, dim3(nblocks(NC)), dim3(256), h->hash,
           (const uint64_t *)ck, NC, h->B, n, h->ckey, h->counters + 1, h->err);
    launch(h, K_NBR_FIX, k_neighbours_fix, dim3(nblocks(27 * n)), dim3(256), h->hash,
           (const uint64_t *)h->key, n, h->nbr27, h->err);
  }
  uint32_t ccounts[16];
  CUDA_TRY(cudaMemcpyAsync(ccounts, h->counters + 1, sizeof ccounts, cudaMemcpyDeviceToHost, h->s));
  AMR_TRY(check_device(h, "amr_create"));
  acc = 0;
  for (int l = 0; l <= kMaxLev; ++l) {
    h->clo[l] = acc;
    acc += ccounts[l];
  }
  h->clo[kMaxLev + 1] = acc;
  h->NE = n + NC;
  h->S = 8 * h->NE;
  AMR_TRY(alloc_n(h, &h->fnb, 6 * h->NE));
  AMR_TRY(alloc_n(h, &h->csrc, 7 * (NC > 0 ? NC : 1)));
  AMR_TRY(alloc_n(h, &h->rslot, 8 * n));
  CUDA_TRY(cudaMemsetAsync(h->rslot, 0xFF, sizeof(int32_t) * 8 * n, h->s));
  AMR_TRY(build_faces_and_sources(h));
  AMR_TRY(check_device(h, "amr_create"));

  // state in mesh order
  const size_t es = h->elem();
  AMR_TRY(dev_alloc(h, &h->U, es * 5 * size_t(h->S)));
  AMR_TRY(dev_alloc(h, &h->Rc, es * 5 * size_t(NC > 0 ? NC : 1)));
  CUDA_TRY(cudaMemsetAsync(h->U, 0, es * 5 * size_t(h->S), h->s));
  CUDA_TRY(cudaMemsetAsync(h->Rc, 0, es * 5 * size_t(NC > 0 ? NC : 1), h->s));
  if (p.precision == 4)
    launch(h, K_GATHER, k_gather_octs<float>, dim3(nblocks(n)), dim3(256), (const uint32_t *)vv,
           (const uint8_t *)d_lvl, (const uint32_t *)d_i, (const uint32_t *)d_j,
           (const uint32_t *)d_k, (const double *)d_U, n, h->key, (float *)h->U, h->S,
           (uint32_t *)nullptr);
  else
    launch(h, K_GATHER, k_gather_octs<double>, dim3(nblocks(n)), dim3(256), (const uint32_t *)vv,
           (const uint8_t *)d_lvl, (const uint32_t *)d_i, (const uint32_t *)d_j,
           (const uint32_t *)d_k, (const double *)d_U, n, h->key, (double *)h->U, h->S,
           (uint32_t *)nullptr);

  // leaf counts (host, from the level sizes: each oct above levelmin splits
  // one cell of the level below)
  for (int l = 0; l <= kMaxLev; ++l) h->leaf[l] = 8 * (h->lo[l + 1] - h->lo[l]);
  for (int l = p.levelmin + 1; l <= kMaxLev; ++l) h->leaf[l - 1] -= h->lo[l + 1] - h->lo[l];

  // scratch for the largest level step
  for (int l = p.levelmin; l <= p.levelmax; ++l) {
    const int64_t ls = 8 * ((h->lo[l + 1] - h->lo[l]) + (h->clo[l + 1] - h->clo[l]));
    h->max_ls = std::max(h->max_ls, ls);
  }
  h->max_cs = 24 * h->NC;
  AMR_TRY(dev_alloc(h, &h->W, es * 5 * size_t(h->max_ls)));
  AMR_TRY(dev_alloc(h, &h->Q, es * 20 * size_t(h->max_ls)));
  AMR_TRY(dev_alloc(h, &h->F, es * 15 * size_t(h->max_ls)));
  AMR_TRY(dev_alloc(h, &h->C, es * 5 * size_t(h->max_cs > 0 ? h->max_cs : 1)));
  if (h->max_cs) CUDA_TRY(cudaMemsetAsync(h->C, 0, es * 5 * size_t(h->max_cs), h->s));
  AMR_TRY(alloc_n(h, &h->dt_dev, 1));
  AMR_TRY(alloc_n(h, &h->dtf_dev, 1));
  AMR_TRY(alloc_n(h, &h->smax, 16));
  CUDA_TRY(cudaMemsetAsync(h->smax, 0, sizeof(unsigned long long) * 16, h->s));

  if (p.precision == 4)
    initial_restriction<float>(h);
  else
    initial_restriction<double>(h);
  AMR_TRY(check_device(h, "amr_create"));
  // release the input staging
  dev_free(h, d_lvl);
  dev_free(h, d_i);
  dev_free(h, d_j);
  dev_free(h, d_k);
  dev_free(h, d_U);
  if (d_hk) dev_free(h, d_hk);
  dev_free(h, perm);
  dev_free(h, perm_alt);
  dev_free(h, comp);
  dev_free(h, comp_alt);
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return AMR_OK;
}

extern "C" amr_status amr_create(const amr_params *p, int64_t n_oct, const uint8_t *level,
                                 const uint32_t *i, const uint32_t *j, const uint32_t *k,
                                 const uint64_t *hilbert_key, const double *U, amr_handle *out) {
  g_last_error.clear();
  if (!out) return fail(AMR_EINVAL, "amr_create: out is NULL");
  *out = nullptr;
  if (!p || !level || !i || !j || !k || !U) return fail(AMR_EINVAL, "amr_create: NULL argument");
  if (p->levelmin < 1 || p->levelmax > kMaxLev || p->levelmin > p->levelmax)
    return fail(AMR_EINVAL, "amr_create: levels must satisfy 1 <= levelmin <= levelmax <= %d", kMaxLev);
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->smallr > 0.0) || !(p->smallc > 0.0))
    return fail(AMR_EINVAL, "amr_create: gamma > 1, cfl > 0, smallr > 0, smallc > 0 required");
  if (p->precision != 4 && p->precision != 8)
    return fail(AMR_EINVAL, "amr_create: precision must be 4 or 8");
  if (n_oct < 1 || n_oct > (int64_t(1) << 26))
    return fail(AMR_EINVAL, "amr_create: n_oct must be in [1, 2^26]");
  amr_mesh *h = new amr_mesh();
  h->p = *p;
  cudaGetDevice(&h->device);
  if (p->stream) {
    h->s = static_cast<cudaStream_t>(p->stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return fail(AMR_ECUDA, "amr_create: cannot create a stream");
    }
    h->own_stream = true;
  }
  amr_status s = create_impl(h, n_oct, level, i, j, k, hilbert_key, U);
  if (s != AMR_OK) {
    std::string msg = g_last_error;
    destroy_all(h);
    g_last_error = msg;
    return s;
  }
  *out = h;
  return AMR_OK;
}

extern "C" amr_status amr_destroy(amr_handle h) {
  if (!h) return AMR_OK;
  destroy_all(h);
  return AMR_OK;
}

// ---------------------------------------------------------------------------
// stepping
// ---------------------------------------------------------------------------
extern "C" amr_status amr_cfl_dt(amr_handle h, double *dt_out) {
  if (!h || !dt_out) return fail(AMR_EINVAL, "amr_cfl_dt: NULL argument");
  cfl_device(h);
  CUDA_TRY(cudaMemcpyAsync(dt_out, h->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  return check_device(h, "amr_cfl_dt");
}

extern "C" amr_status amr_step_level(amr_handle h, int level, double dt) {
  if (!h) return fail(AMR_EINVAL, "amr_step_level: NULL handle");
  if (level < h->p.levelmin || level > h->p.levelmax)
    return fail(AMR_EINVAL, "amr_step_level: level %d outside [%d, %d]", level, h->p.levelmin,
                h->p.levelmax);
  if (!(dt > 0.0)) return fail(AMR_EINVAL, "amr_step_level: dt must be > 0");
  level_step(h, level, nullptr, 1.0, dt);
  if (h->launch_err != cudaSuccess) return check_device(h, "amr_step_level");
  return AMR_OK;
}

static void coarse_step(amr_mesh *h) {
  if (h->p.reindex_every_step) reindex(h);
  cfl_device(h);
  advance_level(h, h->p.levelmin, 1.0);
}

extern "C" amr_status amr_advance(amr_handle h, int n, double *dt_last) {
  if (!h) return fail(AMR_EINVAL, "amr_advance: NULL handle");
  if (n < 0) return fail(AMR_EINVAL, "amr_advance: n must be >= 0");
  const bool graphs = h->p.use_graphs && !h->timing;
  if (graphs && !h->graph && n > 0) {
    h->capturing = true;
    h->capture_kernels = 0;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    coarse_step(h);
    cudaError_t e = cudaStreamEndCapture(h->s, &g);
    h->capturing = false;
    if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_advance: capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_advance: instantiate failed: %s", cudaGetErrorString(e));
    h->graph_kernels = h->capture_kernels;
  }
  for (int t = 0; t < n; ++t) {
    if (graphs) {
      CUDA_TRY(cudaGraphLaunch(h->graph, h->s));
      h->graph_launches++;
      h->launches += h->graph_kernels;
    } else {
      coarse_step(h);
    }
  }
  if (h->launch_err != cudaSuccess) return check_device(h, "amr_advance");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_advance: %s", cudaGetErrorString(e));
  if (dt_last) {
    CUDA_TRY(cudaMemcpyAsync(dt_last, h->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    return check_device(h, "amr_advance");
  }
  return AMR_OK;
}

extern "C" amr_status amr_reindex(amr_handle h) {
  if (!h) return fail(AMR_EINVAL, "amr_reindex: NULL handle");
  AMR_TRY(reindex(h));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_reindex: %s", cudaGetErrorString(e));
  return AMR_OK;
}

extern "C" amr_status amr_sync(amr_handle h) {
  if (!h) return fail(AMR_EINVAL, "amr_sync: NULL handle");
  return check_device(h, "amr_sync");
}

extern "C" amr_status amr_fill_ghosts(amr_handle h, int level) {
  if (!h) return fail(AMR_EINVAL, "amr_fill_ghosts: NULL handle");
  if (level < h->p.levelmin || level > h->p.levelmax) return fail(AMR_EINVAL, "amr_fill_ghosts: bad level");
  if (h->p.precision == 4) {
    LevelArgs<float> a = level_args<float>(h, level, nullptr, 1.0, 0.0);
    if (a.ncl) launch(h, K_PROLONG, k_prolong<float>, dim3(nblocks(5 * a.ncl)), dim3(256), a);
  } else {
    LevelArgs<double> a = level_args<double>(h, level, nullptr, 1.0, 0.0);
    if (a.ncl) launch(h, K_PROLONG, k_prolong<double>, dim3(nblocks(5 * a.ncl)), dim3(256), a);
  }
  return AMR_OK;
}

// ---------------------------------------------------------------------------
// state in / out
// ---------------------------------------------------------------------------
// copy [5][count] values starting at element `first` of each row of a
// device array with row stride `stride` into host doubles
static amr_status rows_to_host(amr_mesh *h, const void *src, int64_t stride, int64_t first,
                               int64_t count, double *dst) {
  if (count == 0) return AMR_OK;
  if (h->p.precision == 8) {
    for (int v = 0; v < 5; ++v)
      CUDA_TRY(cudaMemcpyAsync(dst + v * count, static_cast<const double *>(src) + v * stride + first,
                               sizeof(double) * count, cudaMemcpyDeviceToHost, h->s));
    return AMR_OK;
  }
  double *stage;
  AMR_TRY(alloc_n(h, &stage, 5 * count));
  launch(h, K_CONVERT, k_to_double<float>, dim3(nblocks(5 * count)), dim3(256),
         static_cast<const float *>(src) + first, stride, count, stage);
  CUDA_TRY(cudaMemcpyAsync(dst, stage, sizeof(double) * 5 * count, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  dev_free(h, stage);
  return AMR_OK;
}

extern "C" amr_status amr_read(amr_handle h, int level, int64_t *n_oct_out, uint64_t *keys,
                               double *U, int64_t cap) {
  if (!h) return fail(AMR_EINVAL, "amr_read: NULL handle");
  if (level < 0 || level > kMaxLev) return fail(AMR_EINVAL, "amr_read: bad level");
  const int64_t lo = h->lo[level], nl = h->lo[level + 1] - lo;
  if (n_oct_out) *n_oct_out = nl;
  if ((keys || U) && cap < nl) return fail(AMR_EINVAL, "amr_read: cap %lld < %lld octs", (long long)cap, (long long)nl);
  if (keys && nl)
    CUDA_TRY(cudaMemcpyAsync(keys, h->key + lo, 8 * nl, cudaMemcpyDeviceToHost, h->s));
  if (U) AMR_TRY(rows_to_host(h, h->U, h->S, 8 * lo, 8 * nl, U));
  return check_device(h, "amr_read");
}

extern "C" amr_status amr_read_reflux(amr_handle h, int level, double *R, int64_t cap) {
  if (!h || !R) return fail(AMR_EINVAL, "amr_read_reflux: NULL argument");
  if (level < 0 || level > kMaxLev) return fail(AMR_EINVAL, "amr_read_reflux: bad level");
  const int64_t lo = h->lo[level], nl = h->lo[level + 1] - lo;
  if (cap < nl) return fail(AMR_EINVAL, "amr_read_reflux: cap too small");
  const int64_t n8 = 8 * nl;
  for (int64_t t = 0; t < 5 * n8; ++t) R[t] = 0.0;
  if (nl == 0 || h->NC == 0) return check_device(h, "amr_read_reflux");
  std::vector<int32_t> slot(n8);
  std::vector<double> rc(5 * size_t(h->NC));
  CUDA_TRY(cudaMemcpyAsync(slot.data(), h->rslot + 8 * lo, 4 * n8, cudaMemcpyDeviceToHost, h->s));
  AMR_TRY(rows_to_host(h, h->Rc, h->NC, 0, h->NC, rc.data()));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  for (int64_t t = 0; t < n8; ++t)
    if (slot[t] >= 0)
      for (int v = 0; v < 5; ++v) R[v * n8 + t] = rc[v * size_t(h->NC) + slot[t]];
  return check_device(h, "amr_read_reflux");
}

extern "C" amr_status amr_write(amr_handle h, int level, const double *U, int64_t n) {
  if (!h || !U) return fail(AMR_EINVAL, "amr_write: NULL argument");
  if (level < 0 || level > kMaxLev) return fail(AMR_EINVAL, "amr_write: bad level");
  const int64_t lo = h->lo[level], nl = h->lo[level + 1] - lo;
  if (n != nl) return fail(AMR_EINVAL, "amr_write: level %d holds %lld octs, got %lld", level, (long long)nl, (long long)n);
  if (nl == 0) return AMR_OK;
  const int64_t count = 8 * nl;
  if (h->p.precision == 8) {
    for (int v = 0; v < 5; ++v)
      CUDA_TRY(cudaMemcpyAsync(static_cast<double *>(h->U) + v * h->S + 8 * lo, U + v * count,
                               sizeof(double) * count, cudaMemcpyHostToDevice, h->s));
    return AMR_OK;
  }
  double *stage;
  AMR_TRY(alloc_n(h, &stage, 5 * count));
  CUDA_TRY(cudaMemcpyAsync(stage, U, sizeof(double) * 5 * count, cudaMemcpyHostToDevice, h->s));
  launch(h, K_CONVERT, k_from_double<float>, dim3(nblocks(5 * count)), dim3(256),
         (const double *)stage, count, static_cast<float *>(h->U) + 8 * lo, h->S);
  dev_free(h, stage);
  return AMR_OK;
}

// ---------------------------------------------------------------------------
// introspection
// ---------------------------------------------------------------------------
extern "C" amr_status amr_lookup(amr_handle h, int64_t n, const uint64_t *keys, int64_t *idx_out) {
  if (!h || (n > 0 && (!keys || !idx_out))) return fail(AMR_EINVAL, "amr_lookup: NULL argument");
  if (n <= 0) return AMR_OK;
  uint64_t *dk;
  int64_t *dout;
  AMR_TRY(alloc_n(h, &dk, n));
  AMR_TRY(alloc_n(h, &dout, n));
  CUDA_TRY(cudaMemcpyAsync(dk, keys, 8 * n, cudaMemcpyHostToDevice, h->s));
  launch(h, K_LOOKUP, k_lookup, dim3(nblocks(8 * n)), dim3(256), h->hash, (const uint64_t *)dk, n,
         h->N, dout);
  CUDA_TRY(cudaMemcpyAsync(idx_out, dout, 8 * n, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  dev_free(h, dk);
  dev_free(h, dout);
  return check_device(h, "amr_lookup");
}

extern "C" amr_status amr_read_index(amr_handle h, int level, int64_t *nbr, uint8_t *split,
                                     int64_t cap) {
  if (!h) return fail(AMR_EINVAL, "amr_read_index: NULL handle");
  if (level < 0 || level > kMaxLev) return fail(AMR_EINVAL, "amr_read_index: bad level");
  const int64_t lo = h->lo[level], nl = h->lo[level + 1] - lo;
  if (cap < nl) return fail(AMR_EINVAL, "amr_read_index: cap too small");
  if (nl == 0) return AMR_OK;
  if (nbr) {
    std::vector<int32_t> tmp(27 * size_t(nl));
    for (int e = 0; e < 27; ++e)
      CUDA_TRY(cudaMemcpyAsync(tmp.data() + e * nl, h->nbr27 + e * h->N + lo, 4 * nl,
                               cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    for (int64_t t = 0; t < nl; ++t)
      for (int e = 0; e < 27; ++e) {
        const int64_t x = tmp[e * nl + t];
        nbr[27 * t + e] = x < h->N ? x : -(1 + (x - h->N));
      }
  }
  if (split) {
    std::vector<uint32_t> son(nl);
    CUDA_TRY(cudaMemcpyAsync(son.data(), h->son + lo, 4 * nl, cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    for (int64_t t = 0; t < nl; ++t)
      for (int c = 0; c < 8; ++c) split[8 * t + c] = (son[t] >> c) & 1u;
  }
  return check_device(h, "amr_read_index");
}

extern "C" amr_status amr_read_cache(amr_handle h, int level, int64_t *n_out, int64_t *first_out,
                                     uint64_t *keys, double *Ug, int64_t cap) {
  if (!h) return fail(AMR_EINVAL, "amr_read_cache: NULL handle");
  if (level < 0 || level > kMaxLev) return fail(AMR_EINVAL, "amr_read_cache: bad level");
  const int64_t c0 = h->clo[level], nc = h->clo[level + 1] - c0;
  if (n_out) *n_out = nc;
  if (first_out) *first_out = c0;
  if ((keys || Ug) && cap < nc) return fail(AMR_EINVAL, "amr_read_cache: cap too small");
  if (keys && nc) CUDA_TRY(cudaMemcpyAsync(keys, h->ckey + c0, 8 * nc, cudaMemcpyDeviceToHost, h->s));
  if (Ug) AMR_TRY(rows_to_host(h, h->U, h->S, 8 * (h->N + c0), 8 * nc, Ug));
  return check_device(h, "amr_read_cache");
}

extern "C" amr_status amr_get_info(amr_handle h, amr_info *info) {
  if (!h || !info) return fail(AMR_EINVAL, "amr_get_info: NULL argument");
  std::memset(info, 0, sizeof *info);
  info->n_oct = h->N;
  info->n_cache = h->NC;
  for (int l = 0; l <= kMaxLev; ++l) {
    info->level_octs[l] = h->lo[l + 1] - h->lo[l];
    info->level_cache[l] = h->clo[l + 1] - h->clo[l];
    info->level_leaf_cells[l] = h->leaf[l];
    info->n_leaf_cells += h->leaf[l];
  }
  info->device_bytes = int64_t(h->bytes);
  info->kernel_launches = h->launches;
  info->graph_launches = h->graph_launches;
  info->hash_capacity = int64_t(h->hcap);
  info->precision = h->p.precision;
  return AMR_OK;
}

extern "C" amr_status amr_set_timing(amr_handle h, int on) {
  if (!h) return fail(AMR_EINVAL, "amr_set_timing: NULL handle");
  h->timing = on != 0;
  return AMR_OK;
}

extern "C" amr_status amr_read_timing(amr_handle h, int n, double *ms, int64_t *launches) {
  if (!h) return fail(AMR_EINVAL, "amr_read_timing: NULL handle");
  CUDA_TRY(cudaStreamSynchronize(h->s));
  for (auto &t : h->pending) {
    float x = 0.f;
    cudaEventElapsedTime(&x, t.e0, t.e1);
    h->kernel_ms[t.kid] += x;
    h->kernel_n[t.kid] += 1;
    h->event_pool.push_back(t.e0);
    h->event_pool.push_back(t.e1);
  }
  h->pending.clear();
  for (int t = 0; t < n && t < K_COUNT; ++t) {
    if (ms) ms[t] = h->kernel_ms[t];
    if (launches) launches[t] = h->kernel_n[t];
  }
  return AMR_OK;
}
