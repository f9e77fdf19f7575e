// amr_api.cu -- C ABI of the GB300 level-advance library (see include/amr.h).
// Host orchestration only: every step of the mesh build, index and level
// step runs in the kernels of index_kernels.cuh and hydro_kernels.cuh,
// compiled here as one translation unit.
//
// A handle holds one or more independent member meshes.  Octs are ordered
// by (member, level, Hilbert key), so each (member, level) is a contiguous
// segment; a level-step launch runs over a flattened list of tiles of many
// segments.  A coarse step advances every member by its own CFL time step
// through its own W-cycle; the members' W-cycles are aligned phase by phase
// (phase k runs the k-th level step of every member in one launch per
// kernel), and one coarse step is captured once as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "hydro_kernels.cuh"
#include "rock_kernels.cuh"
#include "regrid_kernels.cuh"
#include "mg_kernels.cuh"
#include "index_kernels.cuh"
#include "deposit_kernels.cuh"

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
  K_CONVERT, K_FLAG, K_REGRID, K_PROLONG_NEW, K_FLAG_RP, K_FLAG_EXPAND, K_FLAG_GRADE,
  K_MG_SMOOTH, K_MG_RESTRICT, K_MG_PROLONG, K_MG_OTHER, K_ROCK, K_COMMIT, K_SWEEP, K_TOTALS,
  K_FNV, K_DEPOSIT, K_SPLIT, K_SORT_GROUPS, K_MERGE, K_FLAG_EXACT, K_COUNT
};
static const char *kKernelNames[K_COUNT] = {
    "sort_keys", "radix_hist", "radix_scatter", "scan", "gather_octs", "hash_insert",
    "father_son", "grading", "neighbours", "claim_comp", "cache_finalize", "neighbours_fix",
    "faces", "cache_sources", "lookup", "prolong", "prim", "predict", "flux", "update",
    "reflux", "reflux_restrict", "cfl", "dt", "convert", "flag", "regrid", "prolong_new",
    "flag_rp", "flag_expand", "flag_grade", "mg_smooth", "mg_restrict", "mg_prolong", "mg_other",
    "rock", "commit", "sweep", "totals", "fnv", "deposit_level", "split_level", "sort_groups",
    "merge_rank", "flag_exact"};

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

// Buffers a regrid's retired mesh leaves for the next regrid: shared by the
// handle and the shells it builds new meshes in, so the next mesh takes its
// arrays from here instead of the allocator (a regrid allocates and frees
// about 60 arrays).  Holds at most `cap` bytes (the live mesh's size, set by
// the regrid; 0 otherwise, when frees go to the allocator).  Handles with a
// device budget do not keep one.
struct BufCache {
  std::vector<DevBuf> v;
  size_t bytes = 0, cap = 0;
};

// page-locked words for small device-to-host reads: several reads queued on
// the stream complete with one synchronisation (a read into pageable memory
// waits for the stream on its own)
struct HostPin {
  uint32_t *w = nullptr;  // w[0]: the device error word; w[1..cap): data
  size_t cap = 0;
  ~HostPin() {
    if (w) cudaFreeHost(w);
  }
};

// level-step launch domains of a segment
enum Dom {
  DOM_CELLS = 0, DOM_REAL = 1, DOM_GHOST5 = 2, DOM_POST = 3, DOM_BLOCKS = 4, DOM_COMMIT = 5, DOM_COUNT = 6
};

// a list of segments and, per domain, its tiles: the offset of its tile
// prefix (nseg + 1 cumulative counts) in the handle's prefix array, and the
// number of tiles
struct SegList {
  int seg0 = 0, nseg = 0;
  int tpre0[DOM_COUNT] = {0, 0, 0, 0, 0, 0}, ntile[DOM_COUNT] = {0, 0, 0, 0, 0, 0};
  int ls = 0;  // scratch cells used
};

struct Member {
  int lmin = 1, lmax = 1;
  double gamma = 1.4, cfl = 0.8, smallr = 1e-10, smallc = 1e-10;
  int64_t n_oct = 0;
  int64_t oct_base = 0, cache_base = 0;  // first mesh index, first ghost slot
  int64_t lo[kMaxLev + 2] = {0};         // member-local level offsets of real octs
  int64_t clo[kMaxLev + 2] = {0};        // member-local level offsets of ghost octs
  int64_t leaf[kMaxLev + 1] = {0};
  std::vector<int> seq;                  // levels of its W-cycle, in order
};

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------
struct amr_mesh {
  amr_params p{};
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int device = 0, sm_count = 152;
  size_t bytes = 0;
  std::vector<DevBuf> bufs;
  std::shared_ptr<BufCache> cache;
  std::shared_ptr<HostPin> pin;  // shared with the handle's regrid shells

  int M = 1, sel = 0, lmax_all = 1;
  std::vector<Member> mem;
  int64_t N = 0, NC = 0, NE = 0, S = 0;
  int B = 1;  // bits per coordinate in ghost sort keys

  // index
  uint64_t *key = nullptr;
  int32_t *nbr27 = nullptr, *fnb = nullptr, *father = nullptr, *csrc = nullptr;
  int32_t *rslot = nullptr;
  uint32_t *son = nullptr;
  uint64_t *ckey = nullptr;
  HashView hash{};
  uint64_t hcap = 0;
  uint64_t *claim = nullptr, *comp0 = nullptr, *comp1 = nullptr;
  uint32_t *val0 = nullptr, *val1 = nullptr;
  int64_t claim_cap = 0;
  uint32_t *counters = nullptr;    // [0] claim count
  uint32_t *seg_count = nullptr;   // [16 M] octs / ghost octs per (member, level)
  uint32_t *table = nullptr, *scan_tmp = nullptr;
  int64_t table_cap = 0, scan_cap = 0;

  // members on the device
  int *mlmin = nullptr, *mlmax = nullptr;
  double *mgamma_d = nullptr, *mcfl_d = nullptr, *msmallr_d = nullptr, *msmallp_d = nullptr;
  void *mgamma_t = nullptr, *migm1_t = nullptr, *msmallr_t = nullptr, *msmallp_t = nullptr;
  float *mflag32 = nullptr;  // per member: gamma - 1, smallr, smallp rounded to FP32 (regrid screen)
  double *dt_dev = nullptr, *dtdx_dev = nullptr;
  float *dtdxf_dev = nullptr;
  int *mrem = nullptr, *mact = nullptr;  // coarse steps left; active this step
  int *merr = nullptr;                   // error bits per member
  unsigned long long *smax = nullptr;
  int *err = nullptr;

  // segments and tiles
  std::vector<Seg> segs_h;
  std::vector<int> tpre_h;
  Seg *segs = nullptr;
  int *tpre = nullptr;
  std::vector<SegList> phases;
  SegList level_list[kMaxLev + 1], restrict_list[kMaxLev + 1], cfl_list;
  int tile_size = 256;
  bool persistent = true;
  bool tuned = false;
  // fused shared-memory level step ("rock" kernel): octs per axis of a block
  // (0: the per-cell passes), block starts (mesh indices) and, on the host,
  // the block of every oct
  int nsub = 0;
  bool planar = false;  // the fused kernel sweeps planes (paper kernel), else stages the cube (rock)
  int32_t *blk = nullptr;
  std::vector<int32_t> blk_first, blk_last;  // block of the first / last oct of each (member, level)
  std::vector<float> tune_ms;  // the autotuner's best step time per candidate
  // asynchronous whole-state copies: copy streams (uploads, downloads; each
  // direction its own, so that one never queues behind the other), input and
  // output staging buffers (doubles, [5][8 n] of the selected member) and
  // their events
  cudaStream_t cs = nullptr, cs_out = nullptr;
  double *st_in = nullptr, *st_out = nullptr;
  int64_t st_n = 0;
  cudaEvent_t ev_in_ready = nullptr, ev_in_free = nullptr, ev_out_ready = nullptr, ev_out_free = nullptr;
  std::vector<std::pair<const void *, int>> occ;  // (kernel, blocks per SM) at tile_size

  // state and scratch
  void *U = nullptr, *Rc = nullptr;
  void *W = nullptr, *Q = nullptr, *F = nullptr, *C = nullptr;
  int64_t max_ls = 0, max_cs = 0;
  int64_t ls_cap = 0, cs_cap = 0;  // elements the scratch arrays hold

  // multigrid (base level of the selected member): dense arrays per level,
  // finest first; the potential of the base cells in mesh order
  struct MGLevel {
    int n = 0;
    double *f = nullptr, *p = nullptr;
  };
  std::vector<MGLevel> mg;
  int mg_member = -1;
  // a mesh built from flags that went through the grading closure skips the
  // (27-probe per oct) grading check, except in the bounds-checked build
  bool graded_by_construction = false;
  // the octs' order came from keys computed here (not from the caller's
  // Hilbert keys), so a regrid's kept octs are already in sorted order
  bool order_computed = false;
  // Poisson on a refined level: per MG level the tables of k_mgl_*, the
  // level's cells (g0: global cell index), their fathers and the coarse cells
  // across boundary faces; the potential of every cell (mesh order)
  struct MGLTab {
    int L = 0;
    int64_t n = 0, nc0 = 0, nc1 = 0;
    int32_t *nb = nullptr, *nbnd = nullptr, *col = nullptr, *child = nullptr, *pro = nullptr;
    double *e = nullptr, *f = nullptr, *r = nullptr;
  };
  struct MGLSet {
    std::vector<MGLTab> tab;
    int32_t *g0 = nullptr, *fatherg = nullptr, *acrossg = nullptr;
    double *bsum = nullptr;
  };
  std::map<int, MGLSet> mgls;  // key: member * 32 + level
  double *mgl_part = nullptr, *mgl_scalar = nullptr;
  double *phil = nullptr;
  int64_t phil_n = 0;
  double *mg_rho = nullptr, *mg_r = nullptr, *mg_part = nullptr, *mg_res = nullptr;
  double *phi = nullptr;

  // particle deposition onto the levels: positions and masses (the handle's
  // precision), two particle lists, split flags and their prefix sums, list
  // lengths per level, and the density of every cell
  void *px = nullptr, *py = nullptr, *pz = nullptr, *pm = nullptr;
  uint32_t *plist0 = nullptr, *plist1 = nullptr, *pflag = nullptr, *ppos = nullptr, *ptmp = nullptr;
  int64_t *pcount = nullptr;
  int64_t pcap = 0;
  void *prho = nullptr;
  int64_t prho_n = 0;
  // oct index of every base-level oct of one member by its coordinates
  // ((x * side + y) * side + z): the complete base level needs no hash probe
  int32_t *btab = nullptr;
  int btab_member = -1;

  // work accounting
  int64_t launches = 0, graph_launches = 0;
  bool capturing = false;
  int64_t capture_kernels = 0;
  int64_t steps_on_mesh = 0;  // coarse steps since this mesh was built
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
  if (h->cache && !h->cache->v.empty()) {  // the smallest cached array that fits, within 2x (or 8 KB)
    std::vector<DevBuf> &v = h->cache->v;
    size_t best = v.size();
    for (size_t t = 0; t < v.size(); ++t)
      if (v[t].bytes >= bytes && v[t].bytes <= std::max(2 * bytes, size_t(8192)) &&
          (best == v.size() || v[t].bytes < v[best].bytes))
        best = t;
    if (best < v.size()) {
      const DevBuf b = v[best];
      v.erase(v.begin() + best);
      h->cache->bytes -= b.bytes;
      h->bufs.push_back(b);
      h->bytes += b.bytes;
      *out = b.p;
      return AMR_OK;
    }
  }
  // a handle that regrids asks for arrays a little larger each time a mesh
  // grows: a fresh array gets 1/8 headroom, so that the next mesh's request
  // still fits the cached array instead of a new allocation
  if (h->cache) {
    const size_t wide = (bytes + bytes / 8 + 4095) & ~size_t(4095);
    if (!h->p.hbm_budget_bytes || h->bytes + wide <= h->p.hbm_budget_bytes) bytes = wide;
  }
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

static void real_free(amr_mesh *h, void *ptr, size_t bytes) {
  if (h->p.free)
    h->p.free(ptr, bytes, (void *)h->s, h->p.alloc_user);
  else
    cudaFreeAsync(ptr, h->s);
}

static void dev_free(amr_mesh *h, void *ptr) {
  if (!ptr) return;
  for (size_t t = 0; t < h->bufs.size(); ++t) {
    if (h->bufs[t].p == ptr) {
      const DevBuf b = h->bufs[t];
      h->bytes -= b.bytes;
      h->bufs.erase(h->bufs.begin() + t);
      if (h->cache && h->cache->bytes + b.bytes <= h->cache->cap) {
        h->cache->v.push_back(b);  // reused in stream order: every use is on h->s
        h->cache->bytes += b.bytes;
      } else {
        real_free(h, b.p, b.bytes);
      }
      return;
    }
  }
}

// hand a buffer from one handle to another (no copy)
static void move_buf(amr_mesh *to, amr_mesh *from, void *ptr) {
  if (!ptr) return;
  for (size_t t = 0; t < from->bufs.size(); ++t)
    if (from->bufs[t].p == ptr) {
      to->bufs.push_back(from->bufs[t]);
      to->bytes += from->bufs[t].bytes;
      from->bytes -= from->bufs[t].bytes;
      from->bufs.erase(from->bufs.begin() + t);
      return;
    }
}

template <class P>
static amr_status alloc_n(amr_mesh *h, P **out, int64_t n) {
  void *p = nullptr;
  AMR_TRY(dev_alloc(h, &p, sizeof(P) * size_t(n > 0 ? n : 1)));
  *out = static_cast<P *>(p);
  return AMR_OK;
}

template <class P>
static amr_status upload(amr_mesh *h, P **out, const std::vector<P> &v) {
  AMR_TRY(alloc_n(h, out, int64_t(v.size())));
  if (!v.empty())
    CUDA_TRY(cudaMemcpyAsync(*out, v.data(), sizeof(P) * v.size(), cudaMemcpyHostToDevice, h->s));
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

// one launch on the handle's stream
template <typename... KArgs, typename... Args>
static void launch_on(amr_mesh *h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                      Args &&...args) {
  kern<<<grid, block, smem, h->s>>>(std::forward<Args>(args)...);
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
  launch_on(h, kern, grid, block, 0, std::forward<Args>(args)...);
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

// launch() with dynamic shared memory
template <class... KArgs, class... Args>
static void launch_smem(amr_mesh *h, int kid, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                        Args &&...args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
  const bool timed = h->timing && !h->capturing;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    e0 = take_event(h);
    cudaEventRecord(e0, h->s);
  }
  launch_on(h, kern, grid, block, smem, std::forward<Args>(args)...);
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

// check_device without a synchronisation: launch errors only (the device
// error word is read at the next check_device)
static amr_status check_launches(amr_mesh *h, const char *where) {
  if (h->launch_err != cudaSuccess) {
    const cudaError_t le = h->launch_err;
    h->launch_err = cudaSuccess;
    return fail(AMR_ECUDA, "%s: launch of kernel %s failed: %s", where,
                h->launch_err_kid >= 0 ? kKernelNames[h->launch_err_kid] : "?", cudaGetErrorString(le));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AMR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
  return AMR_OK;
}

// device error word -> status
static amr_status check_device(amr_mesh *h, const char *where) {
  AMR_TRY(check_launches(h, where));
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
  if (err & kErrIndex)
    return fail(AMR_ECUDA, "%s: an index-table entry out of range (bounds-checked build)", where);
  return fail(AMR_ECUDA, "%s: internal index error (bits 0x%x)", where, err);
}

// the handle's page-locked read-back words, room for n data words (grown at
// need; w[0] is kept for the device error word)
static amr_status pinned_words(amr_mesh *h, size_t n, uint32_t **out) {
  if (!h->pin) h->pin = std::make_shared<HostPin>();
  HostPin &P = *h->pin;
  if (P.cap < n + 1) {
    if (P.w) {
      CUDA_TRY(cudaStreamSynchronize(h->s));  // no read in flight into the old words
      cudaFreeHost(P.w);
      P.w = nullptr;
      P.cap = 0;
    }
    const size_t cap = std::max<size_t>(1024, n + 1);
    void *p = nullptr;
    CUDA_TRY(cudaMallocHost(&p, sizeof(uint32_t) * cap));
    P.w = static_cast<uint32_t *>(p);
    P.cap = cap;
  }
  *out = P.w + 1;
  return AMR_OK;
}

// queue a read of n device words into the data words [at, at + n), within
// the room a pinned_words call made before the first read of the batch
static amr_status read_words(amr_mesh *h, size_t at, const void *src, size_t n) {
  if (!h->pin || !h->pin->w || at + n + 1 > h->pin->cap)
    return fail(AMR_ECUDA, "internal: read-back of %zu words beyond the page-locked room", at + n);
  uint32_t *w = h->pin->w + 1;
  CUDA_TRY(cudaMemcpyAsync(w + at, src, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, h->s));
  return AMR_OK;
}

// check_device with further page-locked reads queued before it: one
// synchronisation for the error word and the reads
static amr_status check_device_after_reads(amr_mesh *h, const char *where) {
  AMR_TRY(check_launches(h, where));
  uint32_t *w = nullptr;
  AMR_TRY(pinned_words(h, 0, &w));
  CUDA_TRY(cudaMemcpyAsync(w - 1, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  if (!w[-1]) return AMR_OK;
  return check_device(h, where);  // decodes (and clears) the error word
}

// ---------------------------------------------------------------------------
// scans and radix sort (host drivers of the index kernels)
// ---------------------------------------------------------------------------
static void scan_exclusive(amr_mesh *h, uint32_t *data, int64_t n, uint32_t *tmp) {
  const int64_t nb = (n + kScanItems - 1) / kScanItems;
  launch(h, K_SCAN, k_scan_block, dim3(unsigned(nb)), dim3(256), data, n, tmp);
  if (nb > 1 && nb <= kScanFlat) {
    launch(h, K_SCAN, k_scan_add_flat, dim3(unsigned(nb - 1)), dim3(256), data, n, (const uint32_t *)tmp);
  } else if (nb > 1) {
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
                       int64_t n, const std::vector<std::pair<int, int>> &digits,
                       uint32_t *table = nullptr, uint32_t *scan_tmp = nullptr) {
  if (n <= 0) return;
  if (!table) table = h->table;
  if (!scan_tmp) scan_tmp = h->scan_tmp;
  const int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
  uint64_t *ka = *k, *kb = k_alt;
  uint32_t *va = *v, *vb = v_alt;
  for (auto &dg : digits) {
    const int shift = dg.first, nbits = dg.second;
    launch(h, K_RADIX_HIST, k_radix_hist, dim3(unsigned(ntiles)), dim3(kRadixTile),
           (const uint64_t *)ka, n, shift, nbits, table, ntiles);
    scan_exclusive(h, table, (int64_t(1) << nbits) * ntiles, scan_tmp);
    launch(h, K_RADIX_SCATTER, k_radix_scatter, dim3(unsigned(ntiles)), dim3(kRadixTile),
           (const uint64_t *)ka, (const uint32_t *)va, kb, vb, n, shift, nbits,
           (const uint32_t *)table, ntiles);
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

static int bits_for(int64_t n) {  // bits to hold values 0..n-1
  int b = 0;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// segment lists
// ---------------------------------------------------------------------------
static int dom_size(const Seg &s, int dom) {
  switch (dom) {
    case DOM_CELLS: return 8 * (s.nl + s.ncl);
    case DOM_REAL: return 8 * s.nl;
    case DOM_GHOST5: return 5 * s.ncl;
    case DOM_BLOCKS: return s.nblk;
    case DOM_COMMIT: return ((s.flags & kSegReflux) ? 5 * s.ncl : 0) + 5 * s.nl;
    default:
      return ((s.flags & kSegReflux) ? 5 * s.ncl : 0) + ((s.flags & kSegRestrict) ? 5 * s.nl : 0);
  }
}

// append the (member, level) segments of `ml` (flags from `mode`: 0 = level
// step, 1 = restriction only) as one list
static SegList make_list(amr_mesh *h, const std::vector<std::pair<int, int>> &ml, int mode) {
  SegList L;
  L.seg0 = int(h->segs_h.size());
  int base = 0;
  for (auto &pr : ml) {
    const Member &m = h->mem[pr.first];
    const int l = pr.second;
    Seg s;
    s.member = pr.first;
    s.level = l;
    s.lo = int(m.oct_base + m.lo[l]);
    s.nl = int(m.lo[l + 1] - m.lo[l]);
    s.clo = int(m.cache_base + m.clo[l]);
    s.ncl = int(m.clo[l + 1] - m.clo[l]);
    s.base = base;
    s.blk0 = 0;
    s.nblk = 0;
    if (h->nsub > 0 && s.nl > 0 && !h->blk_first.empty()) {
      const size_t ml = size_t(pr.first) * (kMaxLev + 1) + size_t(l);
      s.blk0 = h->blk_first[ml];
      s.nblk = h->blk_last[ml] - s.blk0 + 1;
    }
    if (mode == 1)
      s.flags = l > m.lmin ? kSegRestrict : 0;
    else
      s.flags = (h->p.reflux && s.ncl ? kSegReflux : 0) | (l > m.lmin ? kSegRestrict : 0);
    if (s.nl == 0) continue;
    base += 8 * (s.nl + s.ncl);
    h->segs_h.push_back(s);
  }
  L.nseg = int(h->segs_h.size()) - L.seg0;
  L.ls = base;
  for (int d = 0; d < DOM_COUNT; ++d) {
    L.tpre0[d] = int(h->tpre_h.size());
    const int step = d == DOM_BLOCKS ? 1 : h->tile_size;  // one block of octs per tile
    int acc = 0;
    for (int q = 0; q < L.nseg; ++q) {
      h->tpre_h.push_back(acc);
      const int n = dom_size(h->segs_h[L.seg0 + q], d);
      acc += (n + step - 1) / step;
    }
    h->tpre_h.push_back(acc);
    L.ntile[d] = acc;
  }
  return L;
}

static void w_cycle(const Member &m, int l, std::vector<int> &out) {
  if (l + 1 <= kMaxLev && m.lo[l + 2] > m.lo[l + 1]) {
    w_cycle(m, l + 1, out);
    w_cycle(m, l + 1, out);
  }
  out.push_back(l);
}

static void build_lists(amr_mesh *h) {
  h->segs_h.clear();
  h->tpre_h.clear();
  h->phases.clear();
  size_t P = 0;
  for (auto &m : h->mem) {
    m.seq.clear();
    w_cycle(m, m.lmin, m.seq);
    P = std::max(P, m.seq.size());
  }
  // identical (member, level) sets share one list: a W-cycle repeats the
  // phases of its finer levels, and a level list equals its level's phase
  std::map<std::pair<std::vector<std::pair<int, int>>, int>, SegList> memo;
  auto list_of = [&](const std::vector<std::pair<int, int>> &ml, int mode) {
    auto key = std::make_pair(ml, mode);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    const SegList L = make_list(h, ml, mode);
    memo.emplace(std::move(key), L);
    return L;
  };
  for (size_t k = 0; k < P; ++k) {
    std::vector<std::pair<int, int>> ml;
    for (int q = 0; q < h->M; ++q)
      if (k < h->mem[q].seq.size()) ml.push_back({q, h->mem[q].seq[k]});
    h->phases.push_back(list_of(ml, 0));
  }
  for (int l = 0; l <= kMaxLev; ++l) {
    std::vector<std::pair<int, int>> ml;
    for (int q = 0; q < h->M; ++q) ml.push_back({q, l});
    h->level_list[l] = list_of(ml, 0);
    h->restrict_list[l] = list_of(ml, 1);
  }
  std::vector<std::pair<int, int>> all;
  for (int q = 0; q < h->M; ++q)
    for (int l = 0; l <= kMaxLev; ++l) all.push_back({q, l});
  h->cfl_list = make_list(h, all, 0);
  h->max_ls = 0;
  for (auto &L : h->phases) h->max_ls = std::max<int64_t>(h->max_ls, L.ls);
  for (int l = 0; l <= kMaxLev; ++l) h->max_ls = std::max<int64_t>(h->max_ls, h->level_list[l].ls);
}

// ---------------------------------------------------------------------------
// level-step launches
// ---------------------------------------------------------------------------
// the tiles of domain `dom` of list L in the launch arguments
template <class A>
static void set_tiles(amr_mesh *h, A &a, const SegList &L, int dom) {
  a.tpre = h->tpre + L.tpre0[dom];
  a.tseg0 = L.seg0;
  a.tnseg = L.nseg;
  a.tstep = dom == DOM_BLOCKS ? 1 : h->tile_size;
  a.ntiles = L.ntile[dom];
}

template <class T>
static StepArgs<T> step_args(amr_mesh *h, bool device_dt, double dt) {
  StepArgs<T> a{};
  a.N = int(h->N);
  a.NE = int(h->NE);
  a.NC = int(h->NC);
  a.LS = h->max_ls;
  a.S = h->S;
  a.CS = 24 * h->NC;
  a.U = static_cast<T *>(h->U);
  a.Rc = static_cast<T *>(h->Rc);
  a.rslot = h->rslot;
  a.fnb = h->fnb;
  a.nbr27 = h->nbr27;
  a.son = h->son;
  a.father = h->father;
  a.key = h->key;
  a.csrc = h->csrc;
  a.W = static_cast<T *>(h->W);
  a.Q = static_cast<T *>(h->Q);
  a.F = static_cast<T *>(h->F);
  a.C = static_cast<T *>(h->C);
  a.segs = h->segs;
  a.mgamma = static_cast<const T *>(h->mgamma_t);
  a.migm1 = static_cast<const T *>(h->migm1_t);
  a.msmallr = static_cast<const T *>(h->msmallr_t);
  a.msmallp = static_cast<const T *>(h->msmallp_t);
  a.dtdx_dev = device_dt ? h->dtdx_dev : nullptr;
  a.dtdxf_dev = device_dt ? h->dtdxf_dev : nullptr;
  a.dt_host = dt;
  a.mact = device_dt ? h->mact : nullptr;
  a.reflux = h->p.reflux;
  a.err = h->err;
  return a;
}

// persistent grid: enough blocks to fill the GPU once, never more than tiles
template <class T>
static void run_list(amr_mesh *h, int kid, void (*kern)(StepArgs<T>), StepArgs<T> a,
                     const SegList &L, int dom) {
  if (L.ntile[dom] == 0) return;
  set_tiles(h, a, L, dom);
  int grid = a.ntiles;
  if (h->persistent) {
    int per_sm = 0;
    for (auto &o : h->occ)
      if (o.first == (const void *)kern) per_sm = o.second;
    if (per_sm == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, h->tile_size, 0) != cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      h->occ.push_back({(const void *)kern, per_sm});
    }
    grid = std::min(a.ntiles, per_sm * h->sm_count);
  }
  launch(h, kid, kern, dim3(unsigned(grid)), dim3(unsigned(h->tile_size)), a);
}

// the fused kernel over the blocks of a list (dynamic shared memory)
template <class T, int NS>
static void run_rock_ns(amr_mesh *h, StepArgs<T> a, const SegList &L) {
  if (L.ntile[DOM_BLOCKS] == 0) return;
  set_tiles(h, a, L, DOM_BLOCKS);
  constexpr size_t smem = Rock<NS>::template smem<T>();
  auto kern = k_rock<T, NS>;
  int per_sm = 0;
  for (auto &o : h->occ)
    if (o.first == (const void *)kern) per_sm = o.second;
  if (per_sm == 0) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Rock<NS>::THREADS, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    h->occ.push_back({(const void *)kern, per_sm});
  }
  const int grid = h->persistent ? std::min(a.ntiles, per_sm * h->sm_count) : a.ntiles;
  launch_smem(h, K_ROCK, kern, dim3(unsigned(grid)), dim3(unsigned(Rock<NS>::THREADS)), smem, a,
              (const int32_t *)h->blk);
}

template <class T, int NS>
static void run_sweep_ns(amr_mesh *h, StepArgs<T> a, const SegList &L) {
  if (L.ntile[DOM_BLOCKS] == 0) return;
  set_tiles(h, a, L, DOM_BLOCKS);
  constexpr size_t smem = Sweep<NS>::template smem<T>();
  auto kern = k_sweep<T, NS>;
  int per_sm = 0;
  for (auto &o : h->occ)
    if (o.first == (const void *)kern) per_sm = o.second;
  if (per_sm == 0) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sweep<NS>::THREADS, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    h->occ.push_back({(const void *)kern, per_sm});
  }
  const int grid = h->persistent ? std::min(a.ntiles, per_sm * h->sm_count) : a.ntiles;
  launch_smem(h, K_SWEEP, kern, dim3(unsigned(grid)), dim3(unsigned(Sweep<NS>::THREADS)), smem, a,
              (const int32_t *)h->blk);
}

template <class T>
static void run_segments(amr_mesh *h, const SegList &L, bool device_dt, double dt) {
  if (L.nseg == 0) return;
  StepArgs<T> a = step_args<T>(h, device_dt, dt);
  run_list(h, K_PROLONG, k_prolong<T>, a, L, DOM_GHOST5);
  if (h->nsub > 0) {
    // the paper's fused kernels (cube staging or planar sweep): one block of
    // nsub^3 octs per CTA, then the new leaf states from the scratch into U
    if (h->planar) {
      if (h->nsub == 1)
        run_sweep_ns<T, 1>(h, a, L);
      else if (h->nsub == 2)
        run_sweep_ns<T, 2>(h, a, L);
      else
        run_sweep_ns<T, 4>(h, a, L);
    } else if (h->nsub == 1) {
      run_rock_ns<T, 1>(h, a, L);
    } else if (h->nsub == 2) {
      run_rock_ns<T, 2>(h, a, L);
    } else {
      run_rock_ns<T, 4>(h, a, L);
    }
    // new leaf states from the scratch into U, with reflux sums and restriction
    run_list(h, K_COMMIT, k_commit_post<T>, a, L, DOM_COMMIT);
    return;
  } else if constexpr (sizeof(T) == 4) {
    // FP32: primitives recomputed inside the predictor; each leaf cell solves
    // its six faces and updates itself
    run_list(h, K_PREDICT, k_predict_u<T>, a, L, DOM_CELLS);
    run_list(h, K_FLUX, k_flux_update<T>, a, L, DOM_REAL);
  } else {
    // FP64: every predictor and every face solve exactly once
    run_list(h, K_PRIM, k_prim<T>, a, L, DOM_CELLS);
    run_list(h, K_PREDICT, k_predict<T>, a, L, DOM_CELLS);
    run_list(h, K_FLUX, k_flux<T>, a, L, DOM_CELLS);
    run_list(h, K_UPDATE, k_update<T>, a, L, DOM_REAL);
  }
  run_list(h, K_RESTRICT, k_reflux_restrict<T>, a, L, DOM_POST);
}

static void step_segments(amr_mesh *h, const SegList &L, bool device_dt, double dt) {
  if (h->p.precision == 4)
    run_segments<float>(h, L, device_dt, dt);
  else
    run_segments<double>(h, L, device_dt, dt);
}

template <class T>
static void restrict_segments(amr_mesh *h, const SegList &L) {
  if (L.nseg == 0) return;
  run_list(h, K_RESTRICT, k_reflux_restrict<T>, step_args<T>(h, false, 0.0), L, DOM_POST);
}

static CflArgs cfl_args(amr_mesh *h) {
  CflArgs a{};
  a.segs = h->segs;
  set_tiles(h, a, h->cfl_list, DOM_REAL);
  a.S = h->S;
  a.son = h->son;
  a.mgamma = h->mgamma_d;
  a.msmallr = h->msmallr_d;
  a.msmallp = h->msmallp_d;
  a.mcfl = h->mcfl_d;
  a.mgamma_t = h->mgamma_t;
  a.msmallr_t = h->msmallr_t;
  a.msmallp_t = h->msmallp_t;
  a.mlmin = h->mlmin;
  a.nmembers = h->M;
  a.smax = h->smax;
  a.mrem = h->mrem;
  a.mact = h->mact;
  a.dt_dev = h->dt_dev;
  a.dtdx_dev = h->dtdx_dev;
  a.dtdxf_dev = h->dtdxf_dev;
  a.err = h->err;
  a.merr = h->merr;
  return a;
}

static void cfl_device(amr_mesh *h, int consume) {
  CflArgs a = cfl_args(h);
  a.consume = consume;
  const unsigned grid = unsigned(std::min(a.ntiles, 4 * h->sm_count));
  if (grid) {
    if (h->p.precision == 4)
      launch(h, K_CFL, k_cfl<float>, dim3(grid), dim3(unsigned(h->tile_size)), a, (const float *)h->U);
    else
      launch(h, K_CFL, k_cfl<double>, dim3(grid), dim3(unsigned(h->tile_size)), a, (const double *)h->U);
  }
  launch(h, K_DT, k_dt, dim3(nblocks(h->M, 128)), dim3(128), a);
}

// ---------------------------------------------------------------------------
// index build (create and re-index)
// ---------------------------------------------------------------------------
static amr_status build_index(amr_mesh *h, bool first) {
  const int64_t N = h->N;
  cudaMemsetAsync(h->hash.key, 0xFF, sizeof(uint64_t) * h->hcap, h->s);
  cudaMemsetAsync(h->hash.val, 0, sizeof(int32_t) * h->hcap, h->s);
  cudaMemsetAsync(h->son, 0, sizeof(uint32_t) * N, h->s);
  cudaMemsetAsync(h->counters, 0, sizeof(uint32_t) * 4, h->s);
  launch(h, K_HASH_INSERT, k_hash_insert, dim3(nblocks(N)), dim3(256), h->hash,
         (const uint64_t *)h->key, N, h->err);
  launch(h, K_FATHER_SON, k_father_son, dim3(nblocks(N)), dim3(256), h->hash,
         (const uint64_t *)h->key, N, (const int *)h->mlmin, h->father, h->son, h->err);
#ifdef AMR_CHECKED
  const bool check_grading = first;
#else
  const bool check_grading = first && !h->graded_by_construction;
#endif
  if (check_grading)
    launch(h, K_GRADING, k_grading, dim3(nblocks(8 * 27 * N)), dim3(256), h->hash,
           (const uint64_t *)h->key, N, (const int *)h->mlmin, h->err);
  launch(h, K_NEIGHBOURS, k_neighbours, dim3(nblocks(27 * N)), dim3(256), h->hash,
         (const uint64_t *)h->key, N, h->nbr27, h->claim, h->counters, h->claim_cap, h->err);
  if (first) {  // create: stop after the claims; the caller sizes the ghost buffers
    uint32_t *w = nullptr;
    AMR_TRY(pinned_words(h, 1, &w));
    AMR_TRY(read_words(h, 0, h->counters, 1));
    AMR_TRY(check_device_after_reads(h, "amr_create"));
    h->NC = w[0];
    return AMR_OK;
  }
  if (h->NC > 0) {
    launch(h, K_CLAIM, k_claim_to_comp, dim3(nblocks(h->NC)), dim3(256), (const uint64_t *)h->claim,
           h->NC, h->B, h->comp0, h->val0);
    uint64_t *k = h->comp0;
    uint32_t *v = h->val0;
    radix_sort(h, &k, &v, h->comp1, h->val1, h->NC, digits_for(0, 4 + 3 * h->B + bits_for(h->M)));
    launch(h, K_CACHE_FINALIZE, k_cache_finalize, dim3(nblocks(h->NC)), dim3(256), h->hash,
           (const uint64_t *)k, h->NC, h->B, N, h->ckey, (uint32_t *)nullptr, h->err);
    launch(h, K_NBR_FIX, k_neighbours_fix, dim3(nblocks(27 * N)), dim3(256), h->hash,
           (const uint64_t *)h->key, N, h->nbr27, h->err);
  }
  return AMR_OK;
}

static void build_faces_and_sources(amr_mesh *h) {
  launch(h, K_FACES, k_faces_real, dim3(nblocks(6 * h->N)), dim3(256), (const int32_t *)h->nbr27,
         h->N, h->NE, h->fnb);
  cudaMemsetAsync(h->rslot, 0xFF, sizeof(int32_t) * 8 * h->N, h->s);
  if (h->NC) {
    launch(h, K_FACES, k_faces_cache, dim3(nblocks(6 * h->NC)), dim3(256), h->hash,
           (const uint64_t *)h->ckey, h->NC, h->N, h->NE, h->fnb);
    launch(h, K_CACHE_SOURCES, k_cache_sources, dim3(nblocks(h->NC)), dim3(256), h->hash,
           (const uint64_t *)h->ckey, h->NC, h->N, (const int *)h->mlmin, h->csrc, h->rslot, h->err);
  }
}

static amr_status reindex(amr_mesh *h) {
  AMR_TRY(build_index(h, false));
  build_faces_and_sources(h);
  if (h->max_cs) cudaMemsetAsync(h->C, 0, h->elem() * 5 * size_t(h->max_cs), h->s);
  return AMR_OK;
}

// ---------------------------------------------------------------------------
// create / destroy
// ---------------------------------------------------------------------------
extern "C" void amr_params_default(amr_params *p) {
  std::memset(p, 0, sizeof *p);
  p->tile = 0;
  p->schedule = -1;
  p->levelmin = 1;
  p->levelmax = 1;
  p->gamma = 1.4;
  p->cfl = 0.8;
  p->smallr = 1e-10;
  p->smallc = 1e-10;
  p->precision = 8;
  p->reflux = 1;
  p->reindex_every_step = 0;
  p->use_graphs = 1;
  p->regrid_expand = 1;
  p->regrid_every_step = 0;
  p->nsubgrid = -1;
  p->planar = -1;
}

static void destroy_all(amr_mesh *h) {
  if (!h) return;
  if (h->cs) cudaStreamSynchronize(h->cs);
  if (h->cs_out) cudaStreamSynchronize(h->cs_out);
  if (h->s) cudaStreamSynchronize(h->s);
  for (cudaEvent_t e : {h->ev_in_ready, h->ev_in_free, h->ev_out_ready, h->ev_out_free})
    if (e) cudaEventDestroy(e);
  if (h->cs) cudaStreamDestroy(h->cs);
  if (h->cs_out) cudaStreamDestroy(h->cs_out);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (auto &t : h->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  const bool last = h->cache && h->cache.use_count() == 1;
  if (last) h->cache->cap = 0;
  while (!h->bufs.empty()) dev_free(h, h->bufs.back().p);
  if (last) {
    for (const DevBuf &b : h->cache->v) real_free(h, b.p, b.bytes);
    h->cache->v.clear();
    h->cache->bytes = 0;
  }
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->own_stream && h->s) cudaStreamDestroy(h->s);
  delete h;
}

template <class T>
static amr_status upload_member_params(amr_mesh *h) {
  std::vector<T> g(h->M), igm1(h->M), sr(h->M), sp(h->M);
  for (int q = 0; q < h->M; ++q) {
    const Member &m = h->mem[q];
    g[q] = T(m.gamma);
    igm1[q] = T(1.0 / (m.gamma - 1.0));
    sr[q] = T(m.smallr);
    sp[q] = T(m.smallc * m.smallc / m.gamma);
  }
  T *a, *b, *c, *d;
  AMR_TRY(upload(h, &a, g));
  AMR_TRY(upload(h, &b, igm1));
  AMR_TRY(upload(h, &c, sr));
  AMR_TRY(upload(h, &d, sp));
  h->mgamma_t = a;
  h->migm1_t = b;
  h->msmallr_t = c;
  h->msmallp_t = d;
  return AMR_OK;
}

// level-step scratch for max_ls / max_cs: kept when the buffers a regrid
// handed over are large enough, else (re)allocated
static amr_status ensure_scratch(amr_mesh *h) {
  const size_t es = h->elem();
  const int64_t ls = std::max<int64_t>(h->max_ls, 1), cs = std::max<int64_t>(h->max_cs, 1);
  if (!h->W || !h->Q || !h->F || h->ls_cap < ls) {
    dev_free(h, h->W);
    dev_free(h, h->Q);
    dev_free(h, h->F);
    h->W = h->Q = h->F = nullptr;
    h->ls_cap = 0;
    AMR_TRY(dev_alloc(h, &h->W, es * 5 * size_t(ls)));
    AMR_TRY(dev_alloc(h, &h->Q, es * 20 * size_t(ls)));
    AMR_TRY(dev_alloc(h, &h->F, es * 15 * size_t(ls)));
    h->ls_cap = ls;
  }
  if (!h->C || h->cs_cap < cs) {
    dev_free(h, h->C);
    h->C = nullptr;
    h->cs_cap = 0;
    AMR_TRY(dev_alloc(h, &h->C, es * 5 * size_t(cs)));
    h->cs_cap = cs;
  }
  return AMR_OK;
}

// member parameters on the device (from h->mem)
static amr_status upload_members(amr_mesh *h) {
  const int M = h->M;
  std::vector<int> lmin(M), lmax(M);
  std::vector<double> g(M), cfl(M), sr(M), sp(M);
  for (int q = 0; q < M; ++q) {
    const Member &m = h->mem[q];
    lmin[q] = m.lmin;
    lmax[q] = m.lmax;
    g[q] = m.gamma;
    cfl[q] = m.cfl;
    sr[q] = m.smallr;
    sp[q] = m.smallc * m.smallc / m.gamma;
  }
  AMR_TRY(upload(h, &h->mlmin, lmin));
  AMR_TRY(upload(h, &h->mlmax, lmax));
  AMR_TRY(upload(h, &h->mgamma_d, g));
  AMR_TRY(upload(h, &h->mcfl_d, cfl));
  AMR_TRY(upload(h, &h->msmallr_d, sr));
  AMR_TRY(upload(h, &h->msmallp_d, sp));
  std::vector<float> f32(3 * size_t(M));
  for (int q = 0; q < M; ++q) {
    f32[3 * size_t(q)] = float(g[q] - 1.0);
    f32[3 * size_t(q) + 1] = float(sr[q]);
    f32[3 * size_t(q) + 2] = float(sp[q]);
  }
  AMR_TRY(upload(h, &h->mflag32, f32));
  if (h->p.precision == 4) return upload_member_params<float>(h);
  return upload_member_params<double>(h);
}

// a regrid's new mesh nh reads h's member arrays (levels, parameters: fixed
// for a member's life) as they are; h still owns them
static void share_members(amr_mesh *nh, const amr_mesh *h) {
  nh->mlmin = h->mlmin;
  nh->mlmax = h->mlmax;
  nh->mgamma_d = h->mgamma_d;
  nh->mcfl_d = h->mcfl_d;
  nh->msmallr_d = h->msmallr_d;
  nh->msmallp_d = h->msmallp_d;
  nh->mflag32 = h->mflag32;
  nh->mgamma_t = h->mgamma_t;
  nh->migm1_t = h->migm1_t;
  nh->msmallr_t = h->msmallr_t;
  nh->msmallp_t = h->msmallp_t;
}

// after the swap: the new mesh h takes the member arrays over from the old
// mesh old, which then no longer frees them
static void own_members(amr_mesh *h, amr_mesh *old) {
  const void *arrays[] = {h->mlmin,     h->mlmax,   h->mgamma_d, h->mcfl_d,    h->msmallr_d, h->msmallp_d,
                          h->mflag32,   h->mgamma_t, h->migm1_t, h->msmallr_t, h->msmallp_t};
  for (const void *a : arrays) move_buf(h, old, const_cast<void *>(a));
}

static amr_status build_blocks(amr_mesh *h);

// a regrid's state source: the old mesh's state (the handle's precision,
// variable stride S) and, per entry of the new oct list, the old oct it keeps
// (~0 for a new oct); pos is the emit pass's scanned counts over the n_old
// old octs (the new octs of old oct o at [pos[n_old + o], pos[n_old + o + 1]))
struct StateSource {
  const void *U = nullptr;
  int64_t S = 0;
  uint32_t *src = nullptr;
  const uint32_t *pos = nullptr;
  int64_t n_old = 0;
};
static amr_status build_mesh(amr_mesh *h, int64_t n, bool have_hk, uint8_t *d_lvl, uint16_t *d_mem,
                             uint32_t *d_i, uint32_t *d_j, uint32_t *d_k, uint64_t *d_hk,
                             double *d_U, uint8_t *d_new, int64_t sorted_prefix = 0,
                             const StateSource *from = nullptr);

static amr_status create_impl(amr_mesh *h, const amr_member *members) {
  const int M = h->M;
  // --- members and host staging of the concatenated oct list ------------------
  int64_t n = 0;
  int have_hk = 0;
  for (int q = 0; q < M; ++q) {
    const amr_member &a = members[q];
    Member &m = h->mem[q];
    m.lmin = a.levelmin;
    m.lmax = a.levelmax;
    m.gamma = a.gamma;
    m.cfl = a.cfl;
    m.smallr = a.smallr;
    m.smallc = a.smallc;
    m.n_oct = a.n_oct;
    n += a.n_oct;
    have_hk += a.hilbert_key != nullptr;
    h->lmax_all = std::max(h->lmax_all, a.levelmax);
  }
  if (have_hk != 0 && have_hk != M)
    return fail(AMR_EINVAL, "amr_create: give sort keys for every member or for none");
  if (n > (int64_t(1) << 26)) return fail(AMR_EINVAL, "amr_create: more than 2^26 octs in total");
  std::vector<uint8_t> lv(n);
  std::vector<uint32_t> ci(n), cj(n), ck(n);
  std::vector<uint16_t> mm(n);
  std::vector<uint64_t> hk(have_hk ? n : 0);
  std::vector<double> U(40 * size_t(n));
  {
    int64_t off = 0;
    for (int q = 0; q < M; ++q) {
      const amr_member &a = members[q];
      const int64_t nm = a.n_oct;
      std::memcpy(lv.data() + off, a.level, nm);
      std::memcpy(ci.data() + off, a.i, 4 * nm);
      std::memcpy(cj.data() + off, a.j, 4 * nm);
      std::memcpy(ck.data() + off, a.k, 4 * nm);
      for (int64_t t = 0; t < nm; ++t) mm[off + t] = uint16_t(q);
      if (have_hk) std::memcpy(hk.data() + off, a.hilbert_key, 8 * nm);
      for (int v = 0; v < 5; ++v)
        std::memcpy(U.data() + v * 8 * n + 8 * off, a.U + v * 8 * nm, sizeof(double) * 8 * nm);
      off += nm;
    }
  }
  h->N = n;
  AMR_TRY(upload_members(h));
  // --- inputs to the device ------------------------------------------------------
  uint8_t *d_lvl;
  uint16_t *d_mem;
  uint32_t *d_i, *d_j, *d_k;
  uint64_t *d_hk = nullptr;
  double *d_U;
  AMR_TRY(upload(h, &d_lvl, lv));
  AMR_TRY(upload(h, &d_mem, mm));
  AMR_TRY(upload(h, &d_i, ci));
  AMR_TRY(upload(h, &d_j, cj));
  AMR_TRY(upload(h, &d_k, ck));
  AMR_TRY(upload(h, &d_U, U));
  if (have_hk) AMR_TRY(upload(h, &d_hk, hk));
  return build_mesh(h, n, have_hk != 0, d_lvl, d_mem, d_i, d_j, d_k, d_hk, d_U, nullptr);
}

static void mgl_free(amr_mesh *h);

// The mesh from device-resident inputs in any order (create and regrid):
// order, hash, index, ghost cache, state, lists, scratch; the state comes
// from d_U (FP64, variable stride 8 n) or, in a regrid, from the old mesh
// (from); d_new marks octs whose state is to be prolonged from their father
// (regrid), before the restriction.  Frees the inputs.
static amr_status build_mesh(amr_mesh *h, int64_t n, bool have_hk, uint8_t *d_lvl, uint16_t *d_mem,
                             uint32_t *d_i, uint32_t *d_j, uint32_t *d_k, uint64_t *d_hk,
                             double *d_U, uint8_t *d_new, int64_t sorted_prefix,
                             const StateSource *from) {
  const amr_params &p = h->p;
  const int M = h->M;
  // a new set of octs: the refined-level potential and its tables go
  mgl_free(h);
  dev_free(h, h->phil);
  h->phil = nullptr;
  h->phil_n = 0;
  h->N = n;
  uint32_t *perm, *perm_alt;
  uint64_t *comp, *comp_alt;
  AMR_TRY(alloc_n(h, &perm, n));
  AMR_TRY(alloc_n(h, &perm_alt, n));
  AMR_TRY(alloc_n(h, &comp, n));
  AMR_TRY(alloc_n(h, &comp_alt, n));
  AMR_TRY(alloc_n(h, &h->err, 1));
  CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));

  // --- order: Hilbert digits (LSD), the level bucket pass with prefix sums,
  //     then the member digits ----------------------------------------------------
  h->table_cap = 256 * ((n + kRadixTile - 1) / kRadixTile) + 256;
  h->scan_cap = scan_tmp_size(h->table_cap);
  AMR_TRY(alloc_n(h, &h->table, h->table_cap));
  AMR_TRY(alloc_n(h, &h->scan_tmp, h->scan_cap));
  launch(h, K_SORT_KEYS, k_make_sort_keys, dim3(nblocks(n)), dim3(256), (const uint8_t *)d_lvl,
         (const uint32_t *)d_i, (const uint32_t *)d_j, (const uint32_t *)d_k,
         (const uint16_t *)d_mem, (const uint64_t *)d_hk, n, (const int *)h->mlmin,
         (const int *)h->mlmax, comp, perm, h->err);
  // a caller's oct list is validated before it is sorted; a regrid's (d_new
  // set) comes from a checked mesh and is checked with the rest below
  if (!d_new) AMR_TRY(check_device(h, "amr_create"));
  const int hbits = have_hk ? kHilbertBits : 3 * (h->lmax_all - 1);
  std::vector<std::pair<int, int>> digits = digits_for(0, hbits);
  digits.push_back({kHilbertBits, 4});  // level bucket sort
  for (auto &d : digits_for(kHilbertBits + 4, bits_for(M))) digits.push_back(d);
  uint64_t *kk = comp;
  uint32_t *vv = perm;
  const int64_t n_new = n - sorted_prefix;
  if (sorted_prefix > 0 && n_new >= 0 && from && from->pos) {
    // a regrid: the kept octs [0, sorted_prefix) are in order, the new ones
    // are once each father's group is sorted; then the two runs merge by rank
    if (n_new > 0) {
      launch(h, K_SORT_GROUPS, k_sort_groups, dim3(nblocks(from->n_old)), dim3(256), from->pos, from->n_old,
             comp, perm);
      launch(h, K_MERGE, k_merge_rank, dim3(nblocks(sorted_prefix)), dim3(256), (const uint64_t *)comp,
             (const uint32_t *)perm, sorted_prefix, (const uint64_t *)(comp + sorted_prefix), n_new, comp_alt,
             perm_alt);
      launch(h, K_MERGE, k_merge_rank, dim3(nblocks(n_new)), dim3(256),
             (const uint64_t *)(comp + sorted_prefix), (const uint32_t *)(perm + sorted_prefix), n_new,
             (const uint64_t *)comp, sorted_prefix, comp_alt, perm_alt);
      kk = comp_alt;
      vv = perm_alt;
    }
  } else {
    radix_sort(h, &kk, &vv, comp_alt, perm_alt, n, digits);
  }
  h->order_computed = !have_hk;

  // --- keys in mesh order, (member, level) offsets ----------------------------------
  AMR_TRY(alloc_n(h, &h->key, n));
  AMR_TRY(alloc_n(h, &h->counters, 4));
  AMR_TRY(alloc_n(h, &h->seg_count, 16 * int64_t(M)));
  CUDA_TRY(cudaMemsetAsync(h->seg_count, 0, sizeof(uint32_t) * 16 * M, h->s));
  launch(h, K_GATHER, k_gather_octs, dim3(nblocks(n)), dim3(256), (const uint32_t *)vv,
         (const uint8_t *)d_lvl, (const uint32_t *)d_i, (const uint32_t *)d_j,
         (const uint32_t *)d_k, (const uint16_t *)d_mem, n, h->key, h->seg_count);
  std::vector<uint32_t> counts(16 * size_t(M));
  {
    uint32_t *w = nullptr;
    AMR_TRY(pinned_words(h, counts.size(), &w));
    AMR_TRY(read_words(h, 0, h->seg_count, counts.size()));
    AMR_TRY(check_device_after_reads(h, "amr_create"));
    std::memcpy(counts.data(), w, 4 * counts.size());
  }
  {
    int64_t base = 0;
    for (int q = 0; q < M; ++q) {
      Member &m = h->mem[q];
      m.oct_base = base;
      int64_t acc = 0;
      for (int l = 0; l <= kMaxLev; ++l) {
        m.lo[l] = acc;
        acc += counts[16 * q + l];
      }
      m.lo[kMaxLev + 1] = acc;
      base += acc;
      const int64_t side = int64_t(1) << (m.lmin - 1);
      if (int64_t(counts[16 * q + m.lmin]) != side * side * side)
        return fail(AMR_EGRADING, "amr_create: member %d level %d holds %u octs, a complete base needs %lld",
                    q, m.lmin, counts[16 * q + m.lmin], (long long)(side * side * side));
    }
  }

  // --- hash table, father/son, grading, neighbours, ghost cache ---------------------
  h->B = std::max(1, h->lmax_all - 1);
  h->claim_cap = 4 * n + 1024;
  uint64_t cap = 1024;
  while (cap < uint64_t(4 * n)) cap <<= 1;
  AMR_TRY(alloc_n(h, &h->son, n));
  AMR_TRY(alloc_n(h, &h->father, n));
  AMR_TRY(alloc_n(h, &h->nbr27, 27 * n));
  AMR_TRY(alloc_n(h, &h->claim, h->claim_cap));
  for (int attempt = 0; attempt < 3; ++attempt) {
    h->hcap = cap;
    AMR_TRY(alloc_n(h, &h->hash.key, cap));
    AMR_TRY(alloc_n(h, &h->hash.val, cap));
    h->hash.mask = cap - 1;
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
  CUDA_TRY(cudaMemsetAsync(h->seg_count, 0, sizeof(uint32_t) * 16 * M, h->s));
  if (NC > 0) {
    launch(h, K_CLAIM, k_claim_to_comp, dim3(nblocks(NC)), dim3(256), (const uint64_t *)h->claim,
           NC, h->B, h->comp0, h->val0);
    uint64_t *ckk = h->comp0;
    uint32_t *cvv = h->val0;
    radix_sort(h, &ckk, &cvv, h->comp1, h->val1, NC, digits_for(0, 4 + 3 * h->B + bits_for(M)));
    launch(h, K_CACHE_FINALIZE, k_cache_finalize, dim3(nblocks(NC)), dim3(256), h->hash,
           (const uint64_t *)ckk, NC, h->B, n, h->ckey, h->seg_count, h->err);
    launch(h, K_NBR_FIX, k_neighbours_fix, dim3(nblocks(27 * n)), dim3(256), h->hash,
           (const uint64_t *)h->key, n, h->nbr27, h->err);
  }
  {
    uint32_t *w = nullptr;
    AMR_TRY(pinned_words(h, counts.size(), &w));
    AMR_TRY(read_words(h, 0, h->seg_count, counts.size()));
    AMR_TRY(check_device_after_reads(h, "amr_create"));
    std::memcpy(counts.data(), w, 4 * counts.size());
  }
  {
    int64_t base = 0;
    for (int q = 0; q < M; ++q) {
      Member &m = h->mem[q];
      m.cache_base = base;
      int64_t acc = 0;
      for (int l = 0; l <= kMaxLev; ++l) {
        m.clo[l] = acc;
        acc += counts[16 * q + l];
      }
      m.clo[kMaxLev + 1] = acc;
      base += acc;
    }
  }
  // cell indices of real and ghost octs are 32-bit in the kernels and tables
  if (8 * (n + NC) > int64_t(INT32_MAX))
    return fail(AMR_EINVAL, "amr_create: %lld real + %lld ghost octs exceed 2^31 cells",
                (long long)n, (long long)NC);
  h->NE = n + NC;
  h->S = 8 * h->NE;
  AMR_TRY(alloc_n(h, &h->fnb, 6 * h->NE));
  AMR_TRY(alloc_n(h, &h->csrc, 7 * (NC > 0 ? NC : 1)));
  AMR_TRY(alloc_n(h, &h->rslot, 8 * n));
  build_faces_and_sources(h);
  // a caller's mesh is checked here; a regrid's, graded by construction, with
  // its states below
  AMR_TRY(d_new ? check_launches(h, "amr_create") : check_device(h, "amr_create"));

  // --- state in mesh order ---------------------------------------------------------
  const size_t es = h->elem();
  AMR_TRY(dev_alloc(h, &h->U, es * 5 * size_t(h->S)));
  AMR_TRY(dev_alloc(h, &h->Rc, es * 5 * size_t(NC > 0 ? NC : 1)));
  CUDA_TRY(cudaMemsetAsync(h->U, 0, es * 5 * size_t(h->S), h->s));
  CUDA_TRY(cudaMemsetAsync(h->Rc, 0, es * 5 * size_t(NC > 0 ? NC : 1), h->s));
  const unsigned gc = nblocks(8 * n);
  const uint32_t *srcp = from ? (const uint32_t *)from->src : nullptr;
  if (p.precision == 4) {
    if (from)
      launch(h, K_GATHER, k_gather_cells<float, float>, dim3(gc), dim3(256), (const uint32_t *)vv, srcp,
             (const float *)from->U, from->S, n, (float *)h->U, h->S);
    else
      launch(h, K_GATHER, k_gather_cells<double, float>, dim3(gc), dim3(256), (const uint32_t *)vv, srcp,
             (const double *)d_U, 8 * n, n, (float *)h->U, h->S);
  } else {
    launch(h, K_GATHER, k_gather_cells<double, double>, dim3(gc), dim3(256), (const uint32_t *)vv, srcp,
           from ? (const double *)from->U : (const double *)d_U, from ? from->S : 8 * n, n, (double *)h->U,
           h->S);
  }

  // leaf counts: each oct above a member's levelmin splits one cell below
  for (auto &m : h->mem) {
    for (int l = 0; l <= kMaxLev; ++l) m.leaf[l] = 8 * (m.lo[l + 1] - m.lo[l]);
    for (int l = m.lmin + 1; l <= kMaxLev; ++l) m.leaf[l - 1] -= m.lo[l + 1] - m.lo[l];
  }

  // --- work lists, scratch, time-step arrays ------------------------------------------
  if (h->nsub > 0) AMR_TRY(build_blocks(h));
  build_lists(h);
  AMR_TRY(upload(h, &h->segs, h->segs_h));
  AMR_TRY(upload(h, &h->tpre, h->tpre_h));
  h->max_cs = 24 * NC;
  AMR_TRY(ensure_scratch(h));
  if (h->max_cs) CUDA_TRY(cudaMemsetAsync(h->C, 0, es * 5 * size_t(h->max_cs), h->s));
  AMR_TRY(alloc_n(h, &h->dt_dev, M));
  AMR_TRY(alloc_n(h, &h->dtdx_dev, M));
  AMR_TRY(alloc_n(h, &h->dtdxf_dev, M));
  AMR_TRY(alloc_n(h, &h->smax, 16 * int64_t(M)));
  CUDA_TRY(cudaMemsetAsync(h->smax, 0, sizeof(unsigned long long) * 16 * M, h->s));
  AMR_TRY(alloc_n(h, &h->mrem, M));
  AMR_TRY(alloc_n(h, &h->mact, M));
  AMR_TRY(alloc_n(h, &h->merr, M));
  CUDA_TRY(cudaMemsetAsync(h->merr, 0, sizeof(int) * M, h->s));
  CUDA_TRY(cudaMemsetAsync(h->mrem, 0xFF, sizeof(int) * M, h->s));  // -1: unlimited
  CUDA_TRY(cudaMemsetAsync(h->mact, 0, sizeof(int) * M, h->s));

  // regrid: new octs take the prolongation of their father, coarsest first
  if (d_new) {
    uint8_t *isnew = nullptr;
    AMR_TRY(alloc_n(h, &isnew, n));
    launch(h, K_REGRID, k_gather_u8, dim3(nblocks(n)), dim3(256), (const uint32_t *)vv,
           (const uint8_t *)d_new, n, isnew);
    for (auto &m : h->mem)
      for (int l = m.lmin + 1; l <= m.lmax; ++l) {
        const int lo = int(m.oct_base + m.lo[l]), hi = int(m.oct_base + m.lo[l + 1]);
        if (hi <= lo) continue;
        if (p.precision == 4)
          launch(h, K_PROLONG_NEW, k_prolong_new<float>, dim3(nblocks(5 * int64_t(hi - lo))), dim3(256), int(n),
                 int(h->NE), h->S, (const uint64_t *)h->key, (const int32_t *)h->father,
                 (const int32_t *)h->fnb, (const uint8_t *)isnew, (float *)h->U, lo, hi, h->err);
        else
          launch(h, K_PROLONG_NEW, k_prolong_new<double>, dim3(nblocks(5 * int64_t(hi - lo))), dim3(256), int(n),
                 int(h->NE), h->S, (const uint64_t *)h->key, (const int32_t *)h->father,
                 (const int32_t *)h->fnb, (const uint8_t *)isnew, (double *)h->U, lo, hi, h->err);
      }
    dev_free(h, isnew);
    dev_free(h, d_new);
  }

  // split cells carry the mean of their children, finest level first
  for (int l = kMaxLev; l >= 1; --l) {
    if (p.precision == 4)
      restrict_segments<float>(h, h->restrict_list[l]);
    else
      restrict_segments<double>(h, h->restrict_list[l]);
  }
  AMR_TRY(check_device(h, "amr_create"));
  // release the input staging
  dev_free(h, d_lvl);
  dev_free(h, d_mem);
  dev_free(h, d_i);
  dev_free(h, d_j);
  dev_free(h, d_k);
  dev_free(h, d_U);
  if (from) dev_free(h, from->src);
  if (d_hk) dev_free(h, d_hk);
  dev_free(h, perm);
  dev_free(h, perm_alt);
  dev_free(h, comp);
  dev_free(h, comp_alt);
  return AMR_OK;  // the frees are stream-ordered
}

static amr_status check_member(const amr_member &a, int q) {
  if (!a.level || !a.i || !a.j || !a.k || !a.U)
    return fail(AMR_EINVAL, "amr_create: member %d has a NULL array", q);
  if (a.levelmin < 1 || a.levelmax > kMaxLev || a.levelmin > a.levelmax)
    return fail(AMR_EINVAL, "amr_create: levels must satisfy 1 <= levelmin <= levelmax <= %d", kMaxLev);
  if (!(a.gamma > 1.0) || !(a.cfl > 0.0) || !(a.smallr > 0.0) || !(a.smallc > 0.0))
    return fail(AMR_EINVAL, "amr_create: gamma > 1, cfl > 0, smallr > 0, smallc > 0 required");
  if (a.n_oct < 1) return fail(AMR_EINVAL, "amr_create: member %d has no octs", q);
  return AMR_OK;
}

extern "C" amr_status amr_create_batch(const amr_params *p, int n_members,
                                       const amr_member *members, amr_handle *out) {
  g_last_error.clear();
  if (!out) return fail(AMR_EINVAL, "amr_create: out is NULL");
  *out = nullptr;
  if (!p || !members) return fail(AMR_EINVAL, "amr_create: NULL argument");
  if (n_members < 1 || n_members > kMaxMembers)
    return fail(AMR_EINVAL, "amr_create_batch: n_members must be in [1, %d]", kMaxMembers);
  if (p->precision != 4 && p->precision != 8)
    return fail(AMR_EINVAL, "amr_create: precision must be 4 or 8");
  for (int q = 0; q < n_members; ++q) AMR_TRY(check_member(members[q], q));
  {
    int64_t total = 0;
    for (int q = 0; q < n_members; ++q) total += members[q].n_oct;
    if (total > (int64_t(1) << 26)) return fail(AMR_EINVAL, "amr_create: more than 2^26 octs in total");
  }
  amr_mesh *h = new amr_mesh();
  h->p = *p;
  h->M = n_members;
  if (!p->hbm_budget_bytes) h->cache = std::make_shared<BufCache>();
  h->mem.resize(n_members);
  if (p->tile != 0 && p->tile != 64 && p->tile != 128 && p->tile != 256 && p->tile != 512) {
    delete h;
    return fail(AMR_EINVAL, "amr_create: tile must be 0, 64, 128, 256 or 512");
  }
  if (!(p->nsubgrid >= -1 && p->nsubgrid <= 2) && p->nsubgrid != 4) {
    delete h;
    return fail(AMR_EINVAL, "amr_create: nsubgrid must be -1, 0, 1, 2 or 4");
  }
  if (p->planar < -1 || p->planar > 1) {
    delete h;
    return fail(AMR_EINVAL, "amr_create: planar must be -1, 0 or 1");
  }
  h->tile_size = p->tile ? p->tile : 256;
  h->persistent = p->schedule != 0;
  h->nsub = p->nsubgrid > 0 ? p->nsubgrid : 0;
  h->planar = h->nsub > 0 && p->planar == 1;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (h->sm_count < 1) h->sm_count = 1;
  if (p->stream) {
    h->s = static_cast<cudaStream_t>(p->stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return fail(AMR_ECUDA, "amr_create: cannot create a stream");
    }
    h->own_stream = true;
  }
  amr_status s = create_impl(h, members);
  if (s != AMR_OK) {
    std::string msg = g_last_error;
    destroy_all(h);
    g_last_error = msg;
    return s;
  }
  *out = h;
  return AMR_OK;
}

extern "C" amr_status amr_create(const amr_params *p, int64_t n_oct, const uint8_t *level,
                                 const uint32_t *i, const uint32_t *j, const uint32_t *k,
                                 const uint64_t *hilbert_key, const double *U, amr_handle *out) {
  g_last_error.clear();
  if (!out) return fail(AMR_EINVAL, "amr_create: out is NULL");
  *out = nullptr;
  if (!p || !level || !i || !j || !k || !U) return fail(AMR_EINVAL, "amr_create: NULL argument");
  if (n_oct < 1 || n_oct > (int64_t(1) << 26))
    return fail(AMR_EINVAL, "amr_create: n_oct must be in [1, 2^26]");
  amr_member m{};
  m.levelmin = p->levelmin;
  m.levelmax = p->levelmax;
  m.gamma = p->gamma;
  m.cfl = p->cfl;
  m.smallr = p->smallr;
  m.smallc = p->smallc;
  m.n_oct = n_oct;
  m.level = level;
  m.i = i;
  m.j = j;
  m.k = k;
  m.hilbert_key = hilbert_key;
  m.U = U;
  return amr_create_batch(p, 1, &m, out);
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
  cfl_device(h, 0);
  CUDA_TRY(cudaMemcpyAsync(dt_out, h->dt_dev + h->sel, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  return check_device(h, "amr_cfl_dt");
}

extern "C" amr_status amr_member_dt(amr_handle h, double *dt_out, int n) {
  if (!h || !dt_out) return fail(AMR_EINVAL, "amr_member_dt: NULL argument");
  if (n < h->M) return fail(AMR_EINVAL, "amr_member_dt: room for %d members needed", h->M);
  CUDA_TRY(cudaMemcpyAsync(dt_out, h->dt_dev, sizeof(double) * h->M, cudaMemcpyDeviceToHost, h->s));
  return check_device(h, "amr_member_dt");
}

extern "C" amr_status amr_step_level(amr_handle h, int level, double dt) {
  if (!h) return fail(AMR_EINVAL, "amr_step_level: NULL handle");
  if (level < 1 || level > h->lmax_all)
    return fail(AMR_EINVAL, "amr_step_level: level %d outside [1, %d]", level, h->lmax_all);
  if (!(dt > 0.0)) return fail(AMR_EINVAL, "amr_step_level: dt must be > 0");
  step_segments(h, h->level_list[level], false, dt);
  if (h->launch_err != cudaSuccess) return check_device(h, "amr_step_level");
  return AMR_OK;
}

static void coarse_step(amr_mesh *h) {
  if (h->p.reindex_every_step) reindex(h);
  cfl_device(h, 1);
  for (auto &L : h->phases) step_segments(h, L, true, 0.0);
}

static void coarse_step(amr_mesh *h);

// Blocks of the fused kernel: runs of real octs (mesh order) of one (member,
// level) whose coordinates lie in one aligned group of nsub^3 oct positions.
// The level's Hilbert order visits every aligned group in one run; with
// caller-given sort keys a group may come in several runs, which then form
// several blocks (each updates only its own octs).
static amr_status build_blocks(amr_mesh *h) {
  const int64_t N = h->N;
  const unsigned sh = h->nsub == 4 ? 2u : h->nsub == 2 ? 1u : 0u;
  dev_free(h, h->blk);
  h->blk = nullptr;
  AMR_TRY(alloc_n(h, &h->blk, N + 1));
  h->blk_first.assign(size_t(h->M) * (kMaxLev + 1), 0);
  h->blk_last.assign(size_t(h->M) * (kMaxLev + 1), 0);
  if (N == 0) return AMR_OK;
  // block heads (a new (member, level) or aligned group), their exclusive
  // prefix sum = block of every oct, and the blocks' first octs
  uint32_t *head = nullptr, *pos = nullptr, *tmp = nullptr;
  int32_t *ask = nullptr, *got = nullptr;
  std::vector<int32_t> at;  // first and last oct of every (member, level)
  for (int q = 0; q < h->M; ++q)
    for (int l = 0; l <= kMaxLev; ++l) {
      const Member &m = h->mem[q];
      const int64_t lo = m.oct_base + m.lo[l], nl = m.lo[l + 1] - m.lo[l];
      at.push_back(int32_t(nl > 0 ? lo : 0));
      at.push_back(int32_t(nl > 0 ? lo + nl - 1 : 0));
    }
  amr_status st = AMR_OK;
  if ((st = alloc_n(h, &head, N)) == AMR_OK && (st = alloc_n(h, &pos, N)) == AMR_OK &&
      (st = alloc_n(h, &tmp, scan_tmp_size(N))) == AMR_OK && (st = upload(h, &ask, at)) == AMR_OK &&
      (st = alloc_n(h, &got, int64_t(at.size()))) == AMR_OK) {
    launch(h, K_GATHER, k_block_heads, dim3(nblocks(N)), dim3(256), (const uint64_t *)h->key, N, sh, head);
    CUDA_TRY(cudaMemcpyAsync(pos, head, 4 * size_t(N), cudaMemcpyDeviceToDevice, h->s));
    scan_exclusive(h, pos, N, tmp);
    launch(h, K_GATHER, k_block_starts, dim3(nblocks(N)), dim3(256), (const uint32_t *)head,
           (const uint32_t *)pos, N, h->blk);
    launch(h, K_GATHER, k_block_of, dim3(nblocks(int64_t(at.size()))), dim3(256), (const uint32_t *)head,
           (const uint32_t *)pos, (const int32_t *)ask, int64_t(at.size()), got);
    std::vector<int32_t> blk_at(at.size());
    cudaError_t e = cudaMemcpyAsync(blk_at.data(), got, 4 * at.size(), cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = fail(AMR_ECUDA, "block list: %s", cudaGetErrorString(e));
    for (size_t t = 0; 2 * t < blk_at.size(); ++t) {
      h->blk_first[t] = blk_at[2 * t];
      h->blk_last[t] = blk_at[2 * t + 1];
    }
  }
  for (void *b : {(void *)head, (void *)pos, (void *)tmp, (void *)ask, (void *)got}) dev_free(h, b);
  return st;
}

// Rebuild the tile lists for another tile size or fused-kernel block size
// (segments and scratch do not depend on them).
static amr_status set_tile(amr_mesh *h, int tile, int nsub, bool planar = false) {
  h->planar = planar;
  if (tile == h->tile_size && nsub == h->nsub && h->tpre) return AMR_OK;
  h->tile_size = tile;
  if (nsub != h->nsub) {
    h->nsub = nsub;
    if (nsub > 0) AMR_TRY(build_blocks(h));
  }
  h->occ.clear();
  build_lists(h);
  dev_free(h, h->segs);
  dev_free(h, h->tpre);
  h->segs = nullptr;
  h->tpre = nullptr;
  AMR_TRY(upload(h, &h->segs, h->segs_h));
  AMR_TRY(upload(h, &h->tpre, h->tpre_h));
  return AMR_OK;
}

// One coarse step captured as a CUDA graph, the way amr_advance replays it.
static amr_status capture_coarse_step(amr_mesh *h, cudaGraphExec_t *out) {
  *out = nullptr;
  h->capturing = true;
  h->capture_kernels = 0;
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
  coarse_step(h);
  cudaError_t e = cudaStreamEndCapture(h->s, &g);
  h->capturing = false;
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_advance: capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_advance: instantiate failed: %s", cudaGetErrorString(e));
  return AMR_OK;
}

// Time candidate launch shapes on full coarse steps from a snapshot of the
// state, run as they will run (graph replays when graphs are on), the best of
// three steps each; restore the snapshot; keep the fastest.  Candidates: the
// per-cell passes with every tile size x schedule and, unless the tile size
// or the kernel was fixed, the fused kernel with nsubgrid 1, 2 (and 4 in
// FP32) x schedule.
struct LaunchShape {
  int tile, sched, nsub;
  bool planar;
};

static amr_status autotune(amr_mesh *h) {
  h->tuned = true;
  std::vector<int> tiles =
      h->p.tile ? std::vector<int>{h->p.tile} : std::vector<int>{64, 128, 256, 512};
  std::vector<int> scheds = h->p.schedule >= 0 ? std::vector<int>{h->p.schedule} : std::vector<int>{1, 0};
  std::vector<int> nsubs;
  if (h->p.nsubgrid > 0)
    nsubs = {h->p.nsubgrid};
  else if (h->p.nsubgrid == 0 || h->p.tile)
    nsubs = {0};
  else
    nsubs = {0, 1, 2, 4};
  std::vector<LaunchShape> cands;
  for (int ns : nsubs)
    for (int t : (ns == 0 ? tiles : std::vector<int>{tiles[0]}))
      for (int sc : scheds)
        for (int pl = 0; pl < (ns == 0 ? 1 : 2); ++pl) {
          if (h->p.nsubgrid > 0 && h->p.planar >= 0 && pl != h->p.planar) continue;
          cands.push_back({t, sc, ns, pl == 1});
        }
  if (cands.size() == 1) {
    h->persistent = cands[0].sched == 1;
    return set_tile(h, cands[0].tile, cands[0].nsub, cands[0].planar);
  }
  const bool graphs = h->p.use_graphs && !h->timing;
  const size_t ub = h->elem() * 5 * size_t(h->S), rb = h->elem() * 5 * size_t(h->NC > 0 ? h->NC : 1);
  const size_t mb = sizeof(int) * size_t(h->M);
  void *su = nullptr, *sr = nullptr, *sm = nullptr;
  AMR_TRY(dev_alloc(h, &su, ub));
  AMR_TRY(dev_alloc(h, &sr, rb));
  AMR_TRY(dev_alloc(h, &sm, mb));
  CUDA_TRY(cudaMemcpyAsync(su, h->U, ub, cudaMemcpyDeviceToDevice, h->s));
  CUDA_TRY(cudaMemcpyAsync(sr, h->Rc, rb, cudaMemcpyDeviceToDevice, h->s));
  CUDA_TRY(cudaMemcpyAsync(sm, h->mrem, mb, cudaMemcpyDeviceToDevice, h->s));
  // tune with every member stepping
  CUDA_TRY(cudaMemsetAsync(h->mrem, 0xFF, mb, h->s));
  cudaEvent_t e0 = take_event(h), e1 = take_event(h);
  float best = 1e30f;
  LaunchShape pick = cands[0];
  for (const LaunchShape &cd : cands) {
    AMR_TRY(set_tile(h, cd.tile, cd.nsub, cd.planar));
    h->persistent = cd.sched == 1;
    cudaGraphExec_t ge = nullptr;
    if (graphs) AMR_TRY(capture_coarse_step(h, &ge));
    auto step = [&] {
      if (ge)
        cudaGraphLaunch(ge, h->s);
      else
        coarse_step(h);
    };
    step();  // warm-up
    float cand = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0, h->s);
      step();
      cudaEventRecord(e1, h->s);
      CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cand = std::min(cand, ms);
    }
    if (ge) cudaGraphExecDestroy(ge);
    h->tune_ms.push_back(cand);
    if (cand < best) {
      best = cand;
      pick = cd;
    }
    CUDA_TRY(cudaMemcpyAsync(h->U, su, ub, cudaMemcpyDeviceToDevice, h->s));
    CUDA_TRY(cudaMemcpyAsync(h->Rc, sr, rb, cudaMemcpyDeviceToDevice, h->s));
  }
  CUDA_TRY(cudaMemcpyAsync(h->mrem, sm, mb, cudaMemcpyDeviceToDevice, h->s));
  h->event_pool.push_back(e0);
  h->event_pool.push_back(e1);
  AMR_TRY(set_tile(h, pick.tile, pick.nsub, pick.planar));
  h->persistent = pick.sched == 1;
  dev_free(h, su);
  dev_free(h, sr);
  dev_free(h, sm);
  return check_device(h, "amr_advance (autotune)");
}

extern "C" amr_status amr_advance(amr_handle h, int n, double *dt_last) {
  if (!h) return fail(AMR_EINVAL, "amr_advance: NULL handle");
  if (n < 0) return fail(AMR_EINVAL, "amr_advance: n must be >= 0");
  if (!h->tuned && n > 0) AMR_TRY(autotune(h));
  const bool graphs = h->p.use_graphs && !h->timing;
  for (int t = 0; t < n; ++t) {
    if (h->p.regrid_every_step) AMR_TRY(amr_regrid(h, nullptr, nullptr));
    // a mesh's first coarse step runs its launches directly (the device
    // starts at the first one); the graph is captured for the second: a mesh
    // that is regridded before every coarse step never pays for a capture
    if (graphs && !h->graph && h->steps_on_mesh >= 1) {
      AMR_TRY(capture_coarse_step(h, &h->graph));
      h->graph_kernels = h->capture_kernels;
    }
    if (graphs && h->graph) {
      CUDA_TRY(cudaGraphLaunch(h->graph, h->s));
      h->graph_launches++;
      h->launches += h->graph_kernels;
    } else {
      coarse_step(h);
    }
    ++h->steps_on_mesh;
  }
  if (h->launch_err != cudaSuccess) return check_device(h, "amr_advance");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_advance: %s", cudaGetErrorString(e));
  if (dt_last) {
    CUDA_TRY(cudaMemcpyAsync(dt_last, h->dt_dev + h->sel, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    return check_device(h, "amr_advance");
  }
  return AMR_OK;
}

extern "C" amr_status amr_reindex(amr_handle h) {
  if (!h) return fail(AMR_EINVAL, "amr_reindex: NULL handle");
  AMR_TRY(reindex(h));
  if (h->launch_err != cudaSuccess) return check_device(h, "amr_reindex");
  return AMR_OK;
}

extern "C" amr_status amr_sync(amr_handle h) {
  if (!h) return fail(AMR_EINVAL, "amr_sync: NULL handle");
  if (h->cs) CUDA_TRY(cudaStreamSynchronize(h->cs));
  if (h->cs_out) CUDA_TRY(cudaStreamSynchronize(h->cs_out));
  return check_device(h, "amr_sync");
}

// ---------------------------------------------------------------------------
// whole-state copies that overlap the level steps: a copy stream moves host
// data to and from staging buffers while the compute stream steps; the
// compute stream moves staging <-> U (device to device, or a conversion for
// FP32 states).  Events order the reuse of each staging buffer.
// ---------------------------------------------------------------------------
static amr_status state_staging(amr_mesh *h, int64_t n) {
  if (!h->cs) {
    CUDA_TRY(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&h->cs_out, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&h->ev_in_ready, &h->ev_in_free, &h->ev_out_ready, &h->ev_out_free})
      CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  if (h->st_n != n) {
    CUDA_TRY(cudaStreamSynchronize(h->cs));
    CUDA_TRY(cudaStreamSynchronize(h->cs_out));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    dev_free(h, h->st_in);
    dev_free(h, h->st_out);
    h->st_in = h->st_out = nullptr;
    AMR_TRY(alloc_n(h, &h->st_in, 40 * (n > 0 ? n : 1)));
    AMR_TRY(alloc_n(h, &h->st_out, 40 * (n > 0 ? n : 1)));
    h->st_n = n;
  }
  return AMR_OK;
}

extern "C" amr_status amr_load_state_async(amr_handle h, const double *U, int64_t n) {
  if (!h || !U) return fail(AMR_EINVAL, "amr_load_state_async: NULL argument");
  const Member &m = h->mem[h->sel];
  const int64_t octs = m.lo[kMaxLev + 1];
  if (n != octs)
    return fail(AMR_EINVAL, "amr_load_state_async: the member holds %lld octs, got %lld", (long long)octs,
                (long long)n);
  if (n == 0) return AMR_OK;
  AMR_TRY(state_staging(h, n));
  const int64_t count = 8 * n, first = 8 * m.oct_base;
  // copy stream: wait until the previous input has been consumed, upload
  CUDA_TRY(cudaStreamWaitEvent(h->cs, h->ev_in_free, 0));
  CUDA_TRY(cudaMemcpyAsync(h->st_in, U, sizeof(double) * 5 * count, cudaMemcpyHostToDevice, h->cs));
  CUDA_TRY(cudaEventRecord(h->ev_in_ready, h->cs));
  // compute stream: after the work already queued, take the input into U
  CUDA_TRY(cudaStreamWaitEvent(h->s, h->ev_in_ready, 0));
  if (h->p.precision == 8) {  // one copy kernel for the five rows (copy engines ran at about 2.3 TB/s)
    launch(h, K_CONVERT, k_rows_copy, dim3(nblocks(5 * count / 2)), dim3(256), (const double2 *)h->st_in,
           count / 2, count / 2, reinterpret_cast<double2 *>(static_cast<double *>(h->U) + first), h->S / 2);
  } else {
    launch(h, K_CONVERT, k_from_double<float>, dim3(nblocks(5 * count)), dim3(256), (const double *)h->st_in,
           count, static_cast<float *>(h->U) + first, h->S);
  }
  CUDA_TRY(cudaEventRecord(h->ev_in_free, h->s));
  return AMR_OK;
}

extern "C" amr_status amr_store_state_async(amr_handle h, double *U, int64_t cap) {
  if (!h || !U) return fail(AMR_EINVAL, "amr_store_state_async: NULL argument");
  const Member &m = h->mem[h->sel];
  const int64_t n = m.lo[kMaxLev + 1];
  if (cap < n) return fail(AMR_EINVAL, "amr_store_state_async: cap %lld < %lld octs", (long long)cap, (long long)n);
  if (n == 0) return AMR_OK;
  AMR_TRY(state_staging(h, n));
  const int64_t count = 8 * n, first = 8 * m.oct_base;
  // compute stream: once the previous output has left, snapshot U
  CUDA_TRY(cudaStreamWaitEvent(h->s, h->ev_out_free, 0));
  if (h->p.precision == 8) {
    launch(h, K_CONVERT, k_rows_copy, dim3(nblocks(5 * count / 2)), dim3(256),
           reinterpret_cast<const double2 *>(static_cast<const double *>(h->U) + first), h->S / 2, count / 2,
           reinterpret_cast<double2 *>(h->st_out), count / 2);
  } else {
    launch(h, K_CONVERT, k_to_double<float>, dim3(nblocks(5 * count)), dim3(256),
           static_cast<const float *>(h->U) + first, h->S, count, h->st_out);
  }
  CUDA_TRY(cudaEventRecord(h->ev_out_ready, h->s));
  // download stream: the snapshot to the host
  CUDA_TRY(cudaStreamWaitEvent(h->cs_out, h->ev_out_ready, 0));
  CUDA_TRY(cudaMemcpyAsync(U, h->st_out, sizeof(double) * 5 * count, cudaMemcpyDeviceToHost, h->cs_out));
  CUDA_TRY(cudaEventRecord(h->ev_out_free, h->cs_out));
  return AMR_OK;
}

extern "C" amr_status amr_fill_ghosts(amr_handle h, int level) {
  if (!h) return fail(AMR_EINVAL, "amr_fill_ghosts: NULL handle");
  if (level < 1 || level > kMaxLev) return fail(AMR_EINVAL, "amr_fill_ghosts: bad level");
  const SegList &L = h->level_list[level];
  if (h->p.precision == 4)
    run_list(h, K_PROLONG, k_prolong<float>, step_args<float>(h, false, 0.0), L, DOM_GHOST5);
  else
    run_list(h, K_PROLONG, k_prolong<double>, step_args<double>(h, false, 0.0), L, DOM_GHOST5);
  return AMR_OK;
}

extern "C" amr_status amr_set_member_steps(amr_handle h, const int32_t *steps, int n) {
  if (!h || !steps) return fail(AMR_EINVAL, "amr_set_member_steps: NULL argument");
  if (n != h->M) return fail(AMR_EINVAL, "amr_set_member_steps: %d values for %d members", n, h->M);
  for (int q = 0; q < n; ++q)
    if (steps[q] < -1) return fail(AMR_EINVAL, "amr_set_member_steps: steps must be >= -1");
  CUDA_TRY(cudaMemcpyAsync(h->mrem, steps, sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return AMR_OK;
}

extern "C" amr_status amr_member_errors(amr_handle h, int32_t *errs, int n) {
  if (!h || !errs) return fail(AMR_EINVAL, "amr_member_errors: NULL argument");
  if (n < h->M) return fail(AMR_EINVAL, "amr_member_errors: room for %d members needed", h->M);
  CUDA_TRY(cudaMemcpyAsync(errs, h->merr, sizeof(int32_t) * h->M, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  // the per-member bits now carry the news: clear the handle-wide word too
  CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));
  for (int q = 0; q < h->M; ++q) {
    int32_t v = 0;
    if (errs[q] & kErrNaN) v |= 1;
    errs[q] = v;
  }
  return AMR_OK;
}

// ---------------------------------------------------------------------------
// regrid (Sec. 2.2)
// ---------------------------------------------------------------------------
static RegridArgs regrid_args(amr_mesh *h, uint32_t *raw, uint32_t *flag) {
  RegridArgs a{};
  a.N = int(h->N);
  a.NE = int(h->NE);
  a.NC = int(h->NC);
  a.S = h->S;
  a.key = h->key;
  a.son = h->son;
  a.father = h->father;
  a.nbr27 = h->nbr27;
  a.fnb = h->fnb;
  a.csrc = h->csrc;
  a.mlmin = h->mlmin;
  a.mlmax = h->mlmax;
  a.mgamma = h->mgamma_d;
  a.msmallr = h->msmallr_d;
  a.msmallp = h->msmallp_d;
  a.grad_rho = h->p.refine_grad_rho;
  a.grad_p = h->p.refine_grad_p;
  a.mass = h->p.refine_mass;
  a.expand = h->p.regrid_expand ? 1 : 0;
  a.test_r = a.grad_rho > 0.0;
  a.test_p = a.grad_p > 0.0;
  a.test_mass = a.mass > 0.0;
  for (int l = 0; l < 16; ++l) {
    const double t = a.test_mass ? std::ldexp(a.mass, 3 * l) : 0.0;  // +inf past the range
    int64_t b64;
    std::memcpy(&b64, &t, 8);
    a.mass_bits64[l] = b64;
    float f = float(t);  // rounded down to an FP32 value: rho32 > t  <=>  rho32 > f
    if (double(f) > t) f = std::nextafter(f, -INFINITY);
    int32_t b32;
    std::memcpy(&b32, &f, 4);
    a.mass_bits32[l] = b32;
  }
  a.thr_r32 = float(a.grad_rho);
  a.thr_p32 = float(a.grad_p);
  auto thr_ok = [](float t) { return t >= 0x1p-60f && t <= 0x1p60f; };
  a.use32 = (!a.test_r || thr_ok(a.thr_r32)) && (!a.test_p || thr_ok(a.thr_p32));
  a.mflag32 = h->mflag32;
  a.raw = raw;
  a.flag = flag;
  a.err = h->err;
  return a;
}

// flag, expand and grade: final masks in flag[N]
static amr_status compute_flags(amr_mesh *h, uint32_t *raw, uint32_t *flag, const char *where,
                                bool sync = true) {
  const RegridArgs a = regrid_args(h, raw, flag);
  const unsigned g = nblocks(h->N);
  float *rp = nullptr;  // FP32 rho, p and the pressure's error bound per cell
  uint32_t *und = nullptr, *n_und = nullptr;  // cells left to the FP64 tests
  AMR_TRY(alloc_n(h, &rp, 24 * h->N));
  AMR_TRY(alloc_n(h, &und, 8 * h->N));
  AMR_TRY(alloc_n(h, &n_und, 1));
  CUDA_TRY(cudaMemsetAsync(n_und, 0, sizeof(uint32_t), h->s));
  const unsigned g8 = nblocks(8 * h->N);  // 256-thread blocks: whole octs per warp
  const unsigned gx = unsigned(std::max(1, 2 * h->sm_count));
  if (h->p.precision == 4) {
    launch(h, K_FLAG_RP, k_flag_rp<float>, dim3(g8), dim3(256), a, (const float *)h->U, rp);
    launch(h, K_FLAG, k_flag_raw<float>, dim3(g8), dim3(256), a, (const float *)h->U,
           (const float *)rp, und, n_und);
    launch(h, K_FLAG_EXACT, k_flag_exact<float>, dim3(gx), dim3(256), a, (const float *)h->U,
           (const float *)rp, (const uint32_t *)und, (const uint32_t *)n_und);
  } else {
    launch(h, K_FLAG_RP, k_flag_rp<double>, dim3(g8), dim3(256), a, (const double *)h->U, rp);
    launch(h, K_FLAG, k_flag_raw<double>, dim3(g8), dim3(256), a, (const double *)h->U,
           (const float *)rp, und, n_und);
    launch(h, K_FLAG_EXACT, k_flag_exact<double>, dim3(gx), dim3(256), a, (const double *)h->U,
           (const float *)rp, (const uint32_t *)und, (const uint32_t *)n_und);
  }
  dev_free(h, rp);
  dev_free(h, und);
  dev_free(h, n_und);
  launch(h, K_FLAG_EXPAND, k_flag_expand, dim3(g), dim3(256), a);
  for (auto &m : h->mem)
    for (int l = m.lmax - 1; l > m.lmin; --l) {
      const int lo = int(m.oct_base + m.lo[l]), hi = int(m.oct_base + m.lo[l + 1]);
      if (hi > lo) launch(h, K_FLAG_GRADE, k_flag_grade, dim3(nblocks(hi - lo)), dim3(256), a, lo, hi);
    }
  return sync ? check_device(h, where) : check_launches(h, where);
}

extern "C" amr_status amr_flag(amr_handle h, int level, uint8_t *flags, int64_t cap) {
  if (!h || !flags) return fail(AMR_EINVAL, "amr_flag: NULL argument");
  if (level < 0 || level > kMaxLev) return fail(AMR_EINVAL, "amr_flag: level out of range");
  const Member &m = h->mem[h->sel];
  const int64_t lo = m.oct_base + m.lo[level], nl = m.lo[level + 1] - m.lo[level];
  if (cap < 8 * nl) return fail(AMR_EINVAL, "amr_flag: room for %lld cells needed", (long long)(8 * nl));
  uint32_t *raw = nullptr, *flag = nullptr;
  AMR_TRY(alloc_n(h, &raw, h->N));
  AMR_TRY(alloc_n(h, &flag, h->N));
  amr_status st = compute_flags(h, raw, flag, "amr_flag");
  if (st == AMR_OK && nl > 0) {
    std::vector<uint32_t> mk(nl);
    cudaError_t e = cudaMemcpyAsync(mk.data(), flag + lo, 4 * nl, cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = fail(AMR_ECUDA, "amr_flag: %s", cudaGetErrorString(e));
    for (int64_t q = 0; q < nl && st == AMR_OK; ++q)
      for (int c = 0; c < 8; ++c) flags[8 * q + c] = uint8_t((mk[q] >> c) & 1u);
  }
  dev_free(h, raw);
  dev_free(h, flag);
  return st;
}

// The new mesh nh takes over h's stream ownership, events, pending timed
// launches and counters (its own launches, made while it was built, add to
// them); h's captured graph is dropped.
static void take_over(amr_mesh *nh, amr_mesh *h) {
  nh->own_stream = h->own_stream;
  h->own_stream = false;
  nh->event_pool.insert(nh->event_pool.end(), h->event_pool.begin(), h->event_pool.end());
  h->event_pool.clear();
  nh->pending.insert(nh->pending.begin(), h->pending.begin(), h->pending.end());
  h->pending.clear();
  nh->timing = h->timing;
  nh->launches += h->launches;
  nh->graph_launches += h->graph_launches;
  std::memcpy(nh->kernel_ms, h->kernel_ms, sizeof h->kernel_ms);
  std::memcpy(nh->kernel_n, h->kernel_n, sizeof h->kernel_n);
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
}

// A fresh handle shell that shares h's stream, parameters and members.
static amr_mesh *regrid_shell(amr_mesh *h) {
  amr_mesh *nh = new amr_mesh();
  nh->p = h->p;
  nh->s = h->s;
  nh->cache = h->cache;
  nh->pin = h->pin;
  nh->timing = h->timing;  // the new mesh's build is timed with the call that makes it
  nh->own_stream = false;
  nh->device = h->device;
  nh->sm_count = h->sm_count;
  nh->M = h->M;
  nh->sel = h->sel;
  nh->lmax_all = h->lmax_all;
  nh->mem = h->mem;
  nh->tile_size = h->tile_size;
  nh->persistent = h->persistent;
  nh->tuned = h->tuned;
  nh->nsub = h->nsub;
  nh->planar = h->planar;
  return nh;
}

// One regrid; the final flags are computed from the handle's criteria, or
// given (hflags: one byte per cell of the whole handle, mesh order).
static amr_status regrid_impl(amr_mesh *h, const uint8_t *hflags, int64_t *created,
                              int64_t *removed) {
  if (h->cs) CUDA_TRY(cudaStreamSynchronize(h->cs));  // state copies in flight finish first
  if (h->cs_out) CUDA_TRY(cudaStreamSynchronize(h->cs_out));
  if (created) *created = 0;
  if (removed) *removed = 0;
  const int64_t N = h->N;
  uint32_t *raw = nullptr, *flag = nullptr, *pos = nullptr, *tmp = nullptr;
  auto release = [&] {
    for (uint32_t **q : {&raw, &flag, &pos, &tmp})
      if (*q) {
        dev_free(h, *q);
        *q = nullptr;
      }
  };
  amr_status st = AMR_OK;
#define REGRID_TRY(x)        \
  do {                       \
    st = (x);                \
    if (st != AMR_OK) {      \
      release();             \
      return st;             \
    }                        \
  } while (0)
  REGRID_TRY(alloc_n(h, &raw, N));
  REGRID_TRY(alloc_n(h, &flag, N));
  REGRID_TRY(alloc_n(h, &pos, 2 * N + 1));
  REGRID_TRY(alloc_n(h, &tmp, scan_tmp_size(2 * N + 1)));
  if (hflags) {
    std::vector<uint32_t> mk(N);
    for (int64_t q = 0; q < N; ++q) {
      uint32_t b = 0;
      for (int c = 0; c < 8; ++c) b |= uint32_t(hflags[8 * q + c] != 0) << c;
      mk[q] = b;
    }
    cudaError_t e = cudaMemcpyAsync(flag, mk.data(), 4 * N, cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) REGRID_TRY(fail(AMR_ECUDA, "amr_regrid_flags: %s", cudaGetErrorString(e)));
  } else {
    REGRID_TRY(compute_flags(h, raw, flag, "amr_regrid", false));  // checked with the counts
  }
  const RegridArgs a = regrid_args(h, raw, flag);
  launch(h, K_REGRID, k_regrid_count, dim3(nblocks(N)), dim3(256), a, pos);
  scan_exclusive(h, pos, 2 * N + 1, tmp);
  uint32_t *tail = nullptr;
  REGRID_TRY(pinned_words(h, 2, &tail));
  REGRID_TRY(read_words(h, 0, pos + N, 1));      // kept octs
  REGRID_TRY(read_words(h, 1, pos + 2 * N, 1));  // kept + new octs
  REGRID_TRY(check_device_after_reads(h, "amr_regrid"));
  const int64_t K = tail[0], NN = int64_t(tail[1]) - tail[0];
  if (created) *created = NN;
  if (removed) *removed = N - K;
  if (NN == 0 && K == N) {  // nothing changes
    release();
    return AMR_OK;
  }
  const int64_t n_out = K + NN;
  if (n_out > (int64_t(1) << 26)) {
    release();
    return fail(AMR_EINVAL, "amr_regrid: the new mesh would hold more than 2^26 octs");
  }
  // the new oct list, in the new handle's memory
  amr_mesh *nh = regrid_shell(h);
  nh->graded_by_construction = hflags == nullptr;  // caller's flags are checked
  uint8_t *d_lvl = nullptr, *d_new = nullptr;
  uint16_t *d_mem = nullptr;
  uint32_t *d_i = nullptr, *d_j = nullptr, *d_k = nullptr, *d_src = nullptr;
  auto abandon = [&](amr_status e) {
    std::string msg = g_last_error;
    cudaStreamSynchronize(h->s);
    // the old mesh keeps (or gets back) level-step scratch of its own size
    if (nh->W && nh->Q && nh->F) {
      for (void *b : {nh->W, nh->Q, nh->F}) move_buf(h, nh, b);
      h->W = nh->W;
      h->Q = nh->Q;
      h->F = nh->F;
      h->ls_cap = nh->ls_cap;
      nh->W = nh->Q = nh->F = nullptr;
    }
    if (nh->C) {
      move_buf(h, nh, nh->C);
      h->C = nh->C;
      h->cs_cap = nh->cs_cap;
      nh->C = nullptr;
    }
    destroy_all(nh);
    release();
    const amr_status se = ensure_scratch(h);
    g_last_error = msg;
    return se != AMR_OK ? se : e;
  };
  share_members(nh, h);
  if ((st = alloc_n(nh, &d_lvl, n_out)) != AMR_OK ||
      (st = alloc_n(nh, &d_new, n_out)) != AMR_OK || (st = alloc_n(nh, &d_mem, n_out)) != AMR_OK ||
      (st = alloc_n(nh, &d_i, n_out)) != AMR_OK || (st = alloc_n(nh, &d_j, n_out)) != AMR_OK ||
      (st = alloc_n(nh, &d_k, n_out)) != AMR_OK || (st = alloc_n(nh, &d_src, n_out)) != AMR_OK)
    return abandon(st);
  launch(h, K_REGRID, k_regrid_emit, dim3(nblocks(N)), dim3(256), a, (const uint32_t *)pos, d_lvl, d_mem,
         d_i, d_j, d_k, d_src, d_new);
  if ((st = check_launches(h, "amr_regrid")) != AMR_OK) return abandon(st);
  for (uint32_t **q : {&raw, &flag, &tmp}) {  // pos serves the new mesh's build
    dev_free(h, *q);
    *q = nullptr;
  }
  // the level-step scratch goes over to the new mesh (reused if large enough)
  for (void **b : {&h->W, &h->Q, &h->F, &h->C}) move_buf(nh, h, *b);
  nh->W = h->W;
  nh->Q = h->Q;
  nh->F = h->F;
  nh->C = h->C;
  nh->ls_cap = h->ls_cap;
  nh->cs_cap = h->cs_cap;
  h->W = h->Q = h->F = h->C = nullptr;
  h->ls_cap = h->cs_cap = 0;
  const StateSource from{h->U, h->S, d_src, pos, N};  // the old mesh lives until the swap below
  if ((st = build_mesh(nh, n_out, false, d_lvl, d_mem, d_i, d_j, d_k, nullptr, nullptr, d_new,
                       h->order_computed ? K : 0, &from)) != AMR_OK)
    return abandon(st);
  // carry the per-member step counters and last time steps over
  cudaMemcpyAsync(nh->mrem, h->mrem, sizeof(int) * h->M, cudaMemcpyDeviceToDevice, h->s);
  cudaMemcpyAsync(nh->dt_dev, h->dt_dev, sizeof(double) * h->M, cudaMemcpyDeviceToDevice, h->s);
  cudaMemcpyAsync(nh->merr, h->merr, sizeof(int) * h->M, cudaMemcpyDeviceToDevice, h->s);
  // the handle takes the new mesh; the old one is freed
  take_over(nh, h);
  std::swap(*h, *nh);
  own_members(h, nh);
  if (h->cache) h->cache->cap = h->bytes;  // the old mesh's arrays serve the next regrid
  destroy_all(nh);
  return check_launches(h, "amr_regrid");  // the new mesh's error word was read after its build
#undef REGRID_TRY
}

extern "C" amr_status amr_regrid(amr_handle h, int64_t *created, int64_t *removed) {
  if (!h) return fail(AMR_EINVAL, "amr_regrid: NULL handle");
  return regrid_impl(h, nullptr, created, removed);
}

extern "C" amr_status amr_regrid_flags(amr_handle h, const uint8_t *flags, int64_t n_cells,
                                       int64_t *created, int64_t *removed) {
  if (!h || !flags) return fail(AMR_EINVAL, "amr_regrid_flags: NULL argument");
  if (n_cells != 8 * h->N)
    return fail(AMR_EINVAL, "amr_regrid_flags: %lld flags given, the handle has %lld cells",
                (long long)n_cells, (long long)(8 * h->N));
  return regrid_impl(h, flags, created, removed);
}

// ---------------------------------------------------------------------------
// self-gravity: multigrid V-cycles on the base level (Sec. 5)
// ---------------------------------------------------------------------------
constexpr int kMGParts = 1024;  // blocks of the reductions
constexpr int kMGPre = 2, kMGPost = 2, kMGCoarsest = 8;

static amr_status mg_setup(amr_mesh *h, int member, int lmin) {
  if (h->mg_member == member && !h->mg.empty() && h->mg[0].n == (1 << lmin)) return AMR_OK;
  for (auto &L : h->mg) {
    dev_free(h, L.f);
    dev_free(h, L.p);
  }
  h->mg.clear();
  for (void *b : {(void *)h->mg_rho, (void *)h->mg_r, (void *)h->mg_part, (void *)h->mg_res,
                  (void *)h->phi})
    dev_free(h, b);
  const int n0 = 1 << lmin;
  for (int n = n0; n >= 2; n >>= 1) {
    amr_mesh::MGLevel L;
    L.n = n;
    const int64_t m = int64_t(n) * n * n;
    AMR_TRY(alloc_n(h, &L.f, m));
    AMR_TRY(alloc_n(h, &L.p, m));
    CUDA_TRY(cudaMemsetAsync(L.p, 0, sizeof(double) * m, h->s));
    h->mg.push_back(L);
  }
  const int64_t m0 = int64_t(n0) * n0 * n0;
  AMR_TRY(alloc_n(h, &h->mg_rho, m0));
  AMR_TRY(alloc_n(h, &h->mg_r, m0));
  AMR_TRY(alloc_n(h, &h->mg_part, 2 * kMGParts));
  AMR_TRY(alloc_n(h, &h->mg_res, 1024));
  AMR_TRY(alloc_n(h, &h->phi, m0));
  h->mg_member = member;
  return AMR_OK;
}

static unsigned mg_blocks(int64_t m) { return unsigned(std::min<int64_t>((m + 255) / 256, kMGParts)); }

static void mg_vcycle(amr_mesh *h, size_t k, double dx) {
  amr_mesh::MGLevel &L = h->mg[k];
  const int n = L.n;
  const double dx2 = dx * dx;
  if (n <= 2) {
    launch(h, K_MG_OTHER, k_mg_coarsest, dim3(1), dim3(8), dx2, (const double *)L.f, L.p, kMGCoarsest);
    return;
  }
  const int64_t m = int64_t(n) * n * n;
  for (int s = 0; s < kMGPre; ++s)
    for (int colour = 0; colour < 2; ++colour)
      launch(h, K_MG_SMOOTH, k_mg_smooth, dim3(nblocks(m / 2)), dim3(256), n, dx2, (const double *)L.f,
             L.p, colour);
  amr_mesh::MGLevel &C = h->mg[k + 1];
  launch(h, K_MG_RESTRICT, k_mg_restrict, dim3(nblocks(m / 8)), dim3(256), n, 1.0 / dx2,
         (const double *)L.f, (const double *)L.p, C.f, C.p);
  mg_vcycle(h, k + 1, 2.0 * dx);
  launch(h, K_MG_PROLONG, k_mg_prolong, dim3(nblocks(m)), dim3(256), n, (const double *)C.p, L.p);
  for (int s = 0; s < kMGPost; ++s)
    for (int colour = 0; colour < 2; ++colour)
      launch(h, K_MG_SMOOTH, k_mg_smooth, dim3(nblocks(m / 2)), dim3(256), n, dx2, (const double *)L.f,
             L.p, colour);
}

extern "C" amr_status amr_poisson(amr_handle h, double fourpiG, int n_vcycles, double *resid) {
  if (!h) return fail(AMR_EINVAL, "amr_poisson: NULL handle");
  if (n_vcycles < 0 || n_vcycles > 1020) return fail(AMR_EINVAL, "amr_poisson: n_vcycles must be in [0, 1020]");
  const Member &mb = h->mem[h->sel];
  const int lmin = mb.lmin;
  if (lmin > 10) return fail(AMR_EINVAL, "amr_poisson: levelmin above 10 (more than 1024^3 cells)");
  const int n = 1 << lmin;
  const int64_t m0 = int64_t(n) * n * n;
  const int lo = int(mb.oct_base + mb.lo[lmin]), nl = int(mb.lo[lmin + 1] - mb.lo[lmin]);
  if (8 * int64_t(nl) != m0) return fail(AMR_EGRADING, "amr_poisson: the base level is not complete");
  AMR_TRY(mg_setup(h, h->sel, lmin));
  const double dx = std::ldexp(1.0, -lmin);
  if (h->p.precision == 4)
    launch(h, K_MG_OTHER, k_mg_gather<float>, dim3(nblocks(m0)), dim3(256), (const float *)h->U,
           (const uint64_t *)h->key, lo, nl, n, h->mg_rho);
  else
    launch(h, K_MG_OTHER, k_mg_gather<double>, dim3(nblocks(m0)), dim3(256), (const double *)h->U,
           (const uint64_t *)h->key, lo, nl, n, h->mg_rho);
  const unsigned nb = mg_blocks(m0);
  double *mean = h->mg_res + 1022;  // two scalars at the end of the residual array
  launch(h, K_MG_OTHER, k_mg_sum, dim3(nb), dim3(256), (const double *)h->mg_rho, m0, 0, h->mg_part);
  launch(h, K_MG_OTHER, k_mg_total, dim3(1), dim3(32), (const double *)h->mg_part, int(nb),
         1.0 / double(m0), mean);
  launch(h, K_MG_OTHER, k_mg_source, dim3(nb), dim3(256), (const double *)h->mg_rho, m0,
         (const double *)mean, fourpiG, h->mg[0].f);
  for (int c = 0; c < n_vcycles; ++c) {
    mg_vcycle(h, 0, dx);
    if (resid) {
      launch(h, K_MG_OTHER, k_mg_residual, dim3(nblocks(m0)), dim3(256), n, 1.0 / (dx * dx),
             (const double *)h->mg[0].f, (const double *)h->mg[0].p, h->mg_r);
      launch(h, K_MG_OTHER, k_mg_sum, dim3(nb), dim3(256), (const double *)h->mg_r, m0, 1, h->mg_part);
      launch(h, K_MG_OTHER, k_mg_norm, dim3(1), dim3(32), (const double *)h->mg_part, int(nb),
             h->mg_res + c);
    }
  }
  // potential of the base cells, mean removed
  launch(h, K_MG_OTHER, k_mg_sum, dim3(nb), dim3(256), (const double *)h->mg[0].p, m0, 0,
         h->mg_part + kMGParts);
  launch(h, K_MG_OTHER, k_mg_total, dim3(1), dim3(32), (const double *)(h->mg_part + kMGParts),
         int(nb), 1.0 / double(m0), mean + 1);
  launch(h, K_MG_OTHER, k_mg_scatter, dim3(nblocks(m0)), dim3(256), (const double *)h->mg[0].p,
         (const uint64_t *)h->key, lo, nl, n, (const double *)(mean + 1), h->phi);
  if (resid && n_vcycles > 0)
    CUDA_TRY(cudaMemcpyAsync(resid, h->mg_res, sizeof(double) * n_vcycles, cudaMemcpyDeviceToHost, h->s));
  return check_device(h, "amr_poisson");
}

// ---------------------------------------------------------------------------
// Poisson on the refined levels (Sec. 5: the potential built level by level)
// ---------------------------------------------------------------------------
static amr_status ensure_phil(amr_mesh *h) {
  if (h->phil && h->phil_n == 8 * h->N) return AMR_OK;
  dev_free(h, h->phil);
  h->phil = nullptr;
  AMR_TRY(alloc_n(h, &h->phil, 8 * std::max<int64_t>(h->N, 1)));
  CUDA_TRY(cudaMemsetAsync(h->phil, 0, sizeof(double) * size_t(8 * std::max<int64_t>(h->N, 1)), h->s));
  h->phil_n = 8 * h->N;
  return AMR_OK;
}

static bool level_ok(int level) { return level >= 0 && level <= kMaxLev; }

static void mgl_free_set(amr_mesh *h, amr_mesh::MGLSet &S) {
  for (auto &t : S.tab)
    for (void *b : {(void *)t.nb, (void *)t.nbnd, (void *)t.col, (void *)t.child, (void *)t.pro, (void *)t.e,
                    (void *)t.f, (void *)t.r})
      dev_free(h, b);
  S.tab.clear();
  for (void *b : {(void *)S.g0, (void *)S.fatherg, (void *)S.acrossg, (void *)S.bsum}) dev_free(h, b);
  S.g0 = S.fatherg = S.acrossg = nullptr;
  S.bsum = nullptr;
}

static void mgl_free(amr_mesh *h) {
  for (auto &kv : h->mgls) mgl_free_set(h, kv.second);
  h->mgls.clear();
  dev_free(h, h->mgl_part);
  dev_free(h, h->mgl_scalar);
  h->mgl_part = h->mgl_scalar = nullptr;
}

// The MG hierarchy of level L of the selected member, built on the device:
// MG level 0 = the cells of the level-L octs, MG level k = the level-(L-k)
// parents of MG level k-1, down to levelmin; every table in sorted (x, y, z)
// order of the cells (keys with L-k bits per axis).  The cell counts of the
// levels are read back to size them; nothing else leaves the device.
static amr_status mgl_build(amr_mesh *h, int L, amr_mesh::MGLSet &S) {
  const Member &mb = h->mem[h->sel];
  const int lmin = mb.lmin, K = L - lmin;
  const int lo = int(mb.oct_base + mb.lo[L]);
  const int64_t nl = mb.lo[L + 1] - mb.lo[L], n0 = 8 * nl;
  // scratch of the build: keys and values (two copies each for the sort),
  // the sort's digit table and scan space, flags and positions
  const int64_t ntiles = (n0 + kRadixTile - 1) / kRadixTile;
  const int64_t tcap = 256 * ntiles + 256;
  uint64_t *ka = nullptr, *kb = nullptr;
  uint32_t *va = nullptr, *vb = nullptr, *table = nullptr, *stmp = nullptr, *flag = nullptr, *pos = nullptr;
  int64_t *cnt = nullptr;
  std::vector<uint64_t *> keys(size_t(K + 1), nullptr);
  auto release = [&] {
    for (void *b : {(void *)ka, (void *)kb, (void *)va, (void *)vb, (void *)table, (void *)stmp, (void *)flag,
                    (void *)pos, (void *)cnt})
      dev_free(h, b);
    for (uint64_t *b : keys) dev_free(h, b);
  };
  amr_status st = AMR_OK;
#define MGL_TRY(x)      \
  do {                  \
    st = (x);           \
    if (st != AMR_OK) { \
      release();        \
      return st;        \
    }                   \
  } while (0)
  MGL_TRY(alloc_n(h, &ka, n0));
  MGL_TRY(alloc_n(h, &kb, n0));
  MGL_TRY(alloc_n(h, &va, n0));
  MGL_TRY(alloc_n(h, &vb, n0));
  MGL_TRY(alloc_n(h, &table, tcap));
  MGL_TRY(alloc_n(h, &stmp, scan_tmp_size(std::max(tcap, n0))));
  MGL_TRY(alloc_n(h, &flag, n0));
  MGL_TRY(alloc_n(h, &pos, n0));
  MGL_TRY(alloc_n(h, &cnt, 2));
  S.tab.resize(size_t(K + 1));
  // MG level 0: the level's cells, sorted; their global indices are g0
  launch(h, K_MG_OTHER, k_mgl_cells, dim3(nblocks(n0)), dim3(256), (const uint64_t *)h->key, lo, nl, L, ka, va);
  {
    uint64_t *k = ka;
    uint32_t *v = va;
    radix_sort(h, &k, &v, kb, vb, n0, digits_for(0, 3 * L), table, stmp);
    MGL_TRY(alloc_n(h, &keys[0], n0));
    CUDA_TRY(cudaMemcpyAsync(keys[0], k, 8 * size_t(n0), cudaMemcpyDeviceToDevice, h->s));
    MGL_TRY(alloc_n(h, &S.g0, n0));
    CUDA_TRY(cudaMemcpyAsync(S.g0, v, 4 * size_t(n0), cudaMemcpyDeviceToDevice, h->s));
  }
  std::vector<int64_t> n(size_t(K + 1), 0);
  n[0] = n0;
  for (int k = 1; k <= K; ++k) {
    const int b = L - k;
    const int64_t m = n[size_t(k - 1)];
    launch(h, K_MG_OTHER, k_mgl_parents, dim3(nblocks(m)), dim3(256), (const uint64_t *)keys[size_t(k - 1)], m, b,
           ka, va);
    uint64_t *kk = ka;
    uint32_t *vv = va;
    radix_sort(h, &kk, &vv, kb, vb, m, digits_for(0, 3 * b), table, stmp);
    launch(h, K_MG_OTHER, k_mgl_heads, dim3(nblocks(m)), dim3(256), (const uint64_t *)kk, m, flag);
    CUDA_TRY(cudaMemcpyAsync(pos, flag, 4 * size_t(m), cudaMemcpyDeviceToDevice, h->s));
    scan_exclusive(h, pos, m, stmp);
    MGL_TRY(alloc_n(h, &keys[size_t(k)], m));
    launch(h, K_MG_OTHER, k_mgl_unique, dim3(nblocks(m)), dim3(256), (const uint64_t *)kk, (const uint32_t *)flag,
           (const uint32_t *)pos, m, keys[size_t(k)], cnt);
    int64_t c = 0;
    CUDA_TRY(cudaMemcpyAsync(&c, cnt, sizeof c, cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    n[size_t(k)] = c;
  }
  // per MG level: neighbours, colours, children and stencils
  for (int k = 0; k <= K; ++k) {
    const int b = L - k;
    const int64_t m = n[size_t(k)];
    amr_mesh::MGLTab &T = S.tab[size_t(k)];
    T.L = b;
    T.n = m;
    MGL_TRY(alloc_n(h, &T.nb, 6 * m));
    MGL_TRY(alloc_n(h, &T.nbnd, m));
    MGL_TRY(alloc_n(h, &T.col, m));
    MGL_TRY(alloc_n(h, &T.e, m));
    MGL_TRY(alloc_n(h, &T.f, m));
    MGL_TRY(alloc_n(h, &T.r, m));
    launch(h, K_MG_OTHER, k_mgl_faces, dim3(nblocks(m)), dim3(256), (const uint64_t *)keys[size_t(k)], m, b, T.nb,
           T.nbnd, flag);
    CUDA_TRY(cudaMemcpyAsync(pos, flag, 4 * size_t(m), cudaMemcpyDeviceToDevice, h->s));
    scan_exclusive(h, pos, m, stmp);
    launch(h, K_MG_OTHER, k_mgl_colours, dim3(nblocks(m)), dim3(256), (const uint32_t *)flag,
           (const uint32_t *)pos, m, T.col, cnt + 1);
    int64_t c0 = 0;
    CUDA_TRY(cudaMemcpyAsync(&c0, cnt + 1, sizeof c0, cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    T.nc0 = c0;
    T.nc1 = m - c0;
    if (k >= 1) {
      const int64_t mf = n[size_t(k - 1)];
      MGL_TRY(alloc_n(h, &T.child, 8 * m));
      MGL_TRY(alloc_n(h, &S.tab[size_t(k - 1)].pro, 8 * mf));
      launch(h, K_MG_OTHER, k_mgl_children, dim3(nblocks(m)), dim3(256), (const uint64_t *)keys[size_t(k)], m, b,
             (const uint64_t *)keys[size_t(k - 1)], mf, T.child);
      launch(h, K_MG_OTHER, k_mgl_stencils, dim3(nblocks(mf)), dim3(256), (const uint64_t *)keys[size_t(k - 1)], mf,
             b, (const uint64_t *)keys[size_t(k)], m, S.tab[size_t(k - 1)].pro);
    }
  }
  // MG level 0: father cells and the coarse cells across its boundary
  MGL_TRY(alloc_n(h, &S.fatherg, n0));
  MGL_TRY(alloc_n(h, &S.acrossg, 6 * n0));
  MGL_TRY(alloc_n(h, &S.bsum, n0));
  launch(h, K_MG_OTHER, k_mgl_coarse, dim3(nblocks(n0)), dim3(256), h->hash, h->sel, L, int(h->N),
         (const uint64_t *)keys[0], n0, (const int32_t *)S.tab[0].nb, S.fatherg, S.acrossg, h->err);
  st = check_device(h, "amr_poisson_level");
  release();
#undef MGL_TRY
  return st;
}

// the hierarchy of level L of the selected member, built on first use and
// kept until the mesh changes
static amr_status mgl_setup(amr_mesh *h, int L, amr_mesh::MGLSet **out) {
  if (!h->mgl_part) {
    AMR_TRY(alloc_n(h, &h->mgl_part, kMGParts));
    AMR_TRY(alloc_n(h, &h->mgl_scalar, 4));
  }
  const int key = h->sel * 32 + L;
  auto it = h->mgls.find(key);
  if (it == h->mgls.end()) {
    amr_mesh::MGLSet S;
    const amr_status st = mgl_build(h, L, S);
    if (st != AMR_OK) {
      mgl_free_set(h, S);
      return st;
    }
    it = h->mgls.emplace(key, std::move(S)).first;
  }
  *out = &it->second;
  return AMR_OK;
}

static void mgl_sweep(amr_mesh *h, amr_mesh::MGLSet &S, size_t k) {
  amr_mesh::MGLTab &T = S.tab[k];
  const double dx = std::ldexp(1.0, -T.L), dx2 = dx * dx;
  const double *bs = k == 0 ? S.bsum : nullptr;
  if (T.nc0)
    launch(h, K_MG_SMOOTH, k_mgl_smooth, dim3(nblocks(T.nc0)), dim3(256), T.n, (const int32_t *)T.col, T.nc0,
           (const int32_t *)T.nb, (const int32_t *)T.nbnd, bs, (const double *)T.f, T.e, dx2);
  if (T.nc1)
    launch(h, K_MG_SMOOTH, k_mgl_smooth, dim3(nblocks(T.nc1)), dim3(256), T.n, (const int32_t *)(T.col + T.nc0),
           T.nc1, (const int32_t *)T.nb, (const int32_t *)T.nbnd, bs, (const double *)T.f, T.e, dx2);
}

static void mgl_residual(amr_mesh *h, amr_mesh::MGLSet &S, size_t k) {
  amr_mesh::MGLTab &T = S.tab[k];
  const double dx = std::ldexp(1.0, -T.L), dx2 = dx * dx;
  launch(h, K_MG_OTHER, k_mgl_residual, dim3(nblocks(T.n)), dim3(256), T.n, (const int32_t *)T.nb,
         (const int32_t *)T.nbnd, (const double *)(k == 0 ? S.bsum : nullptr), (const double *)T.f,
         (const double *)T.e, dx2, T.r);
}

static void mgl_vcycle(amr_mesh *h, amr_mesh::MGLSet &S, size_t k) {
  const size_t K = S.tab.size() - 1;
  if (k == K) {
    for (int s = 0; s < kMGCoarsest; ++s) mgl_sweep(h, S, k);
    return;
  }
  for (int s = 0; s < kMGPre; ++s) mgl_sweep(h, S, k);
  mgl_residual(h, S, k);
  amr_mesh::MGLTab &T = S.tab[k], &C = S.tab[k + 1];
  launch(h, K_MG_RESTRICT, k_mgl_restrict, dim3(nblocks(C.n)), dim3(256), C.n, (const int32_t *)C.child,
         (const double *)T.r, C.f, C.e);
  mgl_vcycle(h, S, k + 1);
  launch(h, K_MG_PROLONG, k_mgl_prolong, dim3(nblocks(T.n)), dim3(256), T.n, (const int32_t *)T.pro,
         (const double *)C.e, T.e);
  for (int s = 0; s < kMGPost; ++s) mgl_sweep(h, S, k);
}

// one level's solve from the current potential of level L-1 (Dirichlet
// data) and of level L (initial guess); rho_bar host value or, if rho_bar_dev
// is set, read on the device
static amr_status poisson_level(amr_mesh *h, int L, double fourpiG, double rho_bar,
                                const double *rho_bar_dev, int n_vcycles, double *resid) {
  AMR_TRY(ensure_phil(h));
  amr_mesh::MGLSet *Sp = nullptr;
  AMR_TRY(mgl_setup(h, L, &Sp));
  amr_mesh::MGLSet &S = *Sp;
  amr_mesh::MGLTab &T0 = S.tab[0];
  const int64_t n = T0.n;
  launch(h, K_MG_OTHER, k_mgl_bsum, dim3(nblocks(n)), dim3(256), n, (const int32_t *)S.fatherg,
         (const int32_t *)S.acrossg, (const double *)h->phil, S.bsum);
  if (h->p.precision == 4)
    launch(h, K_MG_OTHER, k_mgl_source<float>, dim3(nblocks(n)), dim3(256), n, (const int32_t *)S.g0,
           (const float *)h->U, fourpiG, rho_bar, rho_bar_dev, T0.f);
  else
    launch(h, K_MG_OTHER, k_mgl_source<double>, dim3(nblocks(n)), dim3(256), n, (const int32_t *)S.g0,
           (const double *)h->U, fourpiG, rho_bar, rho_bar_dev, T0.f);
  launch(h, K_MG_OTHER, k_mgl_gather, dim3(nblocks(n)), dim3(256), n, (const int32_t *)S.g0,
         (const double *)h->phil, T0.e);
  const unsigned nb = unsigned(std::min<int64_t>((n + 255) / 256, kMGParts));
  for (int c = 0; c < n_vcycles; ++c) {
    mgl_vcycle(h, S, 0);
    if (resid) {
      mgl_residual(h, S, 0);
      launch(h, K_MG_OTHER, k_mgl_sq, dim3(nb), dim3(256), n, (const double *)T0.r, h->mgl_part);
      launch(h, K_MG_OTHER, k_mgl_norm, dim3(1), dim3(32), (const double *)h->mgl_part, int(nb), h->mgl_scalar);
      CUDA_TRY(cudaMemcpyAsync(resid + c, h->mgl_scalar, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    }
  }
  launch(h, K_MG_OTHER, k_mgl_scatter, dim3(nblocks(n)), dim3(256), n, (const int32_t *)S.g0,
         (const double *)T0.e, h->phil);
  return AMR_OK;
}

static amr_status check_level_solve(amr_mesh *h, int L, int n_vcycles, const char *where) {
  const Member &mb = h->mem[h->sel];
  if (n_vcycles < 0 || n_vcycles > 1020) return fail(AMR_EINVAL, "%s: n_vcycles must be in [0, 1020]", where);
  if (L <= mb.lmin || L > mb.lmax || mb.lo[L + 1] == mb.lo[L])
    return fail(AMR_EINVAL, "%s: level %d is not a populated refined level", where, L);
  return AMR_OK;
}

extern "C" amr_status amr_poisson_level(amr_handle h, int level, double fourpiG, double rho_bar,
                                        int n_vcycles, double *resid) {
  if (!h) return fail(AMR_EINVAL, "amr_poisson_level: NULL handle");
  AMR_TRY(check_level_solve(h, level, n_vcycles, "amr_poisson_level"));
  AMR_TRY(poisson_level(h, level, fourpiG, rho_bar, nullptr, n_vcycles, resid));
  return check_device(h, "amr_poisson_level");
}

// father cell's potential into every cell of level L (the initial guess)
__global__ void k_mgl_inject(int lo, int nl, const uint64_t *__restrict__ key, const int32_t *__restrict__ father,
                             double *phil) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 8 * nl) return;
  const int o = lo + q / 8, c = q & 7;
  const uint64_t k = key[o];
  const int fc = int((ikey_x(k) & 1) | ((ikey_y(k) & 1) << 1) | ((ikey_z(k) & 1) << 2));
  phil[8 * int64_t(o) + c] = phil[8 * int64_t(father[o]) + fc];
}

extern "C" amr_status amr_poisson_levels(amr_handle h, double fourpiG, int n_vcycles, double *resid) {
  if (!h) return fail(AMR_EINVAL, "amr_poisson_levels: NULL handle");
  const Member &mb = h->mem[h->sel];
  std::vector<double> r0(size_t(std::max(n_vcycles, 1)));
  AMR_TRY(amr_poisson(h, fourpiG, n_vcycles, resid ? r0.data() : nullptr));
  AMR_TRY(ensure_phil(h));
  const int64_t blo = mb.oct_base + mb.lo[mb.lmin], bnl = mb.lo[mb.lmin + 1] - mb.lo[mb.lmin];
  CUDA_TRY(cudaMemcpyAsync(h->phil + 8 * blo, h->phi, sizeof(double) * size_t(8 * bnl), cudaMemcpyDeviceToDevice, h->s));
  if (resid)
    for (int c = 0; c < n_vcycles; ++c) resid[size_t(mb.lmin) * n_vcycles + c] = r0[size_t(c)];
  const double *mean = h->mg_res + 1022;  // the base density's mean (amr_poisson)
  for (int L = mb.lmin + 1; L <= mb.lmax; ++L) {
    const int lo = int(mb.oct_base + mb.lo[L]), nl = int(mb.lo[L + 1] - mb.lo[L]);
    if (nl == 0) break;
    launch(h, K_MG_OTHER, k_mgl_inject, dim3(nblocks(8 * int64_t(nl))), dim3(256), lo, nl,
           (const uint64_t *)h->key, (const int32_t *)h->father, h->phil);
    AMR_TRY(poisson_level(h, L, fourpiG, 0.0, mean, n_vcycles,
                          resid ? resid + size_t(L) * n_vcycles : nullptr));
  }
  return check_device(h, "amr_poisson_levels");
}

extern "C" amr_status amr_write_phi(amr_handle h, int level, const double *phi, int64_t n) {
  if (!h || !phi) return fail(AMR_EINVAL, "amr_write_phi: NULL argument");
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_write_phi: bad level");
  const Member &mb = h->mem[h->sel];
  const int64_t lo = mb.oct_base + mb.lo[level], nl = mb.lo[level + 1] - mb.lo[level];
  if (n != 8 * nl) return fail(AMR_EINVAL, "amr_write_phi: %lld values for %lld cells", (long long)n, (long long)(8 * nl));
  AMR_TRY(ensure_phil(h));
  if (nl) CUDA_TRY(cudaMemcpyAsync(h->phil + 8 * lo, phi, sizeof(double) * size_t(8 * nl), cudaMemcpyHostToDevice, h->s));
  return check_device(h, "amr_write_phi");
}

extern "C" amr_status amr_read_phi_level(amr_handle h, int level, double *phi, int64_t cap) {
  if (!h || !phi) return fail(AMR_EINVAL, "amr_read_phi_level: NULL argument");
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_read_phi_level: bad level");
  const Member &mb = h->mem[h->sel];
  const int64_t lo = mb.oct_base + mb.lo[level], nl = mb.lo[level + 1] - mb.lo[level];
  if (cap < 8 * nl)
    return fail(AMR_EINVAL, "amr_read_phi_level: cap %lld < %lld cells", (long long)cap, (long long)(8 * nl));
  if (!h->phil || h->phil_n != 8 * h->N) return fail(AMR_EINVAL, "amr_read_phi_level: no potential on this mesh");
  if (nl) CUDA_TRY(cudaMemcpyAsync(phi, h->phil + 8 * lo, sizeof(double) * size_t(8 * nl), cudaMemcpyDeviceToHost, h->s));
  return check_device(h, "amr_read_phi_level");
}

extern "C" amr_status amr_read_phi(amr_handle h, double *phi, int64_t cap) {
  if (!h || !phi) return fail(AMR_EINVAL, "amr_read_phi: NULL argument");
  const Member &mb = h->mem[h->sel];
  const int64_t nl = mb.lo[mb.lmin + 1] - mb.lo[mb.lmin];
  if (!h->phi || h->mg_member != h->sel) return fail(AMR_EINVAL, "amr_read_phi: no potential (call amr_poisson)");
  if (cap < 8 * nl) return fail(AMR_EINVAL, "amr_read_phi: room for %lld cells needed", (long long)(8 * nl));
  CUDA_TRY(cudaMemcpyAsync(phi, h->phi, sizeof(double) * 8 * nl, cudaMemcpyDeviceToHost, h->s));
  return check_device(h, "amr_read_phi");
}

extern "C" amr_status amr_select_member(amr_handle h, int member) {
  if (!h) return fail(AMR_EINVAL, "amr_select_member: NULL handle");
  if (member < 0 || member >= h->M) return fail(AMR_EINVAL, "amr_select_member: no member %d", member);
  h->sel = member;
  return AMR_OK;
}

// ---------------------------------------------------------------------------
// state in / out (selected member)
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
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_read: bad level");
  const Member &m = h->mem[h->sel];
  const int64_t lo = m.oct_base + m.lo[level], nl = m.lo[level + 1] - m.lo[level];
  if (n_oct_out) *n_oct_out = nl;
  if ((keys || U) && cap < nl) return fail(AMR_EINVAL, "amr_read: cap %lld < %lld octs", (long long)cap, (long long)nl);
  if (keys && nl) {
    CUDA_TRY(cudaMemcpyAsync(keys, h->key + lo, 8 * nl, cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    for (int64_t t = 0; t < nl; ++t) keys[t] = external_key(keys[t]);
  }
  if (U) AMR_TRY(rows_to_host(h, h->U, h->S, 8 * lo, 8 * nl, U));
  return check_device(h, "amr_read");
}

extern "C" amr_status amr_hash(amr_handle h, int64_t n, const uint64_t *keys, uint64_t *hash) {
  if (!h || (n > 0 && (!keys || !hash))) return fail(AMR_EINVAL, "amr_hash: NULL argument");
  if (n < 0 || n > (int64_t(1) << 28)) return fail(AMR_EINVAL, "amr_hash: n outside [0, 2^28]");
  if (n == 0) return AMR_OK;
  uint64_t *buf = nullptr;
  AMR_TRY(alloc_n(h, &buf, 2 * n));
  cudaError_t e = cudaMemcpyAsync(buf, keys, 8 * n, cudaMemcpyHostToDevice, h->s);
  if (e == cudaSuccess) {
    launch(h, K_FNV, k_fnv, dim3(nblocks(n)), dim3(256), (const uint64_t *)buf, n, buf + n);
    e = cudaMemcpyAsync(hash, buf + n, 8 * n, cudaMemcpyDeviceToHost, h->s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  dev_free(h, buf);
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_hash: %s", cudaGetErrorString(e));
  return check_device(h, "amr_hash");
}

extern "C" amr_status amr_read_hash(amr_handle h, int64_t *cap_out, uint64_t *keys, int32_t *vals,
                                    int64_t cap) {
  if (!h || !cap_out) return fail(AMR_EINVAL, "amr_read_hash: NULL argument");
  *cap_out = int64_t(h->hcap);
  if ((keys || vals) && cap < int64_t(h->hcap))
    return fail(AMR_EINVAL, "amr_read_hash: cap %lld < capacity %lld", (long long)cap, (long long)h->hcap);
  if (keys) CUDA_TRY(cudaMemcpyAsync(keys, h->hash.key, 8 * h->hcap, cudaMemcpyDeviceToHost, h->s));
  if (vals) CUDA_TRY(cudaMemcpyAsync(vals, h->hash.val, 4 * h->hcap, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return check_device(h, "amr_read_hash");
}

// ---------------------------------------------------------------------------
// batch repack (continuous batching): a new oct list from the kept members'
// octs (device to device) and the added meshes (from the host), rebuilt as
// by amr_create; per-member step counters, time steps and error bits of the
// kept members carried over
// ---------------------------------------------------------------------------
extern "C" amr_status amr_batch_repack(amr_handle h, int n_keep, const int32_t *keep, int n_add,
                                       const amr_member *added, const int32_t *added_steps) {
  if (!h) return fail(AMR_EINVAL, "amr_batch_repack: NULL handle");
  if (n_keep < 0 || n_add < 0 || n_keep + n_add < 1 || n_keep > h->M ||
      n_keep + n_add > kMaxMembers)
    return fail(AMR_EINVAL, "amr_batch_repack: member counts out of range");
  if ((n_keep && !keep) || (n_add && (!added || !added_steps)))
    return fail(AMR_EINVAL, "amr_batch_repack: NULL argument");
  for (int q = 0; q < n_keep; ++q)
    if (keep[q] < 0 || keep[q] >= h->M || (q && keep[q] <= keep[q - 1]))
      return fail(AMR_EINVAL, "amr_batch_repack: keep must list member indices in increasing order");
  int64_t n_out = 0;
  for (int q = 0; q < n_keep; ++q) n_out += h->mem[keep[q]].lo[kMaxLev + 1];
  const int64_t K = n_out;
  for (int q = 0; q < n_add; ++q) {
    AMR_TRY(check_member(added[q], n_keep + q));
    if (added_steps[q] == 0 || added_steps[q] < -1)
      return fail(AMR_EINVAL, "amr_batch_repack: steps of an added member must be >= 1 or -1");
    n_out += added[q].n_oct;
  }
  if (n_out > (int64_t(1) << 26)) return fail(AMR_EINVAL, "amr_batch_repack: more than 2^26 octs in total");
  if (h->cs) CUDA_TRY(cudaStreamSynchronize(h->cs));  // state copies in flight finish first
  if (h->cs_out) CUDA_TRY(cudaStreamSynchronize(h->cs_out));
  // per-member step counters, time steps and errors of the current members
  std::vector<int> rem(h->M), merr(h->M);
  std::vector<double> dt(h->M);
  CUDA_TRY(cudaMemcpyAsync(rem.data(), h->mrem, sizeof(int) * h->M, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaMemcpyAsync(merr.data(), h->merr, sizeof(int) * h->M, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaMemcpyAsync(dt.data(), h->dt_dev, sizeof(double) * h->M, cudaMemcpyDeviceToHost, h->s));
  AMR_TRY(check_device(h, "amr_batch_repack"));
  // the new handle's members: kept ones in order, then the added ones
  amr_mesh *nh = regrid_shell(h);
  nh->M = n_keep + n_add;
  nh->mem.assign(size_t(nh->M), Member());
  nh->sel = 0;
  nh->lmax_all = 1;
  std::vector<int> remap(size_t(h->M), -1);
  std::vector<int64_t> dst(size_t(h->M), 0), base(size_t(h->M), 0);
  {
    int64_t off = 0;
    for (int q = 0; q < n_keep; ++q) {
      const Member &om = h->mem[keep[q]];
      Member &m = nh->mem[q];
      m.lmin = om.lmin;
      m.lmax = om.lmax;
      m.gamma = om.gamma;
      m.cfl = om.cfl;
      m.smallr = om.smallr;
      m.smallc = om.smallc;
      m.n_oct = om.lo[kMaxLev + 1];
      remap[keep[q]] = q;
      dst[keep[q]] = off;
      base[keep[q]] = om.oct_base;
      off += m.n_oct;
    }
    for (int q = 0; q < n_add; ++q) {
      const amr_member &a = added[q];
      Member &m = nh->mem[n_keep + q];
      m.lmin = a.levelmin;
      m.lmax = a.levelmax;
      m.gamma = a.gamma;
      m.cfl = a.cfl;
      m.smallr = a.smallr;
      m.smallc = a.smallc;
      m.n_oct = a.n_oct;
    }
    for (auto &m : nh->mem) nh->lmax_all = std::max(nh->lmax_all, m.lmax);
  }
  nh->N = n_out;
  uint8_t *d_lvl = nullptr;
  uint16_t *d_mem = nullptr;
  uint32_t *d_i = nullptr, *d_j = nullptr, *d_k = nullptr;
  double *d_U = nullptr;
  int *d_remap = nullptr;
  int64_t *d_dst = nullptr, *d_base = nullptr;
  amr_status st = AMR_OK;
  auto abandon = [&](amr_status e) {
    std::string msg = g_last_error;
    cudaStreamSynchronize(h->s);
    destroy_all(nh);
    g_last_error = msg;
    return e;
  };
  if ((st = upload_members(nh)) != AMR_OK || (st = alloc_n(nh, &d_lvl, n_out)) != AMR_OK ||
      (st = alloc_n(nh, &d_mem, n_out)) != AMR_OK || (st = alloc_n(nh, &d_i, n_out)) != AMR_OK ||
      (st = alloc_n(nh, &d_j, n_out)) != AMR_OK || (st = alloc_n(nh, &d_k, n_out)) != AMR_OK ||
      (st = alloc_n(nh, &d_U, 40 * n_out)) != AMR_OK || (st = upload(nh, &d_remap, remap)) != AMR_OK ||
      (st = upload(nh, &d_dst, dst)) != AMR_OK || (st = upload(nh, &d_base, base)) != AMR_OK)
    return abandon(st);
  if (K > 0) {
    if (h->p.precision == 4)
      launch(h, K_REGRID, k_repack_emit<float>, dim3(nblocks(h->N)), dim3(256), h->N, h->S,
             (const uint64_t *)h->key, (const float *)h->U, (const int *)d_remap,
             (const int64_t *)d_dst, (const int64_t *)d_base, n_out, d_lvl, d_mem, d_i, d_j, d_k, d_U);
    else
      launch(h, K_REGRID, k_repack_emit<double>, dim3(nblocks(h->N)), dim3(256), h->N, h->S,
             (const uint64_t *)h->key, (const double *)h->U, (const int *)d_remap,
             (const int64_t *)d_dst, (const int64_t *)d_base, n_out, d_lvl, d_mem, d_i, d_j, d_k, d_U);
  }
  // the added meshes, staged on the host in the new list's layout
  if (n_add > 0) {
    const int64_t na = n_out - K;
    const size_t nas = static_cast<size_t>(na);
    std::vector<uint8_t> lv(nas);
    std::vector<uint16_t> mm(nas);
    std::vector<uint32_t> ci(nas), cj(nas), ck(nas);
    std::vector<double> U(40 * nas);
    int64_t off = 0;
    for (int q = 0; q < n_add; ++q) {
      const amr_member &a = added[q];
      const int64_t nm = a.n_oct;
      std::memcpy(lv.data() + off, a.level, size_t(nm));
      std::memcpy(ci.data() + off, a.i, 4 * size_t(nm));
      std::memcpy(cj.data() + off, a.j, 4 * size_t(nm));
      std::memcpy(ck.data() + off, a.k, 4 * size_t(nm));
      for (int64_t t = 0; t < nm; ++t) mm[size_t(off + t)] = uint16_t(n_keep + q);
      for (int v = 0; v < 5; ++v)
        std::memcpy(U.data() + v * 8 * na + 8 * off, a.U + v * 8 * nm, sizeof(double) * 8 * size_t(nm));
      off += nm;
    }
    cudaError_t e = cudaMemcpyAsync(d_lvl + K, lv.data(), size_t(na), cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mem + K, mm.data(), 2 * size_t(na), cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_i + K, ci.data(), 4 * size_t(na), cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_j + K, cj.data(), 4 * size_t(na), cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_k + K, ck.data(), 4 * size_t(na), cudaMemcpyHostToDevice, h->s);
    for (int v = 0; v < 5 && e == cudaSuccess; ++v)
      e = cudaMemcpyAsync(d_U + v * 8 * n_out + 8 * K, U.data() + v * 8 * na, sizeof(double) * 8 * size_t(na),
                          cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);  // the host staging goes out of scope
    if (e != cudaSuccess) return abandon(fail(AMR_ECUDA, "amr_batch_repack: %s", cudaGetErrorString(e)));
  }
  if ((st = check_device(h, "amr_batch_repack")) != AMR_OK) return abandon(st);
  dev_free(nh, d_remap);
  dev_free(nh, d_dst);
  dev_free(nh, d_base);
  if ((st = build_mesh(nh, n_out, false, d_lvl, d_mem, d_i, d_j, d_k, nullptr, d_U, nullptr)) != AMR_OK)
    return abandon(st);
  // step counters, last time steps and error bits of the kept members; the
  // added members take their step counts
  {
    std::vector<int> nrem(size_t(nh->M)), nerr(size_t(nh->M), 0);
    std::vector<double> ndt(size_t(nh->M), 0.0);
    for (int q = 0; q < n_keep; ++q) {
      nrem[size_t(q)] = rem[size_t(keep[q])];
      nerr[size_t(q)] = merr[size_t(keep[q])];
      ndt[size_t(q)] = dt[size_t(keep[q])];
    }
    for (int q = 0; q < n_add; ++q) nrem[size_t(n_keep + q)] = added_steps[q];
    cudaError_t e = cudaMemcpyAsync(nh->mrem, nrem.data(), sizeof(int) * nh->M, cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nh->merr, nerr.data(), sizeof(int) * nh->M, cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nh->dt_dev, ndt.data(), sizeof(double) * nh->M, cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return abandon(fail(AMR_ECUDA, "amr_batch_repack: %s", cudaGetErrorString(e)));
  }
  // the handle takes the new mesh; the old one is freed
  take_over(nh, h);
  std::swap(*h, *nh);
  destroy_all(nh);
  return check_device(h, "amr_batch_repack");
}

// ---------------------------------------------------------------------------
// CIC deposition onto the levels of the selected member (Sec. 4)
// ---------------------------------------------------------------------------
__global__ void k_iota_u32(uint32_t *a, int64_t n) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) a[t] = uint32_t(t);
}

static amr_status ensure_particles(amr_mesh *h, int64_t np, bool positions) {
  const size_t es = h->elem();
  if (np > h->pcap || (positions && !h->px)) {
    for (void **b : {&h->px, &h->py, &h->pz, &h->pm}) {
      dev_free(h, *b);
      *b = nullptr;
    }
    for (uint32_t **b : {&h->plist0, &h->plist1, &h->pflag, &h->ppos, &h->ptmp}) {
      dev_free(h, *b);
      *b = nullptr;
    }
    h->pcap = 0;
    const int64_t cap = std::max<int64_t>(np, 1);
    if (positions)
      for (void **b : {&h->px, &h->py, &h->pz, &h->pm}) AMR_TRY(dev_alloc(h, b, es * size_t(cap)));
    for (uint32_t **b : {&h->plist0, &h->plist1, &h->pflag, &h->ppos}) AMR_TRY(alloc_n(h, b, cap));
    AMR_TRY(alloc_n(h, &h->ptmp, scan_tmp_size(cap)));
    h->pcap = cap;
  }
  if (!h->pcount) AMR_TRY(alloc_n(h, &h->pcount, kMaxLev + 2));
  if (h->prho_n != 8 * h->N) {
    dev_free(h, h->prho);
    h->prho = nullptr;
    AMR_TRY(dev_alloc(h, &h->prho, es * size_t(8 * std::max<int64_t>(h->N, 1))));
    h->prho_n = 8 * h->N;
  }
  return AMR_OK;
}

// the base-level table of the selected member (kept until the mesh changes:
// a regrid or repack builds a new handle)
static amr_status ensure_base_table(amr_mesh *h) {
  const Member &mb = h->mem[h->sel];
  if (h->btab && h->btab_member == h->sel) return AMR_OK;
  dev_free(h, h->btab);
  h->btab = nullptr;
  const int64_t side = int64_t(1) << (mb.lmin - 1), nb = side * side * side;
  AMR_TRY(alloc_n(h, &h->btab, nb));
  const int lo = int(mb.oct_base + mb.lo[mb.lmin]);
  launch(h, K_DEPOSIT, k_base_table, dim3(nblocks(nb)), dim3(256), (const uint64_t *)h->key, lo, nb,
         mb.lmin, h->btab);
  h->btab_member = h->sel;
  return AMR_OK;
}

template <class T>
static void deposit_levels(amr_mesh *h, int64_t np, const T *x, const T *y, const T *z, const T *m) {
  const Member &mb = h->mem[h->sel];
  const int N = int(h->N);
  cudaMemsetAsync(h->prho, 0, sizeof(T) * size_t(8 * h->N), h->s);
  std::vector<int64_t> cnt(kMaxLev + 2, 0);
  cnt[size_t(mb.lmin)] = np;
  cudaMemcpyAsync(h->pcount, cnt.data(), sizeof(int64_t) * cnt.size(), cudaMemcpyHostToDevice, h->s);
  if (np == 0) return;
  uint32_t *cur = h->plist0, *nxt = h->plist1;
  for (int l = mb.lmin; l <= mb.lmax; ++l) {
    if (l == mb.lmin)  // every particle, every stencil cell exists: the base table
      launch(h, K_DEPOSIT, k_deposit_base<T>, dim3(nblocks(np)), dim3(256), (const int32_t *)h->btab, l, np,
             x, y, z, m, static_cast<T *>(h->prho));
    else
      launch(h, K_DEPOSIT, k_deposit_level<T>, dim3(nblocks(np)), dim3(256), h->hash, h->sel, l, N, x, y,
             z, m, (const uint32_t *)cur, (const int64_t *)h->pcount, static_cast<T *>(h->prho));
    if (l == mb.lmax) break;
    if (l == mb.lmin) {
      launch(h, K_SPLIT, k_split_base<T>, dim3(nblocks(np)), dim3(256), (const int32_t *)h->btab, l,
             (const uint32_t *)h->son, x, y, z, np, h->pflag);
      launch(h, K_DEPOSIT, k_iota_u32, dim3(nblocks(np)), dim3(256), cur, np);
    } else {
      launch(h, K_SPLIT, k_split_level<T>, dim3(nblocks(np)), dim3(256), h->hash, h->sel, l, N,
             (const uint32_t *)h->son, x, y, z, (const uint32_t *)cur, (const int64_t *)h->pcount, np,
             h->pflag);
    }
    cudaMemcpyAsync(h->ppos, h->pflag, 4 * size_t(np), cudaMemcpyDeviceToDevice, h->s);
    scan_exclusive(h, h->ppos, np, h->ptmp);
    launch(h, K_SPLIT, k_compact_level, dim3(nblocks(np)), dim3(256), (const uint32_t *)cur,
           (const uint32_t *)h->pflag, (const uint32_t *)h->ppos, np, l, nxt, h->pcount);
    std::swap(cur, nxt);
  }
}

static amr_status deposit_counts(amr_mesh *h, int64_t *count) {
  if (!count) return AMR_OK;
  std::vector<int64_t> cnt(kMaxLev + 2, 0);
  CUDA_TRY(cudaMemcpyAsync(cnt.data(), h->pcount, sizeof(int64_t) * cnt.size(), cudaMemcpyDeviceToHost, h->s));
  AMR_TRY(check_device(h, "amr_cic_deposit_levels"));
  const Member &mb = h->mem[h->sel];
  for (int l = 0; l <= kMaxLev; ++l) count[l] = l >= mb.lmin && l <= mb.lmax ? cnt[size_t(l)] : 0;
  return AMR_OK;
}

extern "C" amr_status amr_cic_deposit_levels_device(amr_handle h, int64_t np, const void *x, const void *y,
                                                    const void *z, const void *m, int64_t *count) {
  if (!h) return fail(AMR_EINVAL, "amr_cic_deposit_levels_device: NULL handle");
  if (np < 0 || np >= (int64_t(1) << 32)) return fail(AMR_EINVAL, "amr_cic_deposit_levels_device: np outside [0, 2^32)");
  if (np > 0 && (!x || !y || !z || !m)) return fail(AMR_EINVAL, "amr_cic_deposit_levels_device: NULL array");
  AMR_TRY(ensure_particles(h, np, false));
  AMR_TRY(ensure_base_table(h));
  if (h->p.precision == 4)
    deposit_levels<float>(h, np, (const float *)x, (const float *)y, (const float *)z, (const float *)m);
  else
    deposit_levels<double>(h, np, (const double *)x, (const double *)y, (const double *)z, (const double *)m);
  if (h->launch_err != cudaSuccess) return check_device(h, "amr_cic_deposit_levels_device");
  return deposit_counts(h, count);
}

template <class T>
static amr_status stage_particles(amr_mesh *h, int64_t np, const double *x, const double *y,
                                  const double *z, const double *m) {
  std::vector<T> buf(size_t(std::max<int64_t>(np, 1)));
  const double *src[4] = {x, y, z, m};
  void *dst[4] = {h->px, h->py, h->pz, h->pm};
  for (int a = 0; a < 4; ++a) {
    for (int64_t t = 0; t < np; ++t) buf[size_t(t)] = T(src[a][t]);
    CUDA_TRY(cudaMemcpyAsync(dst[a], buf.data(), sizeof(T) * size_t(np), cudaMemcpyHostToDevice, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));  // buf is reused
  }
  return AMR_OK;
}

extern "C" amr_status amr_cic_deposit_levels(amr_handle h, int64_t np, const double *x, const double *y,
                                             const double *z, const double *m, int64_t *count) {
  if (!h) return fail(AMR_EINVAL, "amr_cic_deposit_levels: NULL handle");
  if (np < 0 || np >= (int64_t(1) << 32)) return fail(AMR_EINVAL, "amr_cic_deposit_levels: np outside [0, 2^32)");
  if (np > 0 && (!x || !y || !z || !m)) return fail(AMR_EINVAL, "amr_cic_deposit_levels: NULL array");
  for (int64_t t = 0; t < np; ++t)
    if (!(x[t] >= 0.0 && x[t] < 1.0 && y[t] >= 0.0 && y[t] < 1.0 && z[t] >= 0.0 && z[t] < 1.0) ||
        !std::isfinite(m[t]))
      return fail(AMR_EINVAL, "amr_cic_deposit_levels: particle %lld outside [0, 1)^3 or with a non-finite mass",
                  (long long)t);
  AMR_TRY(ensure_particles(h, np, true));
  AMR_TRY(ensure_base_table(h));
  if (np > 0) {
    if (h->p.precision == 4)
      AMR_TRY(stage_particles<float>(h, np, x, y, z, m));
    else
      AMR_TRY(stage_particles<double>(h, np, x, y, z, m));
  }
  return amr_cic_deposit_levels_device(h, np, h->px, h->py, h->pz, h->pm, count);
}

extern "C" amr_status amr_read_particle_rho(amr_handle h, int level, double *rho, int64_t cap) {
  if (!h || !rho) return fail(AMR_EINVAL, "amr_read_particle_rho: NULL argument");
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_read_particle_rho: bad level");
  if (!h->prho || h->prho_n != 8 * h->N) return fail(AMR_EINVAL, "amr_read_particle_rho: no deposition on this mesh");
  const Member &mb = h->mem[h->sel];
  const int64_t lo = mb.oct_base + mb.lo[level], nl = mb.lo[level + 1] - mb.lo[level];
  if (cap < nl) return fail(AMR_EINVAL, "amr_read_particle_rho: cap %lld < %lld octs", (long long)cap, (long long)nl);
  if (nl == 0) return AMR_OK;
  if (h->p.precision == 8) {
    CUDA_TRY(cudaMemcpyAsync(rho, static_cast<const double *>(h->prho) + 8 * lo, sizeof(double) * 8 * nl,
                             cudaMemcpyDeviceToHost, h->s));
  } else {
    std::vector<float> f(size_t(8 * nl));
    CUDA_TRY(cudaMemcpyAsync(f.data(), static_cast<const float *>(h->prho) + 8 * lo, sizeof(float) * 8 * nl,
                             cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    for (int64_t t = 0; t < 8 * nl; ++t) rho[t] = double(f[size_t(t)]);
  }
  return check_device(h, "amr_read_particle_rho");
}

// FP64 conservation totals of the selected member's leaf cells (one level, or
// every level added in ascending order); fixed grid per level size, so the
// order of every addition is fixed.
extern "C" amr_status amr_totals(amr_handle h, int level, double *out) {
  if (!h || !out) return fail(AMR_EINVAL, "amr_totals: NULL argument");
  if (level < 0 || level > kMaxLev) return fail(AMR_EINVAL, "amr_totals: level %d outside [0, %d]", level, kMaxLev);
  const Member &m = h->mem[h->sel];
  const int l0 = level ? level : m.lmin, l1 = level ? level : m.lmax;
  constexpr int kMaxG = 1024;
  double *buf = nullptr;
  AMR_TRY(alloc_n(h, &buf, 5 * kMaxG + 5 * (kMaxLev + 1) + 5));
  double *partial = buf, *lev = buf + 5 * kMaxG, *dout = lev + 5 * (kMaxLev + 1);
  for (int l = l0; l <= l1; ++l) {
    const int64_t lo = m.oct_base + m.lo[l], nl = m.lo[l + 1] - m.lo[l];
    const int64_t n = 8 * nl;
    const int G = int(std::max<int64_t>(1, std::min<int64_t>(kMaxG, (n + 2047) / 2048)));
    const int64_t chunk = std::max<int64_t>(256, ((n + G - 1) / G + 255) / 256 * 256);
    if (h->p.precision == 4)
      launch(h, K_TOTALS, k_totals<float>, dim3(unsigned(G)), dim3(256), (const float *)h->U, h->S,
             (const uint32_t *)h->son, 8 * lo, n, chunk, partial, G);
    else
      launch(h, K_TOTALS, k_totals<double>, dim3(unsigned(G)), dim3(256), (const double *)h->U, h->S,
             (const uint32_t *)h->son, 8 * lo, n, chunk, partial, G);
    launch(h, K_TOTALS, k_totals_sum, dim3(1), dim3(32), (const double *)partial, G, l, lev,
           int(level == 0 && l == l1), l0, l1, dout);
  }
  cudaError_t e = cudaMemcpyAsync(out, dout, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  dev_free(h, buf);
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_totals: %s", cudaGetErrorString(e));
  return check_device(h, "amr_totals");
}

extern "C" amr_status amr_read_reflux(amr_handle h, int level, double *R, int64_t cap) {
  if (!h || !R) return fail(AMR_EINVAL, "amr_read_reflux: NULL argument");
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_read_reflux: bad level");
  const Member &m = h->mem[h->sel];
  const int64_t lo = m.oct_base + m.lo[level], nl = m.lo[level + 1] - m.lo[level];
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
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_write: bad level");
  const Member &m = h->mem[h->sel];
  const int64_t lo = m.oct_base + m.lo[level], nl = m.lo[level + 1] - m.lo[level];
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
// introspection (selected member)
// ---------------------------------------------------------------------------
extern "C" amr_status amr_lookup(amr_handle h, int64_t n, const uint64_t *keys, int64_t *idx_out) {
  if (!h || (n > 0 && (!keys || !idx_out))) return fail(AMR_EINVAL, "amr_lookup: NULL argument");
  if (n <= 0) return AMR_OK;
  const Member &m = h->mem[h->sel];
  std::vector<uint64_t> ik(n);
  for (int64_t t = 0; t < n; ++t) {
    const uint64_t k = keys[t];
    const int l = int(k >> 60);
    const uint32_t x = uint32_t(k >> 40) & 0xFFFFF, y = uint32_t(k >> 20) & 0xFFFFF, z = uint32_t(k) & 0xFFFFF;
    // coordinates beyond 15 bits cannot be in any mesh: a key that matches nothing
    ik[t] = (x >> 15 || y >> 15 || z >> 15) ? ~0ull - 1 : ikey(h->sel, l, x, y, z);
  }
  uint64_t *dk;
  int64_t *dout;
  AMR_TRY(upload(h, &dk, ik));
  AMR_TRY(alloc_n(h, &dout, n));
  launch(h, K_LOOKUP, k_lookup, dim3(nblocks(8 * n)), dim3(256), h->hash, (const uint64_t *)dk, n,
         h->N, dout);
  CUDA_TRY(cudaMemcpyAsync(idx_out, dout, 8 * n, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  dev_free(h, dk);
  dev_free(h, dout);
  for (int64_t t = 0; t < n; ++t)
    if (idx_out[t] >= 0) idx_out[t] -= m.oct_base;
  return check_device(h, "amr_lookup");
}

extern "C" amr_status amr_read_index(amr_handle h, int level, int64_t *nbr, uint8_t *split,
                                     int64_t cap) {
  if (!h) return fail(AMR_EINVAL, "amr_read_index: NULL handle");
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_read_index: bad level");
  const Member &m = h->mem[h->sel];
  const int64_t lo = m.oct_base + m.lo[level], nl = m.lo[level + 1] - m.lo[level];
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
        nbr[27 * t + e] = x < h->N ? x - m.oct_base : -(1 + (x - h->N - m.cache_base));
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
  if (!level_ok(level)) return fail(AMR_EINVAL, "amr_read_cache: bad level");
  const Member &m = h->mem[h->sel];
  const int64_t c0 = m.cache_base + m.clo[level], nc = m.clo[level + 1] - m.clo[level];
  if (n_out) *n_out = nc;
  if (first_out) *first_out = m.clo[level];
  if ((keys || Ug) && cap < nc) return fail(AMR_EINVAL, "amr_read_cache: cap too small");
  if (keys && nc) {
    CUDA_TRY(cudaMemcpyAsync(keys, h->ckey + c0, 8 * nc, cudaMemcpyDeviceToHost, h->s));
    CUDA_TRY(cudaStreamSynchronize(h->s));
    for (int64_t t = 0; t < nc; ++t) keys[t] = external_key(keys[t]);
  }
  if (Ug) AMR_TRY(rows_to_host(h, h->U, h->S, 8 * (h->N + c0), 8 * nc, Ug));
  return check_device(h, "amr_read_cache");
}

extern "C" amr_status amr_get_info(amr_handle h, amr_info *info) {
  if (!h || !info) return fail(AMR_EINVAL, "amr_get_info: NULL argument");
  std::memset(info, 0, sizeof *info);
  info->n_oct = h->N;
  info->n_cache = h->NC;
  const Member &m = h->mem[h->sel];
  for (auto &q : h->mem) {
    for (int l = 0; l <= kMaxLev; ++l) {
      info->n_leaf_cells += q.leaf[l];
      if (q.lo[l + 1] > q.lo[l] && l >= q.lmin) info->work_per_step += q.leaf[l] << (l - q.lmin);
    }
  }
  for (int l = 0; l <= kMaxLev; ++l) {
    info->level_octs[l] = m.lo[l + 1] - m.lo[l];
    info->level_cache[l] = m.clo[l + 1] - m.clo[l];
    info->level_leaf_cells[l] = m.leaf[l];
  }
  info->device_bytes = int64_t(h->bytes);
  info->cached_bytes = h->cache ? int64_t(h->cache->bytes) : 0;
  info->kernel_launches = h->launches;
  info->graph_launches = h->graph_launches;
  info->hash_capacity = int64_t(h->hcap);
  info->precision = h->p.precision;
  info->n_members = h->M;
  info->member = h->sel;
  info->phases = int(h->phases.size());
  info->tile = h->tile_size;
  info->schedule = h->persistent ? 1 : 0;
  info->nsubgrid = h->nsub;
  info->planar = h->planar ? 1 : 0;
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

// ---------------------------------------------------------------------------
// FMA rate of this GPU (the denominator of the arithmetic-bound rooflines)
// ---------------------------------------------------------------------------
// Every thread runs 8 independent chains of a <- a x + y for `iters` steps
// (enough independent work per warp to hide the pipe latency); x and y come
// from the arguments, so nothing folds.  One thread writes the sum.
template <class T>
__global__ void k_fma_chains(T x, T y, int iters, T *out) {
  T a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = T(threadIdx.x + q);
  for (int t = 0; t < iters; ++t)
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], x, y);
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == T(-1.2345)) *out = s;  // never true for these inputs; keeps the chains
}

template <class T>
static amr_status fma_rate(int device, int iters, double *flops) {
  CUDA_TRY(cudaSetDevice(device));
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  cudaStream_t s;
  CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  T *out = nullptr;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaMallocAsync(&out, sizeof(T), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const dim3 grid(unsigned(8 * sms)), block(256);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<grid, block, 0, s>>>(T(0.999999), T(1e-7), iters, out);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch warms up
  }
  cudaFreeAsync(out, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return fail(AMR_ECUDA, "amr_fma_rate: %s", cudaGetErrorString(e));
  *flops = 2.0 * 8.0 * double(iters) * double(grid.x) * double(block.x) / (double(best) * 1e-3);
  return AMR_OK;
}

extern "C" amr_status amr_fma_rate(int device, int precision, double *flops) {
  if (!flops) return fail(AMR_EINVAL, "amr_fma_rate: NULL argument");
  if (precision == 8) return fma_rate<double>(device, 2048, flops);
  if (precision == 4) return fma_rate<float>(device, 65536, flops);
  return fail(AMR_EINVAL, "amr_fma_rate: precision must be 4 or 8");
}
