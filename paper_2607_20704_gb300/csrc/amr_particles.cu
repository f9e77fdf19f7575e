// amr_particles.cu -- particle handle of the C ABI in amr_particles.h: CIC
// mass deposition on a periodic n^3 grid (Sec. 4), the source-cell Hilbert
// sort that precedes it, and their host drivers.  Every step runs in the
// kernels of cic_kernels.cuh on the handle's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "amr_particles.h"
#include "cic_kernels.cuh"

void amr_set_error_text(const char *text);

using namespace amr;

namespace {

enum PKid {
  P_KEYS, P_SORT_HIST, P_SORT_SCAN, P_SORT_SCATTER, P_GATHER, P_ZERO, P_CIC_ATOMIC,
  P_SEG_HEADS, P_SEG_SCAN, P_SEG_STARTS, P_SEG_PARTIAL, P_SEG_CARRY, P_SEG_GATHER, P_CONVERT, P_COUNT
};
const char *const kPartKernelNames[P_COUNT] = {
    "part_keys", "psort_hist", "psort_scan", "psort_scatter", "part_gather", "grid_zero",
    "cic_atomic", "seg_heads", "seg_scan", "seg_starts", "seg_partial", "seg_carry", "seg_gather", "convert"};

amr_status set_error(amr_status s, const std::string &msg) {
  amr_set_error_text(msg.c_str());
  return s;
}

struct Timed {
  int kid;
  cudaEvent_t e0, e1;
};

}  // namespace

struct amr_particles {
  int n = 0, bits = 0, precision = 8;
  size_t esize = 8;
  cudaStream_t s = nullptr;
  int64_t np = 0;
  // particle arrays (current order) and the gather targets of the sort
  void *x = nullptr, *y = nullptr, *z = nullptr, *m = nullptr;
  void *x2 = nullptr, *y2 = nullptr, *z2 = nullptr, *m2 = nullptr;
  uint32_t *id = nullptr, *id2 = nullptr;
  // sort: keys and values, their alternates, the digit table and scan scratch
  uint32_t *key = nullptr, *val = nullptr, *key2 = nullptr, *val2 = nullptr;
  uint32_t *table = nullptr, *scan_tmp = nullptr;
  uint32_t *sorted_key = nullptr;  // source-cell keys of the current order (after a sort)
  void *rho = nullptr;
  // segment deposition (allocated on first use)
  uint32_t *flag = nullptr, *start = nullptr, *nseg = nullptr;
  void *sums = nullptr, *carry = nullptr;
  int32_t *cellmap = nullptr;
  double *stage = nullptr;  // device staging of host doubles (FP32 handles)
  bool sorted = false;
  int64_t device_bytes = 0, launches = 0;
  // timing
  bool timing = false;
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> pool;
  double kernel_ms[P_COUNT] = {};
  int64_t kernel_n[P_COUNT] = {};
  cudaError_t launch_err = cudaSuccess;
  int launch_err_kid = 0;
};

namespace {

inline unsigned nblocks(int64_t n, int b = 256) { return unsigned((n + b - 1) / b); }

cudaEvent_t take_event(amr_particles *h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

template <class... KArgs, class... Args>
void launch(amr_particles *h, int kid, void (*kern)(KArgs...), dim3 grid, dim3 block, Args &&...args) {
  if (grid.x == 0) return;
  cudaEvent_t e0 = nullptr;
  if (h->timing) {
    e0 = take_event(h);
    cudaEventRecord(e0, h->s);
  }
  kern<<<grid, block, 0, h->s>>>(std::forward<Args>(args)...);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess && h->launch_err == cudaSuccess) {
    h->launch_err = le;
    h->launch_err_kid = kid;
  }
  if (h->timing) {
    cudaEvent_t e1 = take_event(h);
    cudaEventRecord(e1, h->s);
    h->pending.push_back({kid, e0, e1});
  }
  ++h->launches;
}

// memset as a timed step
void zero(amr_particles *h, int kid, void *p, int byte, size_t bytes) {
  cudaEvent_t e0 = nullptr;
  if (h->timing) {
    e0 = take_event(h);
    cudaEventRecord(e0, h->s);
  }
  cudaMemsetAsync(p, byte, bytes, h->s);
  if (h->timing) {
    cudaEvent_t e1 = take_event(h);
    cudaEventRecord(e1, h->s);
    h->pending.push_back({kid, e0, e1});
  }
}

amr_status launch_status(amr_particles *h, const char *where) {
  if (h->launch_err != cudaSuccess) {
    const cudaError_t e = h->launch_err;
    h->launch_err = cudaSuccess;
    return set_error(AMR_ECUDA, std::string(where) + ": launch of " + kPartKernelNames[h->launch_err_kid] +
                                    " failed: " + cudaGetErrorString(e));
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(AMR_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return AMR_OK;
}

amr_status cuda_status(cudaError_t e, const char *where) {
  if (e == cudaSuccess) return AMR_OK;
  return set_error(e == cudaErrorMemoryAllocation ? AMR_ENOMEM : AMR_ECUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

template <class P>
cudaError_t dalloc(amr_particles *h, P **p, size_t bytes) {
  void *q = nullptr;
  const cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  *p = static_cast<P *>(q);
  h->device_bytes += int64_t(bytes ? bytes : 16);
  return cudaSuccess;
}

void dfree(void *p) {
  if (p) cudaFree(p);
}

int64_t scan_tmp_len(int64_t n) {
  int64_t tot = 0;
  while (n > 1) {
    n = (n + kScanItems - 1) / kScanItems;
    tot += (n + 255) & ~int64_t(255);
  }
  return tot + 256;
}

void scan_exclusive(amr_particles *h, int kid, uint32_t *data, int64_t n, uint32_t *tmp) {
  const int64_t nb = (n + kScanItems - 1) / kScanItems;
  launch(h, kid, k_scan_block, dim3(unsigned(nb)), dim3(256), data, n, tmp);
  if (nb > 1 && nb <= kScanFlat) {
    launch(h, kid, k_scan_add_flat, dim3(unsigned(nb - 1)), dim3(256), data, n, (const uint32_t *)tmp);
  } else if (nb > 1) {
    scan_exclusive(h, kid, tmp, nb, tmp + ((nb + 255) & ~int64_t(255)));
    launch(h, kid, k_scan_add, dim3(nblocks(n)), dim3(256), data, n, (const uint32_t *)tmp);
  }
}

// host checks of one upload
amr_status check_host(int64_t np, const double *x, const double *y, const double *z, const double *m,
                      const char *where) {
  if (np > 0 && (!x || !y || !z || !m)) return set_error(AMR_EINVAL, std::string(where) + ": NULL array");
  for (int64_t t = 0; t < np; ++t) {
    const double a = x[t], b = y[t], c = z[t];
    if (!(a >= 0.0 && a < 1.0) || !(b >= 0.0 && b < 1.0) || !(c >= 0.0 && c < 1.0))
      return set_error(AMR_EINVAL, std::string(where) + ": particle " + std::to_string(t) +
                                       " lies outside [0, 1)^3");
    if (!std::isfinite(m[t]))
      return set_error(AMR_EINVAL, std::string(where) + ": particle " + std::to_string(t) + " has a non-finite mass");
  }
  return AMR_OK;
}

// host doubles -> device arrays of the handle's precision
amr_status upload(amr_particles *h, const double *x, const double *y, const double *z, const double *m,
                  const char *where) {
  const double *src[4] = {x, y, z, m};
  void *dst[4] = {h->x, h->y, h->z, h->m};
  const size_t bytes = size_t(h->np) * sizeof(double);
  for (int a = 0; a < 4 && h->np > 0; ++a) {
    if (h->precision == 8) {
      if (auto st = cuda_status(cudaMemcpyAsync(dst[a], src[a], bytes, cudaMemcpyHostToDevice, h->s), where))
        return st;
    } else {
      if (auto st = cuda_status(cudaMemcpyAsync(h->stage, src[a], bytes, cudaMemcpyHostToDevice, h->s), where))
        return st;
      launch(h, P_CONVERT, k_from_double<float>, dim3(nblocks(h->np)), dim3(256), h->np,
             (const double *)h->stage, static_cast<float *>(dst[a]));
    }
  }
  if (auto st = cuda_status(cudaStreamSynchronize(h->s), where)) return st;
  return launch_status(h, where);
}

void release(amr_particles *h) {
  for (void *p : {h->x, h->y, h->z, h->m, h->x2, h->y2, h->z2, h->m2, (void *)h->id, (void *)h->id2,
                  (void *)h->key, (void *)h->val, (void *)h->key2, (void *)h->val2, (void *)h->table,
                  (void *)h->scan_tmp, h->rho, (void *)h->flag, (void *)h->start, (void *)h->nseg,
                  h->sums, h->carry, (void *)h->cellmap, (void *)h->stage})
    dfree(p);
  for (auto &t : h->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  delete h;
}

int64_t cells(const amr_particles *h) { return int64_t(h->n) * h->n * h->n; }
int64_t ntiles(const amr_particles *h) { return (h->np + kSortTile - 1) / kSortTile; }
int64_t ngroups(const amr_particles *h) { return (h->np + 31) / 32; }

template <class T>
CicGrid<T> grid_of(const amr_particles *h) {
  return CicGrid<T>{h->n, h->bits, T(h->n), T(double(cells(h)))};
}

template <class T>
void sort_impl(amr_particles *h) {
  const int64_t np = h->np, nt = ntiles(h);
  const CicGrid<T> g = grid_of<T>(h);
  const T *px = (const T *)h->x, *py = (const T *)h->y, *pz = (const T *)h->z;
  const dim3 kg(nblocks(np)), kb256(256);
  switch (h->bits) {
    case 1: launch(h, P_KEYS, k_part_keys<T, 1>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 2: launch(h, P_KEYS, k_part_keys<T, 2>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 3: launch(h, P_KEYS, k_part_keys<T, 3>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 4: launch(h, P_KEYS, k_part_keys<T, 4>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 5: launch(h, P_KEYS, k_part_keys<T, 5>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 6: launch(h, P_KEYS, k_part_keys<T, 6>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 7: launch(h, P_KEYS, k_part_keys<T, 7>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 8: launch(h, P_KEYS, k_part_keys<T, 8>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    case 9: launch(h, P_KEYS, k_part_keys<T, 9>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
    default: launch(h, P_KEYS, k_part_keys<T, 10>, kg, kb256, np, g, px, py, pz, h->key, h->val); break;
  }
  uint32_t *ka = h->key, *kb = h->key2, *va = h->val, *vb = h->val2;
  // passes of equal width, at most 8 bits each (27-bit keys of a 512^3 grid:
  // 7, 7, 7, 6): fewer digits per pass keep each digit's run in a tile longer,
  // so the scatter writes stay coalesced
  const int total = 3 * h->bits;
  const int passes = (total + 7) / 8, width = (total + passes - 1) / passes;
  for (int shift = 0; shift < total; shift += width) {
    const int nbits = total - shift < width ? total - shift : width;
    const int64_t len = (int64_t(1) << nbits) * nt;
    const int ndig = 1 << nbits;
    const int64_t nch = (nt + kScanChunk - 1) / kScanChunk;
    uint32_t *pref = h->table + len, *base = pref + len, *dbase = base + int64_t(ndig) * nch;
    launch(h, P_SORT_HIST, k_psort_hist, dim3(unsigned(nt)), dim3(kSortThreads), (const uint32_t *)ka, np,
           shift, nbits, h->table, nt);
    launch(h, P_SORT_SCAN, k_psort_chunks, dim3(unsigned(nch)), dim3(kSortThreads), (const uint32_t *)h->table,
           nt, ndig, pref, base);
    launch(h, P_SORT_SCAN, k_psort_digit_scan, dim3(unsigned(ndig)), dim3(kSortThreads), base, nch, ndig, dbase);
    launch(h, P_SORT_SCAN, k_psort_digit_base, dim3(1), dim3(kSortThreads), dbase, ndig);
    launch(h, P_SORT_SCATTER, k_psort_scatter, dim3(unsigned(nt)), dim3(kSortThreads), (const uint32_t *)ka,
           (const uint32_t *)va, kb, vb, np, shift, nbits, (const uint32_t *)h->table, (const uint32_t *)pref,
           (const uint32_t *)base, (const uint32_t *)dbase);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  launch(h, P_GATHER, k_part_gather<T>, dim3(nblocks(np)), dim3(256), np, (const uint32_t *)va,
         (const T *)h->x, (const T *)h->y, (const T *)h->z, (const T *)h->m, (const uint32_t *)h->id,
         (T *)h->x2, (T *)h->y2, (T *)h->z2, (T *)h->m2, h->id2);
  std::swap(h->x, h->x2);
  std::swap(h->y, h->y2);
  std::swap(h->z, h->z2);
  std::swap(h->m, h->m2);
  std::swap(h->id, h->id2);
  h->sorted_key = ka;
}

template <class T>
void deposit_atomic(amr_particles *h) {
  zero(h, P_ZERO, h->rho, 0, size_t(cells(h)) * sizeof(T));
  launch(h, P_CIC_ATOMIC, k_cic_atomic<T>, dim3(nblocks(h->np)), dim3(256), h->np, grid_of<T>(h),
         (const T *)h->x, (const T *)h->y, (const T *)h->z, (const T *)h->m, (T *)h->rho);
}

template <class T>
void deposit_segment(amr_particles *h) {
  const int64_t np = h->np, cap = np > 0 ? np : 1, ng = ngroups(h) > 0 ? ngroups(h) : 1;
  zero(h, P_ZERO, h->cellmap, 0xFF, size_t(cells(h)) * sizeof(int32_t));
  zero(h, P_ZERO, h->nseg, 0, sizeof(uint32_t));
  if (np > 0) {
    launch(h, P_SEG_HEADS, k_seg_heads, dim3(nblocks(np)), dim3(256), np, (const uint32_t *)h->sorted_key,
           h->flag);
    scan_exclusive(h, P_SEG_SCAN, h->flag, np, h->scan_tmp);
    launch(h, P_SEG_STARTS, k_seg_starts, dim3(nblocks(np)), dim3(256), np, (const uint32_t *)h->sorted_key,
           (const uint32_t *)h->flag, h->start, h->nseg);
    launch(h, P_SEG_PARTIAL, k_seg_partial<T>, dim3(nblocks(np)), dim3(256), np, grid_of<T>(h),
           (const uint32_t *)h->sorted_key, (const uint32_t *)h->flag, (const T *)h->x, (const T *)h->y,
           (const T *)h->z, (const T *)h->m, cap, ng, (T *)h->sums, (T *)h->carry, h->cellmap);
    launch(h, P_SEG_CARRY, k_seg_carry<T>, dim3(nblocks(np)), dim3(256), (const uint32_t *)h->nseg,
           (const uint32_t *)h->start, cap, ng, (const T *)h->carry, (T *)h->sums);
  }
  launch(h, P_SEG_GATHER, k_seg_gather<T>, dim3(nblocks(cells(h))), dim3(256), h->n, cap,
         (const int32_t *)h->cellmap, (const T *)h->sums, (T *)h->rho);
}

}  // namespace

extern "C" amr_status amr_part_create(const amr_part_params *p, int64_t np, const double *x, const double *y,
                                      const double *z, const double *m, amr_part_handle *out) {
  if (!p || !out) return set_error(AMR_EINVAL, "amr_part_create: NULL argument");
  *out = nullptr;
  const int n = p->n;
  if (n < 2 || n > 1024 || (n & (n - 1)))
    return set_error(AMR_EINVAL, "amr_part_create: n must be a power of two in 2..1024");
  if (p->precision != 8 && p->precision != 4)
    return set_error(AMR_EINVAL, "amr_part_create: precision must be 4 or 8");
  if (np < 0 || np >= (int64_t(1) << 32) - 1)
    return set_error(AMR_EINVAL, "amr_part_create: np must be in 0..2^32-2");
  if (auto st = check_host(np, x, y, z, m, "amr_part_create")) return st;
  amr_particles *h = new amr_particles();
  h->n = n;
  h->bits = 0;
  while ((1 << h->bits) < n) ++h->bits;
  h->precision = p->precision;
  h->esize = p->precision == 8 ? 8 : 4;
  h->s = static_cast<cudaStream_t>(p->stream);
  h->np = np;
  const size_t pb = size_t(np) * h->esize, ib = size_t(np) * 4;
  const int64_t nt = (np + kSortTile - 1) / kSortTile;
  // tile counts, their chunk prefixes, the chunk bases and the digit bases
  const int64_t tlen =
      2 * int64_t(kSortBins) * nt + int64_t(kSortBins) * ((nt + kScanChunk - 1) / kScanChunk) + kSortBins + 1;
  cudaError_t e = cudaSuccess;
  for (void **q : {&h->x, &h->y, &h->z, &h->m, &h->x2, &h->y2, &h->z2, &h->m2})
    if (e == cudaSuccess) e = dalloc(h, q, pb);
  for (uint32_t **q : {&h->id, &h->id2, &h->key, &h->val, &h->key2, &h->val2})
    if (e == cudaSuccess) e = dalloc(h, q, ib);
  if (e == cudaSuccess) e = dalloc(h, &h->table, size_t(tlen) * 4);
  if (e == cudaSuccess) e = dalloc(h, &h->scan_tmp, size_t(scan_tmp_len(tlen > np ? tlen : np)) * 4);
  if (e == cudaSuccess) e = dalloc(h, &h->rho, size_t(cells(h)) * h->esize);
  if (e == cudaSuccess && h->precision == 4) e = dalloc(h, &h->stage, size_t(np) * sizeof(double));
  if (e != cudaSuccess) {
    const amr_status st = cuda_status(e, "amr_part_create");
    release(h);
    return st;
  }
  if (np > 0) launch(h, P_CONVERT, k_iota, dim3(nblocks(np)), dim3(256), np, h->id);
  zero(h, P_ZERO, h->rho, 0, size_t(cells(h)) * h->esize);
  if (auto st = upload(h, x, y, z, m, "amr_part_create")) {
    release(h);
    return st;
  }
  *out = h;
  return AMR_OK;
}

extern "C" amr_status amr_part_write(amr_part_handle h, const double *x, const double *y, const double *z,
                                     const double *m) {
  if (!h) return set_error(AMR_EINVAL, "amr_part_write: NULL handle");
  if (auto st = check_host(h->np, x, y, z, m, "amr_part_write")) return st;
  h->sorted = false;
  return upload(h, x, y, z, m, "amr_part_write");
}

extern "C" amr_status amr_part_sort(amr_part_handle h) {
  if (!h) return set_error(AMR_EINVAL, "amr_part_sort: NULL handle");
  if (h->np > 0) {
    if (h->precision == 8)
      sort_impl<double>(h);
    else
      sort_impl<float>(h);
  }
  h->sorted = true;
  return launch_status(h, "amr_part_sort");
}

extern "C" amr_status amr_cic_deposit(amr_part_handle h, int algo) {
  if (!h) return set_error(AMR_EINVAL, "amr_cic_deposit: NULL handle");
  if (algo != AMR_CIC_ATOMIC && algo != AMR_CIC_SEGMENT)
    return set_error(AMR_EINVAL, "amr_cic_deposit: algo must be AMR_CIC_ATOMIC or AMR_CIC_SEGMENT");
  if (algo == AMR_CIC_ATOMIC) {
    if (h->precision == 8)
      deposit_atomic<double>(h);
    else
      deposit_atomic<float>(h);
    return launch_status(h, "amr_cic_deposit");
  }
  if (!h->sorted)
    return set_error(AMR_EINVAL, "amr_cic_deposit: the segment algorithm needs amr_part_sort after the last write");
  if (!h->sums) {
    const size_t cap = size_t(h->np > 0 ? h->np : 1);
    cudaError_t e = dalloc(h, &h->flag, cap * 4);
    if (e == cudaSuccess) e = dalloc(h, &h->start, (cap + 1) * 4);
    if (e == cudaSuccess) e = dalloc(h, &h->nseg, 4);
    if (e == cudaSuccess) e = dalloc(h, &h->cellmap, size_t(cells(h)) * 4);
    if (e == cudaSuccess) e = dalloc(h, &h->sums, 8 * cap * h->esize);
    if (e == cudaSuccess) e = dalloc(h, &h->carry, 8 * size_t(ngroups(h) > 0 ? ngroups(h) : 1) * h->esize);
    if (e != cudaSuccess) {
      for (void **q : {(void **)&h->flag, (void **)&h->start, (void **)&h->nseg, (void **)&h->cellmap, &h->sums,
                       &h->carry}) {
        dfree(*q);
        *q = nullptr;
      }
      return cuda_status(e, "amr_cic_deposit");
    }
  }
  if (h->precision == 8)
    deposit_segment<double>(h);
  else
    deposit_segment<float>(h);
  return launch_status(h, "amr_cic_deposit");
}

extern "C" amr_status amr_part_read_rho(amr_part_handle h, double *rho, int64_t cap) {
  if (!h || !rho) return set_error(AMR_EINVAL, "amr_part_read_rho: NULL argument");
  const int64_t nc = cells(h);
  if (cap < nc) return set_error(AMR_EINVAL, "amr_part_read_rho: cap < n^3");
  const char *where = "amr_part_read_rho";
  if (h->precision == 8) {
    if (auto st = cuda_status(cudaMemcpyAsync(rho, h->rho, size_t(nc) * 8, cudaMemcpyDeviceToHost, h->s), where))
      return st;
  } else {
    double *tmp = nullptr;
    if (auto st = cuda_status(cudaMalloc(&tmp, size_t(nc) * 8), where)) return st;
    launch(h, P_CONVERT, k_to_double<float>, dim3(nblocks(nc)), dim3(256), nc, (const float *)h->rho, tmp);
    cudaMemcpyAsync(rho, tmp, size_t(nc) * 8, cudaMemcpyDeviceToHost, h->s);
    cudaStreamSynchronize(h->s);
    cudaFree(tmp);
  }
  if (auto st = cuda_status(cudaStreamSynchronize(h->s), where)) return st;
  return launch_status(h, where);
}

extern "C" amr_status amr_part_read(amr_part_handle h, double *x, double *y, double *z, double *m, int64_t *id,
                                    int64_t cap) {
  if (!h) return set_error(AMR_EINVAL, "amr_part_read: NULL handle");
  const int64_t np = h->np;
  if ((x || y || z || m || id) && cap < np) return set_error(AMR_EINVAL, "amr_part_read: cap < np");
  const char *where = "amr_part_read";
  if (auto st = cuda_status(cudaStreamSynchronize(h->s), where)) return st;
  if (np == 0) return AMR_OK;
  double *dst[4] = {x, y, z, m};
  const void *src[4] = {h->x, h->y, h->z, h->m};
  double *tmp = nullptr;
  if (h->precision == 4)
    if (auto st = cuda_status(cudaMalloc(&tmp, size_t(np) * 8), where)) return st;
  for (int a = 0; a < 4; ++a) {
    if (!dst[a]) continue;
    if (h->precision == 8) {
      cudaMemcpyAsync(dst[a], src[a], size_t(np) * 8, cudaMemcpyDeviceToHost, h->s);
    } else {
      launch(h, P_CONVERT, k_to_double<float>, dim3(nblocks(np)), dim3(256), np, (const float *)src[a], tmp);
      cudaMemcpyAsync(dst[a], tmp, size_t(np) * 8, cudaMemcpyDeviceToHost, h->s);
      cudaStreamSynchronize(h->s);
    }
  }
  if (id) {
    std::vector<uint32_t> ids(static_cast<size_t>(np));
    cudaMemcpyAsync(ids.data(), h->id, size_t(np) * 4, cudaMemcpyDeviceToHost, h->s);
    cudaStreamSynchronize(h->s);
    for (int64_t t = 0; t < np; ++t) id[t] = int64_t(ids[size_t(t)]);
  }
  const cudaError_t e = cudaStreamSynchronize(h->s);
  if (tmp) cudaFree(tmp);
  if (auto st = cuda_status(e, where)) return st;
  return launch_status(h, where);
}

extern "C" amr_status amr_part_device(amr_part_handle h, void **rho, void **x, void **y, void **z, void **m) {
  if (!h) return set_error(AMR_EINVAL, "amr_part_device: NULL handle");
  if (rho) *rho = h->rho;
  if (x) *x = h->x;
  if (y) *y = h->y;
  if (z) *z = h->z;
  if (m) *m = h->m;
  return AMR_OK;
}

extern "C" amr_status amr_part_get_info(amr_part_handle h, amr_part_info *info) {
  if (!h || !info) return set_error(AMR_EINVAL, "amr_part_get_info: NULL argument");
  info->np = h->np;
  info->n = h->n;
  info->precision = h->precision;
  info->sorted = h->sorted ? 1 : 0;
  info->n_segments = 0;
  if (h->nseg) {
    uint32_t s = 0;
    if (auto st = cuda_status(cudaMemcpyAsync(&s, h->nseg, 4, cudaMemcpyDeviceToHost, h->s), "amr_part_get_info"))
      return st;
    if (auto st = cuda_status(cudaStreamSynchronize(h->s), "amr_part_get_info")) return st;
    info->n_segments = s;
  }
  info->device_bytes = h->device_bytes;
  info->kernel_launches = h->launches;
  return AMR_OK;
}

extern "C" amr_status amr_part_set_timing(amr_part_handle h, int on) {
  if (!h) return set_error(AMR_EINVAL, "amr_part_set_timing: NULL handle");
  h->timing = on != 0;
  return AMR_OK;
}

extern "C" amr_status amr_part_read_timing(amr_part_handle h, int n, double *ms, int64_t *launches) {
  if (!h) return set_error(AMR_EINVAL, "amr_part_read_timing: NULL handle");
  if (auto st = cuda_status(cudaStreamSynchronize(h->s), "amr_part_read_timing")) return st;
  for (auto &t : h->pending) {
    float x = 0.f;
    cudaEventElapsedTime(&x, t.e0, t.e1);
    h->kernel_ms[t.kid] += x;
    h->kernel_n[t.kid] += 1;
    h->pool.push_back(t.e0);
    h->pool.push_back(t.e1);
  }
  h->pending.clear();
  for (int t = 0; t < n && t < P_COUNT; ++t) {
    if (ms) ms[t] = h->kernel_ms[t];
    if (launches) launches[t] = h->kernel_n[t];
  }
  return AMR_OK;
}

extern "C" const char *amr_part_kernel_name(int t) { return t >= 0 && t < P_COUNT ? kPartKernelNames[t] : nullptr; }

extern "C" amr_status amr_part_destroy(amr_part_handle h) {
  if (!h) return AMR_OK;
  cudaStreamSynchronize(h->s);
  release(h);
  return AMR_OK;
}
