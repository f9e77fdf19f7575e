/*
 * amr_particles.h -- C ABI of the particle mass deposition of the GB300
 * library: Cloud-in-Cell (CIC) deposition of particle masses onto a periodic
 * uniform grid (arXiv 2607.20704, Sec. 4, "Mass Deposition"), with the
 * particle sort by the Hilbert key of the source cells that precedes it
 * (Sec. 4, sorting of the particle arrays).
 *
 * One handle owns np particles resident in device memory -- positions
 * (x, y, z) in the periodic unit box [0, 1)^3, masses m, and the particle
 * identifiers 0..np-1 given by the order of the arrays at creation -- and one
 * periodic grid of n^3 cells of size dx = 1/n (n a power of two, 2..1024)
 * holding the density rho of the last deposition, rho[i + n (j + n k)] for
 * the cell centred at ((i + 1/2) dx, (j + 1/2) dx, (k + 1/2) dx).
 *
 * Deposition (CIC, Sec. 4).  Along each axis s = x n - 1/2, i0 = floor(s),
 * f = s - i0; the particle's mass is shared by the 2^3 cells
 * (i0 + cx, j0 + cy, k0 + cz) (periodic) with weights
 * wx wy wz, wx = 1 - f for cx = 0 and f for cx = 1, and
 *   rho(cell) = sum over particles of m wx wy wz / dx^3.
 * The cell (i0, j0, k0) is the particle's source cell (the half-cell-shifted
 * convention of the paper's medium and small kernels).
 *
 * Precision: amr_part_params.precision = 8 holds positions, masses and rho in
 * FP64; 4 holds them in FP32 (host arrays stay double and are converted).
 *
 * Errors.  Every call returns an amr_status (amr.h) and never aborts the
 * process; amr_last_error() gives the text of the calling thread's last
 * error.  Asynchronous calls report CUDA faults at the next synchronising
 * call.  A handle is not thread-safe.
 */
#ifndef AMR_PARTICLES_H
#define AMR_PARTICLES_H
#include <stddef.h>
#include <stdint.h>

#include "amr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amr_particles *amr_part_handle;

typedef enum {
  /* one thread per particle; lanes of a warp whose particles share a source
   * cell combine their contributions before 8 atomic additions (the paper's
   * `medium' kernel, part_dep_algo = 2).  The summation order of a cell
   * depends on timing: the result is reproducible to rounding only. */
  AMR_CIC_ATOMIC = 2,
  /* prefix sums over the sorted particles split them into source-cell
   * segments; each segment's 8 sums (in particle order) are added into the
   * grid once per stencil offset, in offset order (the paper's `small'
   * kernel, part_dep_algo = 3).  Bit-reproducible: the result depends only
   * on the particles and their order.  Needs amr_part_sort since the last
   * amr_part_write. */
  AMR_CIC_SEGMENT = 3
} amr_cic_algo;

typedef struct {
  int n;          /* grid cells per axis: a power of two, 2..1024 */
  int precision;  /* 8 (FP64) or 4 (FP32) */
  void *stream;   /* cudaStream_t of every launch; NULL: the legacy default stream */
} amr_part_params;

/*
 * amr_part_create -- copy np particles from host arrays to the device.
 *   x, y, z   positions, each in [0, 1) (checked: AMR_EINVAL otherwise)
 *   m         masses (finite; checked)
 * np may be 0 (the grid then deposits to zero); np < 2^32.  Particle t of the
 * arrays gets identifier t.  The arrays keep the caller's order until
 * amr_part_sort.  Synchronous.  Errors: AMR_EINVAL, AMR_ENOMEM, AMR_ECUDA.
 */
amr_status amr_part_create(const amr_part_params *p, int64_t np, const double *x, const double *y,
                           const double *z, const double *m, amr_part_handle *out);

/* Replace positions and masses (same count and checks as amr_part_create) in
 * the current order of the handle; identifiers are kept.  Marks the handle
 * unsorted.  Synchronous with respect to the host arrays. */
amr_status amr_part_write(amr_part_handle h, const double *x, const double *y, const double *z,
                          const double *m);

/*
 * amr_part_sort -- sort the particles by the 3-D Hilbert index of their
 * source cells (log2 n bits per axis, x most significant), stably (particles
 * of one source cell keep their order), and reorder positions, masses and
 * identifiers (Sec. 4: Hilbert keys of the source cells, radix sort,
 * reordered particle arrays).  Asynchronous on the handle's stream.
 */
amr_status amr_part_sort(amr_part_handle h);

/*
 * amr_cic_deposit -- overwrite the handle's grid with the CIC density of all
 * particles (Sec. 4, mass deposition) by the given algorithm (amr_cic_algo).
 * AMR_CIC_SEGMENT returns AMR_EINVAL unless the handle has been sorted since
 * its positions were last written.  Asynchronous.
 */
amr_status amr_cic_deposit(amr_part_handle h, int algo);

/* Copy the grid to a host array of n^3 doubles (FP32 grids are widened).
 * Synchronises the stream. */
amr_status amr_part_read_rho(amr_part_handle h, double *rho, int64_t cap);

/* Copy the particles, in the handle's current order, to host arrays of np
 * entries (any pointer may be NULL).  Synchronises the stream. */
amr_status amr_part_read(amr_part_handle h, double *x, double *y, double *z, double *m,
                         int64_t *id, int64_t cap);

/* Device address of the grid (n^3 elements of the handle's precision) and of
 * the position/mass arrays in the current order; valid until the next
 * amr_part_sort (positions) or amr_part_destroy (grid).  Any pointer may be
 * NULL. */
amr_status amr_part_device(amr_part_handle h, void **rho, void **x, void **y, void **z, void **m);

typedef struct {
  int64_t np;
  int n, precision;
  int sorted;                 /* 1 if sorted since the last write */
  int64_t n_segments;         /* source-cell segments of the last segment deposition */
  int64_t device_bytes;       /* bytes held on the device */
  int64_t kernel_launches;    /* kernels launched by the handle so far */
} amr_part_info;

amr_status amr_part_get_info(amr_part_handle h, amr_part_info *info);

/* Per-kernel device time, as amr_set_timing / amr_read_timing of amr.h: ids
 * 0..n-1 named by amr_part_kernel_name (NULL past the last). */
amr_status amr_part_set_timing(amr_part_handle h, int on);
amr_status amr_part_read_timing(amr_part_handle h, int n, double *ms, int64_t *launches);
const char *amr_part_kernel_name(int t);

/* Free the handle and its device memory (synchronises the stream). NULL is a
 * no-op. */
amr_status amr_part_destroy(amr_part_handle h);

#ifdef __cplusplus
}
#endif
#endif /* AMR_PARTICLES_H */
