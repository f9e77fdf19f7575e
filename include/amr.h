/*
 * amr.h -- C ABI of the GB300 level-advance library for compressible Euler on
 * a cell-by-cell octree (the AMR hydro method of RAMSES-GPU, arXiv 2607.20704).
 *
 * One handle owns one graded octree resident in device memory: the oct list
 * (sorted by level, then Hilbert key, Sec. 2.2), an FNV-1a 64 hash table with
 * linear probing keyed by (i,j,k,l) (Sec. 2.1, Sec. 6), the father/neighbour
 * index arrays and the ghost-oct cache (Sec. 2.3), the conservative state
 * U = (rho, rho u, rho v, rho w, E) of every cell and the pending reflux of
 * every coarse cell.  All computation runs in the library's CUDA kernels on
 * the handle's stream; nothing falls back to the CPU.
 *
 * Conventions.  An oct of level l (levelmin <= l <= levelmax <= 15) has
 * integer coordinates (i,j,k) in [0, 2^(l-1))^3 of the periodic unit box and
 * cell size dx_l = 2^-l; its cells are c = cx + 2cy + 4cz.  The father cell
 * of oct (i,j,k,l) is cell (i,j,k) of level l-1, i.e. cell
 * (i&1)+2(j&1)+4(k&1) of oct (i/2,j/2,k/2,l-1) (Sec. 2.1).  Host state
 * arrays are structure-of-arrays: U[v * 8n + 8*oct + c], v = 0..4.  The base
 * level must be complete and the tree graded: every oct of level l > levelmin
 * needs the 27 level-(l-1) cells around its father cell.
 *
 * Errors.  Every call returns an amr_status and never aborts the process.
 * CUDA failures map to AMR_ECUDA.  The text of the last error of the calling
 * thread is returned by amr_last_error().  Asynchronous calls
 * (amr_step_level, amr_advance) report device-side faults at the next
 * synchronising call (amr_cfl_dt, amr_read, amr_sync).
 *
 * Threads.  A handle is not thread-safe; different handles may be used from
 * different threads.
 */
#ifndef AMR_H
#define AMR_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amr_mesh *amr_handle;

typedef enum {
  AMR_OK = 0,
  AMR_EINVAL = 1,   /* bad argument, level, coordinate or size */
  AMR_ENOMEM = 2,   /* allocation refused or over the handle's HBM budget */
  AMR_EGRADING = 3, /* incomplete base level or 2:1 grading violated */
  AMR_EDUP = 4,     /* the same oct listed twice */
  AMR_ECUDA = 5,    /* a CUDA runtime error */
  AMR_ETIMEOUT = 6, /* a bounded device-side wait gave up */
  AMR_ENAN = 7      /* non-finite state met by the time-step reduction */
} amr_status;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns a device pointer aligned to 256 bytes or NULL; free receives
 * the pointer and the size that alloc returned it for.  Both are called with
 * the handle's stream. */
typedef void *(*amr_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*amr_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct {
  int levelmin, levelmax;   /* 1 <= levelmin <= levelmax <= 15 */
  double gamma;             /* ratio of specific heats, > 1 */
  double cfl;               /* Courant number of amr_cfl_dt */
  double smallr, smallc;    /* floors: rho >= smallr, p >= rho smallc^2 / gamma */
  /* refinement criteria of amr_regrid (Sec. 2.2): a cell refines when the
   * relative jump 2|a-b|/(|a|+|b|) of rho (of p) to a face neighbour exceeds
   * refine_grad_rho (refine_grad_p), or when its mass rho dx^3 exceeds
   * refine_mass; a criterion <= 0 is off */
  double refine_grad_rho, refine_grad_p, refine_mass;
  int precision;            /* 8: FP64 state and arithmetic; 4: FP32 state and
                               arithmetic, FP64 time-step reduction */
  int reflux;               /* 1: reflux at coarse-fine faces (default);
                               0: off (a negative control for tests) */
  int reindex_every_step;   /* 1: amr_advance rebuilds the hash table and the
                               neighbour/cache index at the start of every
                               coarse step, as after a regrid (the paper's
                               per-step cache rebuild); 0 (default): the
                               index is rebuilt only where the mesh changes
                               (amr_create, amr_regrid, amr_reindex); the
                               results are the same bit for bit */
  int use_graphs;           /* 1: amr_advance replays a captured CUDA graph of
                               one coarse step (default) */
  size_t hbm_budget_bytes;  /* 0: no limit; else AMR_ENOMEM beyond it */
  void *stream;             /* cudaStream_t; NULL: the legacy default stream */
  amr_alloc_fn alloc;       /* NULL: the library's own stream-ordered pool on
                               the current device (memory a handle frees stays
                               reserved there for later allocations of the
                               process, so regrids and repacks reuse it) */
  amr_free_fn free;
  void *alloc_user;
  int tile;                 /* cells (threads) per work tile: 64, 128, 256 or 512;
                               0: autotune at the first amr_advance (default) */
  int schedule;             /* 1: persistent grids sized by occupancy x SMs;
                               0: one tile per block; -1: autotune (default) */
  int regrid_expand;        /* 1: a refinement flag also flags the 26 cells
                               around it (default); 0: off */
  int regrid_every_step;    /* 1: amr_advance regrids before every coarse
                               step; 0: the mesh only changes by amr_regrid
                               (default) */
  int nsubgrid;             /* level-step kernel (Sec. 3): 0: per-cell passes
                               (primitives, predictor, faces, update, each
                               computed once); 1, 2 or 4: the paper's fused
                               shared-memory kernels on blocks of nsubgrid^3
                               octs with one ring of octs (cubes of 6^3, 8^3
                               or 12^3 cells); -1 (default): picked by the
                               autotuner among these when tile is 0, else the
                               per-cell passes.  All give the same results
                               bit for bit. */
  int planar;               /* with nsubgrid 1, 2 or 4: 0: stage the whole
                               cube (the "rock" kernel); 1: sweep it along z
                               keeping a three-plane window (the "paper"
                               kernel); -1 (default): the autotuner's choice
                               (with a fixed nsubgrid: rock) */
} amr_params;

/* Fills p with the defaults: levelmin = levelmax = 1, gamma = 1.4, cfl = 0.8,
 * smallr = smallc = 1e-10, precision 8, reflux 1, reindex_every_step 0,
 * use_graphs 1, no budget, NULL stream and allocator, tile 0, schedule -1,
 * nsubgrid -1 and planar -1 (picked by the autotuner), refinement criteria
 * off, regrid_expand 1, regrid_every_step 0. */
void amr_params_default(amr_params *p);

/*
 * amr_create -- build a mesh from a host oct list (Sec. 2: oct array;
 * Sec. 2.2: level bucket sort with prefix sums, Hilbert radix sort;
 * Sec. 2.1: FNV-1a 64 hash with linear probing; Sec. 2.3: father/neighbour
 * arrays and ghost cache).
 *   n_oct          number of octs, >= 1 (the base level at least)
 *   level,i,j,k    host arrays of n_oct entries, any order
 *   hilbert_key    optional host array of n_oct sort keys within a level;
 *                  NULL: the library computes the 3-D Hilbert index of
 *                  (i,j,k) with l-1 bits per axis, x most significant
 *   U              host array [5][8*n_oct] in the input order; values of
 *                  split cells are ignored (replaced by the mean of their
 *                  children)
 *   out            receives the handle
 * The inputs are copied; the caller keeps ownership of its buffers.  The call
 * synchronises the stream.  Errors: AMR_EINVAL (arguments, levels,
 * coordinates), AMR_EDUP, AMR_EGRADING, AMR_ENOMEM, AMR_ECUDA.
 */
amr_status amr_create(const amr_params *p, int64_t n_oct, const uint8_t *level,
                      const uint32_t *i, const uint32_t *j, const uint32_t *k,
                      const uint64_t *hilbert_key, const double *U, amr_handle *out);

/* One member mesh of a batched handle: its own levels, gas, floors and oct
 * list, with the same meaning and layout as the arguments of amr_create. */
typedef struct {
  int levelmin, levelmax;
  double gamma, cfl, smallr, smallc;
  int64_t n_oct;
  const uint8_t *level;
  const uint32_t *i, *j, *k;
  const uint64_t *hilbert_key; /* NULL for every member, or given for every member */
  const double *U;             /* [5][8*n_oct] */
} amr_member;

/*
 * amr_create_batch -- one handle over n_members independent meshes (the
 * batched serving of many small solves; the paper's method applies to each
 * mesh unchanged).  Octs are ordered by (member, level, Hilbert key); every
 * level-step launch covers all members (a flattened list of (member, level)
 * tiles), and amr_advance moves each member by its own CFL time step through
 * its own W-cycle, the W-cycles aligned phase by phase.  Results of a member
 * are bit-identical to the same mesh in a handle of its own.  p supplies the
 * shared settings (precision, reflux, reindex_every_step, use_graphs,
 * hbm_budget_bytes, stream, allocator); its per-mesh fields are ignored.
 * amr_create(p, ...) is amr_create_batch with one member built from p.
 * At most 32768 members and 2^26 octs in total.
 */
amr_status amr_create_batch(const amr_params *p, int n_members, const amr_member *members,
                            amr_handle *out);

/* Selects the member that amr_read, amr_write, amr_read_reflux, amr_lookup,
 * amr_read_index, amr_read_cache, amr_cfl_dt and the dt of amr_advance refer
 * to (default 0). */
amr_status amr_select_member(amr_handle h, int member);

/* Coarse steps each member still takes: amr_advance skips members whose
 * count is 0 (their state and dt stay as they are) and counts the others
 * down; -1 means unlimited (the default).  steps holds n = n_members values.
 * Synchronous. */
amr_status amr_set_member_steps(amr_handle h, const int32_t *steps, int n);

/* Per-member error flags (bit 0: a leaf state was not finite), copied into
 * errs[0..n_members), after waiting for the handle's stream; also clears the
 * handle-wide error that the next synchronising call would report. */
amr_status amr_member_errors(amr_handle h, int32_t *errs, int n);

/*
 * amr_batch_repack -- continuous batching of independent meshes (no
 * counterpart in the paper: the serving loop's admission between coarse
 * steps).  The handle is rebuilt with members keep[0..n_keep) of the current
 * ones (indices in increasing order; their states stay on the device and are
 * carried over bit for bit, with their remaining coarse-step counts, last
 * time steps and error bits) followed by n_add new meshes added[] (copied
 * from the host as by amr_create_batch), each to take added_steps[q] coarse
 * steps (-1: unlimited).  Members that are not kept are dropped and their
 * device memory freed.  After the call member q < n_keep is the old member
 * keep[q] and member n_keep + q the added mesh q; member 0 is selected.  A
 * member's results do not depend on the other members, so a kept member
 * continues exactly as it would alone.  Call between coarse steps (no
 * reflux is pending there); the rebuild holds the old and the new mesh for
 * its duration.  Device buffers are replaced (a captured graph is
 * re-captured; the launch shape chosen by the autotuner is kept).
 * Synchronous.  Errors: AMR_EINVAL (counts, unordered keep, bad mesh, more
 * than 2^26 octs), AMR_EGRADING / AMR_EDUP (an added mesh), AMR_ENOMEM,
 * AMR_ECUDA; on error the handle is unchanged.
 */
amr_status amr_batch_repack(amr_handle h, int n_keep, const int32_t *keep, int n_add,
                            const amr_member *added, const int32_t *added_steps);

/* The last coarse time step of every member (from amr_cfl_dt or
 * amr_advance), copied into dt_out[0..n_members) (synchronous). */
amr_status amr_member_dt(amr_handle h, double *dt_out, int n);

/*
 * amr_regrid -- one regrid of the mesh (Sec. 2.2, then the ghost cache of
 * Sec. 2.3).  With the criteria of the handle's amr_params:
 *   flag    cells of level l < levelmax meeting a criterion: the relative
 *           jump 2|a-b|/(|a|+|b|) of rho or p to a face neighbour (the
 *           same-level cell, else the coarser cell covering it) above its
 *           threshold, or the cell mass rho dx^3 above refine_mass; decided
 *           in FP64 in the division-free form 2|a-b| > threshold (|a|+|b|)
 *           with p = (gamma-1)(E - (m.m/2)/rho) and the floors, which equals
 *           the quotient test except for jumps within a few rounding errors
 *           of the threshold
 *   expand  (regrid_expand) also the 26 same-level cells around a flag
 *   grade   finest level first, a flagged cell of level l flags the level
 *           l-1 cells covering its 27 level-l neighbours (2:1 rule)
 * then flagged leaves get a child oct (minmod prolongation of the father
 * from its six face neighbours, coarsest level first), split cells left
 * unflagged lose their child oct, and the mesh is rebuilt as by amr_create
 * (level bucket sort, Hilbert radix sort, hash, index, cache, restriction).
 * A cell refines by at most one level per call.  Call between coarse steps
 * (pending reflux, zero there, is dropped).  Device buffers are replaced:
 * pointers from earlier calls are invalid, a captured graph is re-captured.
 * created/removed (may be NULL): octs added and removed; both 0 leaves the
 * handle untouched.  Synchronous.  Errors: AMR_ENOMEM, AMR_EINVAL (more than
 * 2^26 octs would result), AMR_ECUDA.
 */
amr_status amr_regrid(amr_handle h, int64_t *created, int64_t *removed);

/* amr_regrid with the final flags given instead of computed (the stages
 * after flag, expand and grade): flags[8 * q + c] != 0 splits cell c of oct
 * q, q running over every oct of the handle in mesh order (members, then
 * levels, then amr_read order); n_cells must equal 8 x the handle's octs.
 * The flags must satisfy the 2:1 rule that grading would give them (a
 * violation is reported as AMR_EGRADING by the rebuild).  Host buffer, read
 * before return.  Synchronous; errors as amr_regrid, AMR_EINVAL for a wrong
 * n_cells. */
amr_status amr_regrid_flags(amr_handle h, const uint8_t *flags, int64_t n_cells,
                            int64_t *created, int64_t *removed);

/* Refinement flags of the selected member's cells of one level after the
 * flag, expand and grade stages of amr_regrid, without changing the mesh:
 * flags[8 * n + c] = 1 for cell c of the n-th oct (amr_read order); cap >=
 * 8 * octs of the level.  Synchronous. */
amr_status amr_flag(amr_handle h, int level, uint8_t *flags, int64_t cap);

/*
 * amr_poisson -- self-gravity potential of the selected member's base level
 * (Sec. 5): n_vcycles multigrid V-cycles for
 *     (sum of the 6 face neighbours - 6 phi) / dx^2 = fourpiG (rho - mean rho)
 * on the periodic levelmin grid (complete by construction): red-black
 * Gauss-Seidel smoothing (colour = parity of the cell's index inside its oct;
 * 2 sweeps before and after the coarse correction), residual restriction by
 * the mean of the 8 children, trilinear prolongation with weights
 * (1,3,3,9,3,9,9,27)/64, down to 2^3 cells (8 sweeps there).  The solution
 * of the previous call is the initial guess (zero at first and after a
 * regrid); the potential returned by amr_read_phi has zero mean.  resid
 * (may be NULL) receives the L2 norm of the base-level residual after each
 * V-cycle.  FP64 whatever the precision of the state.  Synchronous.  Errors:
 * AMR_EINVAL (n_vcycles outside [0, 1020], levelmin above 10).
 */
amr_status amr_poisson(amr_handle h, double fourpiG, int n_vcycles, double *resid);

/* Potential of the selected member's base-level cells after amr_poisson,
 * phi[8 * n + c] for cell c of the n-th oct (amr_read order); cap >= 8 *
 * octs of levelmin. */
amr_status amr_read_phi(amr_handle h, double *phi, int64_t cap);

/*
 * amr_poisson_level -- potential of the cells of one refined level L of the
 * selected member (Sec. 5: the Poisson equation is solved level by level,
 * each level taking its boundary values from the level below).  The
 * unknowns are the cells of level L; the operator is the 7-point Laplacian
 *     (sum of the 6 face neighbours - 6 phi) / dx_L^2 = fourpiG (rho - rho_bar)
 * where a face with no level-L cell on the other side takes the Dirichlet
 * value phi_b = (phi of the cell's father + phi of the level-(L-1) cell
 * across the face) / 2 through the ghost value 2 phi_b - phi.  n_vcycles
 * V-cycles over the hierarchy of the level's ancestors down to levelmin
 * (MG level k = the level-(L-k) cells holding a cell of MG level k-1;
 * homogeneous Dirichlet values at every MG level's own boundary), red-black
 * Gauss-Seidel with colour = parity of x + y + z, 2 sweeps before and after
 * the coarse correction and 8 on the coarsest, residuals restricted by the
 * sum of the existing children over 8, corrections prolonged trilinearly
 * with weights (1,3,3,9,3,9,9,27)/64 (coarse cells outside the MG level
 * count 0).  Every FP64 operation is rounded once in a fixed order, so the
 * result does not depend on the launch configuration.
 *
 * Input and output live in the handle's per-cell potential (8 doubles per
 * oct of every member, zero after amr_create and after every regrid): the
 * values of level L-1 are the boundary data, those of level L the initial
 * guess, and level L receives the result (amr_write_phi / amr_read_phi_level
 * move them).  The tables of the level (its cells and their ancestors,
 * sorted, with neighbours, colours, children and prolongation stencils) are
 * built on the device on the first call for a (member, level) and kept
 * until the mesh changes.  resid (may be
 * NULL) receives the L2 norm of the level's residual after each V-cycle.
 * FP64 whatever the precision of the state.  Synchronous.  Errors:
 * AMR_EINVAL (level not a populated level above levelmin, n_vcycles outside
 * [0, 1020]), AMR_EGRADING (a cell of level L without a father cell, or a
 * boundary face without a level-(L-1) cell across).
 */
amr_status amr_poisson_level(amr_handle h, int level, double fourpiG, double rho_bar, int n_vcycles,
                             double *resid);

/*
 * amr_poisson_levels -- the potential of every level of the selected member,
 * coarse to fine: amr_poisson on the base level (its zero-mean result
 * becomes the base level's per-cell potential), then for each populated
 * level L above levelmin the father cell's potential as the initial guess of
 * every cell and amr_poisson_level(L) with rho_bar = the mean density of the
 * base level.  resid (may be NULL) holds n_vcycles values per level:
 * resid[L * n_vcycles + c] for L in [levelmin, levelmax] (size (levelmax + 1)
 * * n_vcycles).  Synchronous.  Errors: those of amr_poisson and
 * amr_poisson_level.
 */
amr_status amr_poisson_levels(amr_handle h, double fourpiG, int n_vcycles, double *resid);

/* Per-cell potential of one level of the selected member from the host,
 * phi[8 * n + c] for cell c of the n-th oct (amr_read order); n must equal
 * 8 * the level's octs.  Errors: AMR_EINVAL (bad level or size). */
amr_status amr_write_phi(amr_handle h, int level, const double *phi, int64_t n);

/* Per-cell potential of one level of the selected member to the host, same
 * order; cap >= 8 * the level's octs.  Errors: AMR_EINVAL (bad level, cap too
 * small, no potential on this mesh since amr_create or the last regrid). */
amr_status amr_read_phi_level(amr_handle h, int level, double *phi, int64_t cap);

/* Frees every device buffer of the handle (after synchronising its stream). */
amr_status amr_destroy(amr_handle h);

/*
 * amr_cfl_dt -- coarse time step (stage "compute dt" of Table 1):
 * dt_l = cfl dx_l / max over leaf cells of level l of sum_d (|u_d| + c),
 * dt = min over levels of dt_l 2^(l - levelmin).  FP64 warp-shuffle max
 * reduction on the device; the result is copied to *dt_out (synchronous).
 * Errors: AMR_ENAN if a leaf state is not finite.
 */
amr_status amr_cfl_dt(amr_handle h, double *dt_out);

/*
 * amr_step_level -- advance every oct of one level by dt (Sec. 3; stages
 * godunov, set uold and upload of Table 1): ghost octs by minmod-limited
 * prolongation from level-1, MUSCL-Hancock predictor, HLLC flux on every
 * face, conservative update of leaf cells plus the pending reflux of the
 * level (which is then cleared), reflux of coarse-fine face fluxes onto the
 * level-1 cells (fixed-order segmented sum, no floating-point atomics), and
 * restriction of the level onto its father cells.  Asynchronous on the
 * handle's stream.  The caller runs levels in the W-cycle order: a level
 * l < finest takes its step after the two half steps of level l+1.
 * In a batched handle the call advances that level of every member with the
 * same dt.  Errors: AMR_EINVAL for a level outside [1, levelmax] or dt <= 0.
 */
amr_status amr_step_level(amr_handle h, int level, double dt);

/*
 * amr_advance -- n coarse steps of the level-by-level W-cycle: per coarse
 * step (optionally) rebuild the index, dt = amr_cfl_dt computed on the device,
 * then advance(levelmin, dt), where advance(l, dt) runs advance(l+1, dt/2)
 * twice when level l+1 holds octs and then amr_step_level(l, dt).  No host
 * synchronisation inside; with use_graphs the coarse step is one graph
 * launch.  If dt_last is not NULL the call synchronises and stores the last
 * coarse dt there.  When the tile size or schedule is left to the autotuner,
 * the first call times each candidate on full coarse steps from a snapshot of
 * the state, restores the snapshot, and keeps the fastest (synchronous, once
 * per handle; the results are the same for every candidate).
 */
amr_status amr_advance(amr_handle h, int n_coarse_steps, double *dt_last);

/* Rebuild the hash table, father/son flags, 27-neighbour array and ghost
 * cache from the oct list (what a regrid triggers, Sec. 2.3).  Async. */
amr_status amr_reindex(amr_handle h);

/*
 * amr_read -- copy out the octs of one level in the mesh order: packed keys
 * key = (l << 60) | (i << 40) | (j << 20) | k, and U [5][8*n] as doubles.
 * *n_oct_out receives the level's oct count; keys and U may be NULL; when not
 * NULL they must hold cap octs (AMR_EINVAL if cap is smaller).  Synchronous.
 */
amr_status amr_read(amr_handle h, int level, int64_t *n_oct_out, uint64_t *keys,
                    double *U, int64_t cap);

/*
 * amr_totals -- conserved totals of the selected member's leaf cells (the
 * per-level conservation check of a cell-by-cell AMR update, Sec. 3: every
 * flux leaves one cell and enters another, reflux closing coarse-fine
 * faces): out[v] = sum over the leaf cells of `level` of U_v dx^3, dx =
 * 2^-level; level 0: the sum over every level, the levels' totals added in
 * ascending level order.  FP64 in both precisions (FP32 states are widened
 * exactly); every addition in a fixed order (fixed blocks per level size, no
 * atomics), so calls repeat bit for bit.  out: 5 doubles, host.  Waits for
 * the handle's stream (synchronous).  Errors: AMR_EINVAL (NULL, level
 * outside [0, 15]), AMR_ENOMEM, AMR_ECUDA.
 */
amr_status amr_totals(amr_handle h, int level, double *out);

/*
 * amr_hash -- FNV-1a 64 as the hash table computes it (Sec. 2.1 keys the
 * table by an "fnv64" hash; Sec. 6 names FNV-1a 64): hash[q] = FNV-1a 64
 * (offset basis 0xcbf29ce484222325, prime 0x100000001b3) over the 8 bytes of
 * keys[q], least significant byte first, evaluated on the device by the
 * function every table insert and probe uses.  keys, hash: n values, host
 * buffers (0 <= n <= 2^28).  Uses the handle's stream and allocator;
 * synchronous.  Errors: AMR_EINVAL, AMR_ENOMEM, AMR_ECUDA.
 */
amr_status amr_hash(amr_handle h, int64_t n, const uint64_t *keys, uint64_t *hash);

/*
 * amr_read_hash -- the handle's hash table as stored (Sec. 2.1: open
 * addressing, linear probing, the home slot of a key is its FNV-1a 64 hash
 * masked by capacity - 1).  *cap_out = capacity (a power of two, at least
 * twice the real + ghost octs).  When keys / vals are not NULL (cap >=
 * capacity) they receive every slot: empty slots hold the key all ones and
 * value 0; an occupied slot holds the internal key
 *     member << 49 | level << 45 | i << 30 | j << 15 | k
 * (member 0 for a single mesh; i, j, k the oct coordinates) and the value
 * 1 + the oct's extended index (real octs in mesh order first, then the
 * ghost octs of the cache).  Synchronous.
 */
amr_status amr_read_hash(amr_handle h, int64_t *cap_out, uint64_t *keys, int32_t *vals,
                         int64_t cap);

/*
 * amr_cic_deposit_levels -- Cloud-in-Cell mass deposition of np particles onto
 * every level of the selected member (Sec. 4, "Mass Deposition": at level l
 * the particles of level l and of every finer level deposit, then the list is
 * split for level l+1).  The list of levelmin holds every particle; at level
 * l each particle of the list adds m (wx wy) wz / dx_l^3 -- the CIC weights
 * at cell size dx_l = 2^-l with the half-cell-shifted stencil: along each
 * axis s = x 2^l - 1/2, i0 = floor(s), f = s - i0, weights 1 - f and f on
 * cells i0 and i0 + 1 (periodic) -- to each of its 8 stencil cells that
 * exists at level l (a cell of a real level-l oct); the list of level l+1
 * keeps, in order, the particles whose host cell at level l (the cell
 * containing the particle) is split.  The result is the density of every
 * cell of the member's levels (split cells included), read with
 * amr_read_particle_rho; count[l] (16 entries, may be NULL) receives the
 * size of each level's list.  One thread per particle of a list, atomic
 * additions: reproducible to rounding only.
 *   x, y, z, m  host arrays of np doubles; positions in [0, 1), finite masses
 *               (checked: AMR_EINVAL); np < 2^32
 * Copies the particles to the device in the handle's precision; synchronous.
 */
amr_status amr_cic_deposit_levels(amr_handle h, int64_t np, const double *x, const double *y,
                                  const double *z, const double *m, int64_t *count);

/* The same deposition from device arrays of the handle's precision (double
 * for precision 8, float for 4), caller-owned, not checked; asynchronous on
 * the handle's stream unless count is not NULL (then synchronous). */
amr_status amr_cic_deposit_levels_device(amr_handle h, int64_t np, const void *x, const void *y,
                                         const void *z, const void *m, int64_t *count);

/* Density of the last deposition for the selected member's cells of one
 * level, [8 n] in amr_read order (FP32 widened).  AMR_EINVAL when the mesh
 * has no deposition or has changed since (regrid, repack).  Synchronous. */
amr_status amr_read_particle_rho(amr_handle h, int level, double *rho, int64_t cap);

/* Same as amr_read for the pending reflux R [5][8*n] of a level. */
amr_status amr_read_reflux(amr_handle h, int level, double *R, int64_t cap);

/*
 * amr_write -- replace the state of one level from a host array [5][8*n] in
 * the mesh order of amr_read (for restarts and end-to-end runs).  Values of
 * split cells are taken as given.  Pinned host memory makes the copy
 * asynchronous; the host buffer must stay valid until the stream passes it.
 */
amr_status amr_write(amr_handle h, int level, const double *U, int64_t n);

/*
 * amr_load_state_async / amr_store_state_async -- the state of every real oct
 * of the selected member, all levels in mesh order (level by level, each as
 * amr_read orders it), as one host array [5][8 n], n = the member's octs.
 * Both return at once and overlap the level steps: two copy streams of the
 * handle (uploads, downloads) move the host data to and from device staging
 * buffers while the handle's stream steps, and the handle's stream moves
 * staging <-> U.  In
 * stream order, a load takes effect after the work queued before it and
 * before the work queued after it; a store captures the state the work
 * queued before it leaves.  So "load, advance, store" per step pipelines the
 * copies of neighbouring steps with the compute.  Host buffers must be
 * pinned to overlap (pageable memory works but blocks) and stay untouched
 * until amr_sync returns: a store's host array is complete only then.
 * Errors: AMR_EINVAL (NULL, n != the member's octs, cap too small),
 * AMR_ENOMEM (staging), AMR_ECUDA.
 */
amr_status amr_load_state_async(amr_handle h, const double *U, int64_t n);
amr_status amr_store_state_async(amr_handle h, double *U, int64_t cap);

/* ---- index introspection (parity tests; not on the hot path) -------------- */

/* hash_get of Sec. 2.1 for n host keys: idx_out[t] = mesh index of the oct
 * (0-based, mesh order) or -1.  Synchronous. */
amr_status amr_lookup(amr_handle h, int64_t n, const uint64_t *keys, int64_t *idx_out);

/* The 27-entry neighbour array of a level, [n][27] in (dz,dy,dx) order
 * (13 = self): >= 0 mesh index of a same-level oct, else -(1 + s) for ghost
 * oct s of the cache; split flags [8n] (1 if the cell has a child oct).
 * Either pointer may be NULL.  Synchronous. */
amr_status amr_read_index(amr_handle h, int level, int64_t *nbr, uint8_t *split,
                          int64_t cap);

/* Ghost (cache) octs of a level: *n_out count, keys (sorted ascending),
 * ghost values Ug [5][8*n] as last filled by a level step or amr_fill_ghosts.
 * cache slot s of the neighbour array counts across levels; the first slot of
 * a level is *first_out.  Synchronous. */
amr_status amr_read_cache(amr_handle h, int level, int64_t *n_out, int64_t *first_out,
                          uint64_t *keys, double *Ug, int64_t cap);

/* Fill the ghost octs of a level from the current coarser levels (the first
 * stage of amr_step_level), asynchronously. */
amr_status amr_fill_ghosts(amr_handle h, int level);

typedef struct {
  int64_t n_oct, n_cache, n_leaf_cells;  /* all members */
  int64_t level_octs[16], level_cache[16], level_leaf_cells[16]; /* selected member */
  int64_t device_bytes;       /* bytes held on the device */
  int64_t kernel_launches;    /* kernels launched by the handle so far */
  int64_t graph_launches;     /* CUDA graph launches so far */
  int64_t hash_capacity;
  int64_t work_per_step;      /* leaf cell-updates of one coarse step, all members */
  int precision;
  int n_members, member;      /* members of the handle; the selected one */
  int phases;                 /* level-step phases of one coarse step */
  int tile, schedule;         /* work-tile size and schedule in use */
  int nsubgrid;               /* level-step kernel in use (amr_params.nsubgrid) */
  int planar;                 /* 1: the fused kernel sweeps planes (amr_params.planar) */
  int64_t cached_bytes;       /* device arrays a regrid retired, kept for the next one
                                 (at most the live mesh's size; 0 with a device budget) */
} amr_info;

/* Counts of the mesh and of the work done so far. */
amr_status amr_get_info(amr_handle h, amr_info *info);

/* Per-kernel device time.  amr_set_timing(h, 1) brackets every later kernel
 * launch (also inside captured graphs) with CUDA events on the handle's
 * stream; amr_read_timing synchronises and, for kernel id t < n, returns the
 * total milliseconds and launch count since timing was enabled.
 * amr_kernel_name(t) names kernel id t (NULL past the last). */
amr_status amr_set_timing(amr_handle h, int on);
amr_status amr_read_timing(amr_handle h, int n, double *ms, int64_t *launches);
const char *amr_kernel_name(int t);

/*
 * amr_fma_rate -- the FMA throughput of GPU `device` in the given precision
 * (8: FP64, 4: FP32), measured by a kernel of independent FMA chains (8 per
 * thread, 8 blocks of 256 threads per SM) timed with CUDA events on a
 * private stream, best of three launches after a warm-up: *flops = 2 x FMAs
 * per second.  The denominator of the arithmetic-bound rooflines, beside
 * the rate derived from the unit counts and the clock.  Synchronous; uses no
 * handle.  Errors: AMR_EINVAL (precision), AMR_ECUDA.
 */
amr_status amr_fma_rate(int device, int precision, double *flops);

/*
 * amr_cfl_dt_static -- the CFL time step of one level of leaf cells held in
 * caller device memory, with no device allocation at all.  It computes the
 * quantity amr_cfl_dt reduces for that level, dt_l = cfl dx_l / max sum_d
 * (|u_d| + c), with three differences: it returns the level's dt_l, not the
 * coarse step's dt; it divides (u_d / rho, gamma p / rho) where amr_cfl_dt
 * multiplies by a Newton-refined reciprocal, so the two can differ in the
 * last bit; and a non-finite cell makes the result NaN, where amr_cfl_dt
 * reports AMR_ENAN.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (device memory pre-reserved by another
 * runtime's pool, allocator-free real-time loops).  Its scratch is fixed
 * device storage inside the library (512 KiB per GPU that loads it, held
 * until the process exits), so n_cells is limited to
 * AMR_CFL_STATIC_MAX_CELLS (AMR_EINVAL beyond it).
 *   U        device array of doubles, variable v of cell t at U[v*stride + t]
 *   n_cells  cells to reduce, all leaves of one level
 *   level    the cells' level l: dx = 2^-l
 *   gamma, cfl, smallr, smallc   as in amr_params
 *   dt_out   device pointer; receives cfl dx / max_t sum_d (|u_d| + c), or
 *            NaN if a cell is not finite
 *   stream   cudaStream_t (NULL: legacy default stream); asynchronous
 * The first call on a device looks up the scratch address (with that device
 * current) and keeps it for the process's life; make that first call before
 * any stream capture, and do not call again after a cudaDeviceReset of that
 * device.  Every call on a
 * device shares the same scratch: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.  The
 * call clears the scratch counter it needs before its kernel runs.
 * Errors: AMR_EINVAL (NULL pointer, sizes, parameters), AMR_ECUDA.
 */
#define AMR_CFL_STATIC_MAX_CELLS ((int64_t)65536 * 256)
amr_status amr_cfl_dt_static(const double *U, int64_t n_cells, int64_t stride, int level,
                             double gamma, double cfl, double smallr, double smallc,
                             double *dt_out, void *stream);

/* ---- serving ------------------------------------------------------------ */
/*
 * A serving loop for many independent solves (the paper has no serving
 * layer; this is the batching of its level advance across requests).
 * amr_server_submit queues a request (its arrays are copied) and returns at
 * once.  A scheduler thread admits queued requests in arrival order whenever
 * the device budget and the wave slots allow; the requests admitted together
 * form a wave -- one batched handle (amr_create_batch) on its own stream, in
 * which each member stops after its own number of coarse steps
 * (amr_set_member_steps).  Waves admitted while others run overlap with them
 * on the GPU.  A finished request's final state is copied to host memory;
 * a wave whose members are all finished frees its device memory.  A
 * request's result is bit-identical to the same solve in a handle of its own.
 * Errors: submit refuses a request that alone exceeds the budget
 * (AMR_ENOMEM) or has bad arguments (AMR_EINVAL); a request whose mesh is
 * invalid (its wave is then rebuilt without it) or whose state turns
 * non-finite fails alone --
 * amr_server_wait returns AMR_ECUDA with the reason in amr_last_error(), and
 * the other requests of its wave carry on.
 */
typedef struct amr_server *amr_server_t;

typedef struct {
  size_t hbm_budget_bytes;  /* device memory the waves may hold; 0: 120e9 */
  int max_waves;            /* waves in flight; <= 0: 8 */
  int max_wave_members;     /* requests per wave; <= 0: 256 */
  int device;               /* CUDA device; -1: the caller's current device */
  int tile, schedule;       /* amr_params.tile / .schedule of the waves;
                               0 and 0: 128-cell tiles, one tile per block */
} amr_server_params;

typedef struct {
  amr_member mesh;          /* the mesh, as for amr_create_batch */
  int n_coarse_steps;       /* >= 1 */
  int precision;            /* 4 or 8 */
} amr_request;

typedef struct {
  int64_t submitted, admitted, completed, failed, queued, running_waves;
  double latency_p50_ms, latency_p99_ms, latency_mean_ms;  /* submit -> result */
  double queue_p50_ms;      /* submit -> admission */
  double cell_updates;      /* leaf cell-updates of the completed requests */
  double span_s;            /* first submission -> last completion */
  int64_t device_bytes;     /* held by the waves in flight */
} amr_server_stats;

amr_status amr_server_create(const amr_server_params *p, amr_server_t *out);
amr_status amr_server_submit(amr_server_t s, const amr_request *req, int64_t *id_out);
/* Wait until request id (or, for id < 0, every submitted request) is
 * finished, at most timeout_s seconds (< 0: no limit); *done = 1 if so. */
amr_status amr_server_wait(amr_server_t s, int64_t id, double timeout_s, int *done);
/* Final state of a finished request, one level at a time, like amr_read. */
amr_status amr_server_read(amr_server_t s, int64_t id, int level, int64_t *n_oct_out,
                           uint64_t *keys, double *U, int64_t cap);
/* Drop a finished request's result. */
amr_status amr_server_release(amr_server_t s, int64_t id);
amr_status amr_server_get_stats(amr_server_t s, amr_server_stats *st);
/* Finish every submitted request, stop the scheduler, free everything. */
amr_status amr_server_destroy(amr_server_t s);

/* Wait for the handle's stream and its state-copy streams, and report any
 * pending device-side error. */
amr_status amr_sync(amr_handle h);

/* Text of the last error on the calling thread ("" if none). */
const char *amr_last_error(void);
const char *amr_status_string(amr_status s);

#ifdef __cplusplus
}
#endif
#endif
