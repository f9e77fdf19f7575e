/*
 * amr_oracle.h -- plain, slow FP64 CPU oracle of one AMR level step of
 * compressible Euler on a cell-by-cell octree (RAMSES-GPU, arXiv 2607.20704).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two are compared
 * element by element on the same seeded inputs.
 *
 * Conventions (paper Sec. 2, "Adaptive Mesh Refinement on the GPU"):
 *   - an oct is a 2x2x2 block of cells; an oct of level l has integer
 *     coordinates (i,j,k) in [0, 2^(l-1))^3 and cell size dx_l = 2^-l in the
 *     unit box; cell c = cx + 2cy + 4cz inside the oct;
 *   - nvar = 5 conservative variables U = (rho, rho u, rho v, rho w, E);
 *   - state arrays are structure-of-arrays: U[v*8n + 8*oct + c];
 *   - octs are held sorted by (level, Hilbert key, input index) (Sec. 2.2).
 *
 * Parity unpinned (any choice is "correct", one is fixed here and mirrored in
 * the CUDA path): the HLLC wave-speed estimate, the floor constants smallr /
 * smallc, the Hilbert orientation, the hash-table slot layout.
 */
#ifndef AMR_ORACLE_H
#define AMR_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NV 5
#define ORC_MAXLEV 15

enum {
  ORC_OK = 0,
  ORC_EINVAL = 1,
  ORC_ENOMEM = 2,
  ORC_EGRADING = 3,
  ORC_EDUP = 4
};

typedef struct {
  int levelmin, levelmax;
  double gamma, cfl;
  double smallr, smallc; /* floors: rho >= smallr, p >= rho*smallc^2/gamma */
  int reflux;            /* 1: reflux at coarse-fine faces; 0: negative control */
} orc_params;

typedef struct orc_mesh orc_mesh;

/* --- keys, hash function, Hilbert key (Sec. 2.1, 2.2, Sec. 6) ------------ */
uint64_t orc_pack_key(int level, uint32_t i, uint32_t j, uint32_t k);
uint64_t orc_fnv1a64_bytes(const uint8_t *bytes, size_t len);
uint64_t orc_fnv1a64_key(uint64_t key);
uint64_t orc_hilbert3(uint32_t x, uint32_t y, uint32_t z, int bits);

/* --- mesh ------------------------------------------------------------------ */
int orc_create(const orc_params *p, int64_t n, const uint8_t *lvl,
               const uint32_t *i, const uint32_t *j, const uint32_t *k,
               const double *U, orc_mesh **out);
void orc_destroy(orc_mesh *m);
int64_t orc_num_octs(const orc_mesh *m, int level);
int64_t orc_level_offset(const orc_mesh *m, int level);
int64_t orc_num_cache(const orc_mesh *m, int level);
int64_t orc_lookup(const orc_mesh *m, uint64_t key);
int orc_read(const orc_mesh *m, int level, uint64_t *keys, double *U);
int orc_read_R(const orc_mesh *m, int level, double *R);
int orc_read_split(const orc_mesh *m, int level, uint8_t *split);
int orc_read_nbr(const orc_mesh *m, int level, int64_t *nbr);
int orc_read_cache(const orc_mesh *m, int level, uint64_t *keys);
int orc_ghost(orc_mesh *m, int level, double *Ug);
int orc_write(orc_mesh *m, int level, const double *U);
void orc_totals(const orc_mesh *m, double tot[ORC_NV]);
/* the same sum over the leaf cells of one level */
void orc_level_totals(const orc_mesh *m, int level, double tot[ORC_NV]);

/* --- time stepping (Sec. 3; stage order of Table 1) ------------------------ */
double orc_cfl_dt(const orc_mesh *m);
int orc_step_level(orc_mesh *m, int level, double dt);
int orc_step_sample(orc_mesh *m, int level, double dt, int64_t ns,
                    const int64_t *octs, double *Unew);
int orc_advance(orc_mesh *m, int nsteps, double *dt_last);

/* --- regrid (Sec. 2.2: refinement, de-refinement, level and Hilbert order;
 *     then the ghost cache of Sec. 2.3) ------------------------------------- */
typedef struct {
  double grad_rho; /* relative jump 2|a-b|/(|a|+|b|) of rho to a face neighbour; <= 0: off */
  double grad_p;   /* the same for the pressure; <= 0: off */
  double mass;     /* cell mass rho dx^3 above which a cell refines; <= 0: off */
  int expand;      /* 1: a flag also flags the 26 same-level neighbours */
} orc_regrid_params;

/* Final refinement flags of every cell of the mesh (flag[8*oct + c], mesh
 * order): criterion, expansion, then the grading closure, finest level
 * first.  A flagged cell is split in the regridded mesh. */
int orc_flags(const orc_mesh *m, const orc_regrid_params *rp, uint8_t *flag);
/* Replace *pm by the regridded mesh: flagged leaves get a child oct whose
 * cells are minmod prolongations of their father, split cells left unflagged
 * lose their child oct, and the mesh is rebuilt in (level, Hilbert) order.
 * Pending reflux is dropped (regrid runs between coarse steps, where it is
 * zero).  created/removed: numbers of octs (may be NULL). */
int orc_regrid(orc_mesh **pm, const orc_regrid_params *rp, int64_t *created, int64_t *removed);
/* The same regrid with the final flags given (flag[8*oct + c], mesh order,
 * as orc_flags writes them): the mesh stages alone. */
int orc_regrid_flags(orc_mesh **pm, const uint8_t *flag, int64_t *created, int64_t *removed);

/* --- self-gravity: multigrid Poisson V-cycles on a periodic level (Sec. 5) --
 * Solves (sum of the 6 neighbours - 6 phi) / dx^2 = fourpiG (rho - mean rho)
 * on an n^3 periodic grid (n a power of two, arrays [x + n (y + n z)]):
 * red-black Gauss-Seidel smoothing (colour = parity of x + y + z, the parity
 * of the cell index inside its oct), residual restricted by the mean of the
 * 8 children, correction prolongated trilinearly with weights
 * (1, 3, 3, 9, 3, 9, 9, 27)/64, down to a 2^3 grid.  phi holds the initial
 * guess and receives the solution (mean subtracted at the end); resid[c]
 * gets the L2 norm of the residual after V-cycle c (may be NULL). */
int orc_mg_solve(int n, double dx, const double *rho, double fourpiG, int ncycles, int nu1,
                 int nu2, double *phi, double *resid);
/* L2 norm of the residual of phi for the source fourpiG (rho - mean rho) */
double orc_mg_residual(int n, double dx, const double *rho, double fourpiG, const double *phi);

/* Poisson on refined level L > levelmin (Sec. 5, level by level): the
 * cells of the level-L octs solve (sum of 6 neighbours - 6 phi) / dx^2 =
 * fourpiG (rho - rho_bar), rho the density of the state; a face to a cell
 * outside the level takes the value phi_b = (phic(father) + phic(cell
 * across the face at level L-1)) / 2 through the ghost 2 phi_b - phi (the
 * diagonal becomes -(6 + b)).  V-cycles over MG levels of the ancestors of
 * the level's cells down to levelmin (homogeneous Dirichlet corrections),
 * red-black Gauss-Seidel (2 + 2 sweeps, 8 on the coarsest), residual
 * restriction by the children's sum over 8 (order cx, cy, cz with cz
 * fastest), trilinear prolongation (1,3,3,9,3,9,9,27)/64.  phic: the
 * potential of level L-1's cells (8 n, read order); phi: in, the initial
 * guess, out, the result (8 n_L, read order); resid[ncycles] (may be NULL):
 * L2 norm of the residual after each cycle. */
int orc_mg_level(const orc_mesh *m, int L, double fourpiG, double rho_bar, const double *phic,
                 int ncycles, double *phi, double *resid);

/* --- particles: cloud-in-cell mass deposition (Sec. 4) ----------------------
 * np particles at positions (x, y, z) in the periodic unit box with masses m
 * deposit onto an n^3 grid of cells of size 1/n (n a power of two; arrays
 * [i + n (j + n k)]): along each axis s = x n - 1/2, i0 = floor(s),
 * f = s - i0, weights 1 - f for cell i0 and f for cell i0 + 1 (periodic);
 * a particle gives m (wx wy) wz to each of its 8 cells, corner order
 * c = cx + 2 cy + 4 cz, particles in index order; rho = sum / dx^3. */
int orc_cic_deposit(int n, int64_t np, const double *x, const double *y, const double *z,
                    const double *m, double *rho);
/* The same deposition onto the levels of a mesh (Sec. 4: at level l the
 * particles of level l and of all finer levels deposit, then the list is
 * split for level l+1).  The list of levelmin holds every particle; at level
 * l each particle of the list gives m (wx wy) wz, the CIC weights at cell
 * size 2^-l, to each of its 8 stencil cells that exists at level l (a cell
 * of a level-l oct); the list of level l+1 keeps, in order, the particles
 * whose host cell at level l (the cell containing the particle) is split.
 * rho[8*oct + c] (mesh order, all levels; split cells included) = sum /
 * dx_l^3; count[l] (16 entries) = particles in the list of level l. */
int orc_cic_deposit_levels(const orc_mesh *m, int64_t np, const double *x, const double *y,
                           const double *z, const double *mass, double *rho, int64_t *count);

/* --- independent cross-check solvers ----------------------------------------- */
int orc_uniform_step(int n, double *U, double gamma, double dt, double smallr,
                     double smallc);
double orc_uniform_cfl_dt(int n, const double *U, double gamma, double cfl,
                          double smallr, double smallc);
int orc_1d_step(int n, double *U, double gamma, double dt, double smallr,
                double smallc);

#ifdef __cplusplus
}
#endif
#endif
