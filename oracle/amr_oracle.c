/*
 * amr_oracle.c -- plain, slow FP64 CPU oracle of one AMR level step
 * (RAMSES-GPU, arXiv 2607.20704).  TEST INFRASTRUCTURE ONLY: loaded by the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark,
 * never by the product path.  Shares no code with the CUDA library.
 *
 * Built with -ffp-contract=off so every expression is evaluated exactly as
 * written, in source order, on every host.
 *
 * Passages followed (section / table of the paper):
 *   Sec. 2   octs of 2x2x2 cells, level-by-level arrays
 *   Sec. 2.1 hash key (i,j,k,l); neighbour (i-1,j,k,l); father (i/2,j/2,k/2,l-1)
 *   Sec. 2.2 octs sorted by level, then along the 3-D Hilbert curve
 *   Sec. 2.3 father/neighbour index arrays; ghost octs for missing neighbours,
 *            filled from the coarser level
 *   Sec. 3   MUSCL-Hancock predictor-corrector, HLLC Riemann solver, two ghost
 *            cells per side: a 6x6x6 stencil of uold -> unew per oct
 *   Table 1  stage order: set unew / godunov / set uold / upload (restriction)
 *   Sec. 6   FNV-1a 64-bit hash (named for the hash table)
 * The paper prints no formulas; each formula below is the cited textbook
 * method (Van Leer 1979 MUSCL-Hancock, Toro HLLC with min/max wave speeds,
 * Teyssier 2002 refluxing and restriction), in the reading documented with
 * the project.
 */
#include "amr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NV ORC_NV

/* ------------------------------------------------------------------------- */
/* keys (Sec. 2.1): 4-bit level, three 20-bit coordinates                    */
/* ------------------------------------------------------------------------- */
uint64_t orc_pack_key(int level, uint32_t i, uint32_t j, uint32_t k) {
  return ((uint64_t)level << 60) | ((uint64_t)i << 40) | ((uint64_t)j << 20) |
         (uint64_t)k;
}

/* FNV-1a 64 (Sec. 6): offset basis 0xcbf29ce484222325, prime 0x100000001b3. */
uint64_t orc_fnv1a64_bytes(const uint8_t *bytes, size_t len) {
  uint64_t h = 0xcbf29ce484222325ULL;
  for (size_t t = 0; t < len; ++t) {
    h ^= (uint64_t)bytes[t];
    h *= 0x100000001b3ULL;
  }
  return h;
}

/* The hash of a key is FNV-1a over its 8 little-endian bytes. */
uint64_t orc_fnv1a64_key(uint64_t key) {
  uint8_t b[8];
  for (int t = 0; t < 8; ++t) b[t] = (uint8_t)(key >> (8 * t));
  return orc_fnv1a64_bytes(b, 8);
}

/*
 * 3-D Hilbert index (Sec. 2.2) by Skilling's transpose method (J. Skilling,
 * "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004): undo the
 * excess work of the inverse transform from the top bit down, Gray-encode
 * across axes, then interleave the transposed bits, x most significant.
 */
uint64_t orc_hilbert3(uint32_t x, uint32_t y, uint32_t z, int bits) {
  if (bits <= 0) return 0;
  uint32_t X[3] = {x, y, z};
  uint32_t top = 1u << (bits - 1);
  for (uint32_t q = top; q > 1; q >>= 1) {
    uint32_t low = q - 1;
    for (int a = 0; a < 3; ++a) {
      if (X[a] & q) {
        X[0] ^= low;
      } else {
        uint32_t t = (X[0] ^ X[a]) & low;
        X[0] ^= t;
        X[a] ^= t;
      }
    }
  }
  X[1] ^= X[0];
  X[2] ^= X[1];
  uint32_t flip = 0;
  for (uint32_t q = top; q > 1; q >>= 1)
    if (X[2] & q) flip ^= q - 1;
  for (int a = 0; a < 3; ++a) X[a] ^= flip;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int a = 0; a < 3; ++a) h = (h << 1) | ((X[a] >> b) & 1u);
  return h;
}

/* ------------------------------------------------------------------------- */
/* mesh                                                                      */
/* ------------------------------------------------------------------------- */
struct orc_mesh {
  orc_params p;
  int64_t n;                   /* real octs, sorted */
  int64_t lo[ORC_MAXLEV + 2];  /* octs of level l are [lo[l], lo[l+1]) */
  uint8_t *lvl;
  uint32_t *ci, *cj, *ck;
  uint64_t *key;
  uint64_t *lk_key; /* all keys ascending, for lookup */
  int64_t *lk_idx;
  double *U;        /* [NV][8n] */
  double *R;        /* [NV][8n] pending reflux */
  uint8_t *split;   /* [8n] */
  int64_t *nbr;     /* [n][27]: >=0 real oct, <0 -(1+cache slot) */
  int64_t nc;       /* cache (ghost) octs, sorted by packed key */
  uint64_t *ckey;
  int64_t clo[ORC_MAXLEV + 2];
  double *Ug;       /* [NV][8nc] ghost values */
};

typedef struct {
  double g, smallr, smallp;
} phys;

static phys make_phys(const orc_params *p) {
  phys ph;
  ph.g = p->gamma;
  ph.smallr = p->smallr;
  ph.smallp = p->smallc * p->smallc / p->gamma;
  return ph;
}

static int key_level(uint64_t key) { return (int)(key >> 60); }
static uint32_t key_i(uint64_t key) { return (uint32_t)((key >> 40) & 0xFFFFF); }
static uint32_t key_j(uint64_t key) { return (uint32_t)((key >> 20) & 0xFFFFF); }
static uint32_t key_k(uint64_t key) { return (uint32_t)(key & 0xFFFFF); }

/* hash_get of Sec. 2.1, as a plain binary search: sorted index or -1. */
int64_t orc_lookup(const orc_mesh *m, uint64_t key) {
  int64_t a = 0, b = m->n;
  while (a < b) {
    int64_t h = a + (b - a) / 2;
    if (m->lk_key[h] < key)
      a = h + 1;
    else
      b = h;
  }
  if (a < m->n && m->lk_key[a] == key) return m->lk_idx[a];
  return -1;
}

static int64_t cache_lookup(const orc_mesh *m, uint64_t key) {
  int64_t a = 0, b = m->nc;
  while (a < b) {
    int64_t h = a + (b - a) / 2;
    if (m->ckey[h] < key)
      a = h + 1;
    else
      b = h;
  }
  if (a < m->nc && m->ckey[a] == key) return a;
  return -1;
}

static uint32_t wrap(int64_t x, int64_t period) {
  int64_t r = x % period;
  if (r < 0) r += period;
  return (uint32_t)r;
}

/* sort helpers */
typedef struct {
  int lvl;
  uint64_t h;
  int64_t idx;
} ord_rec;

static int cmp_ord(const void *a, const void *b) {
  const ord_rec *x = (const ord_rec *)a, *y = (const ord_rec *)b;
  if (x->lvl != y->lvl) return x->lvl < y->lvl ? -1 : 1;
  if (x->h != y->h) return x->h < y->h ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

typedef struct {
  uint64_t key;
  int64_t idx;
} kv_rec;

static int cmp_kv(const void *a, const void *b) {
  const kv_rec *x = (const kv_rec *)a, *y = (const kv_rec *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

void orc_destroy(orc_mesh *m) {
  if (!m) return;
  free(m->lvl);
  free(m->ci);
  free(m->cj);
  free(m->ck);
  free(m->key);
  free(m->lk_key);
  free(m->lk_idx);
  free(m->U);
  free(m->R);
  free(m->split);
  free(m->nbr);
  free(m->ckey);
  free(m->Ug);
  free(m);
}

/* restriction ("upload", Table 1): father cell = mean of its 8 children,
 * summed in child order. */
static void restrict_level(orc_mesh *m, int l) {
  if (l <= m->p.levelmin) return;
  int64_t N8 = 8 * m->n;
  for (int64_t o = m->lo[l]; o < m->lo[l + 1]; ++o) {
    uint64_t fk = orc_pack_key(l - 1, m->ci[o] >> 1, m->cj[o] >> 1, m->ck[o] >> 1);
    int64_t f = orc_lookup(m, fk);
    int fc = (int)((m->ci[o] & 1) + 2 * (m->cj[o] & 1) + 4 * (m->ck[o] & 1));
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
      for (int c = 0; c < 8; ++c) s += m->U[v * N8 + 8 * o + c];
      m->U[v * N8 + 8 * f + fc] = s * 0.125;
    }
  }
}

int orc_create(const orc_params *p, int64_t n, const uint8_t *lvl,
               const uint32_t *i, const uint32_t *j, const uint32_t *k,
               const double *U, orc_mesh **out) {
  *out = NULL;
  if (!p || n < 0 || p->levelmin < 1 || p->levelmax > ORC_MAXLEV ||
      p->levelmin > p->levelmax || !(p->gamma > 1.0))
    return ORC_EINVAL;
  for (int64_t t = 0; t < n; ++t) {
    int l = lvl[t];
    if (l < p->levelmin || l > p->levelmax) return ORC_EINVAL;
    uint32_t side = 1u << (l - 1);
    if (i[t] >= side || j[t] >= side || k[t] >= side) return ORC_EINVAL;
  }
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  if (!m) return ORC_ENOMEM;
  m->p = *p;
  m->n = n;
  size_t n8 = (size_t)(8 * n);
  m->lvl = (uint8_t *)malloc(n ? n : 1);
  m->ci = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  m->cj = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  m->ck = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  m->key = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
  m->lk_key = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
  m->lk_idx = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  m->U = (double *)calloc(NV * n8 + 1, sizeof(double));
  m->R = (double *)calloc(NV * n8 + 1, sizeof(double));
  m->split = (uint8_t *)calloc(n8 + 1, 1);
  m->nbr = (int64_t *)malloc(sizeof(int64_t) * 27 * (n ? n : 1));
  ord_rec *ord = (ord_rec *)malloc(sizeof(ord_rec) * (n ? n : 1));
  kv_rec *kv = (kv_rec *)malloc(sizeof(kv_rec) * (n ? n : 1));
  if (!m->lvl || !m->ci || !m->cj || !m->ck || !m->key || !m->lk_key ||
      !m->lk_idx || !m->U || !m->R || !m->split || !m->nbr || !ord || !kv) {
    free(ord);
    free(kv);
    orc_destroy(m);
    return ORC_ENOMEM;
  }

  /* Sec. 2.2: order by level, then Hilbert key; input index breaks ties. */
  for (int64_t t = 0; t < n; ++t) {
    ord[t].lvl = lvl[t];
    ord[t].h = orc_hilbert3(i[t], j[t], k[t], lvl[t] - 1);
    ord[t].idx = t;
  }
  qsort(ord, (size_t)n, sizeof(ord_rec), cmp_ord);
  for (int64_t t = 0; t < n; ++t) {
    int64_t s = ord[t].idx;
    m->lvl[t] = lvl[s];
    m->ci[t] = i[s];
    m->cj[t] = j[s];
    m->ck[t] = k[s];
    m->key[t] = orc_pack_key(lvl[s], i[s], j[s], k[s]);
    for (int v = 0; v < NV; ++v)
      for (int c = 0; c < 8; ++c)
        m->U[v * n8 + 8 * t + c] = U[v * n8 + 8 * s + c];
  }
  free(ord);
  for (int l = 0; l <= ORC_MAXLEV + 1; ++l) m->lo[l] = 0;
  {
    int64_t t = 0;
    for (int l = 0; l <= ORC_MAXLEV; ++l) {
      m->lo[l] = t;
      while (t < n && m->lvl[t] == l) ++t;
    }
    m->lo[ORC_MAXLEV + 1] = n;
  }

  /* lookup table and duplicate check */
  for (int64_t t = 0; t < n; ++t) {
    kv[t].key = m->key[t];
    kv[t].idx = t;
  }
  qsort(kv, (size_t)n, sizeof(kv_rec), cmp_kv);
  for (int64_t t = 0; t < n; ++t) {
    m->lk_key[t] = kv[t].key;
    m->lk_idx[t] = kv[t].idx;
    if (t > 0 && kv[t].key == kv[t - 1].key) {
      free(kv);
      orc_destroy(m);
      return ORC_EDUP;
    }
  }
  free(kv);

  /* the base level covers the whole box */
  {
    int64_t side = (int64_t)1 << (p->levelmin - 1);
    if (orc_num_octs(m, p->levelmin) != side * side * side) {
      orc_destroy(m);
      return ORC_EGRADING;
    }
  }
  /* grading: the 27 level l-1 cells around the father cell of every oct of
   * level l > levelmin exist (as leaf or split). */
  for (int64_t o = 0; o < n; ++o) {
    int l = m->lvl[o];
    if (l <= p->levelmin) continue;
    int64_t cells = (int64_t)1 << (l - 1); /* cells per side at level l-1 */
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          uint32_t x = wrap((int64_t)m->ci[o] + dx, cells);
          uint32_t y = wrap((int64_t)m->cj[o] + dy, cells);
          uint32_t z = wrap((int64_t)m->ck[o] + dz, cells);
          if (orc_lookup(m, orc_pack_key(l - 1, x >> 1, y >> 1, z >> 1)) < 0) {
            orc_destroy(m);
            return ORC_EGRADING;
          }
        }
  }
  /* split flags (Sec. 2.3 father index) */
  for (int64_t o = 0; o < n; ++o) {
    int l = m->lvl[o];
    if (l <= p->levelmin) continue;
    int64_t f = orc_lookup(m, orc_pack_key(l - 1, m->ci[o] >> 1, m->cj[o] >> 1,
                                           m->ck[o] >> 1));
    int fc = (int)((m->ci[o] & 1) + 2 * (m->cj[o] & 1) + 4 * (m->ck[o] & 1));
    m->split[8 * f + fc] = 1;
  }
  /* neighbour index array over the 3x3x3 block (Sec. 2.3); missing octs
   * become ghost (cache) octs, one per distinct key. */
  uint64_t *miss = (uint64_t *)malloc(sizeof(uint64_t) * (27 * n + 1));
  int64_t nm = 0;
  if (!miss) {
    orc_destroy(m);
    return ORC_ENOMEM;
  }
  for (int64_t o = 0; o < n; ++o) {
    int l = m->lvl[o];
    int64_t side = (int64_t)1 << (l - 1);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          uint64_t nk = orc_pack_key(l, wrap((int64_t)m->ci[o] + dx, side),
                                     wrap((int64_t)m->cj[o] + dy, side),
                                     wrap((int64_t)m->ck[o] + dz, side));
          int64_t e = orc_lookup(m, nk);
          if (e < 0) miss[nm++] = nk;
        }
  }
  qsort(miss, (size_t)nm, sizeof(uint64_t), cmp_u64);
  m->nc = 0;
  for (int64_t t = 0; t < nm; ++t)
    if (t == 0 || miss[t] != miss[t - 1]) miss[m->nc++] = miss[t];
  m->ckey = (uint64_t *)malloc(sizeof(uint64_t) * (m->nc ? m->nc : 1));
  m->Ug = (double *)calloc((size_t)(NV * 8 * m->nc + 1), sizeof(double));
  if (!m->ckey || !m->Ug) {
    free(miss);
    orc_destroy(m);
    return ORC_ENOMEM;
  }
  memcpy(m->ckey, miss, sizeof(uint64_t) * m->nc);
  free(miss);
  for (int l = 0; l <= ORC_MAXLEV + 1; ++l) m->clo[l] = m->nc;
  for (int l = ORC_MAXLEV; l >= 0; --l) {
    int64_t t = m->clo[l + 1];
    while (t > 0 && key_level(m->ckey[t - 1]) >= l) --t;
    m->clo[l] = t;
  }
  for (int64_t o = 0; o < n; ++o) {
    int l = m->lvl[o];
    int64_t side = (int64_t)1 << (l - 1);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          uint64_t nk = orc_pack_key(l, wrap((int64_t)m->ci[o] + dx, side),
                                     wrap((int64_t)m->cj[o] + dy, side),
                                     wrap((int64_t)m->ck[o] + dz, side));
          int64_t e = orc_lookup(m, nk);
          if (e < 0) e = -(1 + cache_lookup(m, nk));
          m->nbr[27 * o + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = e;
        }
  }
  /* split cells carry the restriction of their children */
  for (int l = p->levelmax; l > p->levelmin; --l) restrict_level(m, l);
  *out = m;
  return ORC_OK;
}

int64_t orc_num_octs(const orc_mesh *m, int level) {
  if (level < 0 || level > ORC_MAXLEV) return 0;
  return m->lo[level + 1] - m->lo[level];
}
int64_t orc_level_offset(const orc_mesh *m, int level) {
  if (level < 0 || level > ORC_MAXLEV) return 0;
  return m->lo[level];
}
int64_t orc_num_cache(const orc_mesh *m, int level) {
  if (level < 0 || level > ORC_MAXLEV) return 0;
  return m->clo[level + 1] - m->clo[level];
}

int orc_read(const orc_mesh *m, int level, uint64_t *keys, double *U) {
  int64_t a = m->lo[level], nl = orc_num_octs(m, level), N8 = 8 * m->n;
  for (int64_t t = 0; t < nl; ++t) {
    if (keys) keys[t] = m->key[a + t];
    if (U)
      for (int v = 0; v < NV; ++v)
        for (int c = 0; c < 8; ++c)
          U[v * 8 * nl + 8 * t + c] = m->U[v * N8 + 8 * (a + t) + c];
  }
  return ORC_OK;
}

int orc_read_R(const orc_mesh *m, int level, double *R) {
  int64_t a = m->lo[level], nl = orc_num_octs(m, level), N8 = 8 * m->n;
  for (int v = 0; v < NV; ++v)
    for (int64_t t = 0; t < 8 * nl; ++t) R[v * 8 * nl + t] = m->R[v * N8 + 8 * a + t];
  return ORC_OK;
}

int orc_read_split(const orc_mesh *m, int level, uint8_t *split) {
  int64_t a = m->lo[level], nl = orc_num_octs(m, level);
  memcpy(split, m->split + 8 * a, (size_t)(8 * nl));
  return ORC_OK;
}

int orc_read_nbr(const orc_mesh *m, int level, int64_t *nbr) {
  int64_t a = m->lo[level], nl = orc_num_octs(m, level);
  memcpy(nbr, m->nbr + 27 * a, sizeof(int64_t) * 27 * nl);
  return ORC_OK;
}

int orc_read_cache(const orc_mesh *m, int level, uint64_t *keys) {
  memcpy(keys, m->ckey + m->clo[level], sizeof(uint64_t) * orc_num_cache(m, level));
  return ORC_OK;
}

int orc_write(orc_mesh *m, int level, const double *U) {
  int64_t a = m->lo[level], nl = orc_num_octs(m, level), N8 = 8 * m->n;
  for (int v = 0; v < NV; ++v)
    for (int64_t t = 0; t < 8 * nl; ++t) m->U[v * N8 + 8 * a + t] = U[v * 8 * nl + t];
  return ORC_OK;
}

/* Sum over leaf cells of U dx^3. */
void orc_totals(const orc_mesh *m, double tot[NV]) {
  int64_t N8 = 8 * m->n;
  for (int v = 0; v < NV; ++v) tot[v] = 0.0;
  for (int64_t o = 0; o < m->n; ++o) {
    double dx = ldexp(1.0, -(int)m->lvl[o]);
    double vol = dx * dx * dx;
    for (int c = 0; c < 8; ++c) {
      if (m->split[8 * o + c]) continue;
      for (int v = 0; v < NV; ++v) tot[v] += m->U[v * N8 + 8 * o + c] * vol;
    }
  }
}

void orc_level_totals(const orc_mesh *m, int level, double tot[NV]) {
  int64_t N8 = 8 * m->n;
  double dx = ldexp(1.0, -level);
  double vol = dx * dx * dx;
  for (int v = 0; v < NV; ++v) tot[v] = 0.0;
  if (level < 0 || level > ORC_MAXLEV) return;
  for (int64_t o = m->lo[level]; o < m->lo[level + 1]; ++o)
    for (int c = 0; c < 8; ++c) {
      if (m->split[8 * o + c]) continue;
      for (int v = 0; v < NV; ++v) tot[v] += m->U[v * N8 + 8 * o + c] * vol;
    }
}

/* ------------------------------------------------------------------------- */
/* point-wise pieces of the Godunov scheme (Sec. 3)                          */
/* ------------------------------------------------------------------------- */

/* conservative -> primitive (rho, u, v, w, p) with floors */
static void cons_to_prim(const phys *ph, const double u[NV], double w[NV]) {
  double r = u[0] > ph->smallr ? u[0] : ph->smallr;
  double vx = u[1] / r, vy = u[2] / r, vz = u[3] / r;
  double ek = 0.5 * r * ((vx * vx + vy * vy) + vz * vz);
  double p = (ph->g - 1.0) * (u[4] - ek);
  double pf = r * ph->smallp;
  if (p < pf) p = pf;
  w[0] = r;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = p;
}

/* minmod(a,b) = 0 if ab <= 0, else sign(a) min(|a|,|b|) */
static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  if (a > 0.0) return a < b ? a : b;
  return a > b ? a : b;
}

/* Hancock half-step of the primitive Euler system:
 *   W* = W + dt/(2dx) S,  with dW[d] the limited increment along axis d
 *   S_rho = -sum_d (u_d d_d rho + rho d_d u_d)
 *   S_ua  = -sum_d u_d d_d u_a - d_a p / rho
 *   S_p   = -sum_d (u_d d_d p + gamma p d_d u_d)                            */
static void predict(const phys *ph, double dtdx, const double w[NV],
                    double dw[3][NV], double ws[NV]) {
  double r = w[0], p = w[4], g = ph->g;
  const double *u = w + 1;
  double s[NV];
  s[0] = -(((u[0] * dw[0][0] + r * dw[0][1]) + (u[1] * dw[1][0] + r * dw[1][2])) +
           (u[2] * dw[2][0] + r * dw[2][3]));
  for (int a = 0; a < 3; ++a)
    s[1 + a] = -((u[0] * dw[0][1 + a] + u[1] * dw[1][1 + a]) + u[2] * dw[2][1 + a]) -
               dw[a][4] / r;
  s[4] = -(((u[0] * dw[0][4] + g * p * dw[0][1]) + (u[1] * dw[1][4] + g * p * dw[1][2])) +
           (u[2] * dw[2][4] + g * p * dw[2][3]));
  for (int v = 0; v < NV; ++v) ws[v] = w[v] + 0.5 * dtdx * s[v];
}

/* face state W* +- dW/2 with floors */
static void face_state(const phys *ph, const double ws[NV], const double dw[NV],
                       int plus, double q[NV]) {
  for (int v = 0; v < NV; ++v) q[v] = plus ? ws[v] + 0.5 * dw[v] : ws[v] - 0.5 * dw[v];
  if (q[0] < ph->smallr) q[0] = ph->smallr;
  double pf = q[0] * ph->smallp;
  if (q[4] < pf) q[4] = pf;
}

/* HLLC flux across a face normal to axis d (Toro's HLLC with wave speeds
 * S_L = min(u)-max(c), S_R = max(u)+max(c)); the flux is the physical flux of
 * the state sampled at x/t = 0. */
static void hllc(const phys *ph, const double qL[NV], const double qR[NV], int d,
                 double F[NV]) {
  int in = 1 + d, t1 = 1 + (d + 1) % 3, t2 = 1 + (d + 2) % 3;
  if (t1 > t2) {
    int x = t1;
    t1 = t2;
    t2 = x;
  }
  double g = ph->g;
  double rl = qL[0], ul = qL[in], pl = qL[4];
  double rr = qR[0], ur = qR[in], pr = qR[4];
  double el = pl / (g - 1.0) + 0.5 * rl * ((qL[1] * qL[1] + qL[2] * qL[2]) + qL[3] * qL[3]);
  double er = pr / (g - 1.0) + 0.5 * rr * ((qR[1] * qR[1] + qR[2] * qR[2]) + qR[3] * qR[3]);
  double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
  double cmax = cl > cr ? cl : cr;
  double sl = (ul < ur ? ul : ur) - cmax;
  double sr = (ul > ur ? ul : ur) + cmax;
  double rcl = rl * (ul - sl), rcr = rr * (sr - ur);
  double ustar = ((rcr * ur + rcl * ul) + (pl - pr)) / (rcl + rcr);
  double pstar = ((rcr * pl + rcl * pr) + rcl * rcr * (ul - ur)) / (rcl + rcr);
  double ro, uo, po, eo, v1, v2;
  if (sl > 0.0) {
    ro = rl; uo = ul; po = pl; eo = el; v1 = qL[t1]; v2 = qL[t2];
  } else if (ustar > 0.0) {
    ro = rl * (sl - ul) / (sl - ustar);
    eo = ((sl - ul) * el - pl * ul + pstar * ustar) / (sl - ustar);
    uo = ustar; po = pstar; v1 = qL[t1]; v2 = qL[t2];
  } else if (sr > 0.0) {
    ro = rr * (sr - ur) / (sr - ustar);
    eo = ((sr - ur) * er - pr * ur + pstar * ustar) / (sr - ustar);
    uo = ustar; po = pstar; v1 = qR[t1]; v2 = qR[t2];
  } else {
    ro = rr; uo = ur; po = pr; eo = er; v1 = qR[t1]; v2 = qR[t2];
  }
  F[0] = ro * uo;
  F[in] = ro * uo * uo + po;
  F[t1] = ro * uo * v1;
  F[t2] = ro * uo * v2;
  F[4] = (eo + po) * uo;
}

/* ------------------------------------------------------------------------- */
/* ghost octs (Sec. 2.3): minmod-limited prolongation of the father cell      */
/* ------------------------------------------------------------------------- */

/* value of the cell (x,y,z) of level L, or of the coarser cell covering it
 * when its oct does not exist; returns 0 on success. */
static int cell_value(const orc_mesh *m, int L, int64_t x, int64_t y, int64_t z,
                      double u[NV]) {
  int64_t N8 = 8 * m->n;
  while (L >= m->p.levelmin) {
    int64_t side = (int64_t)1 << L;
    uint32_t X = wrap(x, side), Y = wrap(y, side), Z = wrap(z, side);
    int64_t o = orc_lookup(m, orc_pack_key(L, X >> 1, Y >> 1, Z >> 1));
    if (o >= 0) {
      int c = (int)((X & 1) + 2 * (Y & 1) + 4 * (Z & 1));
      for (int v = 0; v < NV; ++v) u[v] = m->U[v * N8 + 8 * o + c];
      return 0;
    }
    x = X >> 1;
    y = Y >> 1;
    z = Z >> 1;
    --L;
  }
  return 1;
}

static int fill_ghost(orc_mesh *m, int64_t s) {
  uint64_t key = m->ckey[s];
  int l = key_level(key);
  int64_t gi = key_i(key), gj = key_j(key), gk = key_k(key);
  int64_t NC8 = 8 * m->nc;
  double uc[NV], up[NV], um[NV], sl[3][NV];
  /* the father cell of a ghost oct of level l is cell (gi,gj,gk) of l-1 */
  int64_t side = (int64_t)1 << (l - 1);
  int64_t fo = orc_lookup(m, orc_pack_key(l - 1, (uint32_t)gi >> 1, (uint32_t)gj >> 1,
                                          (uint32_t)gk >> 1));
  if (l - 1 < m->p.levelmin || fo < 0) return ORC_EGRADING;
  (void)side;
  if (cell_value(m, l - 1, gi, gj, gk, uc)) return ORC_EGRADING;
  for (int d = 0; d < 3; ++d) {
    int64_t ex = d == 0, ey = d == 1, ez = d == 2;
    if (cell_value(m, l - 1, gi + ex, gj + ey, gk + ez, up)) return ORC_EGRADING;
    if (cell_value(m, l - 1, gi - ex, gj - ey, gk - ez, um)) return ORC_EGRADING;
    for (int v = 0; v < NV; ++v) sl[d][v] = minmod(up[v] - uc[v], uc[v] - um[v]);
  }
  for (int c = 0; c < 8; ++c) {
    double hx = (c & 1) ? 0.25 : -0.25;
    double hy = (c & 2) ? 0.25 : -0.25;
    double hz = (c & 4) ? 0.25 : -0.25;
    for (int v = 0; v < NV; ++v)
      m->Ug[v * NC8 + 8 * s + c] = ((uc[v] + hx * sl[0][v]) + hy * sl[1][v]) + hz * sl[2][v];
  }
  return ORC_OK;
}

int orc_ghost(orc_mesh *m, int level, double *Ug) {
  int64_t a = m->clo[level], nl = orc_num_cache(m, level), NC8 = 8 * m->nc;
  for (int64_t s = a; s < a + nl; ++s) {
    int e = fill_ghost(m, s);
    if (e) return e;
  }
  for (int v = 0; v < NV; ++v)
    for (int64_t t = 0; t < 8 * nl; ++t) Ug[v * 8 * nl + t] = m->Ug[v * NC8 + 8 * a + t];
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Godunov update of one oct on its 6x6x6 stencil (Sec. 3)                    */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t X; /* coarse cell receiving the flux */
  int dir, a, b;
  double v[NV];
} contrib;

typedef struct {
  contrib *c;
  int64_t n, cap;
} contrib_list;

static int push_contrib(contrib_list *L, const contrib *c) {
  if (L->n == L->cap) {
    int64_t nc = L->cap ? 2 * L->cap : 1024;
    contrib *p = (contrib *)realloc(L->c, sizeof(contrib) * nc);
    if (!p) return ORC_ENOMEM;
    L->c = p;
    L->cap = nc;
  }
  L->c[L->n++] = *c;
  return ORC_OK;
}

static int cmp_contrib(const void *a, const void *b) {
  const contrib *x = (const contrib *)a, *y = (const contrib *)b;
  if (x->X != y->X) return x->X < y->X ? -1 : 1;
  if (x->dir != y->dir) return x->dir < y->dir ? -1 : 1;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  return 0;
}

#define T6(x, y, z) (((x) + 2) + 6 * (((y) + 2) + 6 * ((z) + 2)))

/* Computes the new state of the 8 cells of oct o into unew[v*8+c]; when
 * `contribs` is non-NULL, appends the reflux contributions of its coarse-fine
 * faces. */
static int godunov_oct(const orc_mesh *m, int64_t o, double dt, double *unew,
                       contrib_list *contribs) {
  const phys ph = make_phys(&m->p);
  int l = m->lvl[o];
  double dtdx = dt / ldexp(1.0, -l);
  int64_t N8 = 8 * m->n, NC8 = 8 * m->nc;
  double u[216][NV], w[216][NV], dw[216][3][NV], ws[216][NV];
  int split[216], ghost_slot[216];

  /* 1. gather uold on the 6x6x6 stencil: the oct and its 26 neighbours */
  for (int z = -2; z < 4; ++z)
    for (int y = -2; y < 4; ++y)
      for (int x = -2; x < 4; ++x) {
        int ox = x < 0 ? -1 : (x > 1 ? 1 : 0);
        int oy = y < 0 ? -1 : (y > 1 ? 1 : 0);
        int oz = z < 0 ? -1 : (z > 1 ? 1 : 0);
        int c = (x - 2 * ox) + 2 * (y - 2 * oy) + 4 * (z - 2 * oz);
        int64_t e = m->nbr[27 * o + (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
        int t = T6(x, y, z);
        if (e >= 0) {
          for (int v = 0; v < NV; ++v) u[t][v] = m->U[v * N8 + 8 * e + c];
          split[t] = m->split[8 * e + c];
          ghost_slot[t] = -1;
        } else {
          int64_t s = -1 - e;
          for (int v = 0; v < NV; ++v) u[t][v] = m->Ug[v * NC8 + 8 * s + c];
          split[t] = 0;
          ghost_slot[t] = (int)(s - m->clo[l]);
        }
      }
  /* 2. conservative -> primitive on the whole stencil */
  for (int t = 0; t < 216; ++t) cons_to_prim(&ph, u[t], w[t]);
  /* 3. limited slopes and Hancock predictor on [-1,3)^3 */
  for (int z = -1; z < 3; ++z)
    for (int y = -1; y < 3; ++y)
      for (int x = -1; x < 3; ++x) {
        int t = T6(x, y, z);
        int tp[3] = {T6(x + 1, y, z), T6(x, y + 1, z), T6(x, y, z + 1)};
        int tm[3] = {T6(x - 1, y, z), T6(x, y - 1, z), T6(x, y, z - 1)};
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < NV; ++v)
            dw[t][d][v] = minmod(w[tp[d]][v] - w[t][v], w[t][v] - w[tm[d]][v]);
        predict(&ph, dtdx, w[t], dw[t], ws[t]);
      }
  /* 4. HLLC on the 6 faces of each cell of the oct, 5. update */
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        int c = cx + 2 * cy + 4 * cz;
        int t = T6(cx, cy, cz);
        if (split[t]) {
          for (int v = 0; v < NV; ++v) unew[v * 8 + c] = u[t][v];
          continue;
        }
        double F[3][2][NV];
        for (int d = 0; d < 3; ++d)
          for (int side = 0; side < 2; ++side) {
            int dx = d == 0 ? (side ? 1 : -1) : 0;
            int dy = d == 1 ? (side ? 1 : -1) : 0;
            int dz = d == 2 ? (side ? 1 : -1) : 0;
            int tn = T6(cx + dx, cy + dy, cz + dz);
            int tl = side ? t : tn, tr = side ? tn : t;
            if (split[tl] || split[tr]) {
              for (int v = 0; v < NV; ++v) F[d][side][v] = 0.0;
              continue;
            }
            double qL[NV], qR[NV];
            face_state(&ph, ws[tl], dw[tl][d], 1, qL);
            face_state(&ph, ws[tr], dw[tr][d], 0, qR);
            hllc(&ph, qL, qR, d, F[d][side]);
            /* reflux (Teyssier 2002): a face shared with a ghost oct is a
             * coarse-fine face; the coarse cell X covering the ghost gets
             * sigma * dt/dx * F / 8, sigma = +1 when X is on the + side. */
            if (contribs && ghost_slot[tn] >= 0 && m->p.reflux) {
              int64_t s = m->clo[l] + ghost_slot[tn];
              uint64_t gk = m->ckey[s];
              int64_t fo = orc_lookup(m, orc_pack_key(l - 1, key_i(gk) >> 1,
                                                      key_j(gk) >> 1, key_k(gk) >> 1));
              int fc = (int)((key_i(gk) & 1) + 2 * (key_j(gk) & 1) + 4 * (key_k(gk) & 1));
              contrib cb;
              cb.X = 8 * fo + fc;
              /* seen from X the face lies on its -d side when the fine cell
               * is on the - side of the face, i.e. side == 0 */
              cb.dir = 2 * d + (side ? 0 : 1);
              int ccell[3] = {cx, cy, cz};
              int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
              cb.a = ccell[d1];
              cb.b = ccell[d2];
              double sigma = side ? 1.0 : -1.0;
              for (int v = 0; v < NV; ++v) cb.v[v] = sigma * dtdx * F[d][side][v] / 8.0;
              if (push_contrib(contribs, &cb)) return ORC_ENOMEM;
            }
          }
        int64_t gc = 8 * o + c;
        for (int v = 0; v < NV; ++v) {
          double du = ((F[0][0][v] - F[0][1][v]) + (F[1][0][v] - F[1][1][v])) +
                      (F[2][0][v] - F[2][1][v]);
          unew[v * 8 + c] = (u[t][v] + dtdx * du) + m->R[v * N8 + gc];
        }
      }
  return ORC_OK;
}

/* One level step: ghosts, Godunov on every oct of the level, set uold,
 * reflux into level l-1, restriction into level l-1. */
int orc_step_level(orc_mesh *m, int l, double dt) {
  if (l < m->p.levelmin || l > m->p.levelmax) return ORC_EINVAL;
  int64_t a = m->lo[l], nl = orc_num_octs(m, l), N8 = 8 * m->n;
  if (nl == 0) return ORC_OK;
  for (int64_t s = m->clo[l]; s < m->clo[l + 1]; ++s) {
    int e = fill_ghost(m, s);
    if (e) return e;
  }
  double *unew = (double *)malloc(sizeof(double) * NV * 8 * nl);
  if (!unew) return ORC_ENOMEM;
  contrib_list L = {NULL, 0, 0};
  for (int64_t t = 0; t < nl; ++t) {
    double tmp[NV * 8];
    int e = godunov_oct(m, a + t, dt, tmp, l > m->p.levelmin ? &L : NULL);
    if (e) {
      free(unew);
      free(L.c);
      return e;
    }
    for (int v = 0; v < NV; ++v)
      for (int c = 0; c < 8; ++c) unew[v * 8 * nl + 8 * t + c] = tmp[v * 8 + c];
  }
  /* set uold: leaf cells take the new state, their pending reflux is spent */
  for (int64_t t = 0; t < nl; ++t)
    for (int c = 0; c < 8; ++c) {
      int64_t gc = 8 * (a + t) + c;
      if (m->split[gc]) continue;
      for (int v = 0; v < NV; ++v) {
        m->U[v * N8 + gc] = unew[v * 8 * nl + 8 * t + c];
        m->R[v * N8 + gc] = 0.0;
      }
    }
  free(unew);
  /* reflux, in the fixed order (coarse cell, direction, fine face) */
  qsort(L.c, (size_t)L.n, sizeof(contrib), cmp_contrib);
  for (int64_t t = 0; t < L.n; ++t)
    for (int v = 0; v < NV; ++v) m->R[v * N8 + L.c[t].X] += L.c[t].v[v];
  free(L.c);
  restrict_level(m, l);
  return ORC_OK;
}

/* New state of selected octs of level l after one step from the current
 * state, without changing the mesh. */
int orc_step_sample(orc_mesh *m, int level, double dt, int64_t ns, const int64_t *octs,
                    double *Unew) {
  if (level < m->p.levelmin || level > m->p.levelmax) return ORC_EINVAL;
  for (int64_t s = m->clo[level]; s < m->clo[level + 1]; ++s) {
    int e = fill_ghost(m, s);
    if (e) return e;
  }
  for (int64_t t = 0; t < ns; ++t) {
    int64_t o = octs[t];
    if (o < m->lo[level] || o >= m->lo[level + 1]) return ORC_EINVAL;
    double tmp[NV * 8];
    int e = godunov_oct(m, o, dt, tmp, NULL);
    if (e) return e;
    for (int v = 0; v < NV; ++v)
      for (int c = 0; c < 8; ++c) Unew[v * 8 * ns + 8 * t + c] = tmp[v * 8 + c];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* time step (compute dt, Table 1) and the level-by-level W-cycle            */
/* ------------------------------------------------------------------------- */
double orc_cfl_dt(const orc_mesh *m) {
  const phys ph = make_phys(&m->p);
  int64_t N8 = 8 * m->n;
  double dt = INFINITY;
  for (int l = m->p.levelmin; l <= m->p.levelmax; ++l) {
    double smax = 0.0;
    int any = 0;
    for (int64_t o = m->lo[l]; o < m->lo[l + 1]; ++o)
      for (int c = 0; c < 8; ++c) {
        if (m->split[8 * o + c]) continue;
        double u[NV], w[NV];
        for (int v = 0; v < NV; ++v) u[v] = m->U[v * N8 + 8 * o + c];
        cons_to_prim(&ph, u, w);
        double cs = sqrt(ph.g * w[4] / w[0]);
        double s = ((fabs(w[1]) + cs) + (fabs(w[2]) + cs)) + (fabs(w[3]) + cs);
        if (s > smax) smax = s;
        any = 1;
      }
    if (!any) continue;
    double dtl = m->p.cfl * ldexp(1.0, -l) / smax;
    double dtc = dtl * ldexp(1.0, l - m->p.levelmin);
    if (dtc < dt) dt = dtc;
  }
  return dt;
}

static int advance_level(orc_mesh *m, int l, double dt) {
  if (l + 1 <= m->p.levelmax && orc_num_octs(m, l + 1) > 0) {
    int e = advance_level(m, l + 1, 0.5 * dt);
    if (e) return e;
    e = advance_level(m, l + 1, 0.5 * dt);
    if (e) return e;
  }
  return orc_step_level(m, l, dt);
}

int orc_advance(orc_mesh *m, int nsteps, double *dt_last) {
  for (int s = 0; s < nsteps; ++s) {
    double dt = orc_cfl_dt(m);
    if (dt_last) *dt_last = dt;
    int e = advance_level(m, m->p.levelmin, dt);
    if (e) return e;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* independent uniform periodic solvers (cross-checks)                       */
/* ------------------------------------------------------------------------- */

/* One step of the same scheme on an n^3 periodic array U[v][x + n(y + nz)],
 * dx = 1/n, written directly on the array with no octs, hash or ghosts. */
int orc_uniform_step(int n, double *U, double gamma, double dt, double smallr,
                     double smallc) {
  orc_params pp = {0, 0, gamma, 0.0, smallr, smallc, 1};
  phys ph = make_phys(&pp);
  int64_t nn = (int64_t)n * n * n;
  double dtdx = dt * n;
  double *W = (double *)malloc(sizeof(double) * NV * nn);
  double *DW = (double *)malloc(sizeof(double) * 3 * NV * nn);
  double *WS = (double *)malloc(sizeof(double) * NV * nn);
  double *FX = (double *)malloc(sizeof(double) * 3 * NV * nn); /* flux on the - face */
  if (!W || !DW || !WS || !FX) {
    free(W); free(DW); free(WS); free(FX);
    return ORC_ENOMEM;
  }
#define IDX(x, y, z) ((int64_t)wrap((x), n) + (int64_t)n * ((int64_t)wrap((y), n) + (int64_t)n * wrap((z), n)))
  for (int64_t t = 0; t < nn; ++t) {
    double u[NV], w[NV];
    for (int v = 0; v < NV; ++v) u[v] = U[v * nn + t];
    cons_to_prim(&ph, u, w);
    for (int v = 0; v < NV; ++v) W[t * NV + v] = w[v];
  }
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        int64_t t = IDX(x, y, z);
        int64_t tp[3] = {IDX(x + 1, y, z), IDX(x, y + 1, z), IDX(x, y, z + 1)};
        int64_t tm[3] = {IDX(x - 1, y, z), IDX(x, y - 1, z), IDX(x, y, z - 1)};
        double dw[3][NV];
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < NV; ++v)
            dw[d][v] = minmod(W[tp[d] * NV + v] - W[t * NV + v], W[t * NV + v] - W[tm[d] * NV + v]);
        double ws[NV];
        predict(&ph, dtdx, &W[t * NV], dw, ws);
        for (int v = 0; v < NV; ++v) WS[t * NV + v] = ws[v];
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < NV; ++v) DW[(t * 3 + d) * NV + v] = dw[d][v];
      }
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        int64_t t = IDX(x, y, z);
        int64_t tm[3] = {IDX(x - 1, y, z), IDX(x, y - 1, z), IDX(x, y, z - 1)};
        for (int d = 0; d < 3; ++d) {
          double qL[NV], qR[NV], F[NV];
          face_state(&ph, &WS[tm[d] * NV], &DW[(tm[d] * 3 + d) * NV], 1, qL);
          face_state(&ph, &WS[t * NV], &DW[(t * 3 + d) * NV], 0, qR);
          hllc(&ph, qL, qR, d, F);
          for (int v = 0; v < NV; ++v) FX[(t * 3 + d) * NV + v] = F[v];
        }
      }
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        int64_t t = IDX(x, y, z);
        int64_t tp[3] = {IDX(x + 1, y, z), IDX(x, y + 1, z), IDX(x, y, z + 1)};
        for (int v = 0; v < NV; ++v) {
          double du = ((FX[(t * 3 + 0) * NV + v] - FX[(tp[0] * 3 + 0) * NV + v]) +
                       (FX[(t * 3 + 1) * NV + v] - FX[(tp[1] * 3 + 1) * NV + v])) +
                      (FX[(t * 3 + 2) * NV + v] - FX[(tp[2] * 3 + 2) * NV + v]);
          U[v * nn + t] = (U[v * nn + t] + dtdx * du) + 0.0;
        }
      }
#undef IDX
  free(W); free(DW); free(WS); free(FX);
  return ORC_OK;
}

double orc_uniform_cfl_dt(int n, const double *U, double gamma, double cfl, double smallr,
                          double smallc) {
  orc_params pp = {0, 0, gamma, cfl, smallr, smallc, 1};
  phys ph = make_phys(&pp);
  int64_t nn = (int64_t)n * n * n;
  double smax = 0.0;
  for (int64_t t = 0; t < nn; ++t) {
    double u[NV], w[NV];
    for (int v = 0; v < NV; ++v) u[v] = U[v * nn + t];
    cons_to_prim(&ph, u, w);
    double cs = sqrt(ph.g * w[4] / w[0]);
    double s = ((fabs(w[1]) + cs) + (fabs(w[2]) + cs)) + (fabs(w[3]) + cs);
    if (s > smax) smax = s;
  }
  return cfl * (1.0 / n) / smax;
}

/* One step of the scheme along x only, on U[v][x] (n cells, periodic,
 * dx = 1/n): the 1-D restriction of the 3-D scheme to states that do not
 * vary along y and z. */
int orc_1d_step(int n, double *U, double gamma, double dt, double smallr, double smallc) {
  orc_params pp = {0, 0, gamma, 0.0, smallr, smallc, 1};
  phys ph = make_phys(&pp);
  double dtdx = dt * n;
  double *W = (double *)malloc(sizeof(double) * NV * n);
  double *WS = (double *)malloc(sizeof(double) * NV * n);
  double *DW = (double *)malloc(sizeof(double) * NV * n);
  double *F = (double *)malloc(sizeof(double) * NV * (n + 1));
  if (!W || !WS || !DW || !F) {
    free(W); free(WS); free(DW); free(F);
    return ORC_ENOMEM;
  }
  for (int x = 0; x < n; ++x) {
    double u[NV];
    for (int v = 0; v < NV; ++v) u[v] = U[v * n + x];
    cons_to_prim(&ph, u, &W[x * NV]);
  }
  for (int x = 0; x < n; ++x) {
    int xp = (x + 1) % n, xm = (x + n - 1) % n;
    double dw[3][NV];
    for (int v = 0; v < NV; ++v) {
      dw[0][v] = minmod(W[xp * NV + v] - W[x * NV + v], W[x * NV + v] - W[xm * NV + v]);
      dw[1][v] = 0.0;
      dw[2][v] = 0.0;
    }
    predict(&ph, dtdx, &W[x * NV], dw, &WS[x * NV]);
    for (int v = 0; v < NV; ++v) DW[x * NV + v] = dw[0][v];
  }
  for (int x = 0; x < n; ++x) { /* flux on the - face of x */
    int xm = (x + n - 1) % n;
    double qL[NV], qR[NV];
    face_state(&ph, &WS[xm * NV], &DW[xm * NV], 1, qL);
    face_state(&ph, &WS[x * NV], &DW[x * NV], 0, qR);
    hllc(&ph, qL, qR, 0, &F[x * NV]);
  }
  for (int x = 0; x < n; ++x) {
    int xp = (x + 1) % n;
    for (int v = 0; v < NV; ++v)
      U[v * n + x] = U[v * n + x] + dtdx * (F[x * NV + v] - F[xp * NV + v]);
  }
  free(W); free(WS); free(DW); free(F);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* regrid (Sec. 2.2 "Refinement and De-Refinement")                          */
/*                                                                           */
/* The paper names the four stages (refine flagged cells by new child octs,  */
/* remove the child oct of a split cell no longer flagged, level bucket sort,*/
/* Hilbert sort) and leaves the criterion and the grading closure to the    */
/* RAMSES conventions; the readings taken here:                             */
/*   flag   a cell of level l < levelmax is flagged when, to one of its six  */
/*          face neighbours (the same-level cell, else the coarser cell      */
/*          covering it), the relative jump 2|a-b|/(|a|+|b|) of rho exceeds  */
/*          grad_rho or that of p exceeds grad_p, or when rho dx_l^3 exceeds */
/*          mass (rho and p are the primitive variables of the scheme, with */
/*          its floors; a jump between two zeros is 0);                      */
/*   expand with expand = 1 a flag also flags the 26 same-level cells       */
/*          around it that exist;                                            */
/*   grade  finest level first: a flagged cell X of level l flags, at level  */
/*          l-1, the cell covering each of the 27 level-l cells around X, so */
/*          the child oct of X has its 27 level-l neighbours (the 2:1 rule)  */
/*          and the keep rule follows (X's own father is among them);       */
/*   split  in the new mesh the flagged cells are the split ones: children  */
/*          of flagged leaves are created, those of unflagged split cells   */
/*          are removed, so a cell refines by at most one level per regrid;  */
/*   state  new child octs, coarsest level first, are minmod prolongations  */
/*          of their father from the father's six face neighbours in the new */
/*          mesh (the ghost-oct formula); then the mesh is rebuilt as at     */
/*          creation (order, lookup, grading check, cache, restriction).     */
/* ------------------------------------------------------------------------- */

/* relative jump 2|a-b|/(|a|+|b|) of two values (0 when both are 0) */
static double rel_jump(double a, double b) {
  double s = fabs(a) + fabs(b);
  return s > 0.0 ? 2.0 * fabs(a - b) / s : 0.0;
}

/* oct index of the cell (x,y,z) of level L (same level only), or -1 */
static int64_t cell_oct(const orc_mesh *m, int L, int64_t x, int64_t y, int64_t z, int *c) {
  int64_t side = (int64_t)1 << L;
  uint32_t X = wrap(x, side), Y = wrap(y, side), Z = wrap(z, side);
  *c = (int)((X & 1) + 2 * (Y & 1) + 4 * (Z & 1));
  return orc_lookup(m, orc_pack_key(L, X >> 1, Y >> 1, Z >> 1));
}

static int raw_flag(const orc_mesh *m, const phys *ph, const orc_regrid_params *rp, int64_t o,
                    int c) {
  int64_t N8 = 8 * m->n;
  int l = m->lvl[o];
  double uc[NV], wc[NV];
  for (int v = 0; v < NV; ++v) uc[v] = m->U[v * N8 + 8 * o + c];
  if (rp->mass > 0.0 && ldexp(uc[0], -3 * l) > rp->mass) return 1;
  if (!(rp->grad_rho > 0.0) && !(rp->grad_p > 0.0)) return 0;
  cons_to_prim(ph, uc, wc);
  int64_t x = 2 * (int64_t)m->ci[o] + (c & 1), y = 2 * (int64_t)m->cj[o] + ((c >> 1) & 1),
          z = 2 * (int64_t)m->ck[o] + ((c >> 2) & 1);
  for (int d = 0; d < 3; ++d)
    for (int s = -1; s <= 1; s += 2) {
      double un[NV], wn[NV];
      if (cell_value(m, l, x + (d == 0) * s, y + (d == 1) * s, z + (d == 2) * s, un)) continue;
      cons_to_prim(ph, un, wn);
      if (rp->grad_rho > 0.0 && rel_jump(wn[0], wc[0]) > rp->grad_rho) return 1;
      if (rp->grad_p > 0.0 && rel_jump(wn[4], wc[4]) > rp->grad_p) return 1;
    }
  return 0;
}

int orc_flags(const orc_mesh *m, const orc_regrid_params *rp, uint8_t *flag) {
  const phys ph = make_phys(&m->p);
  int64_t n8 = 8 * m->n;
  uint8_t *raw = (uint8_t *)calloc((size_t)n8 + 1, 1);
  if (!raw) return ORC_ENOMEM;
  memset(flag, 0, (size_t)n8);
  for (int64_t o = 0; o < m->n; ++o) {
    if (m->lvl[o] >= m->p.levelmax) continue;
    for (int c = 0; c < 8; ++c) raw[8 * o + c] = (uint8_t)raw_flag(m, &ph, rp, o, c);
  }
  /* expansion over the 3x3x3 same-level block */
  for (int64_t o = 0; o < m->n; ++o) {
    int l = m->lvl[o];
    if (l >= m->p.levelmax) continue;
    for (int c = 0; c < 8; ++c) {
      int64_t x = 2 * (int64_t)m->ci[o] + (c & 1), y = 2 * (int64_t)m->cj[o] + ((c >> 1) & 1),
              z = 2 * (int64_t)m->ck[o] + ((c >> 2) & 1);
      int f = raw[8 * o + c];
      if (rp->expand)
        for (int dz = -1; dz <= 1 && !f; ++dz)
          for (int dy = -1; dy <= 1 && !f; ++dy)
            for (int dx = -1; dx <= 1 && !f; ++dx) {
              int cc;
              int64_t e = cell_oct(m, l, x + dx, y + dy, z + dz, &cc);
              if (e >= 0 && raw[8 * e + cc]) f = 1;
            }
      flag[8 * o + c] = (uint8_t)f;
    }
  }
  free(raw);
  /* grading closure, finest level first */
  for (int l = m->p.levelmax - 1; l > m->p.levelmin; --l) {
    for (int64_t o = m->lo[l]; o < m->lo[l + 1]; ++o)
      for (int c = 0; c < 8; ++c) {
        if (!flag[8 * o + c]) continue;
        int64_t x = 2 * (int64_t)m->ci[o] + (c & 1), y = 2 * (int64_t)m->cj[o] + ((c >> 1) & 1),
                z = 2 * (int64_t)m->ck[o] + ((c >> 2) & 1);
        int64_t side = (int64_t)1 << l;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              /* the level-(l-1) cell covering the level-l cell around X */
              int64_t X = wrap(x + dx, side), Y = wrap(y + dy, side), Z = wrap(z + dz, side);
              int cc;
              int64_t e = cell_oct(m, l - 1, X >> 1, Y >> 1, Z >> 1, &cc);
              if (e < 0) return ORC_EGRADING;
              flag[8 * e + cc] = 1;
            }
      }
  }
  return ORC_OK;
}

/* states of the new child octs of one level, coarsest level first: values
 * at level L are read from the old mesh where the oct is kept, else from the
 * new octs of level L created before */
typedef struct {
  int64_t n;
  uint64_t *key; /* ascending */
  double *U;     /* [n][8][NV] */
} new_level;

static int new_cell_value(const orc_mesh *m, const new_level *nl, int L, int64_t x, int64_t y,
                          int64_t z, double u[NV]) {
  int c;
  int64_t o = cell_oct(m, L, x, y, z, &c);
  if (o >= 0) {
    for (int v = 0; v < NV; ++v) u[v] = m->U[v * 8 * m->n + 8 * o + c];
    return 0;
  }
  int64_t side = (int64_t)1 << L;
  uint64_t k = orc_pack_key(L, wrap(x, side) >> 1, wrap(y, side) >> 1, wrap(z, side) >> 1);
  int64_t a = 0, b = nl[L].n;
  while (a < b) {
    int64_t h = a + (b - a) / 2;
    if (nl[L].key[h] < k)
      a = h + 1;
    else
      b = h;
  }
  if (a >= nl[L].n || nl[L].key[a] != k) return 1;
  for (int v = 0; v < NV; ++v) u[v] = nl[L].U[(8 * a + c) * NV + v];
  return 0;
}

int orc_regrid(orc_mesh **pm, const orc_regrid_params *rp, int64_t *created, int64_t *removed) {
  uint8_t *flag = (uint8_t *)malloc((size_t)(8 * (*pm)->n) + 1);
  if (!flag) return ORC_ENOMEM;
  int e = orc_flags(*pm, rp, flag);
  if (!e) e = orc_regrid_flags(pm, flag, created, removed);
  free(flag);
  return e;
}

int orc_regrid_flags(orc_mesh **pm, const uint8_t *flag, int64_t *created, int64_t *removed) {
  orc_mesh *m = *pm;
  const int64_t n = m->n, n8 = 8 * n;
  const int lmin = m->p.levelmin, lmax = m->p.levelmax;
  int e = 0;
  /* octs of the new mesh: the base level, and the children of flagged cells;
   * an old oct of level l > levelmin is kept when its father is flagged */
  int64_t kept = 0, ncreate = 0, nremove = 0;
  uint8_t *keep = (uint8_t *)calloc((size_t)n + 1, 1);
  new_level nl[ORC_MAXLEV + 1];
  memset(nl, 0, sizeof nl);
  if (!keep) return ORC_ENOMEM;
  for (int64_t o = 0; o < n; ++o) {
    int l = m->lvl[o];
    int k = 1;
    if (l > lmin) {
      int c;
      int64_t f = cell_oct(m, l - 1, m->ci[o], m->cj[o], m->ck[o], &c);
      k = f >= 0 && flag[8 * f + c];
    }
    keep[o] = (uint8_t)k;
    kept += k;
    nremove += !k;
  }
  for (int l = lmin + 1; l <= lmax; ++l) {
    /* flagged leaves of level l-1 whose child oct of level l is new */
    int64_t cnt = 0;
    for (int64_t o = m->lo[l - 1]; o < m->lo[l]; ++o)
      for (int c = 0; c < 8; ++c)
        if (flag[8 * o + c] && !m->split[8 * o + c]) ++cnt;
    nl[l].n = cnt;
    nl[l].key = (uint64_t *)malloc(sizeof(uint64_t) * (cnt ? cnt : 1));
    nl[l].U = (double *)malloc(sizeof(double) * NV * 8 * (cnt ? cnt : 1));
    if (!nl[l].key || !nl[l].U) {
      e = ORC_ENOMEM;
      goto done;
    }
    cnt = 0;
    for (int64_t o = m->lo[l - 1]; o < m->lo[l]; ++o)
      for (int c = 0; c < 8; ++c)
        if (flag[8 * o + c] && !m->split[8 * o + c])
          nl[l].key[cnt++] = orc_pack_key(l, 2 * m->ci[o] + (c & 1), 2 * m->cj[o] + ((c >> 1) & 1),
                                          2 * m->ck[o] + ((c >> 2) & 1));
    qsort(nl[l].key, (size_t)cnt, sizeof(uint64_t), cmp_u64);
    ncreate += cnt;
    /* prolongation of the father cell (level l-1) of each new oct */
    for (int64_t t = 0; t < cnt; ++t) {
      int64_t gi = key_i(nl[l].key[t]), gj = key_j(nl[l].key[t]), gk = key_k(nl[l].key[t]);
      double uc[NV], up[NV], um[NV], sl[3][NV];
      if (new_cell_value(m, nl, l - 1, gi, gj, gk, uc)) {
        e = ORC_EGRADING;
        goto done;
      }
      for (int d = 0; d < 3; ++d) {
        int64_t ex = d == 0, ey = d == 1, ez = d == 2;
        if (new_cell_value(m, nl, l - 1, gi + ex, gj + ey, gk + ez, up) ||
            new_cell_value(m, nl, l - 1, gi - ex, gj - ey, gk - ez, um)) {
          e = ORC_EGRADING;
          goto done;
        }
        for (int v = 0; v < NV; ++v) sl[d][v] = minmod(up[v] - uc[v], uc[v] - um[v]);
      }
      for (int c = 0; c < 8; ++c) {
        double hx = (c & 1) ? 0.25 : -0.25;
        double hy = (c & 2) ? 0.25 : -0.25;
        double hz = (c & 4) ? 0.25 : -0.25;
        for (int v = 0; v < NV; ++v)
          nl[l].U[(8 * t + c) * NV + v] = ((uc[v] + hx * sl[0][v]) + hy * sl[1][v]) + hz * sl[2][v];
      }
    }
  }
  {
    int64_t nn = kept + ncreate, t = 0;
    uint8_t *lv = (uint8_t *)malloc(nn ? nn : 1);
    uint32_t *ii = (uint32_t *)malloc(sizeof(uint32_t) * (nn ? nn : 1));
    uint32_t *jj = (uint32_t *)malloc(sizeof(uint32_t) * (nn ? nn : 1));
    uint32_t *kk = (uint32_t *)malloc(sizeof(uint32_t) * (nn ? nn : 1));
    double *U = (double *)malloc(sizeof(double) * NV * 8 * (nn ? nn : 1));
    if (!lv || !ii || !jj || !kk || !U) {
      free(lv); free(ii); free(jj); free(kk); free(U);
      e = ORC_ENOMEM;
      goto done;
    }
    for (int64_t o = 0; o < n; ++o) {
      if (!keep[o]) continue;
      lv[t] = m->lvl[o];
      ii[t] = m->ci[o];
      jj[t] = m->cj[o];
      kk[t] = m->ck[o];
      for (int v = 0; v < NV; ++v)
        for (int c = 0; c < 8; ++c) U[v * 8 * nn + 8 * t + c] = m->U[v * n8 + 8 * o + c];
      ++t;
    }
    for (int l = lmin + 1; l <= lmax; ++l)
      for (int64_t q = 0; q < nl[l].n; ++q) {
        lv[t] = (uint8_t)l;
        ii[t] = key_i(nl[l].key[q]);
        jj[t] = key_j(nl[l].key[q]);
        kk[t] = key_k(nl[l].key[q]);
        for (int v = 0; v < NV; ++v)
          for (int c = 0; c < 8; ++c) U[v * 8 * nn + 8 * t + c] = nl[l].U[(8 * q + c) * NV + v];
        ++t;
      }
    orc_mesh *out = NULL;
    e = orc_create(&m->p, nn, lv, ii, jj, kk, U, &out);
    free(lv); free(ii); free(jj); free(kk); free(U);
    if (!e) {
      orc_destroy(m);
      *pm = out;
      if (created) *created = ncreate;
      if (removed) *removed = nremove;
    }
  }
done:
  for (int l = 0; l <= ORC_MAXLEV; ++l) {
    free(nl[l].key);
    free(nl[l].U);
  }
  free(keep);
  return e;
}

/* ------------------------------------------------------------------------- */
/* self-gravity: multigrid V-cycles on a periodic level (Sec. 5)             */
/*                                                                           */
/* The paper's solver smooths by red-black Gauss-Seidel over the two parity  */
/* classes of the cells of an oct, restricts residuals by full-weighting     */
/* injection (the mean of the 8 children) and prolongates corrections by    */
/* trilinear interpolation with weights (1,3,3,9,3,9,9,27)/64.  On the      */
/* periodic base level the hierarchy is the same box at half the resolution */
/* per level, down to 2^3 cells; the coarsest grid is smoothed (8 sweeps). */
/* ------------------------------------------------------------------------- */

static int64_t mg_at(int n, int64_t x, int64_t y, int64_t z) {
  return (int64_t)wrap(x, n) + (int64_t)n * ((int64_t)wrap(y, n) + (int64_t)n * wrap(z, n));
}

static double mg_nbsum(int n, const double *phi, int64_t x, int64_t y, int64_t z) {
  return ((phi[mg_at(n, x - 1, y, z)] + phi[mg_at(n, x + 1, y, z)]) +
          (phi[mg_at(n, x, y - 1, z)] + phi[mg_at(n, x, y + 1, z)])) +
         (phi[mg_at(n, x, y, z - 1)] + phi[mg_at(n, x, y, z + 1)]);
}

/* one red-black sweep: colour 0 (x+y+z even) then colour 1 */
static void mg_smooth(int n, double dx2, const double *f, double *phi) {
  for (int colour = 0; colour < 2; ++colour)
    for (int64_t z = 0; z < n; ++z)
      for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x < n; ++x) {
          if ((int)((x + y + z) & 1) != colour) continue;
          int64_t t = mg_at(n, x, y, z);
          phi[t] = (mg_nbsum(n, phi, x, y, z) - dx2 * f[t]) / 6.0;
        }
}

static void mg_residual(int n, double dx2, const double *f, const double *phi, double *r) {
  for (int64_t z = 0; z < n; ++z)
    for (int64_t y = 0; y < n; ++y)
      for (int64_t x = 0; x < n; ++x) {
        int64_t t = mg_at(n, x, y, z);
        r[t] = f[t] - (mg_nbsum(n, phi, x, y, z) - 6.0 * phi[t]) / dx2;
      }
}

static int mg_vcycle(int n, double dx, const double *f, double *phi, int nu1, int nu2) {
  double dx2 = dx * dx;
  if (n <= 2) {
    for (int s = 0; s < 8; ++s) mg_smooth(n, dx2, f, phi);
    return ORC_OK;
  }
  int64_t nn = (int64_t)n * n * n, nc = nn / 8;
  int h = n / 2;
  double *r = (double *)malloc(sizeof(double) * nn);
  double *fc = (double *)calloc((size_t)nc, sizeof(double));
  double *ec = (double *)calloc((size_t)nc, sizeof(double));
  if (!r || !fc || !ec) {
    free(r); free(fc); free(ec);
    return ORC_ENOMEM;
  }
  for (int s = 0; s < nu1; ++s) mg_smooth(n, dx2, f, phi);
  mg_residual(n, dx2, f, phi, r);
  /* restriction: mean of the 8 children, summed in child order */
  for (int64_t Z = 0; Z < h; ++Z)
    for (int64_t Y = 0; Y < h; ++Y)
      for (int64_t X = 0; X < h; ++X) {
        double s = 0.0;
        for (int c = 0; c < 8; ++c)
          s += r[mg_at(n, 2 * X + (c & 1), 2 * Y + ((c >> 1) & 1), 2 * Z + ((c >> 2) & 1))];
        fc[mg_at(h, X, Y, Z)] = s * 0.125;
      }
  int e = mg_vcycle(h, 2.0 * dx, fc, ec, nu1, nu2);
  if (!e) {
    /* trilinear prolongation of the correction: 27/64 from the parent, 9/64
     * from each of its three neighbours towards the fine cell, 3/64 from the
     * three edge neighbours and 1/64 from the corner one */
    for (int64_t z = 0; z < n; ++z)
      for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x < n; ++x) {
          int64_t X = x >> 1, Y = y >> 1, Z = z >> 1;
          int64_t sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
          double v = 27.0 * ec[mg_at(h, X, Y, Z)];
          v += 9.0 * ((ec[mg_at(h, X + sx, Y, Z)] + ec[mg_at(h, X, Y + sy, Z)]) +
                      ec[mg_at(h, X, Y, Z + sz)]);
          v += 3.0 * ((ec[mg_at(h, X + sx, Y + sy, Z)] + ec[mg_at(h, X + sx, Y, Z + sz)]) +
                      ec[mg_at(h, X, Y + sy, Z + sz)]);
          v += ec[mg_at(h, X + sx, Y + sy, Z + sz)];
          phi[mg_at(n, x, y, z)] += v / 64.0;
        }
    for (int s = 0; s < nu2; ++s) mg_smooth(n, dx2, f, phi);
  }
  free(r); free(fc); free(ec);
  return e;
}

static double *mg_source(int n, const double *rho, double fourpiG) {
  int64_t nn = (int64_t)n * n * n;
  double *f = (double *)malloc(sizeof(double) * nn);
  if (!f) return NULL;
  double mean = 0.0;
  for (int64_t t = 0; t < nn; ++t) mean += rho[t];
  mean /= (double)nn;
  for (int64_t t = 0; t < nn; ++t) f[t] = fourpiG * (rho[t] - mean);
  return f;
}

double orc_mg_residual(int n, double dx, const double *rho, double fourpiG, const double *phi) {
  int64_t nn = (int64_t)n * n * n;
  double *f = mg_source(n, rho, fourpiG);
  double *r = (double *)malloc(sizeof(double) * nn);
  if (!f || !r) {
    free(f); free(r);
    return -1.0;
  }
  mg_residual(n, dx * dx, f, phi, r);
  double s = 0.0;
  for (int64_t t = 0; t < nn; ++t) s += r[t] * r[t];
  free(f); free(r);
  return sqrt(s);
}

int orc_mg_solve(int n, double dx, const double *rho, double fourpiG, int ncycles, int nu1,
                 int nu2, double *phi, double *resid) {
  if (n < 2 || (n & (n - 1)) || ncycles < 0 || nu1 < 0 || nu2 < 0) return ORC_EINVAL;
  int64_t nn = (int64_t)n * n * n;
  double *f = mg_source(n, rho, fourpiG);
  if (!f) return ORC_ENOMEM;
  for (int c = 0; c < ncycles; ++c) {
    int e = mg_vcycle(n, dx, f, phi, nu1, nu2);
    if (e) {
      free(f);
      return e;
    }
    if (resid) resid[c] = orc_mg_residual(n, dx, rho, fourpiG, phi);
  }
  double mean = 0.0;
  for (int64_t t = 0; t < nn; ++t) mean += phi[t];
  mean /= (double)nn;
  for (int64_t t = 0; t < nn; ++t) phi[t] -= mean;
  free(f);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* self-gravity on a refined level (Sec. 5: the potential is built level by  */
/* level with V-cycles; the domain boundary takes Dirichlet values through   */
/* an adjusted diagonal).  Readings:                                         */
/*   domain   the cells of the level-L octs; the operator is the 7-point     */
/*            Laplacian (sum of the 6 neighbours - 6 phi) / dx^2 = f, f =    */
/*            fourpiG (rho - rho_bar);                                       */
/*   boundary a face to a cell outside the domain takes phi_b, the mean of   */
/*            the coarse potential of the cell's father and of the level-    */
/*            (L-1) cell across the face, through the ghost value            */
/*            2 phi_b - phi (phi_b on the face): the diagonal becomes        */
/*            -(6 + b) for b such faces and 2 sum phi_b moves to the source; */
/*   cycle    MG level 0 is the domain; MG level k the level-(L-k) cells     */
/*            with a child oct holding a cell of MG level k-1, down to       */
/*            levelmin; the correction equations take homogeneous Dirichlet  */
/*            values at their boundaries; red-black Gauss-Seidel (colour =   */
/*            parity of x+y+z), residuals restricted by the sum of the       */
/*            children in the level below over 8, corrections prolonged      */
/*            trilinearly ((1,3,3,9,3,9,9,27)/64; coarse cells outside the   */
/*            MG level count 0); 2 sweeps before and after, 8 on the         */
/*            coarsest MG level.                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
  int L;                /* AMR level of the cells */
  int64_t n;            /* cells */
  uint64_t *codes;      /* [n] sorted cell codes (x, y, z) */
  int64_t *x, *y, *z;   /* cell coordinates at level L */
  int64_t *nb;          /* [6 n] index of the face neighbour in this MG level, or -1 */
  int *nbnd;            /* faces to the outside */
  double *bsum;         /* 2 sum of phi_b over those faces (MG level 0 only) */
  double *e, *f, *r;
} mg_lvl;

/* index of cell (x,y,z) of level L in the sorted code list of an MG level */
static uint64_t mg_code(int64_t x, int64_t y, int64_t z) {
  return ((uint64_t)x << 42) | ((uint64_t)y << 21) | (uint64_t)z;
}
static int cmp_code(const void *a, const void *b) {
  const uint64_t u = *(const uint64_t *)a, v = *(const uint64_t *)b;
  return u < v ? -1 : u > v;
}
static int64_t mg_find(const uint64_t *codes, int64_t n, uint64_t c) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (codes[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo < n && codes[lo] == c ? lo : -1;
}

static void mg_lvl_free(mg_lvl *g) {
  free(g->codes); free(g->x); free(g->y); free(g->z); free(g->nb); free(g->nbnd); free(g->bsum);
  free(g->e); free(g->f); free(g->r);
  memset(g, 0, sizeof *g);
}

static int64_t mg_find_lvl(const mg_lvl *g, int64_t x, int64_t y, int64_t z) {
  return mg_find(g->codes, g->n, mg_code(x, y, z));
}

/* the cells of the MG level of AMR level L given as sorted codes */
static int mg_lvl_make(mg_lvl *g, int L, const uint64_t *codes, int64_t n) {
  memset(g, 0, sizeof *g);
  g->L = L;
  g->n = n;
  g->codes = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n + 1));
  g->x = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  g->y = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  g->z = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  g->nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(6 * n + 1));
  g->nbnd = (int *)calloc((size_t)(n + 1), sizeof(int));
  g->bsum = (double *)calloc((size_t)(n + 1), sizeof(double));
  g->e = (double *)calloc((size_t)(n + 1), sizeof(double));
  g->f = (double *)calloc((size_t)(n + 1), sizeof(double));
  g->r = (double *)calloc((size_t)(n + 1), sizeof(double));
  if (!g->codes || !g->x || !g->y || !g->z || !g->nb || !g->nbnd || !g->bsum || !g->e || !g->f || !g->r)
    return ORC_ENOMEM;
  memcpy(g->codes, codes, sizeof(uint64_t) * (size_t)n);
  const int64_t side = (int64_t)1 << L;
  for (int64_t t = 0; t < n; ++t) {
    g->x[t] = (int64_t)(codes[t] >> 42);
    g->y[t] = (int64_t)((codes[t] >> 21) & 0x1FFFFF);
    g->z[t] = (int64_t)(codes[t] & 0x1FFFFF);
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        const int64_t dd = s ? 1 : -1;
        const int64_t X = wrap(g->x[t] + (d == 0) * dd, side), Y = wrap(g->y[t] + (d == 1) * dd, side),
                      Z = wrap(g->z[t] + (d == 2) * dd, side);
        const int64_t q = mg_find(codes, n, mg_code(X, Y, Z));
        g->nb[6 * t + 2 * d + s] = q;
        if (q < 0) g->nbnd[t] += 1;
      }
  }
  return ORC_OK;
}

/* red-black Gauss-Seidel sweep: colour 0 (x+y+z even) then colour 1 */
static void mg_lvl_smooth(mg_lvl *g) {
  const double dx = ldexp(1.0, -g->L), dx2 = dx * dx;
  for (int colour = 0; colour < 2; ++colour)
    for (int64_t t = 0; t < g->n; ++t) {
      if ((int)((g->x[t] + g->y[t] + g->z[t]) & 1) != colour) continue;
      double s = 0.0;
      for (int k = 0; k < 6; ++k) {
        const int64_t q = g->nb[6 * t + k];
        if (q >= 0) s += g->e[q];
      }
      g->e[t] = ((s + g->bsum[t]) - dx2 * g->f[t]) / (double)(6 + g->nbnd[t]);
    }
}

static void mg_lvl_residual(mg_lvl *g) {
  const double dx = ldexp(1.0, -g->L), dx2 = dx * dx;
  for (int64_t t = 0; t < g->n; ++t) {
    double s = 0.0;
    for (int k = 0; k < 6; ++k) {
      const int64_t q = g->nb[6 * t + k];
      if (q >= 0) s += g->e[q];
    }
    g->r[t] = g->f[t] - ((s + g->bsum[t]) - (double)(6 + g->nbnd[t]) * g->e[t]) / dx2;
  }
}

static void mg_lvl_cycle(mg_lvl *lv, int k, int K) {
  mg_lvl *g = &lv[k];
  if (k == K) {
    for (int s = 0; s < 8; ++s) mg_lvl_smooth(g);
    return;
  }
  mg_lvl *c = &lv[k + 1];
  for (int s = 0; s < 2; ++s) mg_lvl_smooth(g);
  mg_lvl_residual(g);
  /* restriction: the residuals of the children in the finer MG level,
   * summed in the order (cx, cy, cz) with cz fastest, over 8 */
  for (int64_t t = 0; t < c->n; ++t) {
    double s = 0.0;
    for (int cx = 0; cx < 2; ++cx)
      for (int cy = 0; cy < 2; ++cy)
        for (int cz = 0; cz < 2; ++cz) {
          const int64_t q = mg_find_lvl(g, 2 * c->x[t] + cx, 2 * c->y[t] + cy, 2 * c->z[t] + cz);
          if (q >= 0) s += g->r[q];
        }
    c->f[t] = s / 8.0;
    c->e[t] = 0.0;
  }
  mg_lvl_cycle(lv, k + 1, K);
  /* trilinear prolongation of the correction */
  const int64_t cside = (int64_t)1 << c->L;
  for (int64_t t = 0; t < g->n; ++t) {
    const int64_t X = g->x[t] >> 1, Y = g->y[t] >> 1, Z = g->z[t] >> 1;
    const int64_t sx = (g->x[t] & 1) ? 1 : -1, sy = (g->y[t] & 1) ? 1 : -1, sz = (g->z[t] & 1) ? 1 : -1;
    double e3[2][2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 2; ++d) {
          const int64_t q = mg_find_lvl(c, wrap(X + a * sx, cside), wrap(Y + b * sy, cside), wrap(Z + d * sz, cside));
          e3[a][b][d] = q >= 0 ? c->e[q] : 0.0;
        }
    double v = 27.0 * e3[0][0][0];
    v += 9.0 * ((e3[1][0][0] + e3[0][1][0]) + e3[0][0][1]);
    v += 3.0 * ((e3[1][1][0] + e3[1][0][1]) + e3[0][1][1]);
    v += e3[1][1][1];
    g->e[t] += v / 64.0;
  }
  for (int s = 0; s < 2; ++s) mg_lvl_smooth(g);
}

static uint64_t mg_code_of_cell(const orc_mesh *m, int64_t o, int c) {
  return mg_code(2 * (int64_t)m->ci[o] + (c & 1), 2 * (int64_t)m->cj[o] + ((c >> 1) & 1),
                 2 * (int64_t)m->ck[o] + ((c >> 2) & 1));
}

/* potential of a level-(L-1) cell (x, y, z) from phic (read order of level L-1) */
static double mg_coarse_phi(const orc_mesh *m, int Lc, const double *phic, int64_t x, int64_t y, int64_t z) {
  const int64_t side = (int64_t)1 << Lc;
  const uint32_t X = wrap(x, side), Y = wrap(y, side), Z = wrap(z, side);
  const int64_t o = orc_lookup(m, orc_pack_key(Lc, X >> 1, Y >> 1, Z >> 1));
  const int c = (int)((X & 1) + 2 * (Y & 1) + 4 * (Z & 1));
  return phic[8 * (o - m->lo[Lc]) + c];  /* the cell exists: graded mesh */
}

int orc_mg_level(const orc_mesh *m, int L, double fourpiG, double rho_bar, const double *phic,
                 int ncycles, double *phi, double *resid) {
  const int lmin = m->p.levelmin;
  if (L <= lmin || L > m->p.levelmax || ncycles < 0) return ORC_EINVAL;
  const int64_t no = m->lo[L + 1] - m->lo[L];
  if (no == 0) return ORC_EINVAL;
  const int K = L - lmin;  /* MG levels 0..K: AMR levels L..lmin */
  mg_lvl *lv = (mg_lvl *)calloc((size_t)(K + 1), sizeof(mg_lvl));
  const int64_t n0 = 8 * no;
  uint64_t *codes = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n0);
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n0);  /* read order -> MG index */
  int e = ORC_OK;
  if (!lv || !codes || !pos) {
    e = ORC_ENOMEM;
    goto done;
  }
  for (int64_t q = 0; q < no; ++q)
    for (int c = 0; c < 8; ++c) codes[8 * q + c] = mg_code_of_cell(m, m->lo[L] + q, c);
  qsort(codes, (size_t)n0, sizeof(uint64_t), cmp_code);
  if ((e = mg_lvl_make(&lv[0], L, codes, n0))) goto done;
  for (int64_t q = 0; q < no; ++q)
    for (int c = 0; c < 8; ++c) pos[8 * q + c] = mg_find(codes, n0, mg_code_of_cell(m, m->lo[L] + q, c));
  /* coarser MG levels: the parents of the cells of the level above */
  for (int k = 1; k <= K; ++k) {
    const mg_lvl *g = &lv[k - 1];
    int64_t nc = 0;
    for (int64_t t = 0; t < g->n; ++t) {
      const uint64_t pc = mg_code(g->x[t] >> 1, g->y[t] >> 1, g->z[t] >> 1);
      codes[nc++] = pc;
    }
    qsort(codes, (size_t)nc, sizeof(uint64_t), cmp_code);
    int64_t u = 0;
    for (int64_t t = 0; t < nc; ++t)
      if (t == 0 || codes[t] != codes[t - 1]) codes[u++] = codes[t];
    if ((e = mg_lvl_make(&lv[k], L - k, codes, u))) goto done;
  }
  /* source, boundary values and initial guess of the level */
  {
    mg_lvl *g = &lv[0];
    const int64_t N8 = 8 * m->n;
    const int64_t side = (int64_t)1 << L;
    for (int64_t q = 0; q < no; ++q)
      for (int c = 0; c < 8; ++c) {
        const int64_t t = pos[8 * q + c];
        g->f[t] = fourpiG * (m->U[N8 * 0 + 8 * (m->lo[L] + q) + c] - rho_bar);
        g->e[t] = phi[8 * q + c];
      }
    for (int64_t t = 0; t < g->n; ++t) {
      double bs = 0.0;
      const double pf = mg_coarse_phi(m, L - 1, phic, g->x[t] >> 1, g->y[t] >> 1, g->z[t] >> 1);
      for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
          if (g->nb[6 * t + 2 * d + s] >= 0) continue;
          const int64_t dd = s ? 1 : -1;
          const int64_t X = wrap(g->x[t] + (d == 0) * dd, side), Y = wrap(g->y[t] + (d == 1) * dd, side),
                        Z = wrap(g->z[t] + (d == 2) * dd, side);
          const double pc = mg_coarse_phi(m, L - 1, phic, X >> 1, Y >> 1, Z >> 1);
          bs += 2.0 * (0.5 * (pf + pc));
        }
      g->bsum[t] = bs;
    }
  }
  for (int c = 0; c < ncycles; ++c) {
    mg_lvl_cycle(lv, 0, K);
    if (resid) {
      mg_lvl_residual(&lv[0]);
      double s = 0.0;
      for (int64_t t = 0; t < lv[0].n; ++t) s += lv[0].r[t] * lv[0].r[t];
      resid[c] = sqrt(s);
    }
  }
  for (int64_t q = 0; q < no; ++q)
    for (int c = 0; c < 8; ++c) phi[8 * q + c] = lv[0].e[pos[8 * q + c]];
done:
  if (lv)
    for (int k = 0; k <= K; ++k) mg_lvl_free(&lv[k]);
  free(lv);
  free(codes);
  free(pos);
  return e;
}

/* ------------------------------------------------------------------------- */
/* particles: cloud-in-cell deposition (Sec. 4)                              */
/*                                                                           */
/* The paper deposits particle masses with the Cloud-in-Cell scheme, by     */
/* atomic additions or by prefix sums; the plain definition is written out  */
/* here: each particle spreads its mass over the 8 cells whose centres      */
/* surround it, with the trilinear weights of its offset from them.         */
/* ------------------------------------------------------------------------- */
static void cic_axis(double x, int n, int64_t *i0, double *w0, double *w1) {
  double s = x * (double)n - 0.5;
  double fl = floor(s);
  double f = s - fl;
  *i0 = (int64_t)fl;
  *w0 = 1.0 - f;
  *w1 = f;
}

int orc_cic_deposit(int n, int64_t np, const double *x, const double *y, const double *z,
                    const double *m, double *rho) {
  if (n < 1 || (n & (n - 1)) || np < 0) return ORC_EINVAL;
  int64_t nn = (int64_t)n * n * n;
  for (int64_t t = 0; t < nn; ++t) rho[t] = 0.0;
  for (int64_t p = 0; p < np; ++p) {
    int64_t ix, iy, iz;
    double wx[2], wy[2], wz[2];
    cic_axis(x[p], n, &ix, &wx[0], &wx[1]);
    cic_axis(y[p], n, &iy, &wy[0], &wy[1]);
    cic_axis(z[p], n, &iz, &wz[0], &wz[1]);
    for (int c = 0; c < 8; ++c) {
      int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
      int64_t t = (int64_t)wrap(ix + cx, n) +
                  (int64_t)n * ((int64_t)wrap(iy + cy, n) + (int64_t)n * wrap(iz + cz, n));
      rho[t] += m[p] * ((wx[cx] * wy[cy]) * wz[cz]);
    }
  }
  /* mass -> density: divide by dx^3 = n^-3, an exact scaling */
  for (int64_t t = 0; t < nn; ++t) rho[t] = ldexp(rho[t], 3 * (int)round(log2((double)n)));
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* mass deposition onto the AMR levels (Sec. 4 "Mass Deposition"): the list  */
/* of levelmin holds every particle; at level l each particle of the list    */
/* deposits m (wx wy) wz / dx_l^3, the CIC weights at cell size dx_l = 2^-l  */
/* with the half-cell-shifted stencil, into each of its 8 stencil cells that */
/* exists at level l (a cell of a level-l oct; periodic); then the list of   */
/* level l+1 keeps, in order, the particles whose host cell at level l (the  */
/* cell containing the particle) is split.  Contributions in list order.     */
/* ------------------------------------------------------------------------- */
int orc_cic_deposit_levels(const orc_mesh *m, int64_t np, const double *x, const double *y,
                           const double *z, const double *mass, double *rho, int64_t *count) {
  if (np < 0) return ORC_EINVAL;
  const int64_t N8 = 8 * m->n;
  for (int64_t t = 0; t < N8; ++t) rho[t] = 0.0;
  for (int l = 0; l <= ORC_MAXLEV; ++l) count[l] = 0;
  int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
  if (!list) return ORC_ENOMEM;
  int64_t nl = np;
  for (int64_t p = 0; p < np; ++p) list[p] = p;
  for (int l = m->p.levelmin; l <= m->p.levelmax && nl > 0; ++l) {
    count[l] = nl;
    const int64_t n = (int64_t)1 << l;  /* cells per axis */
    for (int64_t q = 0; q < nl; ++q) {
      const int64_t p = list[q];
      int64_t ix, iy, iz;
      double wx[2], wy[2], wz[2];
      cic_axis(x[p], (int)n, &ix, &wx[0], &wx[1]);
      cic_axis(y[p], (int)n, &iy, &wy[0], &wy[1]);
      cic_axis(z[p], (int)n, &iz, &wz[0], &wz[1]);
      for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        const uint32_t X = wrap(ix + cx, n), Y = wrap(iy + cy, n), Z = wrap(iz + cz, n);
        const int64_t o = orc_lookup(m, orc_pack_key(l, X >> 1, Y >> 1, Z >> 1));
        if (o < 0) continue;  /* no such cell at level l */
        const int cc = (int)((X & 1) + 2 * (Y & 1) + 4 * (Z & 1));
        rho[8 * o + cc] += mass[p] * ((wx[cx] * wy[cy]) * wz[cz]);
      }
    }
    /* the next level's list: particles whose host cell is split */
    int64_t keep = 0;
    for (int64_t q = 0; q < nl; ++q) {
      const int64_t p = list[q];
      const uint32_t X = (uint32_t)floor(x[p] * (double)n), Y = (uint32_t)floor(y[p] * (double)n),
                     Z = (uint32_t)floor(z[p] * (double)n);
      const int64_t o = orc_lookup(m, orc_pack_key(l, X >> 1, Y >> 1, Z >> 1));
      if (o >= 0 && m->split[8 * o + (X & 1) + 2 * (Y & 1) + 4 * (Z & 1)]) list[keep++] = p;
    }
    nl = keep;
  }
  free(list);
  /* mass -> density: divide by dx^3 = 2^(-3l), an exact scaling */
  for (int64_t o = 0; o < m->n; ++o)
    for (int c = 0; c < 8; ++c) rho[8 * o + c] = ldexp(rho[8 * o + c], 3 * (int)m->lvl[o]);
  return ORC_OK;
}
