/*
 * CompaSO oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of the CompaSO group finder
 * (Hadzhiyska et al. 2021, arXiv:2110.11408, Sec. 2.2).  It exists so that the
 * CUDA path can be checked against something written straight from the paper.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it; the product path never does.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Everything is exact integer arithmetic on a periodic grid of 2^21 units per
 * side, so that "same result" can mean bit-for-bit:
 *   - squared distances d are int64 (minimum image);
 *   - the kernel sum Sigma_i = sum_{j != i, d_ij < b2} (b2 - d_ij) is int64,
 *     i.e. b2 times the paper's sum of W(r) = 1 - r^2/b^2 (Sec. 2.2.1, Eq. 1);
 *   - the enclosed-density predicate n^2 u^6 < K d^3 is decided exactly with a
 *     small multi-limb integer (no floating-point decision);
 *   - the competitive test R_new^2 d_old * den >= num * R_old^2 d_new uses int128.
 *
 * Readings of places where the paper is silent (each also listed in the design
 * notes of the repository):
 *   - self term of the kernel sum excluded unless include_self (App. B.2 mean
 *     count is for the other particles);
 *   - thresholds T = floor(Delta * norm), norm = (2/5)(4pi/3) b^3 / u^3 * b2
 *     (App. B.2 normalisation), dense <=> Sigma > T_L0 (Sec. 2.2.1);
 *   - the nucleus stop level is the kernel density at the centre of a singular
 *     isothermal sphere of N_new,min particles inside the radius enclosing
 *     Delta_level times the mean, 5A/b^2 (App. B.2, r < b branch at r -> 0;
 *     Sec. 2.2.2 step 4), applied with the level's own Delta for L2;
 *   - R^2 is the smallest member distance d at which the enclosed count
 *     n(<d) (strictly inside) satisfies n < Delta (4pi/3) (d/u^2)^{3/2}
 *     (Sec. 2.2.2 step 1, Sec. 2.3.3); if no member distance does, the
 *     smallest integer d beyond the farthest member with n = N;
 *   - the local-peak test of step 2 looks at members of the same group only,
 *     within d < b2, with key = (Sigma descending, id ascending);
 *   - ties of Sigma are broken by the smaller particle id.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BOX (1LL << 21)
#define ORC_HALF (1LL << 20)
#define ORC_NONE UINT64_MAX

typedef struct {
  int64_t u;                  /* grid units per mean interparticle spacing l_mean */
  double b_kernel, l_fof;     /* 0.4, 0.25 in units of l_mean (Table 1)          */
  double delta_L0, delta_L1, delta_L2; /* 60, 200, 800 (Sec. 2.2.1, Sec. 2.3.1)  */
  int32_t alpha_num, alpha_den;        /* R_elig / R = 4/5 (step 1)               */
  int32_t roche_num, roche_den;        /* c_Roche = 2/1 (step 3)                  */
  int32_t np_min_density;              /* N_new,min = 35 (step 4)                 */
  int32_t np_min_L1;                   /* catalogue cut (Sec. 2.2.2, last para.)  */
  int32_t include_self;                /* 0: self term not counted                */
  int32_t pad_;
  /* derived by orc_derive() */
  int64_t b2, lfof2, T_L0, T_min_L1, T_min_L2;
  double K_L1, K_L2;
} orc_params;

typedef struct {
  uint64_t nucleus_id;
  int64_t N;
  int64_t R2;
  double R_delta;
  double com[3];
  uint64_t l2max_id;
  int64_t l2max_N;
  double l2max_com[3];
  int64_t l2_top5_N[5];
  int64_t n_l2;
  uint64_t l0_id;
} orc_halo;

/* algorithmic counters, filled by the pipeline entry point */
enum {
  ORC_ST_PAIRS_B = 0,   /* ordered pairs j != i with d < b2                    */
  ORC_ST_PAIRS_FOF,     /* ordered dense pairs with d < lfof2                  */
  ORC_ST_DENSE,         /* particles with Sigma > T_L0                         */
  ORC_ST_L0_GROUPS,
  ORC_ST_L1_NUCLEI,
  ORC_ST_L1_WORK,       /* sum over L1 nuclei of the group size               */
  ORC_ST_L2_NUCLEI,
  ORC_ST_L2_WORK,
  ORC_ST_L1_HALOS_CAT,  /* L1 haloes with N >= np_min_L1                       */
  ORC_ST_COUNT
};

/* ------------------------------------------------------------------------- */
/* geometry                                                                  */
/* ------------------------------------------------------------------------- */

/* minimum-image difference of two grid coordinates in [0, 2^21) */
static int64_t mi(int32_t a, int32_t b) {
  int64_t dx = (int64_t)a - (int64_t)b;
  if (dx >= ORC_HALF) dx -= ORC_BOX;
  else if (dx < -ORC_HALF) dx += ORC_BOX;
  return dx;
}

static int64_t dist2(const int32_t* p, const int32_t* q) {
  int64_t dx = mi(p[0], q[0]), dy = mi(p[1], q[1]), dz = mi(p[2], q[2]);
  return dx * dx + dy * dy + dz * dz;
}

/* ------------------------------------------------------------------------- */
/* derived parameters                                                        */
/* ------------------------------------------------------------------------- */

/* central kernel density of a singular isothermal sphere holding np particles
 * inside the radius whose mean enclosed density is delta (App. B.2: the r < b
 * branch of the smoothed SIS tends to 5A/b^2 as r -> 0; the SIS has
 * M(<R) = 4 pi A R). Lengths in units of l_mean. */
static double sis_central_density(double np, double delta, double b) {
  double R = cbrt(np / (delta * (4.0 * M_PI / 3.0)));
  double A = np / (4.0 * M_PI * R);
  return 5.0 * A / (b * b);
}

int orc_derive(orc_params* p) {
  if (!p || p->u <= 0 || p->b_kernel <= 0 || p->l_fof <= 0) return -1;
  double bu = p->b_kernel * (double)p->u;
  double lu = p->l_fof * (double)p->u;
  p->b2 = llround(bu * bu);
  p->lfof2 = llround(lu * lu);
  /* number of "mean-density particles" a unit-Delta field puts under the
   * kernel, times b2 (App. B.2: N = (2/5)(4pi/3) b^3 Delta) */
  double b2d = (double)p->b2;
  double u3 = (double)p->u * (double)p->u * (double)p->u;
  double norm = 0.4 * (4.0 * M_PI / 3.0) * b2d * b2d * sqrt(b2d) / u3;
  p->T_L0 = (int64_t)floor(p->delta_L0 * norm);
  p->T_min_L1 = (int64_t)floor(sis_central_density(p->np_min_density, p->delta_L1, p->b_kernel) * norm);
  p->T_min_L2 = (int64_t)floor(sis_central_density(p->np_min_density, p->delta_L2, p->b_kernel) * norm);
  double v1 = p->delta_L1 * (4.0 * M_PI / 3.0);
  double v2 = p->delta_L2 * (4.0 * M_PI / 3.0);
  p->K_L1 = v1 * v1;
  p->K_L2 = v2 * v2;
  return 0;
}

/* Thresholds at redshift z of a flat LambdaCDM background (Sec. 2.3.1,
 * Eq. 2): the Bryan & Norman overdensity w.r.t. the critical density,
 * rescaled from 18 pi^2 to 200 (L1) and 800 (L2), divided by Omega_m(z) to
 * be relative to the mean; the L0 cut scales with L1 and l_FoF with the
 * inverse cube root of that change. */
void orc_cosmology(double omega_m0, double z, double out[4]) {
  double a3 = pow(1.0 + z, 3.0);
  double omz = omega_m0 * a3 / (omega_m0 * a3 + 1.0 - omega_m0);
  double x = omz - 1.0;
  double crit = 18.0 * M_PI * M_PI + 82.0 * x - 39.0 * x * x;
  double dl1 = crit * (200.0 / (18.0 * M_PI * M_PI)) / omz;
  out[0] = 60.0 * dl1 / 200.0;          /* Delta_L0 */
  out[1] = dl1;                         /* Delta_L1 */
  out[2] = 4.0 * dl1;                   /* Delta_L2 */
  out[3] = 0.25 / cbrt(dl1 / 200.0);    /* l_FoF    */
}

double orc_sis_central_density(double np, double delta, double b) {
  return sis_central_density(np, delta, b);
}

/* ------------------------------------------------------------------------- */
/* exact enclosed-density predicate                                          */
/* ------------------------------------------------------------------------- */

#define BIG_LIMBS 8
typedef struct { uint64_t w[BIG_LIMBS]; } big_t;

static void big_set(big_t* a, uint64_t v) {
  memset(a, 0, sizeof(*a));
  a->w[0] = v;
}
static void big_mul(big_t* a, uint64_t v) {
  unsigned __int128 carry = 0;
  for (int k = 0; k < BIG_LIMBS; ++k) {
    unsigned __int128 t = (unsigned __int128)a->w[k] * v + carry;
    a->w[k] = (uint64_t)t;
    carry = t >> 64;
  }
}
static void big_shl(big_t* a, int s) {
  while (s >= 64) {
    for (int k = BIG_LIMBS - 1; k > 0; --k) a->w[k] = a->w[k - 1];
    a->w[0] = 0;
    s -= 64;
  }
  if (s > 0) {
    for (int k = BIG_LIMBS - 1; k > 0; --k) a->w[k] = (a->w[k] << s) | (a->w[k - 1] >> (64 - s));
    a->w[0] <<= s;
  }
}
static int big_cmp(const big_t* a, const big_t* b) {
  for (int k = BIG_LIMBS - 1; k >= 0; --k) {
    if (a->w[k] < b->w[k]) return -1;
    if (a->w[k] > b->w[k]) return 1;
  }
  return 0;
}

/* The enclosed count n inside squared radius d is below the level's density:
 *     n < Delta (4 pi / 3) (d / u^2)^{3/2}   <=>   n^2 u^6 < K d^3,
 * K = (Delta 4 pi / 3)^2 as an IEEE double (Sec. 2.2.2 step 1, Sec. 2.3.3).
 * Decided exactly: K = m 2^e with integer m. */
int orc_pred(int64_t n, int64_t d, double K, int64_t u) {
  int E;
  double f = frexp(K, &E);
  uint64_t m = (uint64_t)ldexp(f, 53);
  int e = E - 53;
  big_t lhs, rhs;
  big_set(&lhs, (uint64_t)n);
  big_mul(&lhs, (uint64_t)n);
  for (int k = 0; k < 6; ++k) big_mul(&lhs, (uint64_t)u);
  big_set(&rhs, m);
  for (int k = 0; k < 3; ++k) big_mul(&rhs, (uint64_t)d);
  if (e > 0) big_shl(&rhs, e);
  else if (e < 0) big_shl(&lhs, -e);
  return big_cmp(&lhs, &rhs) < 0;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* Threshold radius search (Sec. 2.2.2 step 1, Sec. 2.3.3): sort the squared
 * distances of all group members to the nucleus and walk outward; the first
 * member distance d whose strictly-enclosed count n(<d) satisfies the
 * predicate is R^2.  If none does, the enclosed count stays N beyond the last
 * member and R^2 is the smallest integer d > max d with N^2 u^6 < K d^3. */
int64_t orc_r_search(const int64_t* d, int64_t n, double K, int64_t u) {
  int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  memcpy(s, d, sizeof(int64_t) * (size_t)n);
  qsort(s, (size_t)n, sizeof(int64_t), cmp_i64);
  int64_t first = 0; /* index of the first element equal to s[k] = n(<s[k]) */
  for (int64_t k = 0; k < n; ++k) {
    if (k > 0 && s[k] != s[k - 1]) first = k;
    if (orc_pred(first, s[k], K, u)) {
      int64_t r = s[k];
      free(s);
      return r;
    }
  }
  int64_t lo = n > 0 ? s[n - 1] : 0; /* predicate false at lo (or lo is 0) */
  free(s);
  int64_t hi = lo + 1;
  while (!orc_pred(n, hi, K, u)) hi = 2 * hi;
  /* smallest D in (lo, hi] with the predicate true; it is monotone in D */
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (orc_pred(n, mid, K, u)) hi = mid;
    else lo = mid;
  }
  return hi;
}

/* ------------------------------------------------------------------------- */
/* cell list (sorted keys + binary search)                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t nc;   /* cells per side; 0 = brute force */
  int64_t n;
  int64_t* key; /* sorted cell keys */
  int64_t* idx; /* particle index for each sorted key */
} orc_grid;

typedef struct { int64_t key, idx; } kv_t;
static int cmp_kv(const void* a, const void* b) {
  const kv_t* x = (const kv_t*)a; const kv_t* y = (const kv_t*)b;
  if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
  return (x->idx > y->idx) - (x->idx < y->idx);
}

static int64_t cell1(int32_t x, int64_t nc) { return ((int64_t)x * nc) >> 21; }

/* cells of side >= reach, so every neighbour within reach lies in the 27 cells
 * around a particle's own; fewer than 3 cells per side -> brute force */
static void grid_build(orc_grid* g, const int32_t* pos, int64_t n, int64_t reach2, int force_brute) {
  g->n = n;
  int64_t reach = (int64_t)floor(sqrt((double)reach2)) + 1;
  g->nc = ORC_BOX / reach;
  if (force_brute || g->nc < 3) g->nc = 0;
  g->key = NULL;
  g->idx = NULL;
  if (g->nc == 0) return;
  kv_t* kv = (kv_t*)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* p = pos + 3 * i;
    kv[i].key = (cell1(p[2], g->nc) * g->nc + cell1(p[1], g->nc)) * g->nc + cell1(p[0], g->nc);
    kv[i].idx = i;
  }
  qsort(kv, (size_t)n, sizeof(kv_t), cmp_kv);
  g->key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  g->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) { g->key[i] = kv[i].key; g->idx[i] = kv[i].idx; }
  free(kv);
}

static void grid_free(orc_grid* g) { free(g->key); free(g->idx); g->key = g->idx = NULL; }

static int64_t lower_bound(const int64_t* a, int64_t n, int64_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) { int64_t m = lo + (hi - lo) / 2; if (a[m] < v) lo = m + 1; else hi = m; }
  return lo;
}

/* ranges [lo, hi) of sorted positions whose particles may lie within reach of
 * a point; returns the number of ranges (<= 27) */
static int grid_ranges(const orc_grid* g, const int32_t* p, int64_t lo_hi[27][2]) {
  if (g->nc == 0) { lo_hi[0][0] = 0; lo_hi[0][1] = g->n; return 1; }
  int64_t nc = g->nc;
  int64_t cx = cell1(p[0], nc), cy = cell1(p[1], nc), cz = cell1(p[2], nc);
  int r = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
        int64_t key = (z * nc + y) * nc + x;
        int64_t lo = lower_bound(g->key, g->n, key);
        int64_t hi = lower_bound(g->key, g->n, key + 1);
        if (hi > lo) { lo_hi[r][0] = lo; lo_hi[r][1] = hi; ++r; }
      }
  return r;
}

static int64_t grid_particle(const orc_grid* g, int64_t s) { return g->nc == 0 ? s : g->idx[s]; }

/* ------------------------------------------------------------------------- */
/* Step: kernel density (Sec. 2.2.1, Eq. 1)                                  */
/* ------------------------------------------------------------------------- */

/* Sigma for the particles listed in `which` (or all if which == NULL).
 * Returns the number of ordered pairs j != i with d < b2 that were summed. */
static int64_t density_on(const orc_grid* g, const int32_t* pos, int64_t n, const orc_params* p,
                          const int64_t* which, int64_t nq, int64_t* sigma) {
  int64_t pairs = 0;
  int64_t rg[27][2];
  for (int64_t q = 0; q < nq; ++q) {
    int64_t i = which ? which[q] : q;
    const int32_t* pi = pos + 3 * i;
    int64_t s = p->include_self ? p->b2 : 0;
    int nr = grid_ranges(g, pi, rg);
    for (int r = 0; r < nr; ++r)
      for (int64_t t = rg[r][0]; t < rg[r][1]; ++t) {
        int64_t j = grid_particle(g, t);
        if (j == i) continue;
        int64_t d = dist2(pi, pos + 3 * j);
        if (d < p->b2) { s += p->b2 - d; ++pairs; }
      }
    sigma[q] = s;
  }
  (void)n;
  return pairs;
}

/* Sigma for every particle; brute = 1 forces the O(N^2) double loop */
int64_t orc_density(const int32_t* pos, int64_t n, const orc_params* p, int brute, int64_t* sigma) {
  orc_grid g;
  grid_build(&g, pos, n, p->b2, brute);
  int64_t pairs = density_on(&g, pos, n, p, NULL, n, sigma);
  grid_free(&g);
  return pairs;
}

/* Sigma for a sample of particles only (full-size spot checks) */
int64_t orc_density_at(const int32_t* pos, int64_t n, const orc_params* p,
                       const int64_t* which, int64_t nq, int64_t* sigma) {
  orc_grid g;
  grid_build(&g, pos, n, p->b2, 0);
  int64_t pairs = density_on(&g, pos, n, p, which, nq, sigma);
  grid_free(&g);
  return pairs;
}

/* ------------------------------------------------------------------------- */
/* Step: L0 groups, modified FoF over dense particles (Sec. 2.2.1)           */
/* ------------------------------------------------------------------------- */

static int64_t uf_find(int64_t* parent, int64_t x) {
  while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
  return x;
}

/* l0[i] = smallest id in i's component of the graph whose vertices are the
 * dense particles (Sigma > T_L0) and whose edges join pairs with d < lfof2;
 * NONE for particles that are not dense.  Returns the number of ordered links. */
int64_t orc_fof(const int32_t* pos, const uint64_t* ids, const int64_t* sigma, int64_t n,
                const orc_params* p, int brute, uint64_t* l0) {
  orc_grid g;
  grid_build(&g, pos, n, p->lfof2, brute);
  int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) parent[i] = i;
  int64_t links = 0;
  int64_t rg[27][2];
  for (int64_t i = 0; i < n; ++i) {
    if (sigma[i] <= p->T_L0) continue;
    const int32_t* pi = pos + 3 * i;
    int nr = grid_ranges(&g, pi, rg);
    for (int r = 0; r < nr; ++r)
      for (int64_t t = rg[r][0]; t < rg[r][1]; ++t) {
        int64_t j = grid_particle(&g, t);
        if (j == i || sigma[j] <= p->T_L0) continue;
        if (dist2(pi, pos + 3 * j) < p->lfof2) {
          ++links;
          int64_t a = uf_find(parent, i), b = uf_find(parent, j);
          if (a != b) parent[a < b ? b : a] = a < b ? a : b;
        }
      }
  }
  uint64_t* minid = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) minid[i] = ORC_NONE;
  for (int64_t i = 0; i < n; ++i)
    if (sigma[i] > p->T_L0) {
      int64_t r = uf_find(parent, i);
      if (ids[i] < minid[r]) minid[r] = ids[i];
    }
  for (int64_t i = 0; i < n; ++i) l0[i] = sigma[i] > p->T_L0 ? minid[uf_find(parent, i)] : ORC_NONE;
  free(minid);
  free(parent);
  grid_free(&g);
  return links;
}

/* ------------------------------------------------------------------------- */
/* Step: CompaSO inside one group (Sec. 2.2.2 steps 1-4, Eq. 3)              */
/* ------------------------------------------------------------------------- */

typedef struct {
  const int32_t* pos;
  const uint64_t* ids;
  const int64_t* sigma;
} orc_view;

/* key order: larger Sigma first, then smaller id */
static int key_before(const orc_view* v, int64_t a, int64_t b) {
  if (v->sigma[a] != v->sigma[b]) return v->sigma[a] > v->sigma[b];
  return v->ids[a] < v->ids[b];
}

static const orc_view* g_sort_view; /* qsort has no context argument */
static int cmp_key(const void* x, const void* y) {
  int64_t a = *(const int64_t*)x, b = *(const int64_t*)y;
  if (a == b) return 0;
  return key_before(g_sort_view, a, b) ? -1 : 1;
}

typedef struct {
  int64_t member;  /* position in the group's member list */
  int64_t R2;
} orc_nucleus;

/* One level of CompaSO over a group whose members (particle indices) are in
 * key order.  `label` gives each particle's group at this level (L0 id for L1,
 * L1 nucleus id for L2); the peak test compares it with `glabel`.
 * Outputs slot[m] (nucleus ordinal or -1) and the nuclei in order. */
static int64_t compaso_level(const orc_view* v, const orc_grid* g, const orc_params* p,
                             const int64_t* members, int64_t n,
                             const uint64_t* label, uint64_t glabel,
                             double K, int64_t T_min,
                             int64_t* slot, orc_nucleus* nuclei, int64_t* work) {
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* dold = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  char* inelig = (char*)calloc((size_t)n, 1);
  int64_t nn = 0;
  int64_t rg[27][2];
  for (int64_t m = 0; m < n; ++m) slot[m] = -1;
  for (int64_t c = 0; c < n; ++c) {
    int64_t pc = members[c];
    /* step 4: stop once the candidate's density is no longer above the level's minimum */
    if (v->sigma[pc] <= T_min) break;
    /* step 2: a nucleus must be eligible ... */
    if (inelig[c]) continue;
    /* ... and denser than every other group member within b */
    int peak = 1;
    int nr = grid_ranges(g, v->pos + 3 * pc, rg);
    for (int r = 0; r < nr && peak; ++r)
      for (int64_t t = rg[r][0]; t < rg[r][1]; ++t) {
        int64_t q = grid_particle(g, t);
        if (q == pc || label[q] != glabel) continue;
        if (dist2(v->pos + 3 * pc, v->pos + 3 * q) < p->b2 && key_before(v, q, pc)) { peak = 0; break; }
      }
    if (!peak) continue;
    /* step 1: distances of all group members to the nucleus, threshold radius */
    for (int64_t m = 0; m < n; ++m) d[m] = dist2(v->pos + 3 * pc, v->pos + 3 * members[m]);
    int64_t R2 = orc_r_search(d, n, K, p->u);
    *work += n;
    /* steps 1 and 3: tentative membership, competitive reassignment, eligibility */
    for (int64_t m = 0; m < n; ++m) {
      if (d[m] >= R2) continue;
      int take = 0;
      if (slot[m] < 0) take = 1;
      else {
        /* Eq. 3: enclosed density Delta R^2 / r^2 w.r.t. the new nucleus is at
         * least c_Roche times that w.r.t. the current one */
        int64_t R2old = nuclei[slot[m]].R2;
        __int128 lhs = (__int128)R2 * dold[m] * p->roche_den;
        __int128 rhs = (__int128)p->roche_num * R2old * d[m];
        take = lhs >= rhs;
      }
      if (take) { slot[m] = nn; dold[m] = d[m]; }
      if ((__int128)p->alpha_den * p->alpha_den * d[m] < (__int128)p->alpha_num * p->alpha_num * R2)
        inelig[m] = 1;
    }
    nuclei[nn].member = c;
    nuclei[nn].R2 = R2;
    ++nn;
  }
  free(d);
  free(dold);
  free(inelig);
  return nn;
}

/* centre of mass: nucleus position plus the mean minimum-image offset,
 * wrapped into the box; offsets are summed exactly in int64 */
static void com_of(const int32_t* pos, const int32_t* nuc, const int64_t* mem, int64_t n, double out[3]) {
  for (int a = 0; a < 3; ++a) {
    int64_t s = 0;
    for (int64_t k = 0; k < n; ++k) s += mi(pos[3 * mem[k] + a], nuc[a]);
    double c = (double)nuc[a] + (double)s / (double)n;
    if (c < 0) c += (double)ORC_BOX;
    if (c >= (double)ORC_BOX) c -= (double)ORC_BOX;
    out[a] = c;
  }
}

static int cmp_desc_i64(const void* a, const void* b) { return -cmp_i64(a, b); }

/* One catalogue row (Sec. 2.2.2 last paragraphs, Table 1) of an L1 halo.
 * hmem[0..nh): the halo's members (particle indices; the nucleus pn among
 * them), R2 its squared L1 radius; the L2 level inside it: slot2[m] is the
 * ordinal of the L2 nucleus that member hmem[m] belongs to (-1: none), and
 * l2nuc[0..n2) the L2 nuclei (particle indices) in the order they were
 * accepted, densest first.  Fills:
 *   N, R2, R_delta = sqrt(R2) / u, com (centre of mass of the members),
 *   l0_id, n_l2 = n2, L2max = the first L2 nucleus with its member count
 *   and centre of mass, l2_top5_N = the five largest L2 member counts in
 *   descending order, zero-padded. */
void orc_halo_row(const int32_t* pos, const uint64_t* ids, const uint64_t* l0, int64_t u, int64_t pn, int64_t R2,
                  const int64_t* hmem, int64_t nh, const int64_t* slot2, int64_t n2, const int64_t* l2nuc,
                  orc_halo* H) {
  memset(H, 0, sizeof(*H));
  H->nucleus_id = ids[pn];
  H->N = nh;
  H->R2 = R2;
  H->R_delta = sqrt((double)R2) / (double)u;
  com_of(pos, pos + 3 * pn, hmem, nh, H->com);
  H->l0_id = l0[pn];
  H->n_l2 = n2;
  H->l2max_id = ORC_NONE;
  int64_t* sizes = (int64_t*)calloc((size_t)(n2 > 0 ? n2 : 1), sizeof(int64_t));
  for (int64_t m = 0; m < nh; ++m) if (slot2[m] >= 0) sizes[slot2[m]]++;
  if (n2 > 0) {
    /* L2max: the first L2 nucleus, i.e. the densest one */
    int64_t pl = l2nuc[0];
    H->l2max_id = ids[pl];
    H->l2max_N = sizes[0];
    int64_t* l2mem = (int64_t*)malloc(sizeof(int64_t) * (size_t)(sizes[0] > 0 ? sizes[0] : 1));
    int64_t k2 = 0;
    for (int64_t m = 0; m < nh; ++m) if (slot2[m] == 0) l2mem[k2++] = hmem[m];
    com_of(pos, pos + 3 * pl, l2mem, k2, H->l2max_com);
    free(l2mem);
  }
  qsort(sizes, (size_t)n2, sizeof(int64_t), cmp_desc_i64);
  for (int k = 0; k < 5; ++k) H->l2_top5_N[k] = k < n2 ? sizes[k] : 0;
  free(sizes);
}

/* CompaSO L1 inside every L0 group, then L2 inside every L1 halo
 * (Sec. 2.2.2), labels and per-halo statistics (Sec. 2.2.2 last paragraphs,
 * Table 1).  Catalogue rows are written for L1 haloes with N >= np_min_L1,
 * in increasing nucleus id.  Returns 0, or -3 if halo_cap is too small (then
 * *n_halos is the number needed). */
int orc_compaso(const int32_t* pos, const uint64_t* ids, const int64_t* sigma, const uint64_t* l0,
                int64_t n, const orc_params* p, uint64_t* l1, uint64_t* l2,
                orc_halo* halos, int64_t halo_cap, int64_t* n_halos, int64_t* stats) {
  orc_view v = {pos, ids, sigma};
  orc_grid g;
  grid_build(&g, pos, n, p->b2, 0);
  for (int64_t i = 0; i < n; ++i) { l1[i] = ORC_NONE; l2[i] = ORC_NONE; }

  /* members of every L0 group, groups ordered by L0 id, members in key order */
  int64_t nd = 0;
  for (int64_t i = 0; i < n; ++i) if (l0[i] != ORC_NONE) ++nd;
  int64_t* dense = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));
  { int64_t k = 0; for (int64_t i = 0; i < n; ++i) if (l0[i] != ORC_NONE) dense[k++] = i; }
  kv_t* kv = (kv_t*)malloc(sizeof(kv_t) * (size_t)(nd > 0 ? nd : 1));
  for (int64_t k = 0; k < nd; ++k) { kv[k].key = (int64_t)l0[dense[k]]; kv[k].idx = dense[k]; }
  /* l0 ids are < 2^63 for any sane input: they are particle ids */
  qsort(kv, (size_t)nd, sizeof(kv_t), cmp_kv);
  for (int64_t k = 0; k < nd; ++k) dense[k] = kv[k].idx;
  free(kv);

  int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));
  orc_nucleus* nuc = (orc_nucleus*)malloc(sizeof(orc_nucleus) * (size_t)(nd > 0 ? nd : 1));
  int64_t* slot2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));
  orc_nucleus* nuc2 = (orc_nucleus*)malloc(sizeof(orc_nucleus) * (size_t)(nd > 0 ? nd : 1));
  int64_t* hmem = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));
  int64_t* l2nuc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));

  int64_t cap_rows = 0, rows = 0;
  orc_halo* tmp = NULL;
  int64_t st[ORC_ST_COUNT] = {0};
  int64_t w1 = 0, w2 = 0;

  for (int64_t a = 0; a < nd;) {
    int64_t b = a;
    while (b < nd && l0[dense[b]] == l0[dense[a]]) ++b;
    int64_t ng = b - a;
    int64_t* M = dense + a;
    g_sort_view = &v;
    qsort(M, (size_t)ng, sizeof(int64_t), cmp_key);
    ++st[ORC_ST_L0_GROUPS];

    int64_t nn = compaso_level(&v, &g, p, M, ng, l0, l0[M[0]], p->K_L1, p->T_min_L1, slot, nuc, &w1);
    st[ORC_ST_L1_NUCLEI] += nn;
    for (int64_t m = 0; m < ng; ++m)
      if (slot[m] >= 0) l1[M[m]] = ids[M[nuc[slot[m]].member]];

    /* L2 inside each L1 halo, in nucleus order */
    for (int64_t h = 0; h < nn; ++h) {
      int64_t nh = 0;
      for (int64_t m = 0; m < ng; ++m) if (slot[m] == h) hmem[nh++] = M[m]; /* still in key order */
      if (nh == 0) continue; /* cannot happen: the nucleus is never stolen */
      uint64_t hid = ids[M[nuc[h].member]];
      int64_t n2 = compaso_level(&v, &g, p, hmem, nh, l1, hid, p->K_L2, p->T_min_L2, slot2, nuc2, &w2);
      st[ORC_ST_L2_NUCLEI] += n2;
      for (int64_t m = 0; m < nh; ++m)
        if (slot2[m] >= 0) l2[hmem[m]] = ids[hmem[nuc2[slot2[m]].member]];

      if (nh < p->np_min_L1) continue;
      if (rows == cap_rows) {
        cap_rows = cap_rows ? 2 * cap_rows : 1024;
        tmp = (orc_halo*)realloc(tmp, sizeof(orc_halo) * (size_t)cap_rows);
      }
      for (int64_t q = 0; q < n2; ++q) l2nuc[q] = hmem[nuc2[q].member];
      orc_halo_row(pos, ids, l0, p->u, M[nuc[h].member], nuc[h].R2, hmem, nh, slot2, n2, l2nuc, tmp + rows++);
    }
    a = b;
  }
  st[ORC_ST_L1_WORK] = w1;
  st[ORC_ST_L2_WORK] = w2;
  st[ORC_ST_L1_HALOS_CAT] = rows;

  /* catalogue in increasing nucleus id */
  for (int64_t i = 1; i < rows; ++i) {
    orc_halo t = tmp[i];
    int64_t j = i - 1;
    while (j >= 0 && tmp[j].nucleus_id > t.nucleus_id) { tmp[j + 1] = tmp[j]; --j; }
    tmp[j + 1] = t;
  }
  int rc = 0;
  *n_halos = rows;
  if (rows > halo_cap) rc = -3;
  else if (rows > 0) memcpy(halos, tmp, sizeof(orc_halo) * (size_t)rows);
  if (stats) for (int k = ORC_ST_L0_GROUPS; k < ORC_ST_COUNT; ++k) if (k != ORC_ST_DENSE) stats[k] = st[k];

  free(tmp); free(dense); free(slot); free(nuc); free(slot2); free(nuc2); free(hmem); free(l2nuc);
  grid_free(&g);
  return rc;
}

/* The whole path for one periodic box: density, L0, L1, L2, catalogue. */
int orc_find_groups(const int32_t* pos, const uint64_t* ids, int64_t n, orc_params* p,
                    int64_t* sigma, uint64_t* l0, uint64_t* l1, uint64_t* l2,
                    orc_halo* halos, int64_t halo_cap, int64_t* n_halos, int64_t* stats) {
  if (orc_derive(p) != 0) return -1;
  for (int64_t i = 0; i < 3 * n; ++i) if (pos[i] < 0 || pos[i] >= ORC_BOX) return -1;
  int64_t st[ORC_ST_COUNT] = {0};
  st[ORC_ST_PAIRS_B] = orc_density(pos, n, p, 0, sigma);
  for (int64_t i = 0; i < n; ++i) if (sigma[i] > p->T_L0) ++st[ORC_ST_DENSE];
  st[ORC_ST_PAIRS_FOF] = orc_fof(pos, ids, sigma, n, p, 0, l0);
  int rc = orc_compaso(pos, ids, sigma, l0, n, p, l1, l2, halos, halo_cap, n_halos, st);
  if (stats) memcpy(stats, st, sizeof(st));
  return rc;
}

int orc_stats_count(void) { return ORC_ST_COUNT; }
int orc_sizeof_halo(void) { return (int)sizeof(orc_halo); }
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }

/* ------------------------------------------------------------------------- */
/* radial statistics of catalogue rows (Table 1: r_XX_L2com,                  */
/* vcirc_max_L2com, rvcirc_max_L2com; Sec. 4)                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t centre[3]; /* grid point nearest the L2max com (the L1 com if no L2) */
  int64_t d_q[4];    /* squared radius enclosing 25, 50, 75, 98 % of members  */
  double r_q[4];     /* sqrt(d_q) / u                                         */
  int64_t vmax_n;    /* members with d <= vmax_d2                             */
  int64_t vmax_d2;   /* squared radius where N(<=r) / r peaks                  */
  double vmax;       /* sqrt(vmax_n / r_vmax), units sqrt(G m_p / l_mean)      */
  double r_vmax;     /* sqrt(vmax_d2) / u                                     */
} orc_radial_t;

static int cmp_kv_key(const void* a, const void* b) {
  const kv_t* x = (const kv_t*)a;
  const kv_t* y = (const kv_t*)b;
  if (x->key != y->key) return (uint64_t)x->key < (uint64_t)y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : x->idx > y->idx;
}

/* For each catalogue row: its members are the particles whose L1 label is
 * the row's nucleus id.  Distances are taken from the grid point nearest the
 * centre of mass of the first L2 halo (L2max com), or of the L1 halo when it
 * has no L2 halo, so that every distance is an exact integer.
 *   r_XX: the k-th smallest member distance with k = ceil(XX N / 100), i.e.
 *         the smallest member radius enclosing at least XX % of the N
 *         members (counting members on the sphere);
 *   V_max: the largest circular velocity v^2 = G m N(<= r) / r over member
 *         radii r > 0, where N(<= r) counts every member at distance <= r
 *         (the value just outside the shell at r); compared exactly as
 *         k_a^2 d_b > k_b^2 d_a; equal values keep the smaller radius.
 * Returns 0, or -1 if a row has no members. */
int orc_radial(const int32_t* pos, const uint64_t* l1, int64_t n, const orc_halo* rows, int64_t nrows,
               double u, orc_radial_t* out) {
  static const int64_t pct[4] = {25, 50, 75, 98};
  kv_t* byl = (kv_t*)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    byl[i].key = (int64_t)l1[i];
    byl[i].idx = i;
  }
  qsort(byl, (size_t)n, sizeof(kv_t), cmp_kv_key);
  for (int64_t r = 0; r < nrows && rc == 0; ++r) {
    const orc_halo* h = &rows[r];
    orc_radial_t* o = &out[r];
    const double* com = h->n_l2 > 0 ? h->l2max_com : h->com;
    int32_t c[3];
    for (int k = 0; k < 3; ++k) {
      o->centre[k] = llround(com[k]) & (ORC_BOX - 1);
      c[k] = (int32_t)o->centre[k];
    }
    /* members: the run of byl with key == nucleus id (binary search) */
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if ((uint64_t)byl[mid].key < h->nucleus_id) lo = mid + 1;
      else hi = mid;
    }
    int64_t m = 0;
    for (int64_t t = lo; t < n && (uint64_t)byl[t].key == h->nucleus_id; ++t)
      d[m++] = dist2(pos + 3 * byl[t].idx, c);
    if (m == 0) {
      rc = -1;
      break;
    }
    qsort(d, (size_t)m, sizeof(int64_t), cmp_i64);
    for (int q = 0; q < 4; ++q) {
      int64_t k = (pct[q] * m + 99) / 100;
      if (k < 1) k = 1;
      o->d_q[q] = d[k - 1];
      o->r_q[q] = sqrt((double)o->d_q[q]) / u;
    }
    int64_t bk = 0, bd = 0;
    for (int64_t j = 0; j < m; ++j) {
      if (d[j] == 0) continue;
      if (j + 1 < m && d[j + 1] == d[j]) continue; /* N(<= r) counts the whole shell */
      const int64_t k = j + 1;
      if (bk == 0) {
        bk = k;
        bd = d[j];
        continue;
      }
      const unsigned __int128 lhs = (unsigned __int128)(k * k) * (uint64_t)bd;
      const unsigned __int128 rhs = (unsigned __int128)(bk * bk) * (uint64_t)d[j];
      if (lhs > rhs) {
        bk = k;
        bd = d[j];
      }
    }
    o->vmax_n = bk;
    o->vmax_d2 = bd;
    o->r_vmax = sqrt((double)bd) / u;
    o->vmax = bk > 0 ? sqrt((double)bk / o->r_vmax) : 0.0;
  }
  free(byl);
  free(d);
  return rc;
}

int orc_sizeof_radial(void) { return (int)sizeof(orc_radial_t); }

/* ------------------------------------------------------------------------- */
/* shrinking-sphere centre of catalogue rows (Sec. 4, Power et al. 2003)      */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t centre[3]; /* final centre (grid point)                                */
  int64_t n;         /* members inside the last sphere tested (below the stop)   */
  int64_t R2;        /* squared radius of that sphere                            */
  int64_t iter;      /* centre-of-mass steps taken                               */
} orc_shrink_t;

/* The centre of the CompaSO sphere followed inwards: starting at the L1
 * nucleus with the L1 radius, the members inside the current sphere
 * (d < R2) give a centre of mass, rounded to the nearest grid point, and the
 * radius shrinks by 5% (R2 <- floor(R2 * 9025 / 10000), exact); this repeats
 * while the sphere holds at least max(ceil(N / 100), n_min) members, N the
 * halo's members (Sec. 4 stops at 1% of the particles or about 700).  Members
 * are the particles whose L1 label is the row's nucleus id.  Returns 0, or -1
 * if a row's nucleus is not among its members. */
int orc_shrink_sphere(const int32_t* pos, const uint64_t* ids, const uint64_t* l1, int64_t n,
                      const orc_halo* rows, int64_t nrows, int64_t n_min, orc_shrink_t* out) {
  kv_t* byl = (kv_t*)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    byl[i].key = (int64_t)l1[i];
    byl[i].idx = i;
  }
  qsort(byl, (size_t)n, sizeof(kv_t), cmp_kv_key);
  for (int64_t r = 0; r < nrows && rc == 0; ++r) {
    const orc_halo* h = &rows[r];
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if ((uint64_t)byl[mid].key < h->nucleus_id) lo = mid + 1;
      else hi = mid;
    }
    int64_t end = lo;
    while (end < n && (uint64_t)byl[end].key == h->nucleus_id) ++end;
    const int64_t N = end - lo;
    int32_t c[3] = {0, 0, 0};
    int found = 0;
    for (int64_t t = lo; t < end; ++t)
      if (ids[byl[t].idx] == h->nucleus_id) {
        memcpy(c, pos + 3 * byl[t].idx, sizeof(c));
        found = 1;
      }
    if (!found) {
      rc = -1;
      break;
    }
    const int64_t stop = (N + 99) / 100 > n_min ? (N + 99) / 100 : n_min;
    int64_t R2 = h->R2, iter = 0, m = 0;
    for (;;) {
      int64_t sum[3] = {0, 0, 0};
      m = 0;
      for (int64_t t = lo; t < end; ++t) {
        const int32_t* q = pos + 3 * byl[t].idx;
        if (dist2(q, c) >= R2) continue;
        ++m;
        for (int a = 0; a < 3; ++a) sum[a] += mi(q[a], c[a]);
      }
      if (m < stop) break;
      for (int a = 0; a < 3; ++a) {
        double f = (double)c[a] + (double)sum[a] / (double)m;
        if (f < 0) f += (double)ORC_BOX;
        if (f >= (double)ORC_BOX) f -= (double)ORC_BOX;
        c[a] = (int32_t)(llround(f) & (ORC_BOX - 1));
      }
      R2 = R2 * 9025 / 10000;
      ++iter;
    }
    orc_shrink_t* o = &out[r];
    for (int a = 0; a < 3; ++a) o->centre[a] = c[a];
    o->n = m;
    o->R2 = R2;
    o->iter = iter;
  }
  free(byl);
  return rc;
}

int orc_sizeof_shrink(void) { return (int)sizeof(orc_shrink_t); }
