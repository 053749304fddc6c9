/*
 * cso.h — C ABI of the GB300 CompaSO hot path.
 *
 * CompaSO (Hadzhiyska et al. 2021, arXiv:2110.11408) finds haloes in a
 * periodic box of equal-mass particles in three nested levels (Sec. 2.2):
 *   L0  friends-of-friends over particles whose kernel density exceeds
 *       Delta_L0 (Sec. 2.2.1, Eq. 1);
 *   L1  competitive spherical-overdensity assignment inside each L0 group
 *       (Sec. 2.2.2 steps 1-4, Eq. 3);
 *   L2  the same assignment, at the higher threshold Delta_L2, inside every
 *       L1 halo (Sec. 2.2.2, last paragraphs).
 *
 * Every step runs in CUDA kernels for sm_103a.  Positions are int32 on a
 * periodic grid of 2^21 units per side; distances, kernel sums and all
 * decisions are exact integers, so results do not depend on the order of the
 * input particles.  Labels are particle ids: L0 = smallest id of the group,
 * L1/L2 = id of the nucleus particle, CSO_NO_GROUP otherwise.
 *
 * Threading: one cso_ctx is used by one host thread at a time.  All device
 * work of a context is issued on the context's CUDA stream.
 *
 * Return codes: CSO_OK (0) or one of the negative CSO_ERR_* values below;
 * cso_last_error() gives a one-line description of the last failure.
 */
#ifndef CSO_H
#define CSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSO_OK 0
#define CSO_ERR_ARG (-1)      /* bad parameters, positions outside [0, 2^21), n too large */
#define CSO_ERR_BUDGET (-2)   /* the request can never fit the context's device-memory budget */
#define CSO_ERR_CAPACITY (-3) /* halo_cap too small; n_halos holds the number needed */
#define CSO_ERR_TIMEOUT (-4)  /* a bounded wait gave up (cso_poll with timeout_us > 0) */
#define CSO_ERR_CUDA (-5)     /* a CUDA runtime call failed */
#define CSO_EAGAIN (-6)       /* cso_submit: queued, not yet admitted (ticket is valid) */
#define CSO_ERR_STATE (-7)    /* unknown ticket or call out of order */

#define CSO_NO_GROUP UINT64_MAX
#define CSO_GRID_BITS 21

/* context flags (cso_init) */
#define CSO_FLAG_BATCHED 1u /* CompaSO levels by group size: warp, 256- and 1024-thread blocks, 8-CTA clusters,
                              16-CTA clusters for huge groups (cso_set_huge_group), largest first, on four
                              concurrent streams */
#define CSO_FLAG_TIMING 2u  /* record per-stage CUDA events (cso_stage_times) */
/* with CSO_FLAG_BATCHED: each CompaSO level stage (size sort, work queue and
 * the five persistent tier kernels) is captured once as a CUDA graph and
 * replayed by later calls with identical launch arguments (a box of the same
 * shape in the same context); the rest of the step is launched directly (its
 * launch sizes are read back from the device between stages) */
#define CSO_FLAG_GRAPH 4u
#define CSO_FLAG_COUNT_PAIRS 8u /* count kernel pairs with d < b2 (cso_last_stats[6]); slows the density pass */
#define CSO_FLAG_SELECT_STRESS 16u /* testing: tiny radius-search tiles so every select branch runs; same results */
/* threshold-radius search by the paper's radial bins (Sec. 2.3.4): members
 * are binned outward in steps of sqrt(3)/3 cell sides and a bin is skipped
 * while the members inside it, placed at its outer edge, still meet the
 * threshold; the default bins by threshold count.  Same R^2 either way. */
#define CSO_FLAG_RADIAL_BINS 32u
/* served path: number of worker slots (concurrent requests), 1..15; 0 = 4 */
#define CSO_FLAG_SLOTS(k) ((uint32_t)((k) & 0xf) << 8)

/*
 * Parameters (Table 1 of the paper; Einstein-de Sitter thresholds of
 * Sec. 2.3.1).  Lengths b_kernel and l_fof are in units of the mean
 * interparticle spacing l_mean; l_mean_grid = u is that spacing in grid units
 * (2^21 / box side in l_mean) and must be an integer value.
 * The derived block is filled by cso_params_derive():
 *   b2    = llround((b_kernel u)^2), lfof2 = llround((l_fof u)^2)   [grid^2]
 *   norm  = 0.4 (4 pi / 3) b2^2 sqrt(b2) / u^3: the kernel sum
 *           Sigma = sum_j (b2 - d_ij) that a unit-density uniform field gives
 *           on average (App. B.2, N = (2/5)(4 pi / 3) b^3 Delta, times b2);
 *   T_L0  = floor(delta_L0 norm)  (dense <=> Sigma > T_L0, Sec. 2.2.1);
 *   T_min_L1/L2 = floor(D norm) with D = 5A/b^2 the kernel density at the
 *           centre of a singular isothermal sphere of np_min_density
 *           particles inside the radius enclosing delta_L1/L2 times the mean
 *           (Sec. 2.2.2 step 4; App. B.2);
 *   K_L1/L2 = (delta (4 pi / 3))^2: a radius whose squared grid length is d
 *           encloses "too little" when n^2 u^6 < K d^3 (Sec. 2.2.2 step 1).
 */
typedef struct cso_params {
  int32_t grid_bits;       /* must be CSO_GRID_BITS */
  int32_t include_self;    /* 1: count the particle itself in its kernel sum */
  double l_mean_grid;      /* u */
  double b_kernel;         /* 0.4 */
  double l_fof;            /* 0.25 */
  double delta_L0;         /* 60 */
  double delta_L1;         /* 200 */
  double delta_L2;         /* 800 */
  int32_t alpha_num;       /* R_elig / R = alpha_num / alpha_den = 4 / 5 */
  int32_t alpha_den;
  int32_t roche_num;       /* c_Roche = roche_num / roche_den = 2 / 1 */
  int32_t roche_den;
  int32_t np_min_density;  /* N_new,min = 35 */
  int32_t np_min_L1;       /* catalogue keeps L1 haloes with N >= this (35) */
  /* derived */
  int64_t b2, lfof2, T_L0, T_min_L1, T_min_L2;
  double K_L1, K_L2;
} cso_params;

/* One row of the L1 catalogue (Table 1 fields).  Positions in grid units. */
typedef struct cso_halo {
  uint64_t nucleus_id;  /* L1 particle (SO_central_particle) */
  int64_t N;            /* members */
  int64_t R2;           /* squared L1 radius, grid^2 */
  double R_delta;       /* sqrt(R2) / u, l_mean units */
  double com[3];        /* L1 centre of mass: nucleus + mean minimum-image offset */
  uint64_t l2max_id;    /* first (densest) L2 nucleus, CSO_NO_GROUP if none */
  int64_t l2max_N;
  double l2max_com[3];
  int64_t l2_top5_N[5]; /* sizes of the five largest L2 haloes, descending, 0-padded */
  int64_t n_l2;         /* number of L2 haloes */
  uint64_t l0_id;       /* L0 group of the halo */
} cso_halo;

/* Input particles.  pos is int32[n][3] (x, y, z), ids is uint64[n]; both host
 * or both device memory (on_device).  The caller owns them and keeps them
 * alive until the call (or, for cso_submit, the ticket) completes.
 * x_lo/x_hi: reserved for slab requests; set both to 0 for a whole box. */
typedef struct cso_input {
  const int32_t* pos;
  const uint64_t* ids;
  int64_t n;
  int32_t on_device;
  int32_t x_lo, x_hi;
  uint64_t request_id;
} cso_input;

/* Radial statistics of one catalogue row (Table 1 fields r_XX_L2com,
 * vcirc_max_L2com and rvcirc_max_L2com; Sec. 4).  Members are the particles
 * of the L1 halo; distances are exact squared grid distances (minimum image)
 * from `centre`, the grid point nearest the L2max centre of mass (the L1
 * centre of mass when the halo has no L2 halo; coordinates rounded half away
 * from zero, then wrapped into [0, 2^21)).
 *   d_q[k]: the m-th smallest member distance, m = ceil(P_k N / 100) with
 *           P = 25, 50, 75, 98: the smallest member radius enclosing at least
 *           P_k % of the N members;
 *   vmax_n, vmax_d2: the member radius r > 0 maximising v^2 = N(<= r) / r,
 *           N(<= r) counting every member at distance <= r (decided exactly
 *           as n_a^2 d_b > n_b^2 d_a; equal values keep the smaller radius);
 *   r_q = sqrt(d_q) / u and r_vmax = sqrt(vmax_d2) / u in l_mean units;
 *   vmax = sqrt(vmax_n / r_vmax) in units of sqrt(G m_particle / l_mean)
 *           (0 when every member sits on the centre).
 * The shrinking-sphere centre (Sec. 4; Power et al. 2003): from the L1
 * nucleus with the L1 radius, the members inside the sphere (d < R2) give a
 * centre of mass, rounded to the nearest grid point, and the radius shrinks
 * by 5% (R2 <- floor(R2 * 9025 / 10000)); this repeats while the sphere holds
 * at least max(ceil(N / 100), 700) members.  ss_centre is the final centre,
 * ss_n and ss_R2 the member count and squared radius of the last sphere
 * tested (the one below the stop count), ss_iter the steps taken. */
typedef struct cso_radial {
  int64_t centre[3];
  int64_t d_q[4];
  double r_q[4];
  int64_t vmax_n;
  int64_t vmax_d2;
  double vmax;
  double r_vmax;
  int64_t ss_centre[3];
  int64_t ss_n;
  int64_t ss_R2;
  int64_t ss_iter;
} cso_radial;

/* Outputs, caller-allocated, length n in input order (NULL = not wanted);
 * halos has room for halo_cap rows and receives the catalogue in increasing
 * nucleus id; n_halos is set to the number of rows (also on CSO_ERR_CAPACITY).
 * All output pointers are host or device memory as on_device says. */
typedef struct cso_output {
  uint64_t* l0;
  uint64_t* l1;
  uint64_t* l2;
  int64_t* sigma;  /* kernel sums Sigma_i = sum_{j != i, d < b2} (b2 - d) */
  cso_halo* halos;
  int64_t halo_cap;
  int64_t n_halos;
  int32_t on_device;
  int32_t pad_;
  cso_radial* radial; /* halo_cap rows, row r describing halos[r]; NULL = not
                         computed.  Whole-box requests only (CSO_ERR_ARG for a
                         slab request). */
} cso_output;

typedef struct cso_ctx cso_ctx;

/* Create a context on `device` with a device-memory budget in bytes
 * (0 = no limit beyond the device).  flags: CSO_FLAG_*.  The context owns its
 * stream, its workspace and its timing events. */
int cso_init(cso_ctx** ctx, int device, size_t hbm_budget_bytes, uint32_t flags);

/* Paper defaults for a box whose mean interparticle spacing is u grid units;
 * the derived block is filled too. */
int cso_params_default(cso_params* p, double l_mean_grid);

/* Fill the derived block from the primary fields (formulas above). */
int cso_params_derive(cso_params* p);

/* Scale the thresholds to redshift z of a flat LambdaCDM background with
 * matter density omega_m0 today (Sec. 2.3.1, Eq. 2, Bryan & Norman 1998):
 * Delta_L1 = (200 / 18 pi^2)(18 pi^2 + 82 x - 39 x^2) / Omega_m(z) with
 * x = Omega_m(z) - 1 (mean-relative), Delta_L2 = 4 Delta_L1, delta_L0 =
 * 60 Delta_L1 / 200, l_fof = 0.25 (Delta_L1 / 200)^(-1/3); b_kernel is kept.
 * Overwrites those four fields and re-derives. */
int cso_params_cosmology(cso_params* p, double omega_m0, double z);

/* Run the whole hot path on one periodic box: kernel density, L0, L1, L2,
 * labels and catalogue.  Synchronous: returns after the outputs are written
 * (and, on an error return, with no copy into them still in flight; their
 * contents are then unspecified). */
int cso_find_groups(cso_ctx* ctx, const cso_input* in, const cso_params* p, cso_output* out);

/* Served path (continuous batching).  Queue a box and return a ticket at
 * once: CSO_OK if it was admitted immediately, CSO_EAGAIN if it waits (the
 * ticket is valid either way), CSO_ERR_BUDGET if it can never fit the
 * context's device-memory budget.  Requests are admitted in submission order
 * onto the context's worker slots (CSO_FLAG_SLOTS, each with its own
 * streams and workspace) while a slot is free and the workspace of all
 * running requests stays within the budget; admitted requests run
 * concurrently and each gives exactly the outputs cso_find_groups gives it
 * alone.  `in`, `out` and every buffer behind them must stay valid until
 * cso_poll reports the ticket done. */
int cso_submit(cso_ctx* ctx, const cso_input* in, const cso_params* p, cso_output* out, uint64_t* ticket);

/* Wait up to timeout_us (0 = just test, <0 = wait forever) for a ticket;
 * *done = 1 when its outputs are complete; returns the request's own status
 * once done.  While the request is still running: CSO_OK for timeout_us == 0,
 * CSO_ERR_TIMEOUT when a positive timeout_us has passed (the ticket stays
 * valid; poll again).  CSO_ERR_STATE: unknown ticket. */
int cso_poll(cso_ctx* ctx, uint64_t ticket, int32_t* done, int32_t timeout_us);

/* Host steady-clock times (seconds, the cso_clock() scale) at which a done
 * ticket was submitted, admitted and completed. */
int cso_ticket_times(cso_ctx* ctx, uint64_t ticket, double* t_submit, double* t_start, double* t_done);

/* The library's host steady clock, seconds. */
double cso_clock(void);

/* Release every resource of the context. */
void cso_free(cso_ctx* ctx);

/* Autotuner of the batched schedule (CSO_FLAG_BATCHED): runs the request
 * under each candidate pair of size bins -- groups above `giant` members on
 * 8-CTA thread-block clusters (4096, 8192, 16384, 65536, 262144), groups of at most
 * `small` members one per warp (32, 64); groups above max(giant / 16, 512)
 * run on 1024-thread blocks and the rest on 256-thread blocks -- times the
 * CompaSO levels, and keeps the fastest pair in the context for every later
 * call.  Outputs are written as by cso_find_groups (identical for every
 * pair).  giant/small (may be NULL) receive the choice. */
int cso_autotune(cso_ctx* ctx, const cso_input* in, const cso_params* p, cso_output* out, int32_t* giant,
                 int32_t* small);

/* Set the batched schedule's size bins directly (giant >= 64, 1 <= small
 * <= 64); the defaults are 16384 and 64. */
int cso_set_schedule(cso_ctx* ctx, int32_t giant, int32_t small);

/* Groups above max(huge, giant) members run on 16-CTA thread-block clusters
 * (a non-portable cluster size) where the device can hold one, instead of
 * 8-CTA clusters: the level passes of the few biggest groups are the batched
 * schedule's critical path.  Default 524288 (2^19); huge >= 64, INT32_MAX
 * keeps every group on 8-CTA clusters.  Outputs do not depend on it.
 * Returns CSO_ERR_ARG for huge < 64. */
int cso_set_huge_group(cso_ctx* ctx, int32_t huge);

/* --- the three steps one at a time --------------------------------------
 *
 * For a caller that distributes one box over several GPUs (each GPU owns
 * x-slabs, the strict slab segmentation of Sec. 2.1) and exchanges ghost
 * particles and cross-boundary groups between the steps.  Each call is
 * synchronous on the context's stream and bins its particles like
 * cso_find_groups; chained on one box they give cso_find_groups' outputs.
 * pos int32[n][3], ids uint64[n] and the per-particle arrays are in input
 * order, host or device memory as on_device (out->on_device for cso_levels)
 * says; the caller owns every buffer.  Errors as cso_find_groups. */

/* Kernel sums Sigma_i = sum_{j != i, d_ij < b2} (b2 - d_ij) (Sec. 2.2.1,
 * Eq. 1 times b2) of the first n_query particles, every one of the n
 * particles counting as a neighbour (the rest are the caller's ghosts). */
int cso_density(cso_ctx* ctx, const int32_t* pos, int64_t n, int64_t n_query, const cso_params* p, int64_t* sigma,
                int32_t on_device);

/* L0 groups (Sec. 2.2.1) of n particles whose kernel sums the caller gives:
 * particles with Sigma > T_L0 link when d < lfof2; l0[i] = smallest id of
 * i's group, CSO_NO_GROUP for the others. */
int cso_fof(cso_ctx* ctx, const int32_t* pos, const uint64_t* ids, const int64_t* sigma, int64_t n,
            const cso_params* p, uint64_t* l0, int32_t on_device);

/* L1 and L2 (Sec. 2.2.2) inside the groups the caller's labels l0 define
 * (equal labels = one group, CSO_NO_GROUP = in none), with the kernel sums
 * sigma: out->l1, out->l2 (either may be NULL) and the catalogue as
 * cso_find_groups writes them; out->l0, out->sigma and out->radial are not
 * used (radial must be NULL). */
int cso_levels(cso_ctx* ctx, const int32_t* pos, const uint64_t* ids, const int64_t* sigma, const uint64_t* l0,
               int64_t n, const cso_params* p, cso_output* out);

/* --- introspection ------------------------------------------------------ */

/* CUDA stream (cudaStream_t) the context issues its work on. */
void* cso_stream(cso_ctx* ctx);

/* Per-stage device times (ms) of the last cso_find_groups when the context
 * has CSO_FLAG_TIMING; names[i] receives a static string.  Returns the
 * number of stages written (<= cap). */
int cso_stage_times(cso_ctx* ctx, double* ms, const char** names, int cap);

/* Counters of the last call: [0] particles, [1] dense particles, [2] L0
 * groups, [3] L1 nuclei, [4] L2 nuclei, [5] catalogue rows, [6] kernel pairs
 * with d < b2 (only with CSO_FLAG_COUNT_PAIRS), [7] sum over L1 nuclei of their
 * group size, [8] sum over L2 nuclei of their L1 halo size, [9] peak device
 * workspace bytes, [10] kernel launches.  Returns the number written. */
int cso_last_stats(cso_ctx* ctx, int64_t* out, int cap);

/* One-line description of the last error of this thread. */
const char* cso_last_error(void);

/* Measured peak rates of the pipes the pair kernels use, on `device`:
 * out[0] integer add/xor lane-ops per second (Tops/s), out[1] integer
 * multiply-add lane-ops per second (Tops/s), out[2] bytes per second
 * delivered to lanes by 128-bit shared-memory loads that a whole warp reads
 * from one address (TB/s).  Each is one timed launch of independent
 * dependency chains over 8 blocks of 256 threads per SM, after one untimed
 * launch.  Allocates and frees a small device buffer; needs n >= 3. */
int cso_probe_peaks(int device, double* out, int n);

/* Sizes in bytes of the structs above as this library was compiled:
 * out[0..4] = sizeof cso_params, cso_halo, cso_input, cso_output, cso_radial
 * (so that a binding can check its own layouts).  Writes min(n, 5) entries
 * and returns 5; needs no GPU. */
int cso_struct_sizes(int64_t* out, int n);

/* --- kernel density without device allocation ---------------------------
 *
 * The paper has no counterpart of this entry point: it exists for callers
 * that cannot allocate device memory where they need the densities (an
 * N-body code that has given all device memory to its own pool, or a
 * time-step loop in which a cudaMalloc would synchronise the device).
 *
 * Computes Sigma_i (as in cso_output.sigma) for n particles.  pos (int32
 * [n][3]) and sigma (int64 [n], input order) are DEVICE pointers owned by
 * the caller; stream is a cudaStream_t (NULL = legacy default stream); the
 * call returns after the work on that stream has completed.  The scratch
 * lives in one fixed 96 MiB array in device memory that every GPU which
 * loads this library holds until the process exits; nothing is allocated or
 * freed.  Limits: n <= CSO_STATIC_MAX_N and at most CSO_STATIC_MAX_CELLS
 * cells (boxes of up to 64 l_mean per side at the default b); larger requests
 * return CSO_ERR_ARG.  The first call on a device looks up the array's
 * device address, so make it before any stream capture; the address is kept
 * for the life of the process, so after a cudaDeviceReset (or any other
 * teardown of the device's primary context) this entry point must not be
 * called again in that process.  All calls share the one array and it keeps
 * the last call's contents (each call clears what must start at zero): calls
 * that overlap on the GPU (other threads, other streams) race and must be
 * serialised by the caller. */
#define CSO_STATIC_MAX_N (1 << 20)
#define CSO_STATIC_MAX_CELLS (1 << 22)
int cso_density_static(const int32_t* pos, int64_t n, const cso_params* p, int64_t* sigma, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CSO_H */
