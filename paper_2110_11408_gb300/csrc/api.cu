// C ABI of the CompaSO hot path: parameters, context, and the pipeline
// density -> L0 -> L1 -> L2 -> labels and catalogue (Sec. 2.2 of the paper).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "cells.cuh"
#include "compaso.cuh"
#include "pipeline.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";
thread_local long long g_cso_launches = 0;

void cso_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* cso_last_error(void) { return g_err; }

int cso_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  if (dev >= 0 && dev < 64) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  if (dev >= 0 && dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
// kernel density at the centre of a singular isothermal sphere holding np
// particles inside the radius of mean enclosed density delta (l_mean units):
// M(<R) = 4 pi A R, and the kernel-smoothed SIS tends to 5A/b^2 at r -> 0
// (App. B.2, r < b branch)
static double sis_centre(double np, double delta, double b) {
  double R = cbrt(np / (delta * (4.0 * M_PI / 3.0)));
  double A = np / (4.0 * M_PI * R);
  return 5.0 * A / (b * b);
}

extern "C" int cso_params_derive(cso_params* p) {
  if (!p) return CSO_ERR_ARG;
  double u = p->l_mean_grid;
  if (p->grid_bits != CSO_GRID_BITS || !(u >= 1.0) || u > (double)(1 << 20) || u != floor(u) || !(p->b_kernel > 0) ||
      !(p->l_fof > 0) || p->alpha_den <= 0 || p->alpha_num < 0 || p->roche_den <= 0 || p->roche_num < 0 ||
      p->np_min_density <= 0 || !(p->delta_L1 >= 1.0) || !(p->delta_L2 >= 1.0)) {
    cso_set_error("invalid CompaSO parameters");
    return CSO_ERR_ARG;
  }
  double bu = p->b_kernel * u;
  double lu = p->l_fof * u;
  p->b2 = llround(bu * bu);
  p->lfof2 = llround(lu * lu);
  double b2 = (double)p->b2;
  // kernel sum of a unit-density uniform field: (2/5)(4 pi/3) (b/u)^3 times b2
  double norm = 0.4 * (4.0 * M_PI / 3.0) * b2 * b2 * sqrt(b2) / (u * u * u);
  p->T_L0 = (int64_t)floor(p->delta_L0 * norm);
  p->T_min_L1 = (int64_t)floor(sis_centre(p->np_min_density, p->delta_L1, p->b_kernel) * norm);
  p->T_min_L2 = (int64_t)floor(sis_centre(p->np_min_density, p->delta_L2, p->b_kernel) * norm);
  double k1 = p->delta_L1 * (4.0 * M_PI / 3.0);
  double k2 = p->delta_L2 * (4.0 * M_PI / 3.0);
  p->K_L1 = k1 * k1;
  p->K_L2 = k2 * k2;
  return CSO_OK;
}

extern "C" int cso_params_default(cso_params* p, double l_mean_grid) {
  if (!p) return CSO_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->grid_bits = CSO_GRID_BITS;
  p->include_self = 0;
  p->l_mean_grid = l_mean_grid;
  p->b_kernel = 0.4;
  p->l_fof = 0.25;
  p->delta_L0 = 60.0;
  p->delta_L1 = 200.0;
  p->delta_L2 = 800.0;
  p->alpha_num = 4;
  p->alpha_den = 5;
  p->roche_num = 2;
  p->roche_den = 1;
  p->np_min_density = 35;
  p->np_min_L1 = 35;
  return cso_params_derive(p);
}

// Thresholds for a flat LambdaCDM background at redshift z (Sec. 2.3.1,
// Eq. 2): Delta_base = 18 pi^2 + 82 x - 39 x^2 with x = Omega_m(z) - 1 is the
// overdensity w.r.t. the critical density; Delta_L1 = (200 / 18 pi^2)
// Delta_base / Omega_m(z) w.r.t. the mean, Delta_L2 = 4 Delta_L1, and the L0
// density cut and l_FoF follow the L1 change (the cut in proportion, l_FoF as
// its inverse cube root); b is unchanged.
extern "C" int cso_params_cosmology(cso_params* p, double omega_m0, double z) {
  if (!p || !(omega_m0 > 0 && omega_m0 <= 1) || !(z > -1)) {
    cso_set_error("invalid cosmology (Omega_m0 = %g, z = %g)", omega_m0, z);
    return CSO_ERR_ARG;
  }
  const double a3 = (1.0 + z) * (1.0 + z) * (1.0 + z);
  const double om = omega_m0 * a3 / (omega_m0 * a3 + (1.0 - omega_m0));
  const double x = om - 1.0;
  const double d18 = 18.0 * M_PI * M_PI;
  const double base = d18 + 82.0 * x - 39.0 * x * x;
  const double l1 = 200.0 / d18 * base / om;
  const double change = l1 / 200.0;
  p->delta_L1 = l1;
  p->delta_L2 = 4.0 * l1;
  p->delta_L0 = 60.0 * change;
  p->l_fof = 0.25 * pow(change, -1.0 / 3.0);
  return cso_params_derive(p);
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int cso_init(cso_ctx** out, int device, size_t budget, uint32_t flags) {
  if (!out) return CSO_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  CSO_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) {
    cso_set_error("no CUDA device %d (found %d)", device, ndev);
    return CSO_ERR_ARG;
  }
  CSO_CUDA(cudaSetDevice(device));
  cso_ctx* c = new cso_ctx();
  c->device = device;
  c->budget = budget;
  c->flags = flags;
  c->served_slots = (int)((flags >> 8) & 0xf);
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side3, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join3, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->out_ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->out_copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->pinned, sizeof(long long) * 64);
  for (int i = 0; e == cudaSuccess && i <= CSO_MAX_STAGES; ++i) e = cudaEventCreate(&c->ev[i]);
  if (e != cudaSuccess) {
    cso_set_error("cso_init: %s", cudaGetErrorString(e));
    cso_free(c);
    return CSO_ERR_CUDA;
  }
  *out = c;
  return CSO_OK;
}

extern "C" void cso_free(cso_ctx* c) {
  if (!c) return;
  served_stop(c);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->ws.base) cudaFree(c->ws.base);
  if (c->pinned) cudaFreeHost(c->pinned);
  for (int i = 0; i <= CSO_MAX_STAGES; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  for (int i = 0; i < CSO_LEVEL_GRAPHS; ++i)
    if (c->graphs[i].exec) cudaGraphExecDestroy(c->graphs[i].exec);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->side2) cudaStreamSynchronize(c->side2);
  if (c->side3) cudaStreamSynchronize(c->side3);
  if (c->join2) cudaEventDestroy(c->join2);
  if (c->side2) cudaStreamDestroy(c->side2);
  if (c->join3) cudaEventDestroy(c->join3);
  if (c->side3) cudaStreamDestroy(c->side3);
  if (c->copy) cudaStreamSynchronize(c->copy);
  if (c->out_ready) cudaEventDestroy(c->out_ready);
  if (c->out_copied) cudaEventDestroy(c->out_copied);
  if (c->copy) cudaStreamDestroy(c->copy);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" void* cso_stream(cso_ctx* c) { return c ? (void*)c->stream : nullptr; }

extern "C" int cso_stage_times(cso_ctx* c, double* ms, const char** names, int cap) {
  if (!c) return 0;
  int k = c->nstages < cap ? c->nstages : cap;
  for (int i = 0; i < k; ++i) {
    if (ms) ms[i] = c->stage_ms[i];
    if (names) names[i] = c->stage_name[i];
  }
  return k;
}

extern "C" int cso_last_stats(cso_ctx* c, int64_t* out, int cap) {
  if (!c) return 0;
  int k = cap < CSO_NSTATS ? cap : CSO_NSTATS;
  for (int i = 0; i < k; ++i) out[i] = c->stats[i];
  return k;
}

// workspace large enough for n particles and ncell cells
size_t workspace_bytes(long long n, long long ncell, bool host_io) {
  size_t need = (size_t)n * CSO_BYTES_PER_PARTICLE + (size_t)(ncell + 1) * 8 + ((size_t)64 << 20);
  if (host_io) need += (size_t)n * (12 + 8 + 32);
  return need;
}

int ctx_reserve(cso_ctx* c, long long n, long long ncell, bool host_io) {
  size_t need = workspace_bytes(n, ncell, host_io);
  if (c->budget && need > c->budget) {
    cso_set_error("request needs %zu bytes of workspace, budget is %zu", need, c->budget);
    return CSO_ERR_BUDGET;
  }
  if (need > c->ws.cap) {
    if (c->ws.base) {
      CSO_CUDA(cudaStreamSynchronize(c->stream));
      CSO_CUDA(cudaFree(c->ws.base));
      c->ws.base = nullptr;
      c->ws.cap = 0;
    }
    CSO_CUDA(cudaMalloc((void**)&c->ws.base, need));
    c->ws.cap = need;
  }
  c->ws.off = 0;
  c->ws.peak = 0;
  c->ws.err = nullptr;  // each request points it at its own device word
  return CSO_OK;
}

// ---------------------------------------------------------------------------
// autotuner of the batched schedule's size bins
// ---------------------------------------------------------------------------
static double level_time(const cso_ctx* c) {
  double t = 0;
  for (int i = 0; i < c->nstages; ++i)
    if (!strcmp(c->stage_name[i], "level1") || !strcmp(c->stage_name[i], "level2")) t += c->stage_ms[i];
  return t;
}

extern "C" int cso_set_schedule(cso_ctx* c, int32_t giant, int32_t small) {
  if (!c || giant < 64 || small < 1 || small > 64) {
    cso_set_error("size bins need giant >= 64 and 1 <= small <= 64");
    return CSO_ERR_ARG;
  }
  c->sched.giant = giant;
  c->sched.small = small;
  return CSO_OK;
}

extern "C" int cso_set_huge_group(cso_ctx* c, int32_t huge) {
  if (!c || huge < 64) {
    cso_set_error("the huge-group bound needs huge >= 64");
    return CSO_ERR_ARG;
  }
  c->sched.huge = huge;
  return CSO_OK;
}

extern "C" int cso_autotune(cso_ctx* c, const cso_input* in, const cso_params* p, cso_output* out,
                            int32_t* giant, int32_t* small) {
  if (!c) return CSO_ERR_ARG;
  static const int giants[] = {4096, 8192, 16384, 65536, 262144};
  static const int smalls[] = {32, 64};
  const uint32_t saved = c->flags;
  c->flags |= CSO_FLAG_TIMING | CSO_FLAG_BATCHED;
  LevelSchedule best = c->sched;
  double best_t = 1e30;
  int rc = CSO_OK;
  for (int gi = 0; gi < 5 && rc == CSO_OK; ++gi)
    for (int si = 0; si < 2 && rc == CSO_OK; ++si) {
      c->sched.giant = giants[gi];
      c->sched.small = smalls[si];
      double t = 1e30;
      for (int rep = 0; rep < 2 && rc == CSO_OK; ++rep) {
        rc = cso_find_groups(c, in, p, out);
        const double lt = level_time(c);
        if (lt < t) t = lt;
      }
      if (rc == CSO_OK && t < best_t) {
        best_t = t;
        best = c->sched;
      }
    }
  c->flags = saved;
  c->sched = best;
  if (giant) *giant = best.giant;
  if (small) *small = best.small;
  return rc;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
int check_io(const cso_input* in, const cso_params* p, cso_output* out) {
  if (!in || !p || !out || in->n < 0 || (in->n > 0 && (!in->pos || !in->ids))) {
    cso_set_error("null or negative argument");
    return CSO_ERR_ARG;
  }
  if (in->n >= (1ll << 31) - 1) {
    cso_set_error("n = %lld is too large for one request (< 2^31)", (long long)in->n);
    return CSO_ERR_ARG;
  }
  if (out->halo_cap < 0 || (out->halo_cap > 0 && !out->halos)) {
    cso_set_error("halo_cap > 0 needs a halos buffer");
    return CSO_ERR_ARG;
  }
  if (out->radial && in->x_hi > 0) {
    cso_set_error("radial statistics are computed for whole-box requests only");
    return CSO_ERR_ARG;
  }
  return CSO_OK;
}

extern "C" int cso_find_groups(cso_ctx* c, const cso_input* in, const cso_params* pin, cso_output* out) {
  if (!c) return CSO_ERR_ARG;
  CSO_TRY(check_io(in, pin, out));
  cso_params p = *pin;
  CSO_TRY(cso_params_derive(&p));
  CSO_CUDA(cudaSetDevice(c->device));
  int rc = pipeline_run(c, in, &p, out);
  return rc;
}

extern "C" int cso_struct_sizes(int64_t* out, int n) {
  const int64_t sz[5] = {(int64_t)sizeof(cso_params), (int64_t)sizeof(cso_halo), (int64_t)sizeof(cso_input),
                         (int64_t)sizeof(cso_output), (int64_t)sizeof(cso_radial)};
  for (int i = 0; i < n && i < 5 && out; ++i) out[i] = sz[i];
  return 5;
}
