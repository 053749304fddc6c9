// Context and pipeline declarations shared by api.cu and pipeline.cu.
#pragma once
#include <utility>
#include <vector>

#include "cso_internal.cuh"

#define CSO_MAX_STAGES 16
#define CSO_NSTATS 11
// device workspace per particle (all stages, worst case), bytes
#define CSO_BYTES_PER_PARTICLE 440

struct ServedRequest {
  cso_input in;
  cso_params p;
  cso_output* out;
  uint64_t ticket = 0;
  size_t need = 0;  // device bytes reserved while it runs
  int status = CSO_OK;
  bool done = false;
  double t_submit = 0, t_start = 0, t_done = 0;  // host steady clock, seconds
};
struct ServedState;

struct cso_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // second stream of the batched schedule (giant groups)
  cudaEvent_t fork = nullptr, join = nullptr;
  size_t budget = 0;
  uint32_t flags = 0;
  Workspace ws;
  long long* pinned = nullptr;  // small pinned host buffer for counter read-backs
  cudaEvent_t ev[CSO_MAX_STAGES + 1] = {};
  int nstages = 0;
  double stage_ms[CSO_MAX_STAGES] = {};
  const char* stage_name[CSO_MAX_STAGES] = {};
  int64_t stats[CSO_NSTATS] = {};
  cso_halo* rows = nullptr;  // per-halo rows (device), grown on demand
  size_t rows_cap = 0;
  uint64_t next_ticket = 0;
  int served_slots = 0;           // worker slots of the served path (0 = 4)
  ServedState* served = nullptr;  // created by the first cso_submit
};

size_t workspace_bytes(long long n, long long ncell, bool host_io);
int ctx_reserve(cso_ctx* c, long long n, long long ncell, bool host_io);
int check_io(const cso_input* in, const cso_params* p, cso_output* out);
void served_stop(cso_ctx* c);
int pipeline_run(cso_ctx* c, const cso_input* in, const cso_params* p, cso_output* out);
