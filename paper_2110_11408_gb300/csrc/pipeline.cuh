// Context and pipeline declarations shared by api.cu and pipeline.cu.
#pragma once
#include <utility>
#include <vector>

#include "cso_internal.cuh"

#define CSO_MAX_STAGES 16
#define CSO_NSTATS 11
// device workspace per particle (all stages, worst case), bytes
#define CSO_BYTES_PER_PARTICLE 440

struct ServedReq {
  cso_input in;
  cso_params p;
  cso_output* out;
  uint64_t ticket;
};

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
  std::vector<ServedReq> queue;
  std::vector<std::pair<uint64_t, int>> finished;
};

int ctx_reserve(cso_ctx* c, long long n, long long ncell, bool host_io);
int pipeline_run(cso_ctx* c, const cso_input* in, const cso_params* p, cso_output* out);
