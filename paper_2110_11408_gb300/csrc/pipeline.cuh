// Context and pipeline declarations shared by api.cu and pipeline.cu.
#pragma once
#include <utility>
#include <vector>

#include "cells.cuh"
#include "compaso.cuh"

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

// a captured level stage of the batched schedule, keyed by its launch
// arguments (the same box gives the same workspace offsets, hence the key)
struct LevelGraph {
  LevelArgs args;
  int giant = 0, small = 0, huge = 0;
  cudaGraphExec_t exec = nullptr;
};
#define CSO_LEVEL_GRAPHS 4

struct cso_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;   // second stream of the batched schedule (giant groups)
  cudaStream_t side2 = nullptr;  // third stream (large groups)
  cudaStream_t side3 = nullptr;  // fourth stream (huge groups on 16-CTA clusters)
  cudaStream_t copy = nullptr;   // device-to-host copies of outputs final before the step ends
  cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr, join3 = nullptr;
  cudaEvent_t out_ready = nullptr, out_copied = nullptr;
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
  LevelSchedule sched;            // size bins of the batched schedule (cso_autotune)
  double level_ms = 0;            // device time of the last call's CompaSO levels
  ServedState* served = nullptr;  // created by the first cso_submit
  LevelGraph graphs[CSO_LEVEL_GRAPHS];  // CSO_FLAG_GRAPH: captured level stages
  int graph_next = 0;
  long long graph_hits = 0, graph_captures = 0;
};

// The batched level stage; with CSO_FLAG_GRAPH captured once per distinct
// argument set and replayed as a CUDA graph.
int level_stage(cso_ctx* c, const LevelArgs& L, const LevelSchedule& sched, unsigned* host_counts);

struct Meta {  // device counters read back by the host
  unsigned long long sigma_max, id_max;
  unsigned long long pairs, work1, work2;
  int bad;
  int tie_overflow;  // a run of equal (group, Sigma) keys too long for k_tie_fix
  int timeout;       // a bounded device wait gave up (Workspace::err points here)
  int pad_;
};

// dense particles taking part (all, or those of selected groups) and group roots
struct Stages {
  cso_ctx* c;
  bool on;
  int k = 0;
  void mark(const char* name) {
    if (!on || k >= CSO_MAX_STAGES) return;
    cudaEventRecord(c->ev[k], c->stream);
    c->stage_name[k] = name;
    ++k;
  }
  void finish() {
    if (!on) return;
    cudaEventRecord(c->ev[k], c->stream);
    cudaEventSynchronize(c->ev[k]);
    for (int i = 0; i < k; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]);
      c->stage_ms[i] = ms;
    }
    c->nstages = k;
  }
};

// inputs of the group stages: cell-sorted particles with their kernel sums
// and L0 roots; with `select`, only dense particles whose select flag is set
// (whole groups) take part.  x0 is added to stored x for the catalogue.
struct GroupsIn {
  const CellGrid* g;
  const int4* spos;
  const long long* sigma;
  const uint64_t* sid;
  const int* root;
  const unsigned long long* minid;
  const uint8_t* select;
  int n;
  int x0;
};

// gather, L1, L2, labels (ol1 / ol2 indexed by spos[s].w, may be null) and
// the catalogue rows (device, increasing nucleus id) of the groups taking
// part; rows_w_out (optional) receives spos[.].w of every row's nucleus
int run_groups(cso_ctx* c, const cso_params* p, const GroupsIn& gi, Stages& S, Meta* meta, uint64_t* ol1,
               uint64_t* ol2, cso_halo** rows_out, int* nrows_out, uint32_t** rows_w_out,
               cso_radial** radial_out = nullptr);

size_t workspace_bytes(long long n, long long ncell, bool host_io);
int ctx_reserve(cso_ctx* c, long long n, long long ncell, bool host_io);
int check_io(const cso_input* in, const cso_params* p, cso_output* out);
void served_stop(cso_ctx* c);
int pipeline_run(cso_ctx* c, const cso_input* in, const cso_params* p, cso_output* out);
