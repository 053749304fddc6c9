// Slab stream state (stream.cu), driven by the served path.
#pragma once
#include <vector>

#include "pipeline.cuh"

struct StreamSlab {
  ServedRequest* req;
  long long n;
  long long pad_;
  cso_output out;
  long long n_halos;
  bool completed = false;
  bool newly_completed = false;
};

struct StreamState {
  uint64_t id = 0;
  cso_params p{};
  int nc = 0;
  long long x_received = 0;  // grid x up to which slabs have arrived
  std::vector<uint8_t> col_fin;  // columns whose kernel sums are final
  // resident particles, double-buffered for compaction (cur is live)
  int cur = 0;
  long long nr = 0, cap = 0;
  int32_t* rpos[2] = {};
  uint64_t* rid[2] = {};
  long long* rsig[2] = {};
  uint8_t* rflag[2] = {};
  uint32_t* rslab[2] = {};
  uint32_t* ridx[2] = {};
  // per-slab output table and counters (device)
  void* dslabs = nullptr;
  unsigned long long* ddone = nullptr;
  unsigned long long* dnrows = nullptr;
  long long slab_cap = 0;
  unsigned* dhist = nullptr;  // resident particles per x column
  int* dbad = nullptr;
  int last_ncols = 0;
  bool failed = false;
  bool busy = false;
  std::vector<StreamSlab> slabs;
};

int stream_begin(StreamState** out, uint64_t id, const cso_params* p);
int stream_step(cso_ctx* c, StreamState& S, const cso_input* in, cso_output* out, ServedRequest* req);
void stream_release(StreamState* S);
