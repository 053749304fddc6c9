// CompaSO level kernels (compaso.cu).
#pragma once
#include "cells.cuh"

// constants of the exact predicate n^2 u^6 < K d^3
struct PredConst {
  double K;                 // (Delta 4 pi / 3)^2
  double u6;                // u^6 (double)
  unsigned long long Km;    // K = Km * 2^Ke exactly
  int Ke;
  unsigned long long u;
  float bin_scale0;         // sqrt(K) / u^3
  int radial;               // first window in radial bins of width sqrt(3)/3 cell sides (Sec. 2.3.4)
  float rbin_inv_w;         // 1 / that width, per grid unit
};
PredConst make_pred_const(double K, long long u);

struct LevelArgs {
  int nseg;
  const uint32_t* seg_off;  // nseg + 1 offsets into the element arrays
  const int4* epos;         // member positions, key order within a segment
  const long long* esig;    // kernel sums (descending within a segment)
  const uint32_t* egs;      // cell-sorted index of each member
  long long T_min;
  PredConst pc;
  int alpha_num, alpha_den, roche_num, roche_den;
  int* eslot;               // out: nucleus ordinal within the segment, or -1
  long long* edold;         // scratch: squared distance to the current nucleus
  uint8_t* einel;           // scratch: ineligible flags
  long long* ed;            // scratch: distances to the nucleus being processed
  // cell-sorted particle data for the local-peak test of step 2
  CellGrid grid;
  const int4* spos;
  const long long* ssig;
  const uint64_t* sid;
  const int* slab;          // group label per cell-sorted particle (-1: none)
  uint32_t b2;
  uint32_t* nuc_member;     // out: [seg_off + q] member offset of nucleus q
  long long* nuc_R2;        // out: [seg_off + q] its squared radius
  uint32_t* nnuc;           // out: nuclei per segment
  unsigned long long* work; // optional: sum over nuclei of the segment size
  int small_n;              // groups up to this size are sorted whole (<= 2048)
  int cap;                  // largest histogram bin sorted in shared memory (<= 2048)
  int nb;                   // histogram bins (<= 1024)
};

// groups above this many members (and above the giant bound) run on 16-CTA
// thread-block clusters where the device can hold one
#define CSO_HUGE_GROUP (1 << 19)

// size bins of the batched schedule: groups above `giant` members run on an
// 8-CTA thread-block cluster, groups above large() on a 1024-thread block,
// groups up to `small` members on one warp, the rest on a 256-thread block;
// largest first within each bin
struct LevelSchedule {
  int giant = 16384;
  int small = 64;
  int huge = CSO_HUGE_GROUP;  // above max(huge, giant): 16-CTA clusters
  int large() const { return giant / 16 > 512 ? giant / 16 : 512; }
};

int level_run(const LevelArgs& a, cudaStream_t st);
// one-time set-up of the batched schedule's launch sizes (occupancy queries),
// kept out of stream capture
void level_prepare();
int level_run_batched(const LevelArgs& a, const LevelSchedule& sc, Workspace& ws, cudaStream_t st,
                      cudaStream_t side, cudaStream_t side2, cudaStream_t side3, cudaEvent_t fork,
                      cudaEvent_t join, cudaEvent_t join2, cudaEvent_t join3, unsigned* host_counts);
// ehalo[j] = global halo of member j (hbase[g] + its nucleus ordinal, or -1)
// and the nucleus records of every halo; n_members = seg_off[nseg] and
// n_halos = hbase[nseg] as the host knows them (launch sizes)
int level_halo(int nseg, const uint32_t* seg_off, const uint32_t* nnuc, const uint32_t* hbase, const int* eslot,
               const uint32_t* nuc_member, const long long* nuc_R2, int* ehalo, uint32_t* hnuc, long long* hR2,
               uint32_t* hseg, long long n_members, long long n_halos, cudaStream_t st);
