// Cell-grid kernels (cells.cu): binning, density, FoF, peak test.
#pragma once
#include "cso_internal.cuh"

struct CellGrid {
  int nc;                 // cells per side
  const uint32_t* start;  // nc^3 + 1 offsets into the cell-sorted arrays
};

int cells_choose(long long b2, int* nc_out);
int cells_bin(const int32_t* pos, const uint64_t* ids, long long n, int nc, uint32_t* start, int4* spos,
              uint64_t* sid, int* bad, Workspace& ws, cudaStream_t st);
int cells_density(const CellGrid& g, const int4* spos, int n, uint32_t b2, int include_self, long long* sigma,
                  unsigned long long* pairs, cudaStream_t st);
int cells_fof(const CellGrid& g, const int4* spos, int n, const long long* sigma, long long T_L0, uint32_t lfof2,
              const uint64_t* sid, int* parent, int* root, unsigned long long* minid, cudaStream_t st);
int cells_peak(const CellGrid& g, const int4* spos, int n, const long long* sigma, const uint64_t* sid,
               const int* label, long long T_min, uint32_t b2, uint8_t* peak, cudaStream_t st);
