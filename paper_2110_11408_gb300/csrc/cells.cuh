// Cell-grid kernels (cells.cu): binning, density, FoF, peak test.
#pragma once
#include "cso_internal.cuh"

struct CellGrid {
  int nc;                 // cells per side
  const uint32_t* start;  // nc^3 + 1 offsets into the cell-sorted arrays
};

// One contiguous run [lo, hi) of the cell-sorted arrays inside the 27-cell
// stencil of a query, with the query coordinates shifted by whole boxes so
// that plain differences give minimum-image offsets for every particle of
// the run.
struct StencilRun {
  uint32_t lo, hi;
  int qx, qy, qz;
};

__device__ __forceinline__ int cell_coord(int x, int nc) {
  return (int)(((unsigned long long)(unsigned)x * (unsigned)nc) >> 21);
}

// The up to 18 runs (9 rows of three x-cells, split where a row wraps).
__device__ __forceinline__ int stencil_runs(const CellGrid& g, int x, int y, int z, StencilRun* out) {
  const int nc = g.nc;
  const int cx = cell_coord(x, nc), cy = cell_coord(y, nc), cz = cell_coord(z, nc);
  int r = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int zz = cz + dz, sz = 0;
    if (zz < 0) { zz += nc; sz = CSO_BOX; } else if (zz >= nc) { zz -= nc; sz = -CSO_BOX; }
    for (int dy = -1; dy <= 1; ++dy) {
      int yy = cy + dy, sy = 0;
      if (yy < 0) { yy += nc; sy = CSO_BOX; } else if (yy >= nc) { yy -= nc; sy = -CSO_BOX; }
      const uint32_t* row = g.start + ((size_t)zz * nc + yy) * nc;
      if (cx >= 1 && cx + 1 < nc) {
        out[r++] = StencilRun{row[cx - 1], row[cx + 2], x, y + sy, z + sz};
      } else if (cx == 0) {
        out[r++] = StencilRun{row[0], row[2], x, y + sy, z + sz};
        out[r++] = StencilRun{row[nc - 1], row[nc], x + CSO_BOX, y + sy, z + sz};
      } else {
        out[r++] = StencilRun{row[nc - 2], row[nc], x, y + sy, z + sz};
        out[r++] = StencilRun{row[0], row[1], x - CSO_BOX, y + sy, z + sz};
      }
    }
  }
  return r;
}

int cells_choose(long long b2, int* nc_out);
int cells_bin(const int32_t* pos, const uint64_t* ids, long long n, int nc, uint32_t* start, int4* spos,
              uint64_t* sid, int* bad, Workspace& ws, cudaStream_t st);
int cells_density(const CellGrid& g, const int4* spos, int n, uint32_t b2, int include_self, long long* sigma,
                  unsigned long long* pairs, cudaStream_t st);
int cells_fof(const CellGrid& g, const int4* spos, int n, const long long* sigma, long long T_L0, uint32_t lfof2,
              const uint64_t* sid, int* parent, int* root, unsigned long long* minid, cudaStream_t st);
