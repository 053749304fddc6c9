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

// first grid coordinate of cell c (cells are [ceil(c 2^21 / nc), ceil((c + 1) 2^21 / nc)))
__device__ __forceinline__ int cell_lo(int c, int nc) {
  return (int)(((long long)c * CSO_BOX + nc - 1) / nc);
}

// Visit every cell-sorted index t that can lie within squared radius r2 of
// the query: the 27-cell stencil, minus the rows and the end cells of rows
// whose nearest possible point is already at r2 or beyond (given the query's
// offset inside its own cell).  f(t, xq, yq, zq) receives the query shifted by
// whole boxes so that plain differences are minimum-image offsets; f returns
// false to stop.  Requires cells at least as wide as the radius.
template <class F>
__device__ __forceinline__ void for_stencil_r(const CellGrid& g, int x, int y, int z, uint32_t r2, F f) {
  const int nc = g.nc;
  const int cx = cell_coord(x, nc), cy = cell_coord(y, nc), cz = cell_coord(z, nc);
  // squared distance from the query to the near faces of the neighbouring cells
  const long long xl = x - cell_lo(cx, nc) + 1, xr = cell_lo(cx + 1, nc) - x;
  const long long yl = y - cell_lo(cy, nc) + 1, yr = cell_lo(cy + 1, nc) - y;
  const long long zl = z - cell_lo(cz, nc) + 1, zr = cell_lo(cz + 1, nc) - z;
  const long long R2 = r2;
  for (int dz = -1; dz <= 1; ++dz) {
    const long long mz = dz < 0 ? zl * zl : (dz > 0 ? zr * zr : 0);
    if (mz >= R2) continue;
    int zz = cz + dz, sz = 0;
    if (zz < 0) { zz += nc; sz = CSO_BOX; } else if (zz >= nc) { zz -= nc; sz = -CSO_BOX; }
    for (int dy = -1; dy <= 1; ++dy) {
      const long long my = mz + (dy < 0 ? yl * yl : (dy > 0 ? yr * yr : 0));
      if (my >= R2) continue;
      int yy = cy + dy, sy = 0;
      if (yy < 0) { yy += nc; sy = CSO_BOX; } else if (yy >= nc) { yy -= nc; sy = -CSO_BOX; }
      const uint32_t* row = g.start + ((size_t)zz * nc + yy) * nc;
      const bool left = my + xl * xl < R2, right = my + xr * xr < R2;
      const int yq = y + sy, zq = z + sz;
      // own cell, plus the x neighbours that can reach; wrapped ones are separate runs
      int a = cx, b = cx;
      int wl = -1, wr = -1;
      if (left) { if (cx > 0) a = cx - 1; else wl = nc - 1; }
      if (right) { if (cx + 1 < nc) b = cx + 1; else wr = 0; }
      for (uint32_t t = row[a], e = row[b + 1]; t < e; ++t)
        if (!f(t, x, yq, zq)) return;
      if (wl >= 0)
        for (uint32_t t = row[wl], e = row[wl + 1]; t < e; ++t)
          if (!f(t, x + CSO_BOX, yq, zq)) return;
      if (wr >= 0)
        for (uint32_t t = row[0], e = row[1]; t < e; ++t)
          if (!f(t, x - CSO_BOX, yq, zq)) return;
    }
  }
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
              const uint64_t* sid, int* parent, int* root, unsigned long long* minid, int* cell_root,
              cudaStream_t st);
