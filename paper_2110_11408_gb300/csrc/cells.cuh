// Cell-grid kernels (cells.cu): binning, density, FoF, peak test.
#pragma once
#include "cso_internal.cuh"

// A cell table over the particles of a whole periodic box, or over a window
// of x columns of one (the served slab stream).  Cells are at least as wide as
// the largest search radius, so every neighbour lies in the 27 cells around a
// particle's own.  Cell (cz, cy, column) starts at
// start[(cz * nc + cy) * ncols + column]; the table has ncols * nc * nc + 1
// entries, x fastest, so the x-cells of one (y, z) row are contiguous.
//
// Whole box: colmap == nullptr, ncols == nc, stored x is the grid x and x
// wraps like y and z.  Window: colmap maps each global x column to its table
// column (-1 if absent), cols maps back, and stored x is (grid x - x0) mod
// 2^21: unwrapped across the window, which never spans half the box, so x
// never wraps inside a window.
struct CellGrid {
  int nc;
  int ncols;
  const uint32_t* start;
  const int* colmap;
  const int* cols;
  int x0;
};

static inline CellGrid whole_box_grid(int nc, const uint32_t* start) {
  return CellGrid{nc, nc, start, nullptr, nullptr, 0};
}

__device__ __forceinline__ int cell_coord(int x, int nc) {
  return (int)(((unsigned long long)(unsigned)x * (unsigned)nc) >> 21);
}

// table column of a stored x
__device__ __forceinline__ int grid_col(const CellGrid& g, int xs) {
  if (!g.colmap) return cell_coord(xs, g.nc);
  return g.colmap[cell_coord((xs + g.x0) & (CSO_BOX - 1), g.nc)];
}

// first grid coordinate of cell c (cells are [ceil(c 2^21 / nc), ceil((c + 1) 2^21 / nc)))
__device__ __forceinline__ int cell_lo(int c, int nc) {
  return (int)(((long long)c * CSO_BOX + nc - 1) / nc);
}

// The x cells around table column tc: columns a..b form one contiguous run
// (a = tc - 1 and b = tc + 1 when those neighbours exist), and in a whole box
// the row may wrap: wl >= 0 is the far-left column (query shifted by +box),
// wr >= 0 the far-right one (query shifted by -box).
struct XCells {
  int a, b, wl, wr;
};

__device__ __forceinline__ XCells x_cells(const CellGrid& g, int tc) {
  XCells r{tc, tc, -1, -1};
  if (!g.colmap) {
    if (tc > 0) r.a = tc - 1; else r.wl = g.nc - 1;
    if (tc + 1 < g.nc) r.b = tc + 1; else r.wr = 0;
  } else {
    const int gc = g.cols[tc];
    if (tc > 0 && g.cols[tc - 1] == (gc + g.nc - 1) % g.nc) r.a = tc - 1;
    if (tc + 1 < g.ncols && g.cols[tc + 1] == (gc + 1) % g.nc) r.b = tc + 1;
  }
  return r;
}

__device__ __forceinline__ int wrap_yz(int c, int nc, int& shift) {
  shift = 0;
  if (c < 0) {
    shift = CSO_BOX;  // neighbour sits at the far end: move the query up by a box
    return c + nc;
  }
  if (c >= nc) {
    shift = -CSO_BOX;
    return c - nc;
  }
  return c;
}

__device__ __forceinline__ const uint32_t* grid_row(const CellGrid& g, int zz, int yy) {
  return g.start + ((size_t)zz * g.nc + yy) * g.ncols;
}

__device__ __forceinline__ size_t grid_cell(const CellGrid& g, int zz, int yy, int tc) {
  return ((size_t)zz * g.nc + yy) * g.ncols + tc;
}

// Visit every cell-sorted index t in the 27-cell stencil of the query, row
// by row; f(t, xq, yq, zq) receives the query shifted by whole boxes so that
// plain differences are minimum-image offsets.  No culling: lanes of a warp
// in one cell walk the same runs, which keeps the warp converged.
template <class F>
__device__ __forceinline__ void for_stencil(const CellGrid& g, int x, int y, int z, F f) {
  const int nc = g.nc;
  const int cy = cell_coord(y, nc), cz = cell_coord(z, nc);
  const XCells X = x_cells(g, grid_col(g, x));
  for (int dz = -1; dz <= 1; ++dz) {
    int sz;
    const int zz = wrap_yz(cz + dz, nc, sz);
    for (int dy = -1; dy <= 1; ++dy) {
      int sy;
      const int yy = wrap_yz(cy + dy, nc, sy);
      const uint32_t* row = grid_row(g, zz, yy);
      const int yq = y + sy, zq = z + sz;
      for (uint32_t t = row[X.a], e = row[X.b + 1]; t < e; ++t) f(t, x, yq, zq);
      if (X.wl >= 0)
        for (uint32_t t = row[X.wl], e = row[X.wl + 1]; t < e; ++t) f(t, x + CSO_BOX, yq, zq);
      if (X.wr >= 0)
        for (uint32_t t = row[X.wr], e = row[X.wr + 1]; t < e; ++t) f(t, x - CSO_BOX, yq, zq);
    }
  }
}

// Cells per side for a kernel radius of sqrt(b2) grid units: the largest nc
// with cells at least b wide, 128 <= nc <= CSO_MAX_NC.
#define CSO_MAX_NC 16384
int cells_choose(long long b2, int* nc_out);
// A whole box keeps one dense table of nc^3 cells (uint32 cell keys, 16 GB at
// most); finer boxes go through the slab stream, whose window tables cover only
// the x columns holding resident particles.
#define CSO_MAX_DENSE_NC 1290
int cells_check_dense(int nc);
// Counting sort of the particles into the cell table, each cell ordered by
// (stored x, input index), so the x cells of a row form one run sorted by x;
// inv (optional, n entries) receives the sorted slot of every input particle.
// spos doubles as scratch for the cell keys and arrival ranks (it must not
// alias pos).
int cells_bin(const int32_t* pos, const uint64_t* ids, long long n, const CellGrid& g, uint32_t* start,
              int4* spos, uint64_t* sid, int* bad, Workspace& ws, cudaStream_t st, uint32_t* inv = nullptr);
int cells_density(const CellGrid& g, const int4* spos, int n, uint32_t b2, int include_self, long long* sigma,
                  unsigned long long* pairs, Workspace& ws, cudaStream_t st, const uint8_t* only = nullptr);
// L0 friends-of-friends over the dense particles (Sigma > T_L0): root[s] (-1
// if not dense) and minid[root] = smallest id of the group.  cell_root is
// scratch of n ints.
int cells_fof(const CellGrid& g, const int4* spos, int n, const long long* sigma, long long T_L0, uint32_t lfof2,
              const uint64_t* sid, int* parent, int* root, unsigned long long* minid, int* cell_root,
              Workspace& ws, cudaStream_t st);
