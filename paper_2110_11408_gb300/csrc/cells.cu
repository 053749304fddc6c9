// Cell binning, kernel density and L0 friends-of-friends.
//
// Particles are binned into nc^3 cells of side 2^21/nc >= b (a counting sort
// into a dense cell table, x fastest, each cell ordered by x inside), so
// every neighbour within b of a particle lies in the 27 cells around its own
// and, for the three cells of one (y, z) row, in one contiguous run of the
// sorted array, itself sorted by x.  Periodic wrap
// is handled per run by shifting the query point by one box length, never
// per pair.  With side <= 2^14 grid units every |dx| inside the stencil is
// below 2^15, so squared distances fit uint32 exactly.
#include <limits.h>
#include <math.h>

#include "cells.cuh"

namespace {

// Table cell of input particle i under the rules of k_cell_count: a position
// outside the box counts as (0, 0, 0) and a window particle outside the
// window's columns is filed under table column 0 with y = z = 0 (both set
// *bad_code).
__device__ __forceinline__ uint32_t bin_key(const int32_t* __restrict__ pos, size_t i, const CellGrid& g,
                                            int* bad_code) {
  int x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  *bad_code = 0;
  if ((unsigned)x >= (unsigned)CSO_BOX || (unsigned)y >= (unsigned)CSO_BOX || (unsigned)z >= (unsigned)CSO_BOX) {
    *bad_code = 1;
    x = y = z = 0;
  }
  // table column from the grid x (whole box or window alike)
  int tc = g.colmap ? g.colmap[cell_coord(x, g.nc)] : cell_coord(x, g.nc);
  if (tc < 0) {
    *bad_code = 2;
    tc = 0;
    y = z = 0;
  }
  return (uint32_t)grid_cell(g, cell_coord(z, g.nc), cell_coord(y, g.nc), tc);
}

// Stored position of input particle i: x relative to the table's x0 (a
// window never wraps), y, z, and w = i.  A particle that k_cell_count
// rejected is stored at the low corner of table column 0, so every later
// kernel derives an in-range cell from it (the request still fails on the bad
// flag, but no kernel indexes past the table).
__device__ __forceinline__ int4 stored_pos(const int32_t* __restrict__ pos, size_t i, const CellGrid& g) {
  int x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  const bool out = (unsigned)x >= (unsigned)CSO_BOX || (unsigned)y >= (unsigned)CSO_BOX ||
                   (unsigned)z >= (unsigned)CSO_BOX || (g.colmap && g.colmap[cell_coord(x, g.nc)] < 0);
  if (out) {
    x = g.colmap ? cell_lo(g.cols[0], g.nc) : 0;
    y = z = 0;
  }
  return make_int4((x - g.x0) & (CSO_BOX - 1), y, z, (int)i);
}

// Cells are sorted by x (k_cell_place), so a run of adjacent x cells is
// sorted by stored x: trim [lo, hi) to the neighbours with xl <= x <= xh by
// two binary searches in lockstep.
__device__ __forceinline__ void x_trim(const int4* __restrict__ spos, uint32_t& lo, uint32_t& hi, int xl, int xh) {
  uint32_t a = lo, b = hi, c = lo, d = hi;
  while (a < b || c < d) {
    if (a < b) {
      const uint32_t m = (a + b) >> 1;
      if (spos[m].x < xl) a = m + 1; else b = m;
    }
    if (c < d) {
      const uint32_t m = (c + d) >> 1;
      if (spos[m].x <= xh) c = m + 1; else d = m;
    }
  }
  lo = a;
  hi = c > a ? c : a;
}

__global__ void k_cell_count(const int32_t* __restrict__ pos, long long n, CellGrid g, uint32_t* __restrict__ key,
                             uint32_t* __restrict__ rank, uint32_t* __restrict__ count, int* __restrict__ bad) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int code;
  const uint32_t k = bin_key(pos, (size_t)i, g, &code);
  if (code) atomicExch(bad, code);
  key[i] = k;
  rank[i] = atomicAdd(&count[k], 1u);
}

// Everything k_cell_place needs of the particle at a provisional slot: its
// sort key (stored x << 32 | input index), its cell's range, its stored y and
// z and its id.  One record is one 32-byte sector, so the scatter writes
// whole sectors and the placement reads nothing from scattered places.
struct __align__(32) BinRec {
  unsigned long long key;
  uint32_t c0, m;
  int y, z;
  unsigned long long id;
};

// Provisional slot of every particle (cell start + arrival rank): the record
// is scattered there, and inv (optional) receives the provisional slot in
// input order.
__global__ void k_cell_scatter(const int32_t* __restrict__ pos, const uint64_t* __restrict__ ids, long long n,
                               CellGrid g, const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
                               const uint32_t* __restrict__ start, BinRec* __restrict__ rec,
                               uint32_t* __restrict__ inv) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 q = stored_pos(pos, (size_t)i, g);
  const uint32_t k = key[i], c0 = start[k], c1 = start[k + 1];
  const uint32_t p = c0 + rank[i];
  // one 256-bit store: the whole sector in one scattered write
  const unsigned long long w0 = ((unsigned long long)(unsigned)q.x << 32) | (unsigned long long)i;
  const unsigned long long w1 = (unsigned long long)c0 | ((unsigned long long)(c1 - c0) << 32);
  const unsigned long long w2 = (unsigned long long)(unsigned)q.y | ((unsigned long long)(unsigned)q.z << 32);
  const unsigned long long w3 = ids[i];
  asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(rec + p), "l"(w0), "l"(w1), "l"(w2), "l"(w3)
               : "memory");
  if (inv) inv[i] = p;
}

// Final slot of every particle: its cell's start plus its rank by (stored x,
// input index) among the cell's particles, so every cell, and with it every
// (y, z) row of adjacent x cells, is sorted by x (the density pass bounds its
// runs by x).  A lane counts a cell of up to 32 particles alone; the warp
// streams each larger cell once through shared memory for all its lanes in
// that cell.  Position and id come with the record and are written into the
// cell's range; fin (optional) maps the provisional slot to the final one
// (k_cell_inv composes it into inv).
constexpr int PLACE_SMALL = 32;
__global__ void __launch_bounds__(256) k_cell_place(long long n, const BinRec* __restrict__ rec,
                                                    int4* __restrict__ spos, uint64_t* __restrict__ sid,
                                                    uint32_t* __restrict__ fin) {
  __shared__ unsigned long long tile[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = t < n;
  unsigned long long kt = 0, id = 0;
  uint32_t c0 = 0, c1 = 0;
  int y = 0, z = 0;
  if (act) {
    unsigned long long w0, w1, w2, w3;
    asm volatile("ld.global.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3) : "l"(rec + t));
    kt = w0;
    c0 = (uint32_t)w1;
    c1 = c0 + (uint32_t)(w1 >> 32);
    y = (int)(uint32_t)w2;
    z = (int)(uint32_t)(w2 >> 32);
    id = w3;
  }
  const bool big = act && c1 - c0 > (uint32_t)PLACE_SMALL;
  uint32_t rk = 0;
  if (act && !big)
    for (uint32_t u = c0; u < c1; ++u) rk += rec[u].key < kt;
  unsigned pend = __ballot_sync(0xffffffffu, big);
  while (pend) {
    const int L = __ffs(pend) - 1;
    const uint32_t b0 = __shfl_sync(0xffffffffu, c0, L), b1 = __shfl_sync(0xffffffffu, c1, L);
    const bool mine = big && c0 == b0;
    for (uint32_t u0 = b0; u0 < b1; u0 += 32) {
      tile[w][lane] = u0 + lane < b1 ? rec[u0 + lane].key : ~0ull;  // past the cell: never below a key
      __syncwarp();
      if (mine) {
#pragma unroll 8
        for (int k = 0; k < 32; ++k) rk += tile[w][k] < kt;
      }
      __syncwarp();
    }
    pend &= ~__ballot_sync(0xffffffffu, mine);
  }
  if (!act) return;
  const uint32_t d = c0 + rk;
  spos[d] = make_int4((int)(kt >> 32), y, z, (int)(uint32_t)kt);
  sid[d] = id;
  if (fin) fin[t] = d;
}

// inv[i] = fin[inv[i]]: the final slot of every input particle (a gather in
// input order instead of a scattered write from the placement)
__global__ void k_cell_inv(long long n, const uint32_t* __restrict__ fin, uint32_t* __restrict__ inv) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) inv[i] = fin[inv[i]];
}

__device__ __forceinline__ uint32_t kern(int4 q, int xq, int yq, int zq, uint32_t b2) {
  const int dx = xq - q.x, dy = yq - q.y, dz = zq - q.z;
  const uint32_t d = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
  return b2 - (d < b2 ? d : b2);  // b2 - d inside the kernel support, else 0
}

// Sigma_s = sum over j != s with d < b2 of (b2 - d)   (Eq. 1 times b2).
//
// A warp takes 32 consecutive cell-sorted particles.  When they all sit in
// one (y, z) row of cells and span at most max_span + 1 adjacent x cells
// (the common case wherever the work is: in and around dense cells), they
// share the nine stencil rows, each the union of their x ranges, which is one
// contiguous run of the sorted array (plus a wrapped run at the periodic x
// edge).  The warp walks each run once, 32 neighbours at a time: every lane
// loads one neighbour of the next 32 (a coalesced int4 load, in flight while
// the current 32 are summed) and stores it, shifted and with |c|^2, into the
// warp's shared tile; each lane then sums its own particle against the tile
// by shared-memory broadcast.  Warps whose particles span more cells walk the
// stencil lane by lane.
//
// In the shared walk, offsets are taken from the warp's first particle o:
// the query is q = p - o, a staged neighbour c = t - shift - o, and
// d = |q|^2 + |c|^2 - 2 q.c.  The staging lane stores |c|^2 beside c, so a
// pair costs three multiply-adds, a min and an add:
//   * in general, d is formed modulo 2^32 and min(d, b2) summed; it is exact
//     because the true d of every staged pair is below 2^32 (max_span is
//     chosen on the host so that ((max_span + 2)^2 + 8) cell^2 < 2^32);
//   * when every true d is below 2^29 (cells below 4,730 grid units), the
//     lane compares t = d - |q|^2 with its own bound b2 - |q|^2 as signed
//     integers, which saves the add of |q|^2.
// Sharing rows over up to three x cells instead of one cell cut the pass by
// 3% on the 16.8M-particle box and 22% on the 2.1M-particle box (GB300); the
// same walk with tiles staged by bulk copies (cp.async.bulk into
// double-buffered shared tiles completing on an mbarrier) measured slower at
// every tile size tried (64, 128, 256 particles), so the lanes load the tiles.
//
// Blocks run heaviest first: a cost pass estimates each block's candidate
// count, files the block under floor(log2(cost)) and the density launch takes
// block order[blockIdx.x], so the dense-halo blocks start in the first wave
// instead of forming the tail.
constexpr int DENS_WARPS = 8;
constexpr int DENS_CLASSES = 33;

__device__ __forceinline__ uint32_t sq3(int x, int y, int z) {
  return (uint32_t)x * (uint32_t)x + (uint32_t)y * (uint32_t)y + (uint32_t)z * (uint32_t)z;
}

// min(d, b2) for the staged neighbour c = (offset, |offset|^2) and the query
// with P = |q|^2 and a = -2 q (modulo 2^32)
__device__ __forceinline__ uint32_t dmin_dot(int4 c, uint32_t P, uint32_t ax, uint32_t ay, uint32_t az, uint32_t b2) {
  const uint32_t d = (uint32_t)c.w + P + ax * (uint32_t)c.x + ay * (uint32_t)c.y + az * (uint32_t)c.z;
  return d < b2 ? d : b2;
}

// min(d - P, b2 - P) as signed integers (every true d below 2^31)
__device__ __forceinline__ int tmin_dot(int4 c, int ax, int ay, int az, int B) {
  const int t = c.w + ax * c.x + ay * c.y + az * c.z;
  return t < B ? t : B;
}

// The shared-walk setup of one warp: whether its valid particles share a
// (y, z) cell row and a short x span, and, for lanes 0-8, the runs of stencil
// row (dz + 1) * 3 + (dy + 1): main run [lo0, hi0) and the wrapped run
// [lo1, hi1) with its x shift sx1.
struct WarpRows {
  bool uniform;
  int src;  // first valid lane
  uint32_t lo0, hi0, lo1, hi1;
  int sy, sz, sx1;
};

__device__ __forceinline__ WarpRows warp_rows(const CellGrid& g, int4 p, bool valid, unsigned vmask, int lane,
                                              int max_span) {
  WarpRows R{};
  const int nc = g.nc;
  const int cy = cell_coord(p.y, nc), cz = cell_coord(p.z, nc), tc = grid_col(g, p.x);
  R.src = __ffs(vmask) - 1;
  const int yz = cz * nc + cy;
  const int yz0 = __shfl_sync(0xffffffffu, yz, R.src);
  const int tmin = __reduce_min_sync(0xffffffffu, valid ? tc : INT_MAX);
  const int tmax = __reduce_max_sync(0xffffffffu, valid ? tc : INT_MIN);
  R.uniform = __all_sync(0xffffffffu, !valid || yz == yz0) && tmax - tmin <= max_span;
  if (!R.uniform) return R;
  int a = tmin, b = tmax, wl = -1, wr = -1;
  if (!g.colmap) {
    if (tmin > 0) a = tmin - 1; else wl = nc - 1;
    if (tmax + 1 < nc) b = tmax + 1; else wr = 0;
  } else {
    // table columns tmin..tmax must be adjacent columns of the box
    const int k = tmin + lane;
    const bool gap = k < tmax && g.cols[k + 1] != (g.cols[k] + 1) % nc;
    if (__any_sync(0xffffffffu, gap)) {
      R.uniform = false;
      return R;
    }
    if (tmin > 0 && g.cols[tmin - 1] == (g.cols[tmin] + nc - 1) % nc) a = tmin - 1;
    if (tmax + 1 < g.ncols && g.cols[tmax + 1] == (g.cols[tmax] + 1) % nc) b = tmax + 1;
  }
  if (lane < 9) {
    const int ccy = yz0 % nc, ccz = yz0 / nc;
    const int zz = wrap_yz(ccz + lane / 3 - 1, nc, R.sz);
    const int yy = wrap_yz(ccy + lane % 3 - 1, nc, R.sy);
    const uint32_t* row = grid_row(g, zz, yy);
    R.lo0 = row[a];
    R.hi0 = row[b + 1];
    if (wl >= 0) { R.lo1 = row[wl]; R.hi1 = row[wl + 1]; R.sx1 = CSO_BOX; }
    if (wr >= 0) { R.lo1 = row[wr]; R.hi1 = row[wr + 1]; R.sx1 = -CSO_BOX; }
  }
  return R;
}

// cost class and in-class rank of every density block
__global__ void __launch_bounds__(DENS_WARPS * 32) k_density_cost(CellGrid g, const int4* __restrict__ spos, int n,
                                                                 const uint8_t* __restrict__ only, int max_span,
                                                                 uint8_t* __restrict__ cls,
                                                                 uint32_t* __restrict__ rank,
                                                                 uint32_t* __restrict__ counts) {
  __shared__ unsigned long long bcost;
  if (threadIdx.x == 0) bcost = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = s < n && (!only || only[s]);
  const int4 p = s < n ? spos[s] : make_int4(0, 0, 0, 0);
  const unsigned vmask = __ballot_sync(0xffffffffu, valid);
  if (vmask) {
    const WarpRows R = warp_rows(g, p, valid, vmask, lane, max_span);
    unsigned long long c;
    if (R.uniform) {
      // candidates the shared walk streams
      c = __reduce_add_sync(0xffffffffu, (R.hi0 - R.lo0) + (R.hi1 - R.lo1));
    } else {
      // lane walks diverge: charge the fullest own cell 27 times
      uint32_t m = 0;
      if (valid) {
        const size_t k = grid_cell(g, cell_coord(p.z, g.nc), cell_coord(p.y, g.nc), grid_col(g, p.x));
        m = g.start[k + 1] - g.start[k];
      }
      c = 27ull * __reduce_max_sync(0xffffffffu, m);
    }
    if (lane == 0) atomicAdd(&bcost, c);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long c = bcost | 1ull;
    const int k = 63 - __clzll(c);
    const int kc = k < DENS_CLASSES - 1 ? k : DENS_CLASSES - 1;
    cls[blockIdx.x] = (uint8_t)kc;
    rank[blockIdx.x] = atomicAdd(&counts[kc], 1u);
  }
}

// order[position] = block, classes in decreasing cost
__global__ void k_density_order(const uint8_t* __restrict__ cls, const uint32_t* __restrict__ rank,
                                const uint32_t* __restrict__ counts, int nb, uint32_t* __restrict__ order) {
  __shared__ uint32_t first[DENS_CLASSES];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int k = DENS_CLASSES - 1; k >= 0; --k) {
      first[k] = acc;
      acc += counts[k];
    }
  }
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) order[first[cls[b]] + rank[b]] = (uint32_t)b;
}

// run r of the shared walk (r = 2 * row + wrapped): [lo, hi) and x shift
__device__ __forceinline__ void run_bounds(const WarpRows& R, int r, uint32_t& lo, uint32_t& hi) {
  lo = __shfl_sync(0xffffffffu, (r & 1) ? R.lo1 : R.lo0, r >> 1);
  hi = __shfl_sync(0xffffffffu, (r & 1) ? R.hi1 : R.hi0, r >> 1);
}

template <bool SMALL>
__global__ void __launch_bounds__(DENS_WARPS * 32, 5) k_density(CellGrid g, const int4* __restrict__ spos, int n,
                                                                 uint32_t b2, int reach, int include_self,
                                                                 long long* __restrict__ sigma,
                                                                 const uint8_t* __restrict__ only,
                                                                 const uint32_t* __restrict__ order, int max_span) {
  __shared__ int4 tile[DENS_WARPS][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int blk = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
  const int s = blk * blockDim.x + threadIdx.x;
  const bool valid = s < n && (!only || only[s]);
  const int4 p = s < n ? spos[s] : make_int4(0, 0, 0, 0);
  const unsigned vmask = __ballot_sync(0xffffffffu, valid);
  if (!vmask) return;
  WarpRows R = warp_rows(g, p, valid, vmask, lane, max_span);
  unsigned long long acc = 0;
  if (R.uniform) {
    // keep the neighbours within reach (the largest e with e^2 < b2) of the
    // warp's x extent in x: a neighbour farther out in x is farther than b
    // from every query of the warp
    const int xmin = __reduce_min_sync(0xffffffffu, valid ? p.x : INT_MAX);
    const int xmax = __reduce_max_sync(0xffffffffu, valid ? p.x : INT_MIN);
    if (lane < 9) {
      // neighbour image x = stored x - shift
      if (R.hi0 - R.lo0 > 16u) x_trim(spos, R.lo0, R.hi0, xmin - reach, xmax + reach);
      if (R.hi1 - R.lo1 > 16u) x_trim(spos, R.lo1, R.hi1, xmin - reach + R.sx1, xmax + reach + R.sx1);
    }
    const int ox = __shfl_sync(0xffffffffu, p.x, R.src), oy = __shfl_sync(0xffffffffu, p.y, R.src),
              oz = __shfl_sync(0xffffffffu, p.z, R.src);
    const int qx = p.x - ox, qy = p.y - oy, qz = p.z - oz;
    const uint32_t P = sq3(qx, qy, qz);
    const int ax = -2 * qx, ay = -2 * qy, az = -2 * qz;
    const int B = (int)(b2 - P);
    int4* tl = tile[w];
#pragma unroll 1
    for (int r = 0; r < 18; ++r) {
      uint32_t lo, hi;
      run_bounds(R, r, lo, hi);
      if (lo >= hi) continue;
      // the neighbour's image nearest the warp: t - shift
      const int bx = ox + ((r & 1) ? __shfl_sync(0xffffffffu, R.sx1, r >> 1) : 0);
      const int by = oy + __shfl_sync(0xffffffffu, R.sy, r >> 1), bz = oz + __shfl_sync(0xffffffffu, R.sz, r >> 1);
      int4 next = lo + lane < hi ? spos[lo + lane] : make_int4(0, 0, 0, 0);
      for (uint32_t t0 = lo; t0 < hi; t0 += 32) {
        {
          const int cx = next.x - bx, cy = next.y - by, cz = next.z - bz;
          tl[lane] = make_int4(cx, cy, cz, (int)sq3(cx, cy, cz));
        }
        __syncwarp();
        const uint32_t t1 = t0 + 32;
        if (t1 + lane < hi) next = spos[t1 + lane];
        const int m = hi - t0 < 32 ? (int)(hi - t0) : 32;
        int k = 0;
        if (SMALL) {
          long long mins = 0;
          for (; k + 4 <= m; k += 4) {
            int part = tmin_dot(tl[k], ax, ay, az, B) + tmin_dot(tl[k + 1], ax, ay, az, B);
            part += tmin_dot(tl[k + 2], ax, ay, az, B) + tmin_dot(tl[k + 3], ax, ay, az, B);
            mins += part;
          }
          for (; k < m; ++k) mins += tmin_dot(tl[k], ax, ay, az, B);
          acc += (unsigned long long)((long long)m * B - mins);
        } else {
          unsigned long long mins = 0;
          const uint32_t uax = (uint32_t)ax, uay = (uint32_t)ay, uaz = (uint32_t)az;
          for (; k + 4 <= m; k += 4) {
            uint32_t part = dmin_dot(tl[k], P, uax, uay, uaz, b2) + dmin_dot(tl[k + 1], P, uax, uay, uaz, b2);
            part += dmin_dot(tl[k + 2], P, uax, uay, uaz, b2) + dmin_dot(tl[k + 3], P, uax, uay, uaz, b2);
            mins += part;
          }
          for (; k < m; ++k) mins += dmin_dot(tl[k], P, uax, uay, uaz, b2);
          acc += (unsigned long long)m * b2 - mins;
        }
        __syncwarp();
      }
    }
  } else if (valid) {
    for_stencil(g, p.x, p.y, p.z, [&](uint32_t t, int xq, int yq, int zq) { acc += kern(spos[t], xq, yq, zq, b2); });
  }
  if (!valid) return;
  if (!include_self) acc -= b2;
  sigma[s] = (long long)acc;
}

// number of ordered pairs j != s with d < b2 (the algorithmic work of the
// density pass; a separate diagnostic launch)
__global__ void __launch_bounds__(256) k_count_pairs(CellGrid g, const int4* __restrict__ spos, int n, uint32_t b2,
                                                     unsigned long long* __restrict__ pairs) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned cnt = 0;
  if (s < n) {
    const int4 p = spos[s];
    for_stencil(g, p.x, p.y, p.z, [&](uint32_t t, int xq, int yq, int zq) { cnt += kern(spos[t], xq, yq, zq, b2) != 0; });
    cnt -= 1;  // the particle itself
  }
  unsigned tot = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0) atomicAdd(pairs, (unsigned long long)tot);
}

// ---------------------------------------------------------------------------
// union-find over sorted indices: parent[x] <= x always, roots are the
// smallest index of their component, hooks go from the larger root to the
// smaller one by compare-and-swap (lock-free; any interleaving ends in the
// same components).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int uf_root(int* parent, int x) {
  int p = parent[x];
  while (p != x) {
    int gp = parent[p];
    if (gp != p) parent[x] = gp;  // halve the path; gp is still an ancestor of x
    x = p;
    p = gp;
  }
  return x;
}

__device__ __forceinline__ void uf_unite(int* parent, int a, int b) {
  a = uf_root(parent, a);
  b = uf_root(parent, b);
  while (a != b) {
    if (a < b) {
      int t = a;
      a = b;
      b = t;
    }
    // hook root a (larger) under b
    int old = atomicCAS(&parent[a], a, b);
    if (old == a) return;
    // a was hooked elsewhere meanwhile: climb and retry
    a = uf_root(parent, old);
    b = uf_root(parent, b);
  }
}

// parent[s] = s for dense particles, -1 for the rest (one load answers both);
// flag[s] = dense, scanned into the positions of the dense list
__global__ void k_fof_init(int* __restrict__ parent, uint32_t* __restrict__ flag, int n,
                           const long long* __restrict__ sigma, long long T_L0) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const bool dense = sigma[s] > T_L0;
  parent[s] = dense ? s : -1;
  flag[s] = dense;
}

// the dense particles in cell order: FoF threads take one each, so a warp
// holds 32 dense particles (consecutive in their cells) instead of 32 slots
// of which only the dense ones work
__global__ void k_dense_list(const uint32_t* __restrict__ pos_in_list, const int* __restrict__ parent, int n,
                             int* __restrict__ didx) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && parent[s] >= 0) didx[pos_in_list[s]] = s;
}

// Pass one (in the spirit of Afforest, Sutton et al. 2018): each dense
// particle tests the W = 32 slots after it in its cell, cyclically, so every
// pair of a cell of up to 33 particles is tested and a big cell is joined by
// a band of links around it.  The band joins almost every dense particle of
// a big cell into one tree; the few it misses are handled one by one later.
//
// A warp whose particles share a cell streams the union of its lanes'
// windows through shared memory; the lane that stages a particle also stages
// its current root (-1 if not dense), so a lane pays a forest update only for
// a link into another tree.  A staged root that has since been hooked
// elsewhere is still a member of its tree, so the test stays correct.
constexpr uint32_t FOF_BAND = 32;

__global__ void __launch_bounds__(256) k_fof_sample(CellGrid g, const int4* __restrict__ spos,
                                                    const int* __restrict__ didx, const uint32_t* __restrict__ nd_ptr,
                                                    uint32_t lfof2, int* __restrict__ parent) {
  __shared__ int4 tile[8][32];
  __shared__ int troot[8][32];
  const int nd = (int)*nd_ptr;
  if ((int)(blockIdx.x * blockDim.x) >= nd) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < nd;
  const unsigned vmask = __ballot_sync(0xffffffffu, valid);
  if (!vmask) return;
  const int s = valid ? didx[i] : -1;
  const int4 p = valid ? spos[s] : make_int4(0, 0, 0, 0);
  const size_t cell = grid_cell(g, cell_coord(p.z, g.nc), cell_coord(p.y, g.nc), grid_col(g, p.x));
  const int src = __ffs(vmask) - 1;
  const size_t cell0 = __shfl_sync(0xffffffffu, cell, src);
  const bool uniform = __all_sync(0xffffffffu, !valid || cell == cell0);
  int rs = valid ? uf_root(parent, s) : -1;
  if (uniform) {
    // cell-relative positions: lane j tests j + 1 .. j + h (mod m)
    const uint32_t c_lo = g.start[cell0], c_hi = g.start[cell0 + 1];
    const uint32_t m = c_hi - c_lo;
    const uint32_t h = m - 1 < FOF_BAND ? m - 1 : FOF_BAND;
    const uint32_t j = valid ? (uint32_t)s - c_lo : 0;
    const uint32_t j_first = __shfl_sync(0xffffffffu, j, src);
    const uint32_t j_last = __shfl_sync(0xffffffffu, j, 31 - __clz(vmask));
    const uint32_t v_end = j_last + h + 1;
    for (uint32_t v0 = j_first + 1; v0 < v_end; v0 += 32) {
      const uint32_t v = v0 + lane;
      int tr = -1;
      if (v < v_end) {
        const uint32_t t = c_lo + (v < m ? v : v - m);  // v < 2m
        tile[w][lane] = spos[t];
        if (parent[t] >= 0) tr = uf_root(parent, (int)t);
      }
      troot[w][lane] = tr;
      __syncwarp();
      const int cnt = v_end - v0 < 32 ? (int)(v_end - v0) : 32;
      if (valid) {
        for (int k = 0; k < cnt; ++k) {
          const int rt = troot[w][k];
          const uint32_t off = v0 + k - j;  // cyclic distance after this lane's slot
          if (rt < 0 || rt == rs || off - 1 >= h) continue;
          const int4 q = tile[w][k];
          const int dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
          const uint32_t d = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
          if (d >= lfof2) continue;
          uf_unite(parent, rs, rt);
          rs = uf_root(parent, rs);
        }
      }
      __syncwarp();
    }
    return;
  }
  if (!valid) return;
  // lanes of several cells: each walks its own band
  const uint32_t c_lo = g.start[cell], m = g.start[cell + 1] - c_lo;
  const uint32_t h = m - 1 < FOF_BAND ? m - 1 : FOF_BAND;
  for (uint32_t o = 1, j = (uint32_t)s - c_lo; o <= h; ++o) {
    const uint32_t v = j + o;
    const uint32_t t = c_lo + (v < m ? v : v - m);
    const int4 q = spos[t];
    const int dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
    const uint32_t d = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
    if (d >= lfof2) continue;
    const int pt = parent[t];
    if (pt < 0 || pt == rs) continue;
    const int rt = uf_root(parent, pt);
    if (rt != rs) {
      uf_unite(parent, rs, rt);
      rs = uf_root(parent, rs);
    }
  }
}

// point every dense particle straight at its current root
__global__ void k_fof_compress(int* __restrict__ parent, int n) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && parent[s] >= 0) parent[s] = uf_root(parent, s);
}

// heads of the cells holding dense particles: position i of the dense list
// starts a cell (the list is in cell order)
__global__ void k_cell_heads(const int4* __restrict__ spos, CellGrid g, const int* __restrict__ didx,
                             const uint32_t* __restrict__ nd_ptr, int n, uint32_t* __restrict__ head) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nd = (int)*nd_ptr;
  uint32_t h = 0;
  if (i < nd) {
    const int4 p = spos[didx[i]];
    const size_t c = grid_cell(g, cell_coord(p.z, g.nc), cell_coord(p.y, g.nc), grid_col(g, p.x));
    if (i == 0) {
      h = 1;
    } else {
      const int4 q = spos[didx[i - 1]];
      h = c != grid_cell(g, cell_coord(q.z, g.nc), cell_coord(q.y, g.nc), grid_col(g, q.x));
    }
  }
  head[i] = h;
}

__global__ void k_cell_list(const uint32_t* __restrict__ head_scan, const int* __restrict__ didx,
                            const uint32_t* __restrict__ nd_ptr, int* __restrict__ clist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int)*nd_ptr) return;
  if (head_scan[i + 1] != head_scan[i]) clist[head_scan[i]] = didx[i];
}

// Every cell that holds dense particles has a main tree: the tree of its
// first dense particle after pass one, kept at slot start[c] of a
// per-particle array (the first slot of every non-empty cell is its own) so
// the summary costs n entries instead of one per cell of the sparse table;
// CELL_EMPTY marks cells without dense particles.  A dense particle outside
// its cell's main tree at that point is a straggler.
constexpr int CELL_EMPTY = -2;

__global__ void k_cell_root_init(int* __restrict__ cell_root, long long n) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) cell_root[c] = CELL_EMPTY;
}

__global__ void k_cell_main(const int4* __restrict__ spos, CellGrid g, const int* __restrict__ clist,
                            const uint32_t* __restrict__ ncl_ptr, const int* __restrict__ parent,
                            int* __restrict__ cell_root, uint2* __restrict__ srange) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int)*ncl_ptr) return;
  const int s0 = clist[i];
  const int4 p = spos[s0];
  const size_t c = grid_cell(g, cell_coord(p.z, g.nc), cell_coord(p.y, g.nc), grid_col(g, p.x));
  cell_root[g.start[c]] = parent[s0];  // a root after compression
  srange[g.start[c]] = make_uint2(0, 0);
}

// srange[start[c]] = the run of cell c in the straggler list (in cell order)
__global__ void k_straggler_ranges(const int4* __restrict__ spos, CellGrid g, const int* __restrict__ slist,
                                   const uint32_t* __restrict__ ns_ptr, uint2* __restrict__ srange) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = (int)*ns_ptr;
  if (i >= ns) return;
  auto cell_of = [&](int s) {
    const int4 p = spos[s];
    return grid_cell(g, cell_coord(p.z, g.nc), cell_coord(p.y, g.nc), grid_col(g, p.x));
  };
  const size_t c = cell_of(slist[i]);
  const uint32_t slot = g.start[c];
  if (i == 0 || cell_of(slist[i - 1]) != c) srange[slot].x = (uint32_t)i;
  if (i == ns - 1 || cell_of(slist[i + 1]) != c) srange[slot].y = (uint32_t)i + 1;
}

__global__ void k_stragglers(const int4* __restrict__ spos, CellGrid g, const int* __restrict__ didx,
                             const uint32_t* __restrict__ nd_ptr, int n, const int* __restrict__ parent,
                             const int* __restrict__ cell_root, uint8_t* __restrict__ strag,
                             uint32_t* __restrict__ sflag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t f = 0;
  if (i < (int)*nd_ptr) {
    const int s = didx[i];
    const int4 p = spos[s];
    const size_t c = grid_cell(g, cell_coord(p.z, g.nc), cell_coord(p.y, g.nc), grid_col(g, p.x));
    f = parent[s] != cell_root[g.start[c]];
    strag[s] = (uint8_t)f;
  }
  sflag[i] = f;
}

// the stragglers in list order (flags scanned in place)
__global__ void k_straggler_list(const uint32_t* __restrict__ sscan, const int* __restrict__ didx,
                                 const uint32_t* __restrict__ nd_ptr, int* __restrict__ slist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int)*nd_ptr) return;
  if (sscan[i + 1] != sscan[i]) slist[sscan[i]] = didx[i];
}

// Pass two, main trees as units: for every cell with dense particles and
// each of its 13 forward neighbours (every adjacent pair of cells once), the
// two main trees are joined if any pair of their members links.  A warp
// holds the cell, 32 slots at a time, streams the neighbour through shared
// memory and stops at the first link, so a pair of dense cells costs one
// tile instead of a test per particle.
__device__ __forceinline__ void fof_cell_pairs(const CellGrid& g, const int4* __restrict__ spos, int s0,
                                               uint32_t lfof2, int lreach, int* __restrict__ parent,
                                               const int* __restrict__ cell_root, const uint8_t* __restrict__ strag,
                                               int4* tile, int* tmain, int4* tileA, int* hit, int lane) {
  const int4 p0 = spos[s0];
  const int nc = g.nc;
  const int cy = cell_coord(p0.y, nc), cz = cell_coord(p0.z, nc), tc = grid_col(g, p0.x);
  const size_t cA = grid_cell(g, cz, cy, tc);
  const uint32_t a_lo = g.start[cA], a_hi = g.start[cA + 1];
  const int crA = cell_root[a_lo];
  const XCells X = x_cells(g, tc);
  // lane r < 13: forward neighbour q = 14 + r, (dz, dy, dx) = (q / 9 - 1, q / 3 % 3 - 1, q % 3 - 1)
  uint32_t b_lo = 0, b_hi = 0;
  int crB = CELL_EMPTY, bsx = 0, bsy = 0, bsz = 0;
  if (lane < 13) {
    const int q = 14 + lane;
    const int dz = q / 9 - 1, dy = q / 3 % 3 - 1, dx = q % 3 - 1;
    int sz, sy;
    const int zz = wrap_yz(cz + dz, nc, sz), yy = wrap_yz(cy + dy, nc, sy);
    const int col = dx < 0 ? (X.a < tc ? X.a : X.wl) : (dx > 0 ? (X.b > tc ? X.b : X.wr) : tc);
    const int sx = dx < 0 ? (X.a < tc ? 0 : CSO_BOX) : (dx > 0 ? (X.b > tc ? 0 : -CSO_BOX) : 0);
    if (col >= 0) {
      const size_t c = grid_cell(g, zz, yy, col);
      b_lo = g.start[c];
      b_hi = g.start[c + 1];
      if (b_lo < b_hi) crB = cell_root[b_lo];
      bsx = sx;
      bsy = sy;
      bsz = sz;
    }
  }
  // every neighbour's tree against ours at once (a stale answer only costs a search)
  const int rootA = uf_root(parent, crA);
  const bool need = crB >= 0 && uf_root(parent, crB) != rootA;
  const uint32_t mA = a_hi - a_lo, mB = b_hi - b_lo;
  const bool small = mA <= 32 && mB <= 32;
  if (mA <= 32 && __any_sync(0xffffffffu, need && small)) {
    // Small pairs together: A's slots staged once, the warp's lanes take
    // (neighbour, slot) pairs of all small neighbours in turn, and every lane
    // tests its neighbour particle against all of A.
    const uint32_t a = a_lo + lane;
    const bool av = a < a_hi && parent[a] >= 0 && !strag[a];
    tileA[lane] = av ? spos[a] : make_int4(0, 0, 0, 0);
    if (lane < 13) hit[lane] = 0;
    const unsigned amask = __ballot_sync(0xffffffffu, av);
    const uint32_t cnt = (need && small) ? mB : 0;
    uint32_t incl = cnt;
    for (int o = 1; o < 16; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 12);
    const uint32_t excl = incl - cnt;
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t gi = base + lane;
      int r = 12;
      for (int q = 11; q >= 0; --q) {
        const uint32_t pr = __shfl_sync(0xffffffffu, incl, q);
        if (gi < pr) r = q;
      }
      const uint32_t bl = __shfl_sync(0xffffffffu, b_lo, r), ex = __shfl_sync(0xffffffffu, excl, r);
      const int sx = __shfl_sync(0xffffffffu, bsx, r), sy = __shfl_sync(0xffffffffu, bsy, r),
                sz = __shfl_sync(0xffffffffu, bsz, r);
      const uint32_t t = bl + (gi - ex);
      if (gi < total && amask && parent[t] >= 0 && !strag[t]) {
        const int4 q = spos[t];
        const int qx = q.x - sx, qy = q.y - sy, qz = q.z - sz;
        for (unsigned m = amask; m; m &= m - 1) {
          const int4 pa = tileA[__ffs(m) - 1];
          const int dx = pa.x - qx, dy = pa.y - qy, dz = pa.z - qz;
          const uint32_t d = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
          if (d < lfof2) {
            hit[r] = 1;
            break;
          }
        }
      }
    }
    __syncwarp();
    if (lane < 13 && hit[lane]) uf_unite(parent, crA, crB);
    __syncwarp();
  }
  // pairs with a big side: the neighbour streamed through shared memory
  for (unsigned todo = __ballot_sync(0xffffffffu, need && !small); todo; todo &= todo - 1) {
    const int r = __ffs(todo) - 1;
    const uint32_t lo = __shfl_sync(0xffffffffu, b_lo, r), hi = __shfl_sync(0xffffffffu, b_hi, r);
    const int cb = __shfl_sync(0xffffffffu, crB, r);
    const int sx = __shfl_sync(0xffffffffu, bsx, r), sy = __shfl_sync(0xffffffffu, bsy, r),
              sz = __shfl_sync(0xffffffffu, bsz, r);
    int same = 0;
    if (lane == 0) same = uf_root(parent, crA) == uf_root(parent, cb);
    if (__shfl_sync(0xffffffffu, same, 0)) continue;
    bool found = false;
    // only our slots within l_FoF in x of the neighbour's x extent can link
    uint32_t ta = a_lo, tb = a_hi;
    if (lane == 0 && tb - ta > 32u) {
      const int bx0 = spos[lo].x - sx, bx1 = spos[hi - 1].x - sx;
      x_trim(spos, ta, tb, bx0 - lreach, bx1 + lreach);
    }
    ta = __shfl_sync(0xffffffffu, ta, 0);
    tb = __shfl_sync(0xffffffffu, tb, 0);
    for (uint32_t a0 = ta; a0 < tb && !found; a0 += 32) {
      const uint32_t a = a0 + lane;
      const bool av = a < tb && parent[a] >= 0 && !strag[a];
      const int4 pa = av ? spos[a] : make_int4(0, 0, 0, 0);
      const int xq = pa.x + sx, yq = pa.y + sy, zq = pa.z + sz;
      if (!__any_sync(0xffffffffu, av)) continue;
      // the neighbour's slots within l_FoF of this tile in x (cells are sorted by x)
      const int xqmin = __reduce_min_sync(0xffffffffu, av ? xq : INT_MAX);
      const int xqmax = __reduce_max_sync(0xffffffffu, av ? xq : INT_MIN);
      uint32_t blo = lo, bhi = hi;
      if (lane == 0 && bhi - blo > 32u) x_trim(spos, blo, bhi, xqmin - lreach, xqmax + lreach);
      blo = __shfl_sync(0xffffffffu, blo, 0);
      bhi = __shfl_sync(0xffffffffu, bhi, 0);
      for (uint32_t b0 = blo; b0 < bhi; b0 += 32) {
        const uint32_t t = b0 + lane;
        const bool tv = t < bhi && parent[t] >= 0 && !strag[t];
        tile[lane] = tv ? spos[t] : make_int4(0, 0, 0, 0);
        tmain[lane] = tv;
        __syncwarp();
        const int m = bhi - b0 < 32 ? (int)(bhi - b0) : 32;
        bool found_here = false;
        if (av) {
          for (int k = 0; k < m; ++k) {
            if (!tmain[k]) continue;
            const int4 qb = tile[k];
            const int dx = xq - qb.x, dy = yq - qb.y, dz = zq - qb.z;
            const uint32_t d = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
            if (d < lfof2) {
              found_here = true;
              break;
            }
          }
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, found_here)) {
          found = true;
          break;
        }
      }
    }
    if (found && lane == 0) uf_unite(parent, crA, cb);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) k_fof_cells(CellGrid g, const int4* __restrict__ spos,
                                                   const int* __restrict__ clist, const uint32_t* __restrict__ ncl_ptr,
                                                   uint32_t lfof2, int lreach, int* __restrict__ parent,
                                                   const int* __restrict__ cell_root,
                                                   const uint8_t* __restrict__ strag) {
  __shared__ int4 tile[8][32];
  __shared__ int4 tileA[8][32];
  __shared__ int tmain[8][32];
  __shared__ int hit[8][16];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ncl = (int)*ncl_ptr;
  for (int wi = blockIdx.x * 8 + w; wi < ncl; wi += gridDim.x * 8)
    fof_cell_pairs(g, spos, clist[wi], lfof2, lreach, parent, cell_root, strag, tile[w], tmain[w], tileA[w], hit[w],
                   lane);
}

// Pass three, the stragglers one by one (a list of them): against every neighbour cell in
// l_FoF reach (its own included), the first link into the cell's main tree
// (skipped when that tree is already the straggler's) and every link to a
// later straggler (each straggler pair once).  Cells out of reach of the
// particle (by its distance to the home cell's faces) are skipped.
__global__ void __launch_bounds__(256) k_fof_stragglers(CellGrid g, const int4* __restrict__ spos,
                                                        const int* __restrict__ didx,
                                                        const uint32_t* __restrict__ nd_ptr, uint32_t lfof2,
                                                        int lreach, int* __restrict__ parent,
                                                        const int* __restrict__ cell_root,
                                                        const uint8_t* __restrict__ strag,
                                                        const uint2* __restrict__ srange) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int)*nd_ptr) return;
  const int s = didx[i];
  const int4 p = spos[s];
  const int nc = g.nc;
  const int cy = cell_coord(p.y, nc), cz = cell_coord(p.z, nc), tc = grid_col(g, p.x);
  const XCells X = x_cells(g, tc);
  const int xcol[3] = {X.a < tc ? X.a : X.wl, tc, X.b > tc ? X.b : X.wr};
  const int xsh[3] = {X.a < tc ? 0 : CSO_BOX, 0, X.b > tc ? 0 : -CSO_BOX};
  const int gx = (p.x + g.x0) & (CSO_BOX - 1), gcx = cell_coord(gx, nc);
  const long long xl = gx - cell_lo(gcx, nc) + 1, xr = cell_lo(gcx + 1, nc) - gx;
  const long long yl = p.y - cell_lo(cy, nc) + 1, yr = cell_lo(cy + 1, nc) - p.y;
  const long long zl = p.z - cell_lo(cz, nc) + 1, zr = cell_lo(cz + 1, nc) - p.z;
  const long long mx[3] = {xl * xl, 0, xr * xr};
  const long long R2 = lfof2;
  int rs = uf_root(parent, s);
  for (int dz = -1; dz <= 1; ++dz) {
    const long long mz = dz < 0 ? zl * zl : (dz > 0 ? zr * zr : 0);
    if (mz >= R2) continue;
    int sz;
    const int zz = wrap_yz(cz + dz, nc, sz);
    for (int dy = -1; dy <= 1; ++dy) {
      const long long my = mz + (dy < 0 ? yl * yl : (dy > 0 ? yr * yr : 0));
      if (my >= R2) continue;
      int sy;
      const int yy = wrap_yz(cy + dy, nc, sy);
      for (int k = 0; k < 3; ++k) {
        if (xcol[k] < 0 || my + mx[k] >= R2) continue;
        const size_t c = grid_cell(g, zz, yy, xcol[k]);
        const uint32_t c_lo = g.start[c], c_hi = g.start[c + 1];
        if (c_lo == c_hi) continue;
        const int cm = cell_root[c_lo];
        if (cm == CELL_EMPTY) continue;
        const int xq = p.x + xsh[k], yq = p.y + sy, zq = p.z + sz;
        // the main tree: the first link joins all of it (only the cell's
        // slots within l_FoF in x can link; cells are sorted by x)
        if (uf_root(parent, cm) != rs) {
          uint32_t t0 = c_lo, t1 = c_hi;
          if (t1 - t0 > 16u) x_trim(spos, t0, t1, xq - lreach, xq + lreach);
          for (uint32_t t = t0; t < t1; ++t) {
            const int pt = parent[t];
            if (pt < 0 || strag[t]) continue;
            const int4 q = spos[t];
            const int ddx = xq - q.x, ddy = yq - q.y, ddz = zq - q.z;
            const uint32_t d = (uint32_t)(ddx * ddx) + (uint32_t)(ddy * ddy) + (uint32_t)(ddz * ddz);
            if (d >= lfof2) continue;
            uf_unite(parent, rs, pt);
            rs = uf_root(parent, rs);
            break;
          }
        }
        // the cell's stragglers after this one, from its run of the list
        const uint2 sr = srange[c_lo];
        for (uint32_t j = sr.x; j < sr.y; ++j) {
          const int t = didx[j];
          if (t <= s) continue;
          const int4 q = spos[t];
          const int ddx = xq - q.x, ddy = yq - q.y, ddz = zq - q.z;
          const uint32_t d = (uint32_t)(ddx * ddx) + (uint32_t)(ddy * ddy) + (uint32_t)(ddz * ddz);
          if (d >= lfof2) continue;
          const int rt = uf_root(parent, t);
          if (rt != rs) {
            uf_unite(parent, rs, rt);
            rs = uf_root(parent, rs);
          }
        }
      }
    }
  }
}

// root of every dense particle (-1 otherwise); smallest id per root
__global__ void k_fof_finish(int* __restrict__ parent, int n, const long long* __restrict__ sigma, long long T_L0,
                             const uint64_t* __restrict__ sid, int* __restrict__ root,
                             unsigned long long* __restrict__ minid) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int r = parent[s] < 0 ? -1 : uf_root(parent, s);
  root[s] = r;
  // smallest id per root: reduce over the lanes that share a root first
  const unsigned peers = __match_any_sync(__activemask(), r);
  unsigned long long v = r >= 0 ? (unsigned long long)sid[s] : ~0ull;
  for (unsigned m = peers; m; m &= m - 1) {
    const unsigned long long o = __shfl_sync(peers, v, __ffs(m) - 1);
    v = o < v ? o : v;
  }
  if (r >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMin(&minid[r], v);
}

}  // namespace

// the largest e >= 0 with e^2 < v (v >= 1): the farthest x offset at which
// a pair can still be closer than sqrt(v)
static int reach_below(long long v) {
  long long e = (long long)sqrt((double)v);
  while (e > 0 && e * e >= v) --e;
  while ((e + 1) * (e + 1) < v) ++e;
  return (int)e;
}

int cells_choose(long long b2, int* nc_out) {
  // largest nc with (2^21 / nc)^2 >= b2: cells at least as wide as b
  double b = sqrt((double)b2);
  long long nc = (long long)floor((double)CSO_BOX / b);
  while (nc > 1 && (long double)CSO_BOX * CSO_BOX < (long double)b2 * nc * nc) --nc;
  while ((long double)CSO_BOX * CSO_BOX >= (long double)b2 * (nc + 1) * (nc + 1)) ++nc;
  if (nc < 128) {
    cso_set_error("kernel radius b = %.0f grid units is too large (cells must be <= 2^14 units, u <= 40960)", b);
    return CSO_ERR_ARG;
  }
  if (nc > CSO_MAX_NC) {
    cso_set_error("kernel radius b = %.0f grid units is too small (more than %d cells per side)", b, CSO_MAX_NC);
    return CSO_ERR_ARG;
  }
  *nc_out = (int)nc;
  return CSO_OK;
}

int cells_check_dense(int nc) {
  if (nc > CSO_MAX_DENSE_NC) {
    cso_set_error("box too fine for one dense cell table (%d cells per side > %d): deliver it as x-slabs", nc,
                  CSO_MAX_DENSE_NC);
    return CSO_ERR_ARG;
  }
  return CSO_OK;
}

int cells_bin(const int32_t* pos, const uint64_t* ids, long long n, const CellGrid& g, uint32_t* start,
              int4* spos, uint64_t* sid, int* bad, Workspace& ws, cudaStream_t st, uint32_t* inv) {
  long long ncell = (long long)g.ncols * g.nc * g.nc;
  size_t mark = ws.off;
  // the cell keys and arrival ranks live in the output spos (16 bytes per
  // particle) until k_cell_place overwrites it; the records (and the slot map
  // when inv is wanted) take workspace
  uint32_t* key = reinterpret_cast<uint32_t*>(spos);
  uint32_t* rank = key + n;
  BinRec* rec = ws.get<BinRec>(n);
  uint32_t* fin = inv ? ws.get<uint32_t>(n) : nullptr;
  if (!rec || (inv && !fin)) {
    cso_set_error("workspace exhausted in binning");
    return CSO_ERR_BUDGET;
  }
  CSO_CUDA(cudaMemsetAsync(start, 0, sizeof(uint32_t) * (ncell + 1), st));
  if (n > 0) {
    k_cell_count<<<CL(cdiv(n, 256)), 256, 0, st>>>(pos, n, g, key, rank, start, bad);
    CSO_CUDA(cudaGetLastError());
  }
  CSO_TRY(scan_u32(start, ncell + 1, nullptr, ws, st));
  if (n > 0) {
    CellGrid gs = g;
    gs.start = start;
    k_cell_scatter<<<CL(cdiv(n, 256)), 256, 0, st>>>(pos, ids, n, gs, key, rank, start, rec, inv);
    k_cell_place<<<CL(cdiv(n, 256)), 256, 0, st>>>(n, rec, spos, sid, fin);
    if (inv) k_cell_inv<<<CL(cdiv(n, 256)), 256, 0, st>>>(n, fin, inv);
    CSO_CUDA(cudaGetLastError());
  }
  ws.off = mark;
  return CSO_OK;
}

// Widest x span of a warp's shared walk for cells of nc per side, and whether
// every staged squared distance stays below 2^29 (the signed form).  A staged
// pair is at most (span + 2) cells apart in x and 2 cells in y and z.
static void density_span(int nc, int* max_span, bool* small) {
  const double side = ceil((double)CSO_BOX / nc);
  int sp = 0;
  for (int s = 2; s >= 0; --s)
    if (((s + 2.0) * (s + 2.0) + 8.0) * side * side < 4294967296.0) {
      sp = s;
      break;
    }
  *max_span = sp;
  *small = ((sp + 2.0) * (sp + 2.0) + 8.0) * side * side < 536870912.0;
}

int cells_density(const CellGrid& g, const int4* spos, int n, uint32_t b2, int include_self, long long* sigma,
                  unsigned long long* pairs, Workspace& ws, cudaStream_t st, const uint8_t* only) {
  if (n <= 0) return CSO_OK;
  const int nb = cdiv(n, DENS_WARPS * 32);
  const size_t mark = ws.off;
  uint32_t* order = ws.get<uint32_t>(nb);
  uint32_t* rank = ws.get<uint32_t>(nb);
  uint32_t* counts = ws.get<uint32_t>(DENS_CLASSES);
  uint8_t* cls = ws.get<uint8_t>(nb);
  if (!order || !rank || !counts || !cls) {
    cso_set_error("workspace exhausted in the density pass");
    return CSO_ERR_BUDGET;
  }
  int max_span;
  bool small;
  density_span(g.nc, &max_span, &small);
  const int reach = reach_below(b2);
  CSO_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * DENS_CLASSES, st));
  k_density_cost<<<CL(nb), DENS_WARPS * 32, 0, st>>>(g, spos, n, only, max_span, cls, rank, counts);
  k_density_order<<<CL(cdiv(nb, 256)), 256, 0, st>>>(cls, rank, counts, nb, order);
  if (small)
    k_density<true><<<CL(nb), DENS_WARPS * 32, 0, st>>>(g, spos, n, b2, reach, include_self, sigma, only, order,
                                                         max_span);
  else
    k_density<false><<<CL(nb), DENS_WARPS * 32, 0, st>>>(g, spos, n, b2, reach, include_self, sigma, only, order,
                                                          max_span);
  if (pairs) k_count_pairs<<<CL(cdiv(n, 256)), 256, 0, st>>>(g, spos, n, b2, pairs);
  CSO_CUDA(cudaGetLastError());
  ws.off = mark;
  return CSO_OK;
}

int cells_fof(const CellGrid& g, const int4* spos, int n, const long long* sigma, long long T_L0, uint32_t lfof2,
              const uint64_t* sid, int* parent, int* root, unsigned long long* minid, int* cell_root,
              Workspace& ws, cudaStream_t st) {
  if (n <= 0) return CSO_OK;
  const size_t mark = ws.off;
  uint32_t* flag = ws.get<uint32_t>((size_t)n + 1);
  int* didx = ws.get<int>(n);
  uint32_t* head = ws.get<uint32_t>((size_t)n + 1);
  int* clist = ws.get<int>(n);
  uint8_t* strag = ws.get<uint8_t>(n);
  uint32_t* sflag = ws.get<uint32_t>((size_t)n + 1);
  int* slist = ws.get<int>(n);
  uint2* srange = ws.get<uint2>(n);
  if (!flag || !didx || !head || !clist || !strag || !sflag || !slist || !srange) {
    cso_set_error("workspace exhausted in the FoF pass");
    return CSO_ERR_BUDGET;
  }
  // the dense list and the cells that hold dense particles; launches over
  // them are sized by n and blocks past the counts (read on the device)
  // return at once
  k_fof_init<<<CL(cdiv(n, 256)), 256, 0, st>>>(parent, flag, n, sigma, T_L0);
  CSO_TRY(scan_u32(flag, n, flag + n, ws, st));
  k_dense_list<<<CL(cdiv(n, 256)), 256, 0, st>>>(flag, parent, n, didx);
  const uint32_t* nd = flag + n;
  k_cell_heads<<<CL(cdiv(n, 256)), 256, 0, st>>>(spos, g, didx, nd, n, head);
  CSO_TRY(scan_u32(head, n, head + n, ws, st));
  k_cell_list<<<CL(cdiv(n, 256)), 256, 0, st>>>(head, didx, nd, clist);
  const uint32_t* ncl = head + n;
  // pass one: bands inside cells; main trees and stragglers
  k_fof_sample<<<CL(cdiv(n, 256)), 256, 0, st>>>(g, spos, didx, nd, lfof2, parent);
  k_fof_compress<<<CL(cdiv(n, 256)), 256, 0, st>>>(parent, n);
  k_cell_root_init<<<CL(cdiv(n, 256)), 256, 0, st>>>(cell_root, n);
  k_cell_main<<<CL(cdiv(n, 256)), 256, 0, st>>>(spos, g, clist, ncl, parent, cell_root, srange);
  k_stragglers<<<CL(cdiv(n, 256)), 256, 0, st>>>(spos, g, didx, nd, n, parent, cell_root, strag, sflag);
  CSO_TRY(scan_u32(sflag, n, sflag + n, ws, st));
  k_straggler_list<<<CL(cdiv(n, 256)), 256, 0, st>>>(sflag, didx, nd, slist);
  k_straggler_ranges<<<CL(cdiv(n, 256)), 256, 0, st>>>(spos, g, slist, sflag + n, srange);
  // pass two: main trees of adjacent cells; pass three: stragglers
  const int lreach = reach_below(lfof2);
  k_fof_cells<<<CL(cso_sm_count() * 8), 256, 0, st>>>(g, spos, clist, ncl, lfof2, lreach, parent, cell_root, strag);
  k_fof_stragglers<<<CL(cdiv(n, 256)), 256, 0, st>>>(g, spos, slist, sflag + n, lfof2, lreach, parent, cell_root, strag,
                                                     srange);
  CSO_CUDA(cudaMemsetAsync(minid, 0xff, sizeof(unsigned long long) * n, st));
  k_fof_finish<<<CL(cdiv(n, 256)), 256, 0, st>>>(parent, n, sigma, T_L0, sid, root, minid);
  CSO_CUDA(cudaGetLastError());
  ws.off = mark;
  return CSO_OK;
}
