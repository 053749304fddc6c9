// CompaSO levels (Sec. 2.2.2): one thread block per group runs the nucleus
// loop of steps 1-4 over the group's members in key order (Sigma desc, id asc).
//
// Per nucleus:
//   pass A  squared distances d_j of all members to the nucleus;
//   select  R^2 = the smallest member distance d with n(<d)^2 u^6 < K d^3
//           (exact), found without a full sort: a 1024-bin histogram over a
//           window of d (first window binned by the threshold count
//           sqrt(K) d^1.5 / u^3, later windows linearly), the first bin that
//           could hold the answer (its interior count at its largest d) is
//           sorted in shared memory and scanned, or narrowed further when it
//           holds more than 2048 members; small groups are sorted whole;
//   pass B  tentative membership / competitive reassignment (Eq. 3) and
//           eligibility marking.
#include <cooperative_groups.h>
#include <atomic>
#include <float.h>
#include <limits.h>

#include "cells.cuh"
#include "compaso.cuh"

namespace {

constexpr int NB = 1024;      // histogram bins
constexpr int CAP = 2048;     // largest bin resolved by an in-block sort
constexpr int COUNT_N = 512;  // groups whose enclosed counts are counted directly

// ---------------------------------------------------------------------------
// exact predicate n^2 u^6 < K d^3 with K = Km 2^Ke (256-bit integers),
// behind a double-precision filter whose rounding error is far below 1e-12
// ---------------------------------------------------------------------------
struct U256 {
  unsigned long long w[4];
};

__device__ __forceinline__ void u256_mul(U256& a, unsigned long long b) {
  unsigned long long carry = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned long long lo = a.w[i] * b;
    unsigned long long hi = __umul64hi(a.w[i], b);
    lo += carry;
    hi += lo < carry;
    a.w[i] = lo;
    carry = hi;
  }
}

__device__ __forceinline__ void u256_shl(U256& a, int s) {
  while (s >= 64) {
    a.w[3] = a.w[2];
    a.w[2] = a.w[1];
    a.w[1] = a.w[0];
    a.w[0] = 0;
    s -= 64;
  }
  if (s) {
    a.w[3] = (a.w[3] << s) | (a.w[2] >> (64 - s));
    a.w[2] = (a.w[2] << s) | (a.w[1] >> (64 - s));
    a.w[1] = (a.w[1] << s) | (a.w[0] >> (64 - s));
    a.w[0] <<= s;
  }
}

__device__ __forceinline__ bool u256_less(const U256& a, const U256& b) {
  for (int i = 3; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  return false;
}

__device__ __noinline__ bool pred_exact(unsigned long long n, unsigned long long d, const PredConst& c) {
  U256 L = {{n, 0, 0, 0}}, R = {{c.Km, 0, 0, 0}};
  u256_mul(L, n);
#pragma unroll
  for (int i = 0; i < 6; ++i) u256_mul(L, c.u);
  u256_mul(R, d);
  u256_mul(R, d);
  u256_mul(R, d);
  if (c.Ke > 0) u256_shl(R, c.Ke);
  else if (c.Ke < 0) u256_shl(L, -c.Ke);
  return u256_less(L, R);
}

// the enclosed count n inside squared radius d is below the level's density
__device__ __forceinline__ bool pred(unsigned long long n, unsigned long long d, const PredConst& c) {
  double L = (double)n * (double)n * c.u6;
  double dd = (double)d;
  double R = c.K * (dd * dd * dd);
  if (L < R * (1.0 - 1e-12)) return true;
  if (L > R * (1.0 + 1e-12)) return false;
  return pred_exact(n, d, c);
}

// smallest D > dmax with pred(n, D): the enclosed count stays n beyond the
// farthest member (single thread)
__device__ long long exhaust_radius(unsigned long long n, long long dmax, const PredConst& c) {
  unsigned long long lo = (unsigned long long)dmax, hi = lo + 1;
  while (!pred(n, hi, c)) hi *= 2;
  while (hi - lo > 1) {
    unsigned long long mid = lo + (hi - lo) / 2;
    if (pred(n, mid, c)) hi = mid;
    else lo = mid;
  }
  return (long long)hi;
}

__device__ __forceinline__ int mi(int v) {
  if (v >= CSO_HALF) return v - CSO_BOX;
  if (v < -CSO_HALF) return v + CSO_BOX;
  return v;
}

__device__ __forceinline__ long long dist2(int4 a, int4 b) {
  long long dx = mi(a.x - b.x), dy = mi(a.y - b.y), dz = mi(a.z - b.z);
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ unsigned warp_incl(unsigned v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// block exclusive scan (NT threads), returns total
template <int NT>
__device__ unsigned block_scan(unsigned v, unsigned& excl, unsigned* sw) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned inc = warp_incl(v);
  if (lane == 31) sw[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned s = lane < NT / 32 ? sw[lane] : 0;
    unsigned si = warp_incl(s);
    if (lane < NT / 32) sw[lane] = si - s;
    if (lane == 31) sw[32] = si;
  }
  __syncthreads();
  excl = inc - v + sw[w];
  unsigned tot = sw[32];
  __syncthreads();
  return tot;
}

__device__ void bitonic_sort(long long* a, int m) {  // m power of two
  for (int k = 2; k <= m; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          long long x = a[i], y = a[l];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
}

struct SelShared {
  unsigned cnt[NB];
  unsigned clo[NB];
  unsigned long long dmn[NB];
  unsigned long long dmx[NB];
  long long list[CAP];
  unsigned sw[33];
  int best;
  int nlist;
  unsigned long long dmax_all;
};

// In the sorted list s[0..m) with n(<s[0]) = base, the first element whose
// strictly-enclosed count satisfies the predicate; returns its index or m.
__device__ int scan_sorted(const long long* s, int m, unsigned long long base, const PredConst& c, int* best) {
  if (threadIdx.x == 0) *best = m;
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    int f = k;
    while (f > 0 && s[f - 1] == s[k]) --f;
    if (pred(base + (unsigned long long)f, (unsigned long long)s[k], c)) atomicMin(best, k);
  }
  __syncthreads();
  int r = *best;
  __syncthreads();
  return r;
}

__device__ __forceinline__ int pow2_at_least(int m) {
  int p = 1;
  while (p < m) p <<= 1;
  return p;
}

// Bin of distance d in the first window of the select.  Both binnings are
// monotone in d, and the select only prunes with the exact predicate at each
// bin's largest member distance, so both give the same R^2:
//   * threshold-count bins (default): bin = sqrt(K) d^1.5 / u^3 / w with
//     w = n / (nb - 1) members of threshold count per bin;
//   * radial bins (the paper's cell-bounded search, Sec. 2.3.4): bins of
//     width sqrt(3)/3 cell sides in r; a bin is skipped when the members
//     inside it, placed at its outer edge, still meet the threshold.
__device__ __forceinline__ int first_bin(unsigned long long d, const PredConst& c, float scale0, int nb) {
  const float f = (float)d;
  const float g = c.radial ? sqrtf(f) * c.rbin_inv_w : f * sqrtf(f) * scale0;
  return g < (float)(nb - 1) ? (int)g : nb - 1;
}

// R^2 of nucleus pc over the n members at epos[0..n); distances left in ed.
// The bin's smallest and largest distance.  A bound read without the atomic
// can only be stale in the safe direction (the minimum only falls, the
// maximum only rises), so a member that does not beat it is skipped: per bin
// only the few members that move a bound pay a 64-bit shared atomic, not
// every member.
__device__ __forceinline__ void bin_minmax(SelShared& S, int b, unsigned long long d) {
  if (d < *(volatile unsigned long long*)&S.dmn[b]) atomicMin(&S.dmn[b], d);
  if (d > *(volatile unsigned long long*)&S.dmx[b]) atomicMax(&S.dmx[b], d);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  return v;
}

template <int NT>
__device__ long long r_search(const int4* __restrict__ epos, long long* __restrict__ ed, int n, int4 pc,
                              const PredConst& c, SelShared& S, const int small_n, const int cap, const int nb) {
  const int tid = threadIdx.x;
  if (n <= small_n && n <= COUNT_N) {
    // every member's strictly enclosed count, counted directly: n(<d_i) =
    // #{j : d_j < d_i}; R^2 is the smallest d_i whose count satisfies the
    // predicate (2 barriers instead of a sort)
    for (int j = tid; j < n; j += blockDim.x) {
      long long d = dist2(pc, epos[j]);
      ed[j] = d;
      S.list[j] = d;
    }
    if (tid == 0) S.dmax_all = ~0ull;
    __syncthreads();
    unsigned long long best = ~0ull, dmax = 0;
    for (int i = tid; i < n; i += blockDim.x) {
      const long long di = S.list[i];
      unsigned cnt = 0;
      for (int j = 0; j < n; ++j) cnt += S.list[j] < di;
      if (pred(cnt, (unsigned long long)di, c) && (unsigned long long)di < best) best = (unsigned long long)di;
      dmax = (unsigned long long)di > dmax ? (unsigned long long)di : dmax;
    }
    atomicMin(&S.dmax_all, best);
    if (tid == 0) S.dmn[0] = 0;
    __syncthreads();
    atomicMax(&S.dmn[0], dmax);
    __syncthreads();
    long long r = (long long)S.dmax_all;
    const long long far = (long long)S.dmn[0];
    __syncthreads();
    if (S.dmax_all == ~0ull || r < 0) {
      if (tid == 0) S.list[0] = exhaust_radius((unsigned long long)n, far, c);
      __syncthreads();
      r = S.list[0];
      __syncthreads();
    }
    return r;
  }
  if (n <= small_n) {
    for (int j = tid; j < n; j += blockDim.x) {
      long long d = dist2(pc, epos[j]);
      ed[j] = d;
      S.list[j] = d;
    }
    int m = pow2_at_least(n);
    for (int j = n + tid; j < m; j += blockDim.x) S.list[j] = LLONG_MAX;
    __syncthreads();
    bitonic_sort(S.list, m);
    int k = scan_sorted(S.list, n, 0, c, &S.best);
    long long r;
    if (k < n) r = S.list[k];
    else r = S.list[n - 1];  // sentinel: exhaustion below
    __syncthreads();
    if (k >= n) {
      if (tid == 0) S.list[0] = exhaust_radius((unsigned long long)n, r, c);
      __syncthreads();
      r = S.list[0];
      __syncthreads();
    }
    return r;
  }

  // ---- windowed histogram select ----
  // window [wlo, whi] of d; base = members with d < wlo; mode 0 = threshold-count bins
  unsigned long long wlo = 0, whi = ~0ull, base = 0;
  int mode = 0;
  const float scale0 = c.bin_scale0 / (float)((n + nb - 2) / (nb - 1));  // n/(nb-1) members of threshold per bin
  bool first_pass = true;
  while (true) {
    for (int b = tid; b < NB; b += blockDim.x) {
      S.cnt[b] = 0;
      S.dmn[b] = ~0ull;
      S.dmx[b] = 0;
    }
    if (tid == 0 && first_pass) S.dmax_all = 0;
    __syncthreads();
    unsigned long long span = whi - wlo + 1;  // mode 1 only
    unsigned long long dmax = 0;              // this thread's farthest member (first pass)
    for (int j = tid; j < n; j += blockDim.x) {
      unsigned long long d;
      if (first_pass) {
        d = (unsigned long long)dist2(pc, epos[j]);
        ed[j] = (long long)d;
        dmax = d > dmax ? d : dmax;
      } else {
        d = (unsigned long long)ed[j];
      }
      if (d < wlo || d > whi) continue;
      int b;
      if (mode == 0) {
        b = first_bin(d, c, scale0, nb);
      } else {
        b = (int)(((d - wlo) * (unsigned long long)nb) / span);
      }
      atomicAdd(&S.cnt[b], 1u);
      bin_minmax(S, b, d);
    }
    if (first_pass) {
      // one shared atomic per warp (per member it serialised on one address)
      const unsigned long long m = warp_max_u64(dmax);
      if ((tid & 31) == 0) atomicMax(&S.dmax_all, m);
    }
    __syncthreads();
    first_pass = false;
    // interior counts
    {
      constexpr int per = NB / NT;
      unsigned loc[per];
      unsigned s = 0;
#pragma unroll
      for (int q = 0; q < per; ++q) {
        loc[q] = S.cnt[tid * per + q];
        s += loc[q];
      }
      unsigned excl;
      unsigned tot = block_scan<NT>(s, excl, S.sw);
      unsigned run = excl;
#pragma unroll
      for (int q = 0; q < per; ++q) {
        S.clo[tid * per + q] = run;
        run += loc[q];
      }
      if (tid == 0) S.nlist = (int)tot;  // members in the window
      __syncthreads();
    }
    const unsigned in_window = (unsigned)S.nlist;
    int from = 0;
    bool narrowed = false;
    while (true) {
      // first bin >= from that could hold the answer
      if (tid == 0) S.best = NB;
      __syncthreads();
      for (int b = from + tid; b < NB; b += blockDim.x)
        if (S.cnt[b] && pred(base + S.clo[b], S.dmx[b], c)) atomicMin(&S.best, b);
      __syncthreads();
      // read the chosen bin before the barrier: the next window pass rewrites it
      const int b = S.best;
      unsigned long long lo = 0, hi = 0, cb = 0;
      unsigned cntb = 0;
      if (b < NB) {
        lo = S.dmn[b];
        hi = S.dmx[b];
        cb = base + S.clo[b];
        cntb = S.cnt[b];
      }
      __syncthreads();
      if (b == NB) break;  // nothing in this window
      if (lo == hi) {
        // one distinct value: its enclosed count is cb, and the bin test above
        // was the exact predicate at that value
        return (long long)lo;
      }
      if (cntb <= (unsigned)cap) {
        if (tid == 0) S.nlist = 0;
        __syncthreads();
        for (int j = tid; j < n; j += blockDim.x) {
          unsigned long long d = (unsigned long long)ed[j];
          if (d >= lo && d <= hi) S.list[atomicAdd(&S.nlist, 1)] = (long long)d;
        }
        __syncthreads();
        int m = S.nlist;
        int p2 = pow2_at_least(m);
        for (int j = m + tid; j < p2; j += blockDim.x) S.list[j] = LLONG_MAX;
        __syncthreads();
        bitonic_sort(S.list, p2);
        int k = scan_sorted(S.list, m, cb, c, &S.best);
        if (k < m) {
          long long r = S.list[k];
          __syncthreads();
          return r;
        }
        from = b + 1;
        continue;
      }
      // too many members in the bin: narrow the window to it
      wlo = lo;
      whi = hi;
      base = cb;
      mode = 1;
      narrowed = true;
      break;
    }
    if (narrowed) continue;
    // nothing in [wlo, whi]: move past it
    base += in_window;
    if (whi >= S.dmax_all) break;
    wlo = whi + 1;
    whi = S.dmax_all;
    mode = 1;
  }
  long long r = 0;
  if (tid == 0) S.list[0] = exhaust_radius((unsigned long long)n, (long long)S.dmax_all, c);
  __syncthreads();
  r = S.list[0];
  __syncthreads();
  return r;
}

// Step 2's density criterion for cell-sorted particle se of group glabel: no
// particle of the same group within d < b2 comes before it in key order
// (Sigma desc, id asc).  The neighbours are the runs of the 27-cell stencil,
// nine rows (own row first, where a denser neighbour usually sits), each one
// run plus one where the row wraps; rows and end cells that cannot reach
// within b are dropped.
struct PeakRows {
  uint32_t lo0, hi0, lo1, hi1;  // lanes 0-8: row lane's runs (rows in walk order)
  int qx1, qy, qz;              // the query in that row's image
  uint32_t pre;                 // lanes 0-9: neighbours in the rows before this one
};

__device__ __forceinline__ int peak_row_of(int o) { return o == 0 ? 4 : (o <= 4 ? o - 1 : o); }

__device__ PeakRows peak_rows(const LevelArgs& a, int4 p) {
  const int lane = threadIdx.x & 31;
  const CellGrid& g = a.grid;
  const int nc = g.nc;
  const int cy = cell_coord(p.y, nc), cz = cell_coord(p.z, nc);
  const int tc = grid_col(g, p.x);
  const XCells X = x_cells(g, tc);
  PeakRows R{0, 0, 0, 0, p.x, p.y, p.z, 0};
  if (lane < 9) {
    const int r = peak_row_of(lane);
    const int dz = r / 3 - 1, dy = r % 3 - 1;
    const int gx = (p.x + g.x0) & (CSO_BOX - 1), gcx = cell_coord(gx, nc);
    const long long zl = p.z - cell_lo(cz, nc) + 1, zr = cell_lo(cz + 1, nc) - p.z;
    const long long yl = p.y - cell_lo(cy, nc) + 1, yr = cell_lo(cy + 1, nc) - p.y;
    const long long xl = gx - cell_lo(gcx, nc) + 1, xr = cell_lo(gcx + 1, nc) - gx;
    const long long m = (dz < 0 ? zl * zl : (dz > 0 ? zr * zr : 0)) + (dy < 0 ? yl * yl : (dy > 0 ? yr * yr : 0));
    if (m < (long long)a.b2) {
      int sz, sy;
      const int zz = wrap_yz(cz + dz, nc, sz), yy = wrap_yz(cy + dy, nc, sy);
      R.qz += sz;
      R.qy += sy;
      const uint32_t* row = grid_row(g, zz, yy);
      const bool left = m + xl * xl < (long long)a.b2, right = m + xr * xr < (long long)a.b2;
      const int ca = left ? X.a : tc, cb = right ? X.b : tc;
      if (left && X.wl >= 0) { R.lo1 = row[X.wl]; R.hi1 = row[X.wl + 1]; R.qx1 = p.x + CSO_BOX; }
      if (right && X.wr >= 0) { R.lo1 = row[X.wr]; R.hi1 = row[X.wr + 1]; R.qx1 = p.x - CSO_BOX; }
      R.lo0 = row[ca];
      R.hi0 = row[cb + 1];
    }
  }
  // exclusive prefix of the rows' neighbour counts (lane 9 holds the total)
  const uint32_t cnt = lane < 9 ? (R.hi0 - R.lo0) + (R.hi1 - R.lo1) : 0u;
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  R.pre = inc - cnt;
  return R;
}

// One load step of the peak test: neighbours f0 + k * 32 + lane (k < U) of
// the flattened rows; true if any lane found a beater.  Every load of the
// step is issued before any comparison, so a step costs one memory round trip.
constexpr int PEAK_U = 4;
__device__ __forceinline__ bool peak_step(const LevelArgs& a, const PeakRows& R, uint32_t f0, uint32_t total, uint32_t se,
                                          int glabel, int4 p, long long sp, uint64_t idp) {
  const int lane = threadIdx.x & 31;
  int4 q[PEAK_U];
  int lab[PEAK_U];
  long long st[PEAK_U];
  uint32_t tt[PEAK_U];
  int ow[PEAK_U];  // row (walk order) | 16 for the wrapped run
#pragma unroll
  for (int k = 0; k < PEAK_U; ++k) {
    const uint32_t f = f0 + k * 32 + lane;
    // the row holding f: the last o with pre[o] <= f
    int o = 0;
#pragma unroll
    for (int oo = 1; oo < 9; ++oo)
      if (__shfl_sync(0xffffffffu, R.pre, oo) <= f) o = oo;
    const uint32_t r = f - __shfl_sync(0xffffffffu, R.pre, o);
    const uint32_t l0 = __shfl_sync(0xffffffffu, R.lo0, o), n0 = __shfl_sync(0xffffffffu, R.hi0, o) - l0;
    const uint32_t l1 = __shfl_sync(0xffffffffu, R.lo1, o);
    tt[k] = f < total ? (r < n0 ? l0 + r : l1 + (r - n0)) : se;
    ow[k] = o | (r < n0 ? 0 : 16);
    q[k] = a.spos[tt[k]];
    lab[k] = a.slab[tt[k]];
    st[k] = a.ssig[tt[k]];
  }
  bool beat = false;
#pragma unroll
  for (int k = 0; k < PEAK_U; ++k) {
    const int o = ow[k] & 15;
    const int x1 = __shfl_sync(0xffffffffu, R.qx1, o), yq = __shfl_sync(0xffffffffu, R.qy, o),
              zq = __shfl_sync(0xffffffffu, R.qz, o);
    if (tt[k] == se || lab[k] != glabel) continue;  // past the end (tt = se), self, or another group
    const int dx = (ow[k] & 16 ? x1 : p.x) - q[k].x, dy = yq - q[k].y, dz = zq - q[k].z;
    const uint32_t d = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
    if (d < a.b2) beat = beat || st[k] > sp || (st[k] == sp && a.sid[tt[k]] < idp);
  }
  return __any_sync(0xffffffffu, beat);
}

enum : int { PEAK_NO = 0, PEAK_YES = 1, PEAK_OPEN = 2 };

// The test by one warp, at most `steps` load steps: PEAK_NO (a beater was
// found), PEAK_YES (no beater among all neighbours) or PEAK_OPEN (not
// finished; peak_part finishes it with many warps).
__device__ __forceinline__ int warp_peak(const LevelArgs& a, uint32_t se, int glabel, int steps) {
  const int4 p = a.spos[se];
  const long long sp = a.ssig[se];
  const uint64_t idp = a.sid[se];
  const PeakRows R = peak_rows(a, p);
  const uint32_t total = __shfl_sync(0xffffffffu, R.pre, 9);
  for (uint32_t f0 = 0; f0 < total; f0 += 32 * PEAK_U) {
    if (steps-- <= 0) return PEAK_OPEN;
    if (peak_step(a, R, f0, total, se, glabel, p, sp, idp)) return PEAK_NO;
  }
  return PEAK_YES;
}

// Part `part` of `parts` of the test (warps of a block or of a cluster
// share the neighbours step by step): true if this part holds a beater.
__device__ __forceinline__ bool peak_part_beaten(const LevelArgs& a, uint32_t se, int glabel, int part, int parts) {
  const int4 p = a.spos[se];
  const long long sp = a.ssig[se];
  const uint64_t idp = a.sid[se];
  const PeakRows R = peak_rows(a, p);
  const uint32_t total = __shfl_sync(0xffffffffu, R.pre, 9);
  for (uint32_t f0 = (uint32_t)part * 32 * PEAK_U; f0 < total; f0 += (uint32_t)parts * 32 * PEAK_U)
    if (peak_step(a, R, f0, total, se, glabel, p, sp, idp)) return true;
  return false;
}

// load steps a warp spends on a candidate before the test goes to all warps
constexpr int PEAK_STEPS = 4;

__device__ bool warp_is_peak(const LevelArgs& a, uint32_t se, int glabel) {
  return warp_peak(a, se, glabel, INT_MAX) == PEAK_YES;
}

template <int NT>
__device__ void level_block(const LevelArgs& a, const int seg) {
  constexpr int NW = NT / 32;
  __shared__ SelShared S;
  __shared__ int sP;
  __shared__ int list[NT];
  __shared__ int peak_of[NW];
  __shared__ int coop_beat;
  const unsigned base = a.seg_off[seg];
  const int n = (int)(a.seg_off[seg + 1] - base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4* epos = a.epos + base;
  const long long* esig = a.esig + base;
  const uint32_t* egs = a.egs + base;
  int* eslot = a.eslot + base;
  long long* edold = a.edold + base;
  uint8_t* einel = a.einel + base;
  long long* ed = a.ed + base;

  for (int j = tid; j < n; j += blockDim.x) {
    eslot[j] = -1;
    einel[j] = 0;
  }
  // step 4: candidates are the members above the stop level: a prefix in key order
  if (tid == 0) {
    int lo = 0, hi = n;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (esig[mid] > a.T_min) lo = mid + 1;
      else hi = mid;
    }
    sP = lo;
  }
  __syncthreads();
  const int P = sP;
  const int glabel = a.slab[egs[0]];  // every member carries the group's label
  const long long anum2 = (long long)a.alpha_num * a.alpha_num, aden2 = (long long)a.alpha_den * a.alpha_den;
  int nn = 0;
  for (int c0 = 0; c0 < P; c0 += NT) {
    // the eligible candidates of this chunk, in key order
    const int j = c0 + tid;
    const unsigned f = (j < P && !einel[j]) ? 1u : 0u;
    unsigned excl;
    const unsigned m = block_scan<NT>(f, excl, S.sw);
    if (f) list[excl] = j;
    __syncthreads();
    for (int g0 = 0; g0 < (int)m; g0 += NW) {
      // step 2 for up to NW of them at once, one warp each for at most
      // PEAK_STEPS load steps (peak-ness never changes)
      const int k = g0 + warp;
      if (k < (int)m) {
        const int e = list[k];
        const int st = einel[e] ? PEAK_NO : warp_peak(a, egs[e], glabel, PEAK_STEPS);
        if (lane == 0) peak_of[warp] = st;
      }
      __syncthreads();
      const int kmax = min(NW, (int)m - g0);
      for (int kk = 0; kk < kmax; ++kk) {
        const int e = list[g0 + kk];
        // eligibility may have been lost to a nucleus found earlier in this walk
        if (peak_of[kk] == PEAK_NO || einel[e]) continue;
        if (peak_of[kk] == PEAK_OPEN) {
          // a test one warp did not finish: every warp of the block takes a share
          if (tid == 0) coop_beat = 0;
          __syncthreads();
          if (peak_part_beaten(a, egs[e], glabel, warp, NW) && lane == 0) coop_beat = 1;
          __syncthreads();
          const bool beaten = coop_beat != 0;
          __syncthreads();
          if (beaten) continue;
        }
        const int4 pc = epos[e];
        const long long R2 = r_search<NT>(epos, ed, n, pc, a.pc, S, a.small_n, a.cap, a.nb);
        // steps 1 and 3
        for (int jj = tid; jj < n; jj += blockDim.x) {
          long long d = ed[jj];
          if (d >= R2) continue;
          int s = eslot[jj];
          bool take;
          if (s < 0) {
            take = true;
          } else {
            long long R2old = a.nuc_R2[base + s];
            __int128 lhs = (__int128)R2 * edold[jj] * a.roche_den;
            __int128 rhs = (__int128)a.roche_num * R2old * d;
            take = lhs >= rhs;
          }
          if (take) {
            eslot[jj] = nn;
            edold[jj] = d;
          }
          if ((__int128)aden2 * d < (__int128)anum2 * R2) einel[jj] = 1;
        }
        if (tid == 0) {
          a.nuc_member[base + nn] = (uint32_t)e;
          a.nuc_R2[base + nn] = R2;
        }
        ++nn;
        __syncthreads();
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    a.nnuc[seg] = (uint32_t)nn;
    if (a.work && nn) atomicAdd(a.work, (unsigned long long)nn * (unsigned long long)n);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_level(LevelArgs a, const uint32_t* __restrict__ segs) {
  level_block<NT>(a, segs ? (int)segs[blockIdx.x] : (int)blockIdx.x);
}

// ---------------------------------------------------------------------------
// Giant groups: one thread-block cluster of CS CTAs per group.  CTA r owns
// the members [r n / CS, (r + 1) n / CS) for the distance, histogram, gather
// and assignment passes; CTA 0 (the leader) runs the nucleus loop and the
// select decisions and broadcasts them through its shared memory, which the
// other CTAs read (and add their histograms into) over DSMEM.  Every CTA
// passes every cluster barrier, in the same order: all control decisions are
// read from the leader after a barrier.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

constexpr int CL_CS = 8;      // CTAs per cluster (giant groups)
constexpr int CL_HUGE_CS = 16;  // CTAs per cluster for huge groups (non-portable size, where it fits)
constexpr int CL_NT = 1024;   // threads per CTA

enum : int { OP_DONE = 0, OP_HIST = 1, OP_GATHER = 2 };

struct ClusterCtl {
  int op;
  int e;                    // next nucleus (member index) or -1
  int mode;                 // histogram binning of the window
  int P;                    // members above the stop level
  long long R2;
  unsigned long long wlo, whi, base;  // window and members below it
  unsigned long long lo, hi, cb;      // bin to gather and its enclosed count
  int from;                 // next bin to examine after a gather
  int bin;                  // bin being gathered
  unsigned in_window;
  int blo, bn, bend;        // candidate batch of the nucleus walk
  int coop;                 // batch entry whose peak test every warp shares, or -1
  int cbeat;                // that test found a beater
};

struct ClusterGen {  // the leader's resumable walk over eligible candidates
  int list[CL_NT];
  int8_t peak_of[CL_NT];
  int m, pos, c0;
};

// Leader only: refill the candidate list when it is used up (the eligible
// members among the next CL_NT above the stop level, in key order) and
// publish the next batch of up to cs * 32 untested candidates in C.blo /
// C.bn, or C.bend = 1 when none remain.  Every CTA of the cluster then tests
// one candidate of the batch per warp.
__device__ void leader_next_batch(const uint8_t* einel, int P, ClusterGen& G, ClusterCtl& C, SelShared& S, int cs) {
  const int tid = threadIdx.x;
  while (G.pos >= G.m && G.c0 < P) {
    const int j = G.c0 + tid;
    const unsigned f = (j < P && !einel[j]) ? 1u : 0u;
    unsigned excl;
    const unsigned m = block_scan<CL_NT>(f, excl, S.sw);
    if (f) G.list[excl] = j;
    __syncthreads();
    if (tid == 0) {
      G.m = (int)m;
      G.pos = 0;
      G.c0 += CL_NT;
    }
    __syncthreads();
  }
  if (tid == 0) {
    C.bend = G.pos >= G.m;
    C.blo = G.pos;
    C.bn = min(G.m - G.pos, cs * 32);
  }
}

// leader only: decide the next step of the select from bin `from` of the
// merged histogram (S.cnt / S.dmn / S.dmx / S.clo, window in Ctl)
__device__ void leader_decide(ClusterCtl& C, SelShared& S, int from, int nb, int cap, int n, const PredConst& c) {
  const int tid = threadIdx.x;
  if (tid == 0) S.best = NB;
  __syncthreads();
  for (int b = from + tid; b < NB; b += blockDim.x)
    if (S.cnt[b] && pred(C.base + S.clo[b], S.dmx[b], c)) atomicMin(&S.best, b);
  __syncthreads();
  if (tid == 0) {
    const int b = S.best;
    if (b < NB) {
      const unsigned long long lo = S.dmn[b], hi = S.dmx[b], cb = C.base + S.clo[b];
      if (lo == hi) {  // one distinct value: the bin test was the exact predicate
        C.op = OP_DONE;
        C.R2 = (long long)lo;
      } else if (S.cnt[b] <= (unsigned)cap) {
        C.op = OP_GATHER;
        C.lo = lo;
        C.hi = hi;
        C.cb = cb;
        C.bin = b;
      } else {  // narrow the window to the bin
        C.op = OP_HIST;
        C.wlo = lo;
        C.whi = hi;
        C.base = cb;
        C.mode = 1;
      }
    } else {  // nothing in the window: move past it
      C.base += C.in_window;
      if (C.whi >= S.dmax_all) {
        C.op = OP_DONE;
        C.R2 = exhaust_radius((unsigned long long)n, (long long)S.dmax_all, c);
      } else {
        C.op = OP_HIST;
        C.wlo = C.whi + 1;
        C.whi = S.dmax_all;
        C.mode = 1;
      }
    }
  }
  __syncthreads();
}

// R^2 of nucleus pc over the group, computed by the whole cluster.  Every CTA
// builds its histogram (and, for a gather, its list) in its own shared
// memory; after the barrier the leader reads the others' with plain DSMEM
// loads and combines them.
__device__ long long cluster_r_search(cg::cluster_group& cluster, const int4* __restrict__ epos,
                                      long long* __restrict__ ed, int n, int lo_r, int hi_r, int4 pc,
                                      const PredConst& c, SelShared& S, ClusterCtl& C, int cap, int nb) {
  const int tid = threadIdx.x;
  const bool leader = cluster.block_rank() == 0;
  const int cs = (int)cluster.num_blocks();
  ClusterCtl* LC = cluster.map_shared_rank(&C, 0);
  const float scale0 = c.bin_scale0 / (float)((n + nb - 2) / (nb - 1));
  // the first pass: threshold-count bins over every distance
  unsigned long long wlo = 0, whi = ~0ull;
  int mode = 0;
  bool first = true;
  if (leader && tid == 0) {
    C.base = 0;
    C.wlo = 0;
    C.whi = ~0ull;
    C.mode = 0;
  }
  int op = OP_HIST;
  while (true) {
    if (op == OP_HIST) {
      for (int b = tid; b < NB; b += blockDim.x) {
        S.cnt[b] = 0;
        S.dmn[b] = ~0ull;
        S.dmx[b] = 0;
      }
      if (tid == 0 && first) S.dmax_all = 0;
      __syncthreads();
      const unsigned long long span = whi - wlo + 1;
      unsigned long long dmax = 0;  // this thread's farthest member (first pass)
      for (int j = lo_r + tid; j < hi_r; j += blockDim.x) {
        unsigned long long d;
        if (first) {
          d = (unsigned long long)dist2(pc, epos[j]);
          ed[j] = (long long)d;
          dmax = d > dmax ? d : dmax;
        } else {
          d = (unsigned long long)ed[j];
        }
        if (d < wlo || d > whi) continue;
        int b;
        if (mode == 0) {
          b = first_bin(d, c, scale0, nb);
        } else {
          b = (int)(((d - wlo) * (unsigned long long)nb) / span);
        }
        atomicAdd(&S.cnt[b], 1u);
        bin_minmax(S, b, d);
      }
      if (first) {
        const unsigned long long m = warp_max_u64(dmax);
        if ((tid & 31) == 0) atomicMax(&S.dmax_all, m);
      }
      __syncthreads();
      cluster.sync();  // every CTA's histogram of its members is complete
      if (leader) {
        // combine the CTAs' histograms (the leader's own is the first share)
        for (int b = tid; b < NB; b += blockDim.x) {
          unsigned cn = S.cnt[b];
          unsigned long long mn = S.dmn[b], mx = S.dmx[b];
          for (int r = 1; r < cs; ++r) {
            const SelShared* R = cluster.map_shared_rank(&S, r);
            cn += R->cnt[b];
            const unsigned long long a1 = R->dmn[b], a2 = R->dmx[b];
            mn = a1 < mn ? a1 : mn;
            mx = a2 > mx ? a2 : mx;
          }
          S.cnt[b] = cn;
          S.dmn[b] = mn;
          S.dmx[b] = mx;
        }
        if (first && tid == 0) {
          unsigned long long m = S.dmax_all;
          for (int r = 1; r < cs; ++r) {
            const unsigned long long v = cluster.map_shared_rank(&S, r)->dmax_all;
            m = v > m ? v : m;
          }
          S.dmax_all = m;
        }
        __syncthreads();
        constexpr int per = NB / CL_NT;
        unsigned loc[per > 0 ? per : 1];
        unsigned sum = 0;
#pragma unroll
        for (int q = 0; q < per; ++q) {
          loc[q] = S.cnt[tid * per + q];
          sum += loc[q];
        }
        unsigned excl;
        const unsigned tot = block_scan<CL_NT>(sum, excl, S.sw);
        unsigned run = excl;
#pragma unroll
        for (int q = 0; q < per; ++q) {
          S.clo[tid * per + q] = run;
          run += loc[q];
        }
        if (tid == 0) C.in_window = tot;
        __syncthreads();
        leader_decide(C, S, 0, nb, cap, n, c);
      }
      first = false;
    } else {  // OP_GATHER: every CTA lists its members of the bin, the leader collects them
      const unsigned long long glo = LC->lo, ghi = LC->hi;
      if (tid == 0) S.nlist = 0;
      __syncthreads();
      for (int j = lo_r + tid; j < hi_r; j += blockDim.x) {
        const unsigned long long d = (unsigned long long)ed[j];
        if (d >= glo && d <= ghi) S.list[atomicAdd(&S.nlist, 1)] = (long long)d;
      }
      __syncthreads();
      cluster.sync();  // every CTA's list is complete
      if (leader) {
        int off = S.nlist;
        for (int r = 1; r < cs; ++r) {
          const SelShared* R = cluster.map_shared_rank(&S, r);
          const int mr = R->nlist;
          for (int j = tid; j < mr; j += blockDim.x) S.list[off + j] = R->list[j];
          off += mr;
        }
        __syncthreads();
        const int m = off;
        const int p2 = pow2_at_least(m);
        for (int j = m + tid; j < p2; j += blockDim.x) S.list[j] = LLONG_MAX;
        __syncthreads();
        bitonic_sort(S.list, p2);
        const int k = scan_sorted(S.list, m, C.cb, c, &S.best);
        if (k < m) {
          if (tid == 0) {
            C.op = OP_DONE;
            C.R2 = S.list[k];
          }
          __syncthreads();
        } else {
          leader_decide(C, S, C.bin + 1, nb, cap, n, c);
        }
      }
    }
    cluster.sync();  // the leader's decision is published (and it has read everyone's shares)
    op = LC->op;
    if (op == OP_DONE) break;
    wlo = LC->wlo;
    whi = LC->whi;
    mode = LC->mode;
    cluster.sync();  // everyone has read it before the leader writes the next one
  }
  const long long R2 = LC->R2;
  cluster.sync();
  return R2;
}

// Step 2 walk of the cluster tier: the next candidate in key order that is
// eligible and a local peak (member index), or -1.  The leader hands out
// batches; every warp of every CTA peak-tests one candidate for at most
// PEAK_STEPS load steps and stores the state in the leader's shared memory;
// the leader's thread 0 takes the first candidate of the batch still in
// play, and a test no warp finished is finished by every warp of the cluster
// before it is decided (no nucleus is accepted during the walk, so a batch
// is settled in order).  Every CTA passes the same barriers: the exits are
// read from the leader after a barrier.
__device__ __forceinline__ int cluster_walk(const LevelArgs& a, const uint32_t* __restrict__ egs,
                                         const uint8_t* __restrict__ einel, int glabel, SelShared& S,
                                         ClusterCtl& C, ClusterGen& G) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const bool leader = rank == 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cs = (int)cluster.num_blocks();
  ClusterCtl* LC = cluster.map_shared_rank(&C, 0);
  ClusterGen* LG = cluster.map_shared_rank(&G, 0);
  int e = -1;
  while (true) {
    if (leader) leader_next_batch(einel, C.P, G, C, S, cs);
    cluster.sync();  // batch published
    if (LC->bend) break;
    const int blo = LC->blo, bn = LC->bn;
    const int k = blo + rank * 32 + warp;
    if (k < blo + bn) {
      const int ek = LG->list[k];
      const int st = einel[ek] ? PEAK_NO : warp_peak(a, egs[ek], glabel, PEAK_STEPS);
      if (lane == 0) LG->peak_of[k] = (int8_t)st;
    }
    cluster.sync();  // peak states in the leader's shared memory
    int from = blo;
    while (true) {
      // the leader takes the first candidate of the batch still in play: a
      // settled peak is the nucleus; an open test goes to every warp of
      // the cluster first
      if (leader && tid == 0) {
        int kk = from, found = -1, coop = -1;
        for (const int kend = C.blo + C.bn; kk < kend; ++kk) {
          const int ec = G.list[kk];
          if (G.peak_of[kk] == PEAK_NO || einel[ec]) continue;
          if (G.peak_of[kk] == PEAK_OPEN) {
            coop = kk;
            break;
          }
          found = ec;
          ++kk;
          break;
        }
        G.pos = kk;
        C.e = found;
        C.coop = coop;
        C.cbeat = 0;
      }
      cluster.sync();  // walk decision (or the shared test) published
      const int kc = LC->coop;
      if (kc < 0) break;
      if (peak_part_beaten(a, egs[LG->list[kc]], glabel, rank * 32 + warp, cs * 32) && lane == 0)
        atomicExch(&LC->cbeat, 1);
      cluster.sync();  // every share of the shared test done
      if (leader && tid == 0) G.peak_of[kc] = (int8_t)(C.cbeat ? PEAK_NO : PEAK_YES);
      from = kc;
    }
    e = LC->e;
    if (e >= 0) break;
  }
  return e;
}

__device__ void cluster_level(const LevelArgs& a, const int seg, SelShared& S, ClusterCtl& C, ClusterGen& G) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const bool leader = rank == 0;
  const unsigned base = a.seg_off[seg];
  const int n = (int)(a.seg_off[seg + 1] - base);
  const int tid = threadIdx.x;
  const int cs = (int)cluster.num_blocks();
  const int lo_r = (int)((long long)n * rank / cs), hi_r = (int)((long long)n * (rank + 1) / cs);
  const int4* epos = a.epos + base;
  const long long* esig = a.esig + base;
  const uint32_t* egs = a.egs + base;
  int* eslot = a.eslot + base;
  long long* edold = a.edold + base;
  uint8_t* einel = a.einel + base;
  long long* ed = a.ed + base;
  ClusterCtl* LC = cluster.map_shared_rank(&C, 0);

  for (int j = lo_r + tid; j < hi_r; j += blockDim.x) {
    eslot[j] = -1;
    einel[j] = 0;
  }
  if (leader && tid == 0) {
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (esig[mid] > a.T_min) lo = mid + 1;
      else hi = mid;
    }
    C.P = lo;
    G.m = 0;
    G.pos = 0;
    G.c0 = 0;
  }
  ClusterGen* LG = cluster.map_shared_rank(&G, 0);
  const int warp = tid >> 5, lane = tid & 31;
  const int glabel = a.slab[egs[0]];
  const long long anum2 = (long long)a.alpha_num * a.alpha_num, aden2 = (long long)a.alpha_den * a.alpha_den;
  cluster.sync();  // slots and flags initialised everywhere
  int nn = 0;
  while (true) {
    const int e = cluster_walk(a, egs, einel, glabel, S, C, G);
    if (e < 0) break;
    const int4 pc = epos[e];
    const long long R2 = cluster_r_search(cluster, epos, ed, n, lo_r, hi_r, pc, a.pc, S, C, a.cap, a.nb);
    // steps 1 and 3 on this CTA's share of the members
    for (int j = lo_r + tid; j < hi_r; j += blockDim.x) {
      const long long d = ed[j];
      if (d >= R2) continue;
      const int sl = eslot[j];
      bool take;
      if (sl < 0) {
        take = true;
      } else {
        const long long R2old = a.nuc_R2[base + sl];
        take = (__int128)R2 * edold[j] * a.roche_den >= (__int128)a.roche_num * R2old * d;
      }
      if (take) {
        eslot[j] = nn;
        edold[j] = d;
      }
      if ((__int128)aden2 * d < (__int128)anum2 * R2) einel[j] = 1;
    }
    if (leader && tid == 0) {
      a.nuc_member[base + nn] = (uint32_t)e;
      a.nuc_R2[base + nn] = R2;
    }
    ++nn;
    cluster.sync();  // assignments and eligibility visible to the leader's next walk
  }
  if (leader && tid == 0) {
    a.nnuc[seg] = (uint32_t)nn;
    if (a.work && nn) atomicAdd(a.work, (unsigned long long)nn * (unsigned long long)n);
  }
  // no CTA may exit while another can still read its shared memory (the last
  // read of the leader's C.e happens after the final barrier of the loop)
  cluster.sync();
}

// ---------------------------------------------------------------------------
// The batched schedule's work queue: the groups sorted by size (largest
// first) and cut into four size bins on the device -- giants, large, medium
// and small -- with one fetch counter per bin.  Four persistent kernels pull
// from it concurrently: 8-CTA clusters take giants, 1024-thread blocks large
// groups, 256-thread blocks medium ones and warps the small ones, each taking
// the next group of its bin when it finishes one, so no launch size depends
// on a count read back by the host.
// ---------------------------------------------------------------------------
struct TierQueue {
  unsigned count[4];  // giant (huge included), large, small, huge (from k_seg_sizes)
  unsigned next[5];   // fetch counters: giant, large, medium, small, huge
  unsigned nseg;
};

// first index in the size-sorted order and count of bin t
__device__ __forceinline__ void tier_range(const TierQueue& q, int t, unsigned& first, unsigned& cnt) {
  const unsigned ng = q.count[0], nl = q.count[1], ns = q.count[2], nh = q.count[3];
  const unsigned nm = q.nseg - ng - nl - ns;
  if (t == 4) { first = 0; cnt = nh; }
  else if (t == 0) { first = nh; cnt = ng - nh; }
  else if (t == 1) { first = ng; cnt = nl; }
  else if (t == 2) { first = ng + nl; cnt = nm; }
  else { first = q.nseg - ns; cnt = ns; }
}

// tier 0 (giants) on 8-CTA clusters, tier 4 (huge groups) on 16-CTA clusters
template <int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(CL_NT)
    k_level_cluster_q(LevelArgs a, const uint32_t* __restrict__ order, TierQueue* q, int tier) {
  __shared__ SelShared S;
  __shared__ ClusterCtl C;
  __shared__ ClusterGen G;
  __shared__ unsigned item;
  cg::cluster_group cluster = cg::this_cluster();
  const bool leader = cluster.block_rank() == 0;
  unsigned first, cnt;
  tier_range(*q, tier, first, cnt);
  for (;;) {
    if (leader && threadIdx.x == 0) item = atomicAdd(&q->next[tier], 1u);
    cluster.sync();
    const unsigned it = *cluster.map_shared_rank(&item, 0);
    cluster.sync();  // every CTA has read the leader's item before it changes
    if (it >= cnt) return;
    cluster_level(a, (int)order[first + it], S, C, G);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_level_q(LevelArgs a, const uint32_t* __restrict__ order, TierQueue* q,
                                                int tier) {
  __shared__ unsigned item;
  unsigned first, cnt;
  tier_range(*q, tier, first, cnt);
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(&q->next[tier], 1u);
    __syncthreads();
    const unsigned it = item;
    __syncthreads();
    if (it >= cnt) return;
    level_block<NT>(a, (int)order[first + it]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// One small group (n <= 64 members) per warp.  Members live in registers
// (lane l holds members l and l + 32).  The enclosed count n(<d_i) of every
// member is counted directly over all members (n^2 compares), so R^2 =
// min{d_i : pred(n(<d_i), d_i)} needs no sort.
// ---------------------------------------------------------------------------
constexpr long long D_INF = LLONG_MAX;

__device__ __forceinline__ long long warp_min_ll(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t < v ? t : v;
  }
  return v;
}

__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  return v;
}

__device__ void level_warp(const LevelArgs& a, const int seg) {
  const int lane = threadIdx.x & 31;
  const unsigned base = a.seg_off[seg];
  const int n = (int)(a.seg_off[seg + 1] - base);
  const bool v0 = lane < n, v1 = lane + 32 < n;
  const int4 p0 = v0 ? a.epos[base + lane] : make_int4(0, 0, 0, 0);
  const int4 p1 = v1 ? a.epos[base + lane + 32] : make_int4(0, 0, 0, 0);
  const long long s0 = v0 ? a.esig[base + lane] : LLONG_MIN;
  const long long s1 = v1 ? a.esig[base + lane + 32] : LLONG_MIN;
  const uint32_t g0 = v0 ? a.egs[base + lane] : 0, g1 = v1 ? a.egs[base + lane + 32] : 0;
  int slot0 = -1, slot1 = -1;
  bool in0 = false, in1 = false;
  long long do0 = 0, do1 = 0;
  // step 4: the members above the stop level form a prefix in key order
  const int P = __popc(__ballot_sync(0xffffffffu, s0 > a.T_min)) + __popc(__ballot_sync(0xffffffffu, s1 > a.T_min));
  const int glabel = a.slab[__shfl_sync(0xffffffffu, g0, 0)];
  const long long anum2 = (long long)a.alpha_num * a.alpha_num, aden2 = (long long)a.alpha_den * a.alpha_den;
  int nn = 0;
  for (int c = 0; c < P; ++c) {
    const int src = c & 31;
    const bool hi = c >= 32;
    const bool inel = __shfl_sync(0xffffffffu, hi ? in1 : in0, src);
    if (inel) continue;
    const uint32_t se = __shfl_sync(0xffffffffu, hi ? g1 : g0, src);
    if (!warp_is_peak(a, se, glabel)) continue;
    int4 pc;
    pc.x = __shfl_sync(0xffffffffu, hi ? p1.x : p0.x, src);
    pc.y = __shfl_sync(0xffffffffu, hi ? p1.y : p0.y, src);
    pc.z = __shfl_sync(0xffffffffu, hi ? p1.z : p0.z, src);
    const long long d0 = v0 ? dist2(pc, p0) : D_INF, d1 = v1 ? dist2(pc, p1) : D_INF;
    // strictly enclosed counts
    unsigned k0 = 0, k1 = 0;
    for (int j = 0; j < n; ++j) {
      const long long dj = __shfl_sync(0xffffffffu, j >= 32 ? d1 : d0, j & 31);
      k0 += dj < d0;
      k1 += dj < d1;
    }
    const bool ok0 = v0 && pred(k0, (unsigned long long)d0, a.pc);
    const bool ok1 = v1 && pred(k1, (unsigned long long)d1, a.pc);
    long long R2 = warp_min_ll(min(ok0 ? d0 : D_INF, ok1 ? d1 : D_INF));
    if (R2 == D_INF) {
      const long long dmax = warp_max_ll(max(v0 ? d0 : 0ll, v1 ? d1 : 0ll));
      long long r = 0;
      if (lane == 0) r = exhaust_radius((unsigned long long)n, dmax, a.pc);
      R2 = __shfl_sync(0xffffffffu, r, 0);
    }
    // steps 1 and 3 on the two members of this lane
    if (v0 && d0 < R2) {
      bool take = slot0 < 0;
      if (!take) {
        const long long R2old = a.nuc_R2[base + slot0];
        take = (__int128)R2 * do0 * a.roche_den >= (__int128)a.roche_num * R2old * d0;
      }
      if (take) {
        slot0 = nn;
        do0 = d0;
      }
      if ((__int128)aden2 * d0 < (__int128)anum2 * R2) in0 = true;
    }
    if (v1 && d1 < R2) {
      bool take = slot1 < 0;
      if (!take) {
        const long long R2old = a.nuc_R2[base + slot1];
        take = (__int128)R2 * do1 * a.roche_den >= (__int128)a.roche_num * R2old * d1;
      }
      if (take) {
        slot1 = nn;
        do1 = d1;
      }
      if ((__int128)aden2 * d1 < (__int128)anum2 * R2) in1 = true;
    }
    if (lane == 0) {
      a.nuc_member[base + nn] = (uint32_t)c;
      a.nuc_R2[base + nn] = R2;
    }
    __syncwarp();
    ++nn;
  }
  if (v0) a.eslot[base + lane] = slot0;
  if (v1) a.eslot[base + lane + 32] = slot1;
  if (lane == 0) {
    a.nnuc[seg] = (uint32_t)nn;
    if (a.work && nn) atomicAdd(a.work, (unsigned long long)nn * (unsigned long long)n);
  }
}

__global__ void __launch_bounds__(256) k_level_warp_q(LevelArgs a, const uint32_t* __restrict__ order, TierQueue* q) {
  unsigned first, cnt;
  tier_range(*q, 3, first, cnt);
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(&q->next[3], 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= cnt) return;  // whole warps leave together
    level_warp(a, (int)order[first + it]);
  }
}

// segment sizes as descending sort keys, and the size-bin counts
__global__ void k_seg_sizes(const uint32_t* __restrict__ seg_off, int nseg, int huge, int giant, int large, int small,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ val, unsigned* __restrict__ counts,
                            unsigned* __restrict__ nseg_out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) *nseg_out = (unsigned)nseg;
  if (g >= nseg) return;
  const uint32_t sz = seg_off[g + 1] - seg_off[g];
  key[g] = 0xffffffffu - sz;
  val[g] = (uint32_t)g;
  if (sz > (uint32_t)huge) atomicAdd(&counts[3], 1u);
  if (sz > (uint32_t)giant) atomicAdd(&counts[0], 1u);
  else if (sz > (uint32_t)large) atomicAdd(&counts[1], 1u);
  else if (sz <= (uint32_t)small) atomicAdd(&counts[2], 1u);
}

// largest g with off[g] <= k (off ascending, off[0] = 0)
__device__ __forceinline__ int seg_of(const uint32_t* __restrict__ off, int nseg, unsigned k) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// global halo index of every member (or -1): one thread per member
__global__ void k_level_halo_members(const uint32_t* __restrict__ seg_off, int nseg, const uint32_t* __restrict__ hbase,
                                     const int* __restrict__ eslot, int* __restrict__ ehalo) {
  const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= seg_off[nseg]) return;
  const int s = eslot[j];
  ehalo[j] = s < 0 ? -1 : (int)(hbase[seg_of(seg_off, nseg, j)] + s);
}

// per-halo nucleus records: one thread per halo (halos of segment g start at
// hbase[g])
__global__ void k_level_halo_nuclei(const uint32_t* __restrict__ seg_off, int nseg, const uint32_t* __restrict__ hbase,
                                    const uint32_t* __restrict__ nuc_member, const long long* __restrict__ nuc_R2,
                                    uint32_t* __restrict__ hnuc, long long* __restrict__ hR2,
                                    uint32_t* __restrict__ hseg) {
  const unsigned h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= hbase[nseg]) return;
  const int g = seg_of(hbase, nseg, h);  // hbase ascending; segments without nuclei repeat a value
  const unsigned base = seg_off[g], q = h - hbase[g];
  hnuc[h] = base + nuc_member[base + q];
  hR2[h] = nuc_R2[base + q];
  hseg[h] = (uint32_t)g;
}

}  // namespace

// resident blocks per SM of the persistent level kernels (same for every
// device of one build; queried once)
static std::atomic<int> g_occ_l{0}, g_occ_m{0}, g_occ_w{0};
// 16-CTA clusters that can be resident at once (0: that size does not fit
// this device, and huge groups stay on 8-CTA clusters)
static std::atomic<int> g_cl16{0};

void level_prepare() {
  if (g_occ_l.load()) return;
  int l = 0, m = 0, w = 0;
  int c16 = 0;
  if (cudaFuncSetAttribute(k_level_cluster_q<CL_HUGE_CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
      cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL_HUGE_CS, 1, 1);
    cfg.blockDim = dim3(CL_NT, 1, 1);
    if (cudaOccupancyMaxActiveClusters(&c16, k_level_cluster_q<CL_HUGE_CS>, &cfg) != cudaSuccess) c16 = 0;
  }
  cudaGetLastError();  // an unsupported size leaves only the answer 0
  g_cl16.store(c16 > 0 ? c16 : 0);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l, k_level_q<1024>, 1024, 0) != cudaSuccess || l < 1) l = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_level_q<256>, 256, 0) != cudaSuccess || m < 1) m = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&w, k_level_warp_q, 256, 0) != cudaSuccess || w < 1) w = 1;
  g_occ_m.store(m);
  g_occ_w.store(w);
  g_occ_l.store(l);
  cso_sm_count();
}

int level_run(const LevelArgs& a, cudaStream_t st) {
  if (a.nseg <= 0) return CSO_OK;
  k_level<256><<<CL(a.nseg), 256, 0, st>>>(a, nullptr);
  CSO_CUDA(cudaGetLastError());
  return CSO_OK;
}

int level_run_batched(const LevelArgs& a, const LevelSchedule& sc, Workspace& ws, cudaStream_t st,
                      cudaStream_t side, cudaStream_t side2, cudaStream_t side3, cudaEvent_t fork,
                      cudaEvent_t join, cudaEvent_t join2, cudaEvent_t join3, unsigned* host_counts) {
  (void)host_counts;
  if (a.nseg <= 0) return CSO_OK;
  size_t mark = ws.off;
  uint32_t* key = ws.get<uint32_t>(a.nseg);
  uint32_t* val = ws.get<uint32_t>(a.nseg);
  uint32_t* key2 = ws.get<uint32_t>(a.nseg);
  uint32_t* val2 = ws.get<uint32_t>(a.nseg);
  TierQueue* q = ws.get<TierQueue>(1);
  if (!key || !val || !key2 || !val2 || !q) {
    cso_set_error("workspace exhausted in the batched schedule");
    return CSO_ERR_BUDGET;
  }
  CSO_CUDA(cudaMemsetAsync(q, 0, sizeof(TierQueue), st));
  level_prepare();
  const int c16 = g_cl16;
  // groups above the huge bound (and the giant bound) run on 16-CTA clusters
  // where the device holds them
  const int huge = c16 > 0 ? std::max(sc.giant, sc.huge) : INT_MAX;
  k_seg_sizes<<<CL(cdiv(a.nseg, 256)), 256, 0, st>>>(a.seg_off, a.nseg, huge, sc.giant, sc.large(), sc.small, key,
                                                     val, q->count, &q->nseg);
  // largest groups first: giants start at once, the rest fill in behind them
  uint32_t *pk = key, *pv = val;
  CSO_TRY(radix_sort_32(&pk, &pv, key2, val2, a.nseg, 32, ws, st));
  CSO_CUDA(cudaGetLastError());
  // persistent grids sized to the device; blocks of a bin leave when its
  // queue is empty
  const int occ_l = g_occ_l, occ_m = g_occ_m, occ_w = g_occ_w;
  const int sms = cso_sm_count();
  const int n_clusters = sms / CL_CS > 0 ? sms / CL_CS : 1;
  const int nseg = a.nseg;
  // no bin can hold more groups than there are: grids never exceed nseg
  auto cap = [nseg](long long g) { return (unsigned)(g < nseg ? g : nseg); };
  CSO_CUDA(cudaEventRecord(fork, st));
  CSO_CUDA(cudaStreamWaitEvent(side, fork, 0));
  k_level_cluster_q<CL_CS><<<CL(cap(n_clusters) * CL_CS), CL_NT, 0, side>>>(a, pv, q, 0);
  CSO_CUDA(cudaGetLastError());
  if (c16 > 0) {
    // at most two: huge groups are few, and every 16-CTA cluster holds 16 SMs
    CSO_CUDA(cudaStreamWaitEvent(side3, fork, 0));
    k_level_cluster_q<CL_HUGE_CS><<<CL(cap(c16 < 2 ? c16 : 2) * CL_HUGE_CS), CL_NT, 0, side3>>>(a, pv, q, 4);
    CSO_CUDA(cudaGetLastError());
  }
  CSO_CUDA(cudaStreamWaitEvent(side2, fork, 0));
  k_level_q<1024><<<CL(cap((long long)sms * occ_l)), 1024, 0, side2>>>(a, pv, q, 1);
  k_level_q<256><<<CL(cap((long long)sms * occ_m)), 256, 0, st>>>(a, pv, q, 2);
  k_level_warp_q<<<CL(cdiv(cap((long long)sms * occ_w * 8), 8)), 256, 0, st>>>(a, pv, q);
  CSO_CUDA(cudaGetLastError());
  CSO_CUDA(cudaEventRecord(join, side));
  CSO_CUDA(cudaStreamWaitEvent(st, join, 0));
  CSO_CUDA(cudaEventRecord(join2, side2));
  CSO_CUDA(cudaStreamWaitEvent(st, join2, 0));
  if (c16 > 0) {
    CSO_CUDA(cudaEventRecord(join3, side3));
    CSO_CUDA(cudaStreamWaitEvent(st, join3, 0));
  }
  ws.off = mark;
  return CSO_OK;
}

int level_halo(int nseg, const uint32_t* seg_off, const uint32_t* nnuc, const uint32_t* hbase, const int* eslot,
               const uint32_t* nuc_member, const long long* nuc_R2, int* ehalo, uint32_t* hnuc, long long* hR2,
               uint32_t* hseg, long long n_members, long long n_halos, cudaStream_t st) {
  (void)nnuc;
  if (nseg <= 0) return CSO_OK;
  if (n_members > 0)
    k_level_halo_members<<<CL(cdiv(n_members, 256)), 256, 0, st>>>(seg_off, nseg, hbase, eslot, ehalo);
  if (n_halos > 0)
    k_level_halo_nuclei<<<CL(cdiv(n_halos, 256)), 256, 0, st>>>(seg_off, nseg, hbase, nuc_member, nuc_R2, hnuc, hR2,
                                                                hseg);
  CSO_CUDA(cudaGetLastError());
  return CSO_OK;
}

PredConst make_pred_const(double K, long long u) {
  PredConst c{};  // zeroed padding: level stages are cached by their argument bytes
  c.K = K;
  int E;
  double f = frexp(K, &E);
  c.Km = (unsigned long long)ldexp(f, 53);
  c.Ke = E - 53;
  c.u = (unsigned long long)u;
  double ud = (double)u;
  c.u6 = ud * ud * ud * ud * ud * ud;
  // bin of the first window: threshold count sqrt(K) d^1.5 / u^3 (before /w)
  c.bin_scale0 = (float)(sqrt(K) / (ud * ud * ud));
  c.radial = 0;
  c.rbin_inv_w = 0.0f;
  return c;
}
