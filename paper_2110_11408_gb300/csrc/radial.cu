// Radial statistics of L1 haloes (Table 1: r_XX_L2com, vcirc_max_L2com,
// rvcirc_max_L2com; Sec. 4).
//
// Every member's squared distance to its halo's centre (the grid point
// nearest the L2max centre of mass) is an exact integer, so the statistics are
// order statistics of integers: the members of all haloes are sorted once by
// (halo, d) with the device radix sort, which leaves each halo's distances
// ascending in the halo's own segment.  A block per halo then reads the four
// enclosed-fraction radii by index and finds the circular-velocity peak
// max N(<= r) / r with an exact 128-bit comparison.
#include "radial.cuh"

namespace {

constexpr int RAD_NT = 256;

__device__ __forceinline__ long long min_image(int dx) {
  long long d = dx;
  if (d >= (1ll << 20)) d -= CSO_BOX;
  else if (d < -(1ll << 20)) d += CSO_BOX;
  return d;
}

// centre of halo h: nearest grid point of the L2max com (L1 com without L2
// haloes); cen holds it in stored coordinates (x relative to x0)
__global__ void k_radial_centre(const cso_halo* __restrict__ rows, int H, int x0, int4* __restrict__ cen,
                                cso_radial* __restrict__ out) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  const cso_halo r = rows[h];
  const double* com = r.n_l2 > 0 ? r.l2max_com : r.com;
  int c[3];
  for (int k = 0; k < 3; ++k) {
    c[k] = (int)(llround(com[k]) & (CSO_BOX - 1));
    out[h].centre[k] = c[k];
  }
  cen[h] = make_int4((c[0] - x0) & (CSO_BOX - 1), c[1], c[2], 0);
}

__global__ void k_radial_dist(const int4* __restrict__ epos, const uint32_t* __restrict__ ehal, long long na,
                              const int4* __restrict__ cen, uint64_t* __restrict__ d,
                              unsigned long long* __restrict__ dmax) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (j < na) {
    const int4 q = epos[j];
    const int4 c = cen[ehal[j]];
    const long long dx = min_image(q.x - c.x), dy = min_image(q.y - c.y), dz = min_image(q.z - c.z);
    v = (unsigned long long)(dx * dx + dy * dy + dz * dz);
    d[j] = v;
  }
  unsigned long long best = v;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(dmax, best);
}

__global__ void k_radial_pack(uint64_t* __restrict__ key, const uint32_t* __restrict__ ehal, long long na,
                              int dbits) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < na) key[j] |= (unsigned long long)ehal[j] << dbits;
}

__global__ void k_radial_hi(uint64_t* __restrict__ hi, const uint32_t* __restrict__ ehal, long long na) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < na) hi[j] = ehal[j];
}

// (n_a, d_a) beats (n_b, d_b) when n_a^2 / d_a > n_b^2 / d_b, or the values
// are equal and d_a is smaller; n_b = 0 marks "none yet"
__device__ __forceinline__ bool vbetter(unsigned long long na_, unsigned long long da, unsigned long long nb,
                                        unsigned long long db) {
  if (na_ == 0) return false;
  if (nb == 0) return true;
  const unsigned __int128 l = (unsigned __int128)(na_ * na_) * db;
  const unsigned __int128 r = (unsigned __int128)(nb * nb) * da;
  return l > r || (l == r && da < db);
}

__global__ void __launch_bounds__(RAD_NT) k_radial_stats(const uint64_t* __restrict__ key,
                                                         unsigned long long dmask, const uint32_t* __restrict__ seg,
                                                         double u, cso_radial* __restrict__ out) {
  __shared__ unsigned long long sn[RAD_NT / 32], sd[RAD_NT / 32];
  const int h = blockIdx.x;
  const uint32_t b = seg[h];
  const uint32_t n = seg[h + 1] - b;
  const uint64_t* D = key + b;
  unsigned long long bn = 0, bd = 0;
  for (uint32_t i = threadIdx.x; i < n; i += RAD_NT) {
    const unsigned long long di = D[i] & dmask;
    if (di == 0) continue;
    if (i + 1 < n && (D[i + 1] & dmask) == di) continue;  // N(<= r) takes the whole shell
    if (vbetter(i + 1, di, bn, bd)) {
      bn = i + 1;
      bd = di;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long tn = __shfl_xor_sync(0xffffffffu, bn, o);
    const unsigned long long td = __shfl_xor_sync(0xffffffffu, bd, o);
    if (vbetter(tn, td, bn, bd)) {
      bn = tn;
      bd = td;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sn[w] = bn;
    sd[w] = bd;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int k = 1; k < RAD_NT / 32; ++k)
    if (vbetter(sn[k], sd[k], bn, bd)) {
      bn = sn[k];
      bd = sd[k];
    }
  cso_radial& r = out[h];
  const int pct[4] = {25, 50, 75, 98};
  for (int q = 0; q < 4; ++q) {
    long long m = ((long long)pct[q] * n + 99) / 100;
    if (m < 1) m = 1;
    const unsigned long long dq = n > 0 ? (D[m - 1] & dmask) : 0;
    r.d_q[q] = (int64_t)dq;
    r.r_q[q] = sqrt((double)dq) / u;
  }
  r.vmax_n = (int64_t)bn;
  r.vmax_d2 = (int64_t)bd;
  r.r_vmax = sqrt((double)bd) / u;
  r.vmax = bn > 0 ? sqrt((double)bn / r.r_vmax) : 0.0;
}

// Shrinking-sphere centre, a block per halo: every step is one pass over the
// halo's members (count and summed minimum-image offsets of those inside the
// sphere, reduced over the block in one step), then thread 0 moves the
// centre to the rounded centre of mass and shrinks the radius, or stops.  The
// sums are exact integers, so the reduction order is free.  Haloes of at
// least SS_BIG members (the ones that take many steps over many members) run
// on 1024-thread blocks, the rest on 256-thread blocks; each launch skips the
// other's haloes.
constexpr long long SS_N_MIN = 700;
constexpr long long SS_BIG = 16384;

template <int NT>
__global__ void __launch_bounds__(NT) k_shrink_sphere(const int4* __restrict__ epos, const uint32_t* __restrict__ seg,
                                                      const int4* __restrict__ nuc_pos,
                                                      const uint32_t* __restrict__ hnuc,
                                                      const cso_halo* __restrict__ rows, int x0,
                                                      cso_radial* __restrict__ out) {
  __shared__ long long sh[NT / 32][4];
  __shared__ int sc[3];
  __shared__ long long sR2, sm, siter;
  __shared__ int sgo;
  const int h = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t b = seg[h];
  const long long N = seg[h + 1] - b;
  if ((N >= SS_BIG) != (NT == 1024)) return;
  const long long stop = (N + 99) / 100 > SS_N_MIN ? (N + 99) / 100 : SS_N_MIN;
  if (threadIdx.x == 0) {
    const int4 p = nuc_pos[hnuc[h]];
    sc[0] = p.x;
    sc[1] = p.y;
    sc[2] = p.z;
    sR2 = rows[h].R2;
    siter = 0;
  }
  __syncthreads();
  for (;;) {
    const int cx = sc[0], cy = sc[1], cz = sc[2];
    const long long R2 = sR2;
    long long v[4] = {0, 0, 0, 0};  // count, summed dx, dy, dz
    for (long long j = threadIdx.x; j < N; j += blockDim.x) {
      const int4 q = epos[b + j];
      const long long dx = min_image(q.x - cx), dy = min_image(q.y - cy), dz = min_image(q.z - cz);
      if (dx * dx + dy * dy + dz * dz >= R2) continue;
      v[0] += 1;
      v[1] += dx;
      v[2] += dy;
      v[3] += dz;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
      for (int k = 0; k < 4; ++k) sh[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t[4] = {0, 0, 0, 0};
      for (int x = 0; x < (int)(blockDim.x >> 5); ++x)
        for (int k = 0; k < 4; ++k) t[k] += sh[x][k];
      const long long m = t[0];
      sm = m;
      if (m < stop) {
        sgo = 0;
      } else {
        for (int a = 0; a < 3; ++a) {
          double f = (double)sc[a] + (double)t[a + 1] / (double)m;
          if (f < 0) f += (double)CSO_BOX;
          if (f >= (double)CSO_BOX) f -= (double)CSO_BOX;
          sc[a] = (int)(llround(f) & (CSO_BOX - 1));
        }
        sR2 = R2 * 9025 / 10000;
        ++siter;
        sgo = 1;
      }
    }
    __syncthreads();
    if (!sgo) break;
  }
  if (threadIdx.x == 0) {
    cso_radial& r = out[h];
    r.ss_centre[0] = (sc[0] + x0) & (CSO_BOX - 1);
    r.ss_centre[1] = sc[1];
    r.ss_centre[2] = sc[2];
    r.ss_n = sm;
    r.ss_R2 = sR2;
    r.ss_iter = siter;
  }
}

}  // namespace

int radial_run(const uint32_t* seg, const uint32_t* ehal, const int4* epos, long long na, const cso_halo* rows,
               int H, int x0, double u, const uint32_t* hnuc, const int4* nuc_pos, cso_radial* out, void* pinned,
               Workspace& ws, cudaStream_t st) {
  if (H <= 0) return CSO_OK;
  const size_t mark = ws.off;
  int4* cen = ws.get<int4>(H);
  uint64_t* key = ws.get<uint64_t>(na);
  uint64_t* key2 = ws.get<uint64_t>(na);
  uint32_t* val = ws.get<uint32_t>(na);
  uint32_t* val2 = ws.get<uint32_t>(na);
  unsigned long long* dmax = ws.get<unsigned long long>(1);
  if (!cen || !key || !key2 || !val || !val2 || !dmax) {
    cso_set_error("workspace exhausted in the radial statistics");
    return CSO_ERR_BUDGET;
  }
  k_radial_centre<<<CL(cdiv(H, 256)), 256, 0, st>>>(rows, H, x0, cen, out);
  CSO_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st));
  if (na > 0) {
    k_radial_dist<<<CL(cdiv(na, 256)), 256, 0, st>>>(epos, ehal, na, cen, key, dmax);
    CSO_CUDA(cudaMemsetAsync(val, 0, sizeof(uint32_t) * na, st));
  }
  CSO_CUDA(cudaMemcpyAsync(pinned, dmax, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaStreamSynchronize(st));
  const unsigned long long dm = *(unsigned long long*)pinned;
  const int dbits = bit_length_u64(dm) > 0 ? bit_length_u64(dm) : 1;
  const int hbits = bit_length_u64((unsigned long long)(H - 1));
  const uint64_t* sorted = key;
  unsigned long long dmask = ~0ull;
  if (na > 0) {
    uint32_t* pv = val;
    if (dbits + hbits <= 64) {
      // one 64-bit key: halo above the distance
      k_radial_pack<<<CL(cdiv(na, 256)), 256, 0, st>>>(key, ehal, na, dbits);
      uint64_t* ph = nullptr;
      uint64_t* pl = key;
      CSO_TRY(radix_sort_128(&ph, &pl, &pv, nullptr, key2, val2, na, dbits + hbits, ws, st));
      sorted = pl;
      dmask = dbits == 64 ? ~0ull : ((1ull << dbits) - 1);
    } else {
      uint64_t* hi = ws.get<uint64_t>(na);
      uint64_t* hi2 = ws.get<uint64_t>(na);
      if (!hi || !hi2) {
        cso_set_error("workspace exhausted in the radial statistics");
        return CSO_ERR_BUDGET;
      }
      k_radial_hi<<<CL(cdiv(na, 256)), 256, 0, st>>>(hi, ehal, na);
      uint64_t* ph = hi;
      uint64_t* pl = key;
      CSO_TRY(radix_sort_128(&ph, &pl, &pv, hi2, key2, val2, na, 64 + hbits, ws, st));
      sorted = pl;
    }
  }
  k_radial_stats<<<CL(H), RAD_NT, 0, st>>>(sorted, dmask, seg, u, out);
  k_shrink_sphere<1024><<<CL(H), 1024, 0, st>>>(epos, seg, nuc_pos, hnuc, rows, x0, out);
  k_shrink_sphere<256><<<CL(H), 256, 0, st>>>(epos, seg, nuc_pos, hnuc, rows, x0, out);
  CSO_CUDA(cudaGetLastError());
  ws.off = mark;
  return CSO_OK;
}
