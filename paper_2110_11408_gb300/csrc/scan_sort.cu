// Device-wide exclusive scan (single pass, decoupled look-back) and stable
// LSD radix sorts (8-bit digits).
//
// Both sorts rank elements inside a tile with warp-level matching
// (__match_any_sync): warp w owns a contiguous run of the tile and keeps a
// running per-digit counter in shared memory, so ranks are stable; per-warp
// counts are then prefixed across warps.  Keys of up to 64 bits go through
// the one-sweep sort (one kernel per digit, tile offsets by look-back); keys
// wider than 64 bits (two words) through a histogram / scan / scatter
// sequence per digit whose tile offsets come from the scanned [digit][tile]
// histogram.
#include <algorithm>

#include "cso_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* smem_warp, uint32_t& excl) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) smem_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < nw ? smem_warp[lane] : 0;
    uint32_t si = warp_incl_scan(s);
    if (lane < nw) smem_warp[lane] = si - s;
    if (lane == 31) smem_warp[32] = si;
  }
  __syncthreads();
  excl = inc - v + smem_warp[w];
  uint32_t total = smem_warp[32];
  __syncthreads();
  return total;
}

// Single-pass exclusive scan with decoupled look-back (Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).  Tiles
// take their index from an atomic counter in the order they start, so every
// predecessor of a tile is already running; each tile publishes its aggregate
// (flag A), then warp 0 walks back over 32 predecessors at a time, adding
// aggregates until it meets an inclusive prefix (flag P), and publishes its
// own inclusive prefix.  A status word is flag << 32 | value.
constexpr int SP_THREADS = 256;
// values per thread: 16 (tiles of 4,096), or 32 for arrays of more than
// SP_BIG values (half the tiles and look-backs, twice the loads in flight)
constexpr long long SP_BIG = 1ll << 22;
constexpr unsigned long long SP_A = 1ull << 32, SP_P = 2ull << 32;
constexpr long long SP_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ unsigned long long sp_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void sp_store(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// status[0 .. ntiles) and the tile counter status[ntiles] start at zero
template <int SP_ITEMS>
__global__ void __launch_bounds__(SP_THREADS) k_scan_onepass(uint32_t* __restrict__ d, long long n,
                                                             unsigned long long* __restrict__ status, long long ntiles,
                                                             uint32_t* __restrict__ total, int* __restrict__ err) {
  constexpr int SP_TILE = SP_THREADS * SP_ITEMS;
  constexpr int R = SP_ITEMS / 4;  // rounds of four consecutive values per lane
  __shared__ uint32_t sw[33];
  __shared__ long long tile_sh;
  __shared__ uint32_t prefix_sh;
  if (threadIdx.x == 0) tile_sh = (long long)atomicAdd(&status[ntiles], 1ull);
  __syncthreads();
  const long long tile = tile_sh;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // warp w holds a contiguous run of the tile; in round q its lanes hold 32
  // consecutive groups of four values, so every load moves 512 contiguous bytes
  const long long wb = tile * SP_TILE + (long long)w * 32 * SP_ITEMS;
  const bool vec = wb + 32 * SP_ITEMS <= n && ((reinterpret_cast<uintptr_t>(d) & 15) == 0);
  uint4 v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const long long i = wb + ((long long)q * 32 + lane) * 4;
    if (vec) {
      v[q] = *reinterpret_cast<const uint4*>(d + i);
    } else {
      v[q].x = i < n ? d[i] : 0u;
      v[q].y = i + 1 < n ? d[i + 1] : 0u;
      v[q].z = i + 2 < n ? d[i + 2] : 0u;
      v[q].w = i + 3 < n ? d[i + 3] : 0u;
    }
  }
  // each round's exclusive prefix within the warp's run
  uint32_t base[R];
  uint32_t carry = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const uint32_t sq = v[q].x + v[q].y + v[q].z + v[q].w;
    const uint32_t inc = warp_incl_scan(sq);
    base[q] = carry + inc - sq;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  // the warps' runs in order: lane 0 carries its warp's total into the block scan
  uint32_t excl;
  const uint32_t agg = block_excl_scan(lane == 0 ? carry : 0u, sw, excl);
  const uint32_t woff = __shfl_sync(0xffffffffu, excl, 0);
  if (threadIdx.x < 32) {
    uint32_t prefix = 0;
    if (tile > 0) {
      if (lane == 0) sp_store(&status[tile], SP_A | agg);
      long long top = tile - 1;
      long long spins = 0;
      for (;;) {
        const long long j = top - lane;
        const unsigned long long wv = j >= 0 ? sp_load(&status[j]) : SP_P;  // before tile 0: prefix 0
        const unsigned long long flag = wv & ~0xffffffffull;
        const unsigned pmask = __ballot_sync(0xffffffffu, flag == SP_P);
        const unsigned xmask = __ballot_sync(0xffffffffu, flag == 0);
        const int firstP = pmask ? __ffs(pmask) - 1 : 31;
        const unsigned need = firstP == 31 ? 0xffffffffu : ((2u << firstP) - 1u);
        if (xmask & need) {  // a predecessor has not published yet
          if (++spins > SP_SPIN_LIMIT) {
            if (lane == 0) atomicExch(err, 1);
            break;
          }
          continue;
        }
        prefix += __reduce_add_sync(0xffffffffu, lane <= firstP ? (uint32_t)wv : 0u);
        if (pmask) break;
        top -= 32;
      }
    }
    if (lane == 0) {
      sp_store(&status[tile], SP_P | (uint32_t)(prefix + agg));
      prefix_sh = prefix;
      if (total && tile == ntiles - 1) *total = prefix + agg;
    }
  }
  __syncthreads();
  const uint32_t off = prefix_sh + woff;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const long long i = wb + ((long long)q * 32 + lane) * 4;
    const uint32_t b0 = off + base[q], b1 = b0 + v[q].x, b2 = b1 + v[q].y, b3 = b2 + v[q].z;
    if (vec) {
      *reinterpret_cast<uint4*>(d + i) = make_uint4(b0, b1, b2, b3);
    } else {
      if (i < n) d[i] = b0;
      if (i + 1 < n) d[i + 1] = b1;
      if (i + 2 < n) d[i + 2] = b2;
      if (i + 3 < n) d[i + 3] = b3;
    }
  }
}

// --------------------------------------------------------------------------
// radix sort
// --------------------------------------------------------------------------
constexpr int RS_WARPS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;
constexpr int RS_ITEMS = 8;                       // per lane
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;    // 2048
constexpr int RS_RADIX = 256;

struct Key128 {
  const uint64_t* hi;
  const uint64_t* lo;
  // shifts are multiples of 8, so a digit never straddles the two words
  __device__ __forceinline__ uint32_t digit(long long i, int shift) const {
    if (shift < 64) return (uint32_t)(lo[i] >> shift) & 0xffu;
    return (uint32_t)(hi[i] >> (shift - 64)) & 0xffu;
  }
};


template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(K key, long long n, int shift, uint32_t* __restrict__ hist,
                                                      int ntiles) {
  __shared__ uint32_t h[RS_RADIX];
  for (int t = threadIdx.x; t < RS_RADIX; t += RS_THREADS) h[t] = 0;
  __syncthreads();
  long long base = (long long)blockIdx.x * RS_TILE;
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    long long i = base + (long long)k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[key.digit(i, shift)], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < RS_RADIX; t += RS_THREADS) hist[(long long)t * ntiles + blockIdx.x] = h[t];
}

template <class K, class MoveFn>
__device__ __forceinline__ void rs_scatter_body(K key, long long n, int shift, const uint32_t* __restrict__ hist,
                                                int ntiles, MoveFn move) {
  __shared__ uint32_t wh[RS_WARPS][RS_RADIX];
  __shared__ uint32_t gb[RS_RADIX];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < RS_WARPS * RS_RADIX; t += RS_THREADS) (&wh[0][0])[t] = 0;
  for (int t = threadIdx.x; t < RS_RADIX; t += RS_THREADS) gb[t] = hist[(long long)t * ntiles + blockIdx.x];
  __syncthreads();
  long long base = (long long)blockIdx.x * RS_TILE + (long long)w * 32 * RS_ITEMS;
  uint32_t dig[RS_ITEMS], rk[RS_ITEMS];
  unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    long long i = base + k * 32 + lane;
    uint32_t d = i < n ? key.digit(i, shift) : RS_RADIX;  // RS_RADIX: past the end
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (d < RS_RADIX) before = wh[w][d];
    __syncwarp();
    int leader = __ffs(peers) - 1;
    if (d < RS_RADIX && lane == leader) wh[w][d] = before + __popc(peers);
    __syncwarp();
    dig[k] = d;
    rk[k] = before + __popc(peers & lt);
  }
  __syncthreads();
  // exclusive prefix across warps, per digit
  for (int t = threadIdx.x; t < RS_RADIX; t += RS_THREADS) {
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) {
      uint32_t c = wh[q][t];
      wh[q][t] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    long long i = base + k * 32 + lane;
    if (i < n) move(i, (long long)gb[dig[k]] + wh[w][dig[k]] + rk[k]);
  }
}

__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scatter128(const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo, const uint32_t* __restrict__ v,
                    uint64_t* __restrict__ hi2, uint64_t* __restrict__ lo2, uint32_t* __restrict__ v2, long long n,
                    int shift, const uint32_t* __restrict__ hist, int ntiles) {
  Key128 key{hi, lo};
  rs_scatter_body(key, n, shift, hist, ntiles, [&](long long i, long long dst) {
    if (hi) hi2[dst] = hi[i];
    lo2[dst] = lo[i];
    v2[dst] = v[i];
  });
}

// --------------------------------------------------------------------------
// one-sweep radix sort (keys of up to 64 bits)
//
// In the spirit of Adinets and Merrill, "Onesweep: A Faster Least Significant
// Digit Radix Sort for GPUs" (2022): the digit histograms of every pass come
// from one upfront read of the keys, and each pass is a single kernel.  Its
// tiles take their index from an atomic counter (every predecessor of a tile
// is already running), rank their elements per 8-bit digit with warp-level
// matching (stable), publish per-digit counts and find each digit's
// exclusive prefix over the earlier tiles by a decoupled look-back (one
// thread per digit), then stage the tile in digit order in shared memory so
// that the writes to each digit's run are coalesced.  Status words are
// flag << 32 | count; the flags carry the pass number (2p + 1: tile count,
// 2p + 2: inclusive prefix), so one clearing serves every pass of a sort.
// --------------------------------------------------------------------------
constexpr int OS_THREADS = 256;
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_RADIX = 256;
constexpr int OS_MAX_PASSES = 8;
constexpr long long OS_SPIN_LIMIT = 1ll << 22;
constexpr int OS_LB = 8;  // predecessors read per look-back round trip

template <class K>
struct OsItems;
template <>
struct OsItems<uint64_t> {  // 3072-element tiles: 36 KB of staging
  static constexpr int v = 12;
};
template <>
struct OsItems<uint32_t> {  // 4096-element tiles: 32 KB of staging
  static constexpr int v = 16;
};

template <class K>
__global__ void __launch_bounds__(OS_THREADS) k_os_hist(const K* __restrict__ key, long long n, int passes,
                                                      uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[OS_MAX_PASSES][OS_RADIX];
  for (int t = threadIdx.x; t < OS_MAX_PASSES * OS_RADIX; t += OS_THREADS) (&h[0][0])[t] = 0;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * OS_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * OS_THREADS) {
    const K k = key[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(k >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < passes * OS_RADIX; t += OS_THREADS) {
    const uint32_t v = (&h[0][0])[t];
    if (v) atomicAdd(&ghist[t], v);
  }
}

// each pass's histogram to exclusive digit bases (one block per pass)
__global__ void __launch_bounds__(OS_RADIX) k_os_bases(uint32_t* __restrict__ ghist) {
  __shared__ uint32_t sw[33];
  uint32_t* h = ghist + (size_t)blockIdx.x * OS_RADIX;
  uint32_t excl;
  block_excl_scan(h[threadIdx.x], sw, excl);
  h[threadIdx.x] = excl;
}

template <class K>
__global__ void __launch_bounds__(OS_THREADS, 4) k_os_pass(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      K* __restrict__ kout, uint32_t* __restrict__ vout, long long n,
                                                      int pass, const uint32_t* __restrict__ gbase,
                                                      unsigned long long* __restrict__ status,
                                                      unsigned* __restrict__ ctr, int* __restrict__ err) {
  constexpr int ITEMS = OsItems<K>::v;
  constexpr int TILE = OS_THREADS * ITEMS;
  __shared__ K skey[TILE];
  __shared__ uint32_t sval[TILE];
  __shared__ uint32_t wh[OS_WARPS][OS_RADIX];
  __shared__ uint32_t dpre[OS_RADIX];
  __shared__ long long gofs[OS_RADIX];
  __shared__ uint32_t sw[33];
  __shared__ unsigned tile_sh;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) tile_sh = atomicAdd(ctr, 1u);
  for (int t = threadIdx.x; t < OS_WARPS * OS_RADIX; t += OS_THREADS) (&wh[0][0])[t] = 0;
  __syncthreads();
  const long long tile = tile_sh;
  const int shift = 8 * pass;
  // warp w holds a contiguous run of the tile, 32 consecutive elements per item
  const long long base = tile * TILE + (long long)w * 32 * ITEMS;
  K key[ITEMS];
  uint32_t val[ITEMS], dr[ITEMS];  // dr: rank in the warp's run << 9 | digit (256: past the end)
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const long long e = base + k * 32 + lane;
    const bool v = e < n;
    key[k] = v ? kin[e] : K(0);
    val[k] = v ? vin[e] : 0u;
    const uint32_t d = v ? ((uint32_t)(key[k] >> shift) & 255u) : (uint32_t)OS_RADIX;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (d < OS_RADIX) before = wh[w][d];
    __syncwarp();
    if (d < OS_RADIX && lane == __ffs(peers) - 1) wh[w][d] = before + __popc(peers);
    __syncwarp();
    dr[k] = ((before + __popc(peers & lt)) << 9) | d;
  }
  __syncthreads();
  // thread d: digit d's per-warp prefix and the tile's count
  const int d = threadIdx.x;
  uint32_t cnt = 0;
#pragma unroll
  for (int q = 0; q < OS_WARPS; ++q) {
    const uint32_t c = wh[q][d];
    wh[q][d] = cnt;
    cnt += c;
  }
  // publish the tile's count of digit d, then stage the tile in digit order
  // (tile-local offsets only) before the look-back, so the keys leave the
  // registers before the wait
  const unsigned long long FA = (unsigned long long)(2 * pass + 1) << 32;
  const unsigned long long FP = (unsigned long long)(2 * pass + 2) << 32;
  if (tile > 0) sp_store(&status[tile * OS_RADIX + d], FA | cnt);
  uint32_t dex;
  block_excl_scan(cnt, sw, dex);
  dpre[d] = dex;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint32_t dk = dr[k] & 511u;
    if (dk < OS_RADIX) {
      const uint32_t pos = dpre[dk] + wh[w][dk] + (dr[k] >> 9);
      skey[pos] = key[k];
      sval[pos] = val[k];
    }
  }
  // decoupled look-back over the earlier tiles' counts of digit d: OS_LB
  // predecessors per round trip, nearest first, adding counts up to the first
  // inclusive prefix; a predecessor that has not published yet is read again
  uint32_t excl = 0;
  if (tile > 0) {
    long long j = tile - 1, spins = 0;
    while (j >= 0) {
      unsigned long long wv[OS_LB];
#pragma unroll
      for (int q = 0; q < OS_LB; ++q) wv[q] = j - q >= 0 ? sp_load(&status[(j - q) * OS_RADIX + d]) : FP;
      int used = 0;
      bool done = false, wait = false;
#pragma unroll
      for (int q = 0; q < OS_LB; ++q) {
        if (done || wait) continue;
        const unsigned long long f = wv[q] & 0xffffffff00000000ull;
        if (f < FA) {  // not yet published in this pass
          wait = true;
          continue;
        }
        excl += (uint32_t)wv[q];
        ++used;
        done = f == FP;
      }
      if (done) break;
      j -= used;
      if (wait && ++spins > OS_SPIN_LIMIT) {
        atomicExch(err, 1);
        break;  // excl stays below the true prefix: every write stays in range
      }
    }
  }
  sp_store(&status[tile * OS_RADIX + d], FP | (excl + cnt));
  gofs[d] = (long long)gbase[d] + excl - dex;
  __syncthreads();
  const long long left = n - tile * TILE;
  const int tn = left < TILE ? (int)left : TILE;
  for (int pos = threadIdx.x; pos < tn; pos += OS_THREADS) {
    const K kk = skey[pos];
    const long long dst = gofs[(uint32_t)(kk >> shift) & 255u] + pos;
    kout[dst] = kk;
    vout[dst] = sval[pos];
  }
}

}  // namespace

int scan_u32(uint32_t* data, long long n, uint32_t* total, Workspace& ws, cudaStream_t st) {
  if (n <= 0) {
    if (total) CSO_CUDA(cudaMemsetAsync(total, 0, sizeof(uint32_t), st));
    return CSO_OK;
  }
  if (!ws.err) {
    cso_set_error("scan without a device error word");
    return CSO_ERR_STATE;
  }
  const bool big = n > SP_BIG;
  const long long ntiles = cdiv(n, (long long)SP_THREADS * (big ? 32 : 16));
  size_t mark = ws.off;
  unsigned long long* status = ws.get<unsigned long long>(ntiles + 1);
  if (!status) {
    cso_set_error("workspace exhausted in scan");
    return CSO_ERR_BUDGET;
  }
  CSO_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (ntiles + 1), st));
  if (big)
    k_scan_onepass<32><<<CL((unsigned)ntiles), SP_THREADS, 0, st>>>(data, n, status, ntiles, total, ws.err);
  else
    k_scan_onepass<16><<<CL((unsigned)ntiles), SP_THREADS, 0, st>>>(data, n, status, ntiles, total, ws.err);
  CSO_CUDA(cudaGetLastError());
  ws.off = mark;
  return CSO_OK;
}

template <class K>
static int onesweep(K** key, uint32_t** val, K* key_alt, uint32_t* val_alt, long long n, int bits, Workspace& ws,
                    cudaStream_t st) {
  if (!ws.err) {
    cso_set_error("sort without a device error word");
    return CSO_ERR_STATE;
  }
  constexpr int TILE = OS_THREADS * OsItems<K>::v;
  const int passes = (bits + 7) / 8;
  const long long ntiles = cdiv(n, TILE);
  const size_t mark = ws.off;
  unsigned long long* status = ws.get<unsigned long long>((size_t)ntiles * OS_RADIX);
  uint32_t* aux = ws.get<uint32_t>((size_t)passes * OS_RADIX + passes);  // histograms, then tile counters
  if (!status || !aux) {
    cso_set_error("workspace exhausted in radix sort");
    return CSO_ERR_BUDGET;
  }
  CSO_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * ntiles * OS_RADIX, st));
  CSO_CUDA(cudaMemsetAsync(aux, 0, sizeof(uint32_t) * ((size_t)passes * OS_RADIX + passes), st));
  const long long hb = std::min<long long>(cdiv(n, (long long)OS_THREADS * 16), (long long)cso_sm_count() * 8);
  k_os_hist<K><<<CL((unsigned)hb), OS_THREADS, 0, st>>>(*key, n, passes, aux);
  k_os_bases<<<passes, OS_RADIX, 0, st>>>(aux);
  for (int p = 0; p < passes; ++p) {
    k_os_pass<K><<<CL((unsigned)ntiles), OS_THREADS, 0, st>>>(*key, *val, key_alt, val_alt, n, p,
                                                               aux + (size_t)p * OS_RADIX, status,
                                                               aux + (size_t)passes * OS_RADIX + p, ws.err);
    K* t1 = *key;
    *key = key_alt;
    key_alt = t1;
    uint32_t* t2 = *val;
    *val = val_alt;
    val_alt = t2;
  }
  CSO_CUDA(cudaGetLastError());
  ws.off = mark;
  return CSO_OK;
}

int radix_sort_128(uint64_t** khi, uint64_t** klo, uint32_t** val, uint64_t* khi_alt, uint64_t* klo_alt,
                   uint32_t* val_alt, long long n, int bits, Workspace& ws, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return CSO_OK;
  // keys of up to 64 bits: the low word alone, one kernel per pass
  if (bits <= 64) return onesweep<uint64_t>(klo, val, klo_alt, val_alt, n, bits, ws, st);
  int ntiles = (int)cdiv(n, RS_TILE);
  size_t mark = ws.off;
  uint32_t* hist = ws.get<uint32_t>((size_t)ntiles * RS_RADIX);
  if (!hist) {
    cso_set_error("workspace exhausted in radix sort");
    return CSO_ERR_BUDGET;
  }
  bool with_hi = bits > 64;
  for (int shift = 0; shift < bits; shift += 8) {
    Key128 key{with_hi ? *khi : nullptr, *klo};
    k_rs_hist<<<CL(ntiles), RS_THREADS, 0, st>>>(key, n, shift, hist, ntiles);
    CSO_TRY(scan_u32(hist, (long long)ntiles * RS_RADIX, nullptr, ws, st));
    k_rs_scatter128<<<CL(ntiles), RS_THREADS, 0, st>>>(with_hi ? *khi : nullptr, *klo, *val, khi_alt, klo_alt, val_alt, n,
                                                   shift, hist, ntiles);
    CSO_CUDA(cudaGetLastError());
    uint64_t* t1 = *khi; *khi = khi_alt; khi_alt = t1;
    uint64_t* t2 = *klo; *klo = klo_alt; klo_alt = t2;
    uint32_t* t3 = *val; *val = val_alt; val_alt = t3;
  }
  ws.off = mark;
  return CSO_OK;
}

int radix_sort_32(uint32_t** key, uint32_t** val, uint32_t* key_alt, uint32_t* val_alt, long long n, int bits,
                  Workspace& ws, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return CSO_OK;
  return onesweep<uint32_t>(key, val, key_alt, val_alt, n, bits, ws, st);
}
