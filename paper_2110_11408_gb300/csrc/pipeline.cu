// The pipeline of one box, stage by stage on the context's stream (the
// batched schedule adds two side streams inside the level stages):
//
//   bin      counting sort of particles into the dense cell table
//   density  Sigma per particle (Eq. 1)
//   fof      L0 groups over dense particles (Sec. 2.2.1)
//   gather   dense particles sorted by (L0 group, Sigma desc, id asc)
//   level1   CompaSO L1 per L0 group (steps 1-4; the local-peak test of
//            step 2 runs inside, only for eligible candidates): a block per
//            group, or by size a warp, block or thread-block cluster
//   prep2    members of each L1 halo in key order and their L1 labels
//   level2   CompaSO L2 per L1 halo, scheduled as level1
//   halos    per-halo statistics and the catalogue (optionally the radial
//            statistics and the shrinking-sphere centre)
//   output   labels and kernel sums in input order
#include <math.h>
#include <string.h>

#include "cells.cuh"
#include "compaso.cuh"
#include "pipeline.cuh"
#include "radial.cuh"

namespace {

constexpr unsigned long long NONE = ~0ull;

__global__ void k_flags(const int* __restrict__ root, int n, const uint8_t* __restrict__ select,
                        uint32_t* __restrict__ dflag, uint32_t* __restrict__ rflag) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int r = root[s];
  const bool in = r >= 0 && (!select || select[s]);
  dflag[s] = in;
  rflag[s] = in && r == s;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v = sh[i] > v ? sh[i] : v;
  __syncthreads();
  return v;
}

// compact the dense particles; block maxima of Sigma and id, one atomic per block
__global__ void __launch_bounds__(256) k_compact_dense(const int* __restrict__ root, const uint8_t* __restrict__ select,
                                                       int n, const uint32_t* __restrict__ dscan,
                                                       const long long* __restrict__ sigma,
                                                       const uint64_t* __restrict__ sid, uint32_t* __restrict__ dl,
                                                       Meta* meta) {
  __shared__ unsigned long long sh[8];
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long ms = 0, mid = 0;
  if (s < n && root[s] >= 0 && (!select || select[s])) {
    dl[dscan[s]] = (uint32_t)s;
    ms = (unsigned long long)sigma[s];
    mid = (unsigned long long)sid[s];
  }
  ms = block_max_u64(ms, sh);
  mid = block_max_u64(mid, sh);
  if (threadIdx.x == 0) {
    atomicMax(&meta->sigma_max, ms);
    atomicMax(&meta->id_max, mid);
  }
}

// key = group | (Sigma_max - Sigma) | id, packed low to high: id, Sigma', group
__global__ void k_make_keys(const uint32_t* __restrict__ dl, int nd, const int* __restrict__ root,
                            const uint32_t* __restrict__ rscan, const long long* __restrict__ sigma,
                            const uint64_t* __restrict__ sid, unsigned long long sigma_max, int bits_id,
                            int bits_sig, uint64_t* __restrict__ khi, uint64_t* __restrict__ klo,
                            uint32_t* __restrict__ val) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  uint32_t s = dl[k];
  unsigned __int128 g = rscan[root[s]];
  unsigned __int128 sp = sigma_max - (unsigned long long)sigma[s];
  unsigned __int128 key = (g << (bits_sig + bits_id)) | (sp << bits_id) | (unsigned __int128)sid[s];
  khi[k] = (uint64_t)(key >> 64);
  klo[k] = (uint64_t)key;
  val[k] = s;
}

// (group, Sigma desc) in one 64-bit key; the id tie-break is settled after
// the sort by k_tie_fix
__global__ void k_make_keys64(const uint32_t* __restrict__ dl, int nd, const int* __restrict__ root,
                              const uint32_t* __restrict__ rscan, const long long* __restrict__ sigma,
                              unsigned long long sigma_max, int bits_sig, uint64_t* __restrict__ key,
                              uint32_t* __restrict__ val) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  uint32_t s = dl[k];
  key[k] = ((uint64_t)rscan[root[s]] << bits_sig) | (sigma_max - (unsigned long long)sigma[s]);
  val[k] = s;
}

// Runs of equal (group, Sigma) keys, ordered by id: the first thread of a run
// sorts it by insertion (runs are almost always single elements).  A run
// longer than TIE_RUN_MAX is left alone and raises *overflow, and the caller
// sorts again with the id inside the key.
constexpr int TIE_RUN_MAX = 64;

__global__ void k_tie_fix(const uint64_t* __restrict__ key, uint32_t* __restrict__ val, int nd,
                          const uint64_t* __restrict__ sid, int* __restrict__ overflow) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k + 1 >= nd || key[k + 1] != key[k] || (k > 0 && key[k - 1] == key[k])) return;
  int e = k + 1;
  while (e < nd && key[e] == key[k] && e - k <= TIE_RUN_MAX) ++e;
  if (e - k > TIE_RUN_MAX) {
    atomicExch(overflow, 1);
    return;
  }
  for (int i = k + 1; i < e; ++i) {
    const uint32_t v = val[i];
    const uint64_t id = sid[v];
    int j = i - 1;
    while (j >= k && sid[val[j]] > id) {
      val[j + 1] = val[j];
      --j;
    }
    val[j + 1] = v;
  }
}

__global__ void k_seg_bounds128(const uint64_t* __restrict__ khi, const uint64_t* __restrict__ klo, int nd,
                                int gshift, int nseg, uint32_t* __restrict__ seg_off) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  auto grp = [&](int i) -> unsigned long long {
    unsigned __int128 key = ((unsigned __int128)(khi ? khi[i] : 0) << 64) | klo[i];
    return (unsigned long long)(key >> gshift);
  };
  unsigned long long g = grp(k);
  if (k == 0 || grp(k - 1) != g) seg_off[g] = k;
  if (k == nd - 1) seg_off[nseg] = nd;
}

__global__ void k_seg_bounds32(const uint32_t* __restrict__ key, int m, int nseg, uint32_t* __restrict__ seg_off) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  uint32_t g = key[k];
  if (k == 0 || key[k - 1] != g) seg_off[g] = k;
  if (k == m - 1) seg_off[nseg] = m;
}

__global__ void k_gather1(const uint32_t* __restrict__ val, int nd, const int4* __restrict__ spos,
                          const long long* __restrict__ sigma, const uint64_t* __restrict__ sid,
                          int4* __restrict__ epos, long long* __restrict__ esig, uint64_t* __restrict__ eid) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  uint32_t s = val[k];
  epos[k] = spos[s];
  esig[k] = sigma[s];
  eid[k] = sid[s];
}

__global__ void k_flag_assigned(const int* __restrict__ ehalo, int nd, uint32_t* __restrict__ f) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nd) f[k] = ehalo[k] >= 0;
}

__global__ void k_compact_assigned(const int* __restrict__ ehalo, int nd, const uint32_t* __restrict__ scan,
                                   const uint32_t* __restrict__ gs, uint32_t* __restrict__ key,
                                   uint32_t* __restrict__ val, int* __restrict__ lab1) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  int h = ehalo[k];
  if (h < 0) return;
  key[scan[k]] = (uint32_t)h;
  val[scan[k]] = (uint32_t)k;
  lab1[gs[k]] = h;
}

__global__ void k_gather2(const uint32_t* __restrict__ ek, int m, const int4* __restrict__ epos,
                          const long long* __restrict__ esig, const uint32_t* __restrict__ gs,
                          int4* __restrict__ epos2, long long* __restrict__ esig2, uint32_t* __restrict__ egs2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint32_t k = ek[i];
  epos2[i] = epos[k];
  esig2[i] = esig[k];
  egs2[i] = gs[k];
}

__global__ void k_fill_u64(uint64_t* p, long long n, uint64_t v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// kernel sums and L0 labels in input order: thread i reads its particle's
// sorted slot (scattered reads, coalesced writes)
__global__ void k_out_cells(const uint32_t* __restrict__ inv, int n, const long long* __restrict__ sigma,
                            const int* __restrict__ root, const unsigned long long* __restrict__ minid,
                            int64_t* __restrict__ osig, uint64_t* __restrict__ ol0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t s = inv[i];
  if (osig) osig[i] = sigma[s];
  if (ol0) {
    int r = root[s];
    ol0[i] = r >= 0 ? minid[r] : NONE;
  }
}

__global__ void k_out_l1(const int* __restrict__ ehalo, int nd, const uint32_t* __restrict__ gs,
                         const int4* __restrict__ spos, const uint32_t* __restrict__ hnuc,
                         const uint64_t* __restrict__ eid, uint64_t* __restrict__ ol1) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  int h = ehalo[k];
  if (h >= 0) ol1[spos[gs[k]].w] = eid[hnuc[h]];
}

__global__ void k_out_l2(const int* __restrict__ ehalo2, int m, const uint32_t* __restrict__ ek2,
                         const uint32_t* __restrict__ gs, const int4* __restrict__ spos,
                         const uint32_t* __restrict__ hnuc2, const uint64_t* __restrict__ eid,
                         uint64_t* __restrict__ ol2, unsigned* __restrict__ h2size) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int h = ehalo2[i];
  // one atomic per distinct halo in the warp (members of a halo are mostly adjacent)
  const unsigned peers = __match_any_sync(__activemask(), h);
  if (h >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h2size[h], (unsigned)__popc(peers));
  if (h < 0) return;
  if (ol2) ol2[spos[gs[ek2[i]]].w] = eid[ek2[hnuc2[h]]];
}

__device__ __forceinline__ int mi(int v) {
  if (v >= CSO_HALF) return v - CSO_BOX;
  if (v < -CSO_HALF) return v + CSO_BOX;
  return v;
}

__device__ __forceinline__ double wrap_box(double c) {
  if (c < 0) c += (double)CSO_BOX;
  if (c >= (double)CSO_BOX) c -= (double)CSO_BOX;
  return c;
}

// Statistics of every L1 halo over its members (the L2-level segments).
// Pass one (k_summary_sums): the minimum-image offsets of every member from
// its halo's nucleus, and from the halo's first L2 nucleus for members of
// that L2 halo, summed exactly per halo in int64; pass two, one thread per
// halo, forms the row.
// Per-halo sums of the members' minimum-image offsets from the L1 nucleus
// (and, for members of the halo's first L2 subhalo, from that nucleus).  The
// members come sorted by halo; a warp takes 32 x SUM_ITEMS consecutive ones,
// sums each halo's lanes with one warp reduction per component, carries the
// halo that runs on across items in registers, and adds a halo's partial sums
// to acc once per warp (per-warp atomics on the accumulators of the biggest
// halos serialised).  One offset is below 2^20 in magnitude, so 32 of them
// sum exactly in 32 bits.
constexpr int SUM_ITEMS = 16;
__global__ void __launch_bounds__(256) k_summary_sums(const uint32_t* __restrict__ ehal2, int na,
                                                      const int4* __restrict__ epos2, const int* __restrict__ ehalo2,
                                                      const uint32_t* __restrict__ hnuc, const int4* __restrict__ epos,
                                                      const uint32_t* __restrict__ nnuc2,
                                                      const uint32_t* __restrict__ hbase2,
                                                      const uint32_t* __restrict__ hnuc2,
                                                      unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32 * SUM_ITEMS;
  int open_h = -1;  // the halo carried over from earlier items
  long long run[6] = {0, 0, 0, 0, 0, 0};
  for (int it = 0; it < SUM_ITEMS; ++it) {
    const long long i = w0 + (long long)it * 32 + lane;
    const bool v = i < na;
    const int h = v ? (int)ehal2[i] : -1;
    int s[6] = {0, 0, 0, 0, 0, 0};
    if (v) {
      const int4 q = epos2[i];
      const int4 pn = epos[hnuc[h]];
      s[0] = mi(q.x - pn.x);
      s[1] = mi(q.y - pn.y);
      s[2] = mi(q.z - pn.z);
      if (nnuc2[h] > 0 && ehalo2[i] == (int)hbase2[h]) {
        const int4 p2 = epos2[hnuc2[hbase2[h]]];
        s[3] = mi(q.x - p2.x);
        s[4] = mi(q.y - p2.y);
        s[5] = mi(q.z - p2.z);
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, h);
    const bool lead = lane == __ffs(peers) - 1;
    const int last_h = __shfl_sync(0xffffffffu, h, 31);
    const unsigned omask = __ballot_sync(0xffffffffu, h == open_h && open_h >= 0);
    const int olane = omask ? __ffs(omask) - 1 : 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int t = __reduce_add_sync(peers, s[k]);
      const long long t_open = (long long)__shfl_sync(0xffffffffu, t, olane);
      const long long t_last = (long long)__shfl_sync(0xffffffffu, t, 31);
      // a halo wholly inside this item: its leader adds it
      if (v && lead && h != open_h && h != last_h && t)
        atomicAdd(&acc[6 * (size_t)h + k], (unsigned long long)(long long)t);
      if (omask) run[k] += t_open;
      if (last_h != open_h) {
        // the carried halo ended: flush it and carry the last lane's halo
        if (lane == 0 && open_h >= 0 && run[k]) atomicAdd(&acc[6 * (size_t)open_h + k], (unsigned long long)run[k]);
        run[k] = t_last;
      }
    }
    open_h = last_h;
  }
  if (lane == 0 && open_h >= 0)
    for (int k = 0; k < 6; ++k)
      if (run[k]) atomicAdd(&acc[6 * (size_t)open_h + k], (unsigned long long)run[k]);
}

__global__ void k_summary(const uint32_t* __restrict__ seg2, int H1, const int4* __restrict__ epos2,
                          const uint32_t* __restrict__ hnuc, const long long* __restrict__ hR2,
                          const int4* __restrict__ epos, const uint64_t* __restrict__ eid,
                          const uint32_t* __restrict__ gs, const int* __restrict__ root,
                          const unsigned long long* __restrict__ minid, const uint32_t* __restrict__ nnuc2,
                          const uint32_t* __restrict__ hbase2, const uint32_t* __restrict__ hnuc2,
                          const unsigned* __restrict__ h2size, const unsigned long long* __restrict__ acc,
                          const uint32_t* __restrict__ ek2, double inv_u, int np_min, int x0,
                          cso_halo* __restrict__ rows, uint32_t* __restrict__ keep) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H1) return;
  const int n = (int)(seg2[h + 1] - seg2[h]);
  const uint32_t kn = hnuc[h];
  const int4 pn = epos[kn];
  const int nl2 = (int)nnuc2[h];
  const int first2 = (int)hbase2[h];
  const long long sx = (long long)acc[6 * (size_t)h], sy = (long long)acc[6 * (size_t)h + 1],
                  sz = (long long)acc[6 * (size_t)h + 2], tx = (long long)acc[6 * (size_t)h + 3],
                  ty = (long long)acc[6 * (size_t)h + 4], tz = (long long)acc[6 * (size_t)h + 5];
  cso_halo r;
  r.nucleus_id = eid[kn];
  r.N = n;
  r.R2 = hR2[h];
  r.R_delta = sqrt((double)r.R2) * inv_u;
  r.com[0] = wrap_box((double)((pn.x + x0) & (CSO_BOX - 1)) + (double)sx / (double)n);
  r.com[1] = wrap_box((double)pn.y + (double)sy / (double)n);
  r.com[2] = wrap_box((double)pn.z + (double)sz / (double)n);
  r.l0_id = minid[root[gs[kn]]];
  r.n_l2 = nl2;
  for (int k = 0; k < 5; ++k) r.l2_top5_N[k] = 0;
  if (nl2 > 0) {
    const int4 p2 = epos2[hnuc2[first2]];
    long long n2 = h2size[first2];
    r.l2max_id = eid[ek2[hnuc2[first2]]];
    r.l2max_N = n2;
    r.l2max_com[0] = wrap_box((double)((p2.x + x0) & (CSO_BOX - 1)) + (double)tx / (double)n2);
    r.l2max_com[1] = wrap_box((double)p2.y + (double)ty / (double)n2);
    r.l2max_com[2] = wrap_box((double)p2.z + (double)tz / (double)n2);
    for (int q = 0; q < nl2; ++q) {  // five largest sizes, descending
      long long v = h2size[first2 + q];
      for (int k = 0; k < 5; ++k)
        if (v > r.l2_top5_N[k]) {
          long long t = r.l2_top5_N[k];
          r.l2_top5_N[k] = v;
          v = t;
        }
    }
  } else {
    r.l2max_id = NONE;
    r.l2max_N = 0;
    r.l2max_com[0] = r.l2max_com[1] = r.l2max_com[2] = 0.0;
  }
  rows[h] = r;
  keep[h] = n >= np_min;
}

__global__ void k_catalogue_keys(const cso_halo* __restrict__ rows, const uint32_t* __restrict__ keep,
                                 const uint32_t* __restrict__ kscan, int H, uint64_t* __restrict__ key,
                                 uint32_t* __restrict__ val) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H || !keep[h]) return;
  key[kscan[h]] = rows[h].nucleus_id;
  val[kscan[h]] = (uint32_t)h;
}

// rows in nucleus-id order; optionally the input index of each row's nucleus
__global__ void k_catalogue_write(const cso_halo* __restrict__ rows, const uint32_t* __restrict__ order, int m,
                                  const uint32_t* __restrict__ hnuc, const int4* __restrict__ epos,
                                  cso_halo* __restrict__ out, uint32_t* __restrict__ out_w,
                                  const cso_radial* __restrict__ rad, cso_radial* __restrict__ rad_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t h = order[i];
  out[i] = rows[h];
  if (out_w) out_w[i] = (uint32_t)epos[hnuc[h]].w;
  if (rad_out) rad_out[i] = rad[h];
}

int readback(cso_ctx* c, const void* dev, size_t bytes) {
  CSO_CUDA(cudaMemcpyAsync(c->pinned, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  CSO_CUDA(cudaStreamSynchronize(c->stream));
  return CSO_OK;
}

#define G1(n) CL(cdiv((n), 256)), 256, 0, st

}  // namespace

int level_stage(cso_ctx* c, const LevelArgs& L, const LevelSchedule& sched, unsigned* host_counts) {
  cudaStream_t st = c->stream;
  if (!(c->flags & CSO_FLAG_GRAPH))
    return level_run_batched(L, sched, c->ws, st, c->side, c->side2, c->side3, c->fork, c->join, c->join2, c->join3,
                             host_counts);
  for (int i = 0; i < CSO_LEVEL_GRAPHS; ++i) {
    LevelGraph& G = c->graphs[i];
    if (G.exec && G.giant == sched.giant && G.small == sched.small && G.huge == sched.huge &&
        !memcmp(&G.args, &L, sizeof(LevelArgs))) {
      ++c->graph_hits;
      CSO_CUDA(cudaGraphLaunch(G.exec, st));
      return CSO_OK;
    }
  }
  // capture this stage (thread-local mode: the served path's other threads
  // keep issuing work) and keep it in the oldest slot
  level_prepare();
  CSO_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int rc = level_run_batched(L, sched, c->ws, st, c->side, c->side2, c->side3, c->fork, c->join, c->join2,
                                   c->join3, host_counts);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc != CSO_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  CSO_CUDA(e);
  LevelGraph& G = c->graphs[c->graph_next];
  c->graph_next = (c->graph_next + 1) % CSO_LEVEL_GRAPHS;
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  CSO_CUDA(ei);
  memcpy(&G.args, &L, sizeof(LevelArgs));
  G.giant = sched.giant;
  G.small = sched.small;
  G.huge = sched.huge;
  ++c->graph_captures;
  CSO_CUDA(cudaGraphLaunch(G.exec, st));
  return CSO_OK;
}

int run_groups(cso_ctx* c, const cso_params* p, const GroupsIn& gi, Stages& S, Meta* meta, uint64_t* ol1,
               uint64_t* ol2, cso_halo** rows_out, int* nrows_out, uint32_t** rows_w_out, cso_radial** radial_out) {
  cudaStream_t st = c->stream;
  Workspace& ws = c->ws;
  const CellGrid& g = *gi.g;
  const int4* spos = gi.spos;
  const long long* sigma = gi.sigma;
  const uint64_t* sid = gi.sid;
  const int* root = gi.root;
  const unsigned long long* minid = gi.minid;
  const int N = gi.n;
  const long long n = gi.n;
#define ALLOC(T, name, cnt)                              \
  T* name = ws.get<T>(cnt);                              \
  if (!name) {                                           \
    cso_set_error("workspace exhausted (%s)", #name);    \
    return CSO_ERR_BUDGET;                               \
  }
  // ---- gather: dense particles by (group, Sigma desc, id asc) ----
  S.mark("gather");
  ALLOC(uint32_t, dscan, n + 1);
  ALLOC(uint32_t, rscan, n + 1);
  k_flags<<<G1(n)>>>(root, N, gi.select, dscan, rscan);
  CSO_TRY(scan_u32(dscan, n, dscan + n, ws, st));
  CSO_TRY(scan_u32(rscan, n, rscan + n, ws, st));
  ALLOC(uint32_t, dl, n);
  k_compact_dense<<<G1(n)>>>(root, gi.select, N, dscan, sigma, sid, dl, meta);
  CSO_CUDA(cudaGetLastError());
  // counters: n_dense, G, sigma_max, id_max, bad
  {
    CSO_CUDA(cudaMemcpyAsync(c->pinned, dscan + n, 4, cudaMemcpyDeviceToHost, st));
    CSO_CUDA(cudaMemcpyAsync((char*)c->pinned + 4, rscan + n, 4, cudaMemcpyDeviceToHost, st));
    CSO_CUDA(cudaMemcpyAsync(c->pinned + 1, meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
    CSO_CUDA(cudaStreamSynchronize(st));
  }
  const int nd = (int)((uint32_t*)c->pinned)[0];
  const int G = (int)((uint32_t*)c->pinned)[1];
  Meta hm;
  memcpy(&hm, c->pinned + 1, sizeof(Meta));
  if (hm.bad) {
    cso_set_error("positions outside [0, 2^21)");
    return CSO_ERR_ARG;
  }
  if (hm.timeout) {
    cso_set_error("a bounded device wait gave up");
    return CSO_ERR_TIMEOUT;
  }
  c->stats[1] = nd;
  c->stats[2] = G;

  const int bits_id = bit_length_u64(hm.id_max);
  const int bits_sig = nd ? bit_length_u64(hm.sigma_max - (unsigned long long)(p->T_L0 + 1)) : 0;
  const int bits_g = bit_length_u64(G > 0 ? (unsigned long long)(G - 1) : 0);
  if (bits_id + bits_sig + bits_g > 128) {
    cso_set_error("sort key of %d bits exceeds 128", bits_id + bits_sig + bits_g);
    return CSO_ERR_ARG;
  }
  ALLOC(uint64_t, khi, nd);
  ALLOC(uint64_t, klo, nd);
  ALLOC(uint32_t, kval, nd);
  ALLOC(uint64_t, khi2, nd);
  ALLOC(uint64_t, klo2, nd);
  ALLOC(uint32_t, kval2, nd);
  ALLOC(uint32_t, seg1, G + 1);
  ALLOC(int4, epos, nd);
  ALLOC(long long, esig, nd);
  ALLOC(uint64_t, eid, nd);
  uint32_t* gs = kval;
  if (nd > 0) {
    // (group, Sigma desc) fits one 64-bit key in every box the cell table
    // admits: sort by it, then order the rare runs of equal sums by id
    bool full = bits_sig + bits_g > 64;
    uint64_t *ph = nullptr, *pl = klo;
    uint32_t* pv = kval;
    if (!full) {
      k_make_keys64<<<G1(nd)>>>(dl, nd, root, rscan, sigma, hm.sigma_max, bits_sig, klo, kval);
      CSO_TRY(radix_sort_128(&ph, &pl, &pv, nullptr, klo2, kval2, nd, bits_sig + bits_g, ws, st));
      int* overflow = &meta->tie_overflow;
      k_tie_fix<<<G1(nd)>>>(pl, pv, nd, sid, overflow);
      CSO_CUDA(cudaMemcpyAsync(c->pinned, overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
      CSO_CUDA(cudaStreamSynchronize(st));
      full = *(int*)c->pinned != 0;
      if (full) CSO_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int), st));
      else k_seg_bounds128<<<G1(nd)>>>(nullptr, pl, nd, bits_sig, G, seg1);
    }
    if (full) {
      k_make_keys<<<G1(nd)>>>(dl, nd, root, rscan, sigma, sid, hm.sigma_max, bits_id, bits_sig, khi, klo, kval);
      ph = khi;
      pl = klo;
      pv = kval;
      int bits = bits_id + bits_sig + bits_g;
      CSO_TRY(radix_sort_128(&ph, &pl, &pv, khi2, klo2, kval2, nd, bits, ws, st));
      k_seg_bounds128<<<G1(nd)>>>(bits > 64 ? ph : nullptr, pl, nd, bits_sig + bits_id, G, seg1);
    }
    gs = pv;
    k_gather1<<<G1(nd)>>>(gs, nd, spos, sigma, sid, epos, esig, eid);
    CSO_CUDA(cudaGetLastError());
  }

  // ---- level1 ----
  S.mark("level1");
  ALLOC(int, eslot, nd);
  ALLOC(long long, edold, nd);
  ALLOC(uint8_t, einel, nd);
  ALLOC(long long, ed, nd);
  ALLOC(uint32_t, nucm, nd);
  ALLOC(long long, nucR2, nd);
  ALLOC(uint32_t, nnuc, G + 1);
  LevelArgs L1{};
  L1.nseg = G;
  L1.seg_off = seg1;
  L1.epos = epos;
  L1.esig = esig;
  L1.egs = gs;
  L1.T_min = p->T_min_L1;
  L1.pc = make_pred_const(p->K_L1, (long long)p->l_mean_grid);
  const bool radial_bins = (c->flags & CSO_FLAG_RADIAL_BINS) != 0;
  // radial bins of sqrt(3)/3 cell sides (cells of 2^21 / nc grid units)
  const float rbin_inv_w = (float)(sqrt(3.0) * g.nc / (double)CSO_BOX);
  L1.pc.radial = radial_bins;
  L1.pc.rbin_inv_w = rbin_inv_w;
  L1.alpha_num = p->alpha_num;
  L1.alpha_den = p->alpha_den;
  L1.roche_num = p->roche_num;
  L1.roche_den = p->roche_den;
  L1.eslot = eslot;
  L1.edold = edold;
  L1.einel = einel;
  L1.ed = ed;
  L1.grid = g;
  L1.spos = spos;
  L1.ssig = sigma;
  L1.sid = sid;
  L1.slab = root;
  L1.b2 = (uint32_t)p->b2;
  L1.nuc_member = nucm;
  L1.nuc_R2 = nucR2;
  L1.nnuc = nnuc;
  L1.work = &meta->work1;
  const bool stress = (c->flags & CSO_FLAG_SELECT_STRESS) != 0;
  L1.small_n = stress ? 8 : 2048;
  L1.cap = stress ? 8 : 2048;
  L1.nb = stress ? 16 : 1024;
  const bool batched = (c->flags & CSO_FLAG_BATCHED) != 0;
  const LevelSchedule sched = c->sched;
  unsigned* hcounts = (unsigned*)(c->pinned + 32);
  if (batched) CSO_TRY(level_stage(c, L1, sched, hcounts));
  else CSO_TRY(level_run(L1, st));

  // ---- prep2: L1 haloes, their members in key order, peaks within L1 ----
  S.mark("prep2");
  ALLOC(uint32_t, hbase, G + 1);
  if (G > 0) CSO_CUDA(cudaMemcpyAsync(hbase, nnuc, sizeof(uint32_t) * G, cudaMemcpyDeviceToDevice, st));
  CSO_TRY(scan_u32(hbase, G, hbase + G, ws, st));
  ALLOC(uint32_t, aflag, nd + 1);
  ALLOC(int, ehalo, nd);
  if (nd > 0) k_flag_assigned<<<G1(nd)>>>(eslot, nd, aflag);  // slot >= 0 <=> assigned
  CSO_TRY(scan_u32(aflag, nd, aflag + nd, ws, st));
  CSO_CUDA(cudaMemcpyAsync(c->pinned, hbase + G, 4, cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaMemcpyAsync((char*)c->pinned + 4, aflag + nd, 4, cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaStreamSynchronize(st));
  const int H1 = (int)((uint32_t*)c->pinned)[0];
  const int na = (int)((uint32_t*)c->pinned)[1];
  c->stats[3] = H1;
  ALLOC(uint32_t, hnuc, H1);
  ALLOC(long long, hR2, H1);
  ALLOC(uint32_t, hseg, H1);
  CSO_TRY(level_halo(G, seg1, nnuc, hbase, eslot, nucm, nucR2, ehalo, hnuc, hR2, hseg, nd, H1, st));
  ALLOC(int, lab1, n);
  CSO_CUDA(cudaMemsetAsync(lab1, 0xff, sizeof(int) * n, st));
  ALLOC(uint32_t, akey, na);
  ALLOC(uint32_t, aval, na);
  ALLOC(uint32_t, akey2, na);
  ALLOC(uint32_t, aval2, na);
  ALLOC(uint32_t, seg2, H1 + 1);
  uint32_t* ek2 = aval;
  uint32_t* ehal2 = akey;  // L1 halo of each member element, ascending
  if (nd > 0) k_compact_assigned<<<G1(nd)>>>(ehalo, nd, aflag, gs, akey, aval, lab1);
  if (na > 0) {
    uint32_t *pk = akey, *pv = aval;
    CSO_TRY(radix_sort_32(&pk, &pv, akey2, aval2, na, bit_length_u64(H1 > 0 ? H1 - 1 : 0), ws, st));
    k_seg_bounds32<<<G1(na)>>>(pk, na, H1, seg2);
    ek2 = pv;
    ehal2 = pk;
  }
  ALLOC(int4, epos2, na);
  ALLOC(long long, esig2, na);
  ALLOC(uint32_t, egs2, na);
  if (na > 0) k_gather2<<<G1(na)>>>(ek2, na, epos, esig, gs, epos2, esig2, egs2);
  CSO_CUDA(cudaGetLastError());

  // ---- level2 ----
  S.mark("level2");
  ALLOC(int, eslot2, na);
  ALLOC(uint32_t, nucm2, na);
  ALLOC(long long, nucR22, na);
  ALLOC(uint32_t, nnuc2, H1 + 1);
  LevelArgs L2 = L1;
  L2.nseg = H1;
  L2.seg_off = seg2;
  L2.epos = epos2;
  L2.esig = esig2;
  L2.egs = egs2;
  L2.slab = lab1;
  L2.T_min = p->T_min_L2;
  L2.pc = make_pred_const(p->K_L2, (long long)p->l_mean_grid);
  L2.pc.radial = radial_bins;
  L2.pc.rbin_inv_w = rbin_inv_w;
  L2.eslot = eslot2;
  L2.nuc_member = nucm2;
  L2.nuc_R2 = nucR22;
  L2.nnuc = nnuc2;
  L2.work = &meta->work2;
  // edold / einel / ed are reused (na <= nd)
  if (batched) CSO_TRY(level_stage(c, L2, sched, hcounts));
  else CSO_TRY(level_run(L2, st));

  // ---- output ----
  S.mark("halos");
  ALLOC(uint32_t, hbase2, H1 + 1);
  if (H1 > 0) CSO_CUDA(cudaMemcpyAsync(hbase2, nnuc2, sizeof(uint32_t) * H1, cudaMemcpyDeviceToDevice, st));
  CSO_TRY(scan_u32(hbase2, H1, hbase2 + H1, ws, st));
  CSO_TRY(readback(c, hbase2 + H1, 4));
  const int H2 = (int)((uint32_t*)c->pinned)[0];
  c->stats[4] = H2;
  ALLOC(int, ehalo2, na);
  ALLOC(uint32_t, hnuc2, H2);
  ALLOC(long long, hR2b, H2);
  ALLOC(uint32_t, hseg2, H2);
  ALLOC(unsigned, h2size, H2);
  CSO_TRY(level_halo(H1, seg2, nnuc2, hbase2, eslot2, nucm2, nucR22, ehalo2, hnuc2, hR2b, hseg2, na, H2, st));
  if (H2 > 0) CSO_CUDA(cudaMemsetAsync(h2size, 0, sizeof(unsigned) * H2, st));

  if (ol1 && nd > 0) k_out_l1<<<G1(nd)>>>(ehalo, nd, gs, spos, hnuc, eid, ol1);
  if (na > 0) k_out_l2<<<G1(na)>>>(ehalo2, na, ek2, gs, spos, hnuc2, eid, ol2, h2size);
  CSO_CUDA(cudaGetLastError());

  // per-halo rows and the catalogue
  if ((size_t)H1 * 2 + 1024 > c->rows_cap) {
    if (c->rows) {
      CSO_CUDA(cudaStreamSynchronize(st));
      CSO_CUDA(cudaFree(c->rows));
      c->rows = nullptr;
    }
    size_t cap = (size_t)H1 * 2 + 1024;
    CSO_CUDA(cudaMalloc((void**)&c->rows, sizeof(cso_halo) * cap));
    c->rows_cap = cap;
  }
  cso_halo* rows = c->rows;
  cso_halo* sorted_rows = c->rows + H1;
  ALLOC(uint32_t, keep, H1 + 1);
  int nrows = 0;
  if (H1 > 0) {
    {
      ALLOC(unsigned long long, acc, 6 * (size_t)H1);
      CSO_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 6 * (size_t)H1, st));
      if (na > 0)
        k_summary_sums<<<CL(cdiv(na, 256 * SUM_ITEMS)), 256, 0, st>>>(ehal2, na, epos2, ehalo2, hnuc, epos, nnuc2,
                                                                      hbase2, hnuc2, acc);
      k_summary<<<G1(H1)>>>(seg2, H1, epos2, hnuc, hR2, epos, eid, gs, root, minid, nnuc2, hbase2, hnuc2, h2size,
                            acc, ek2, 1.0 / p->l_mean_grid, p->np_min_L1, gi.x0, rows, keep);
    }
    CSO_CUDA(cudaGetLastError());
    cso_radial* rad = nullptr;
    if (radial_out) {
      S.mark("radial");
      ALLOC(cso_radial, r1, H1);
      rad = r1;
      CSO_TRY(radial_run(seg2, ehal2, epos2, na, rows, H1, gi.x0, p->l_mean_grid, hnuc, epos, rad, c->pinned, ws,
                         st));
      S.mark("catalogue");
    }
    ALLOC(uint32_t, kscan, H1 + 1);
    CSO_CUDA(cudaMemcpyAsync(kscan, keep, sizeof(uint32_t) * H1, cudaMemcpyDeviceToDevice, st));
    CSO_TRY(scan_u32(kscan, H1, kscan + H1, ws, st));
    CSO_TRY(readback(c, kscan + H1, 4));
    nrows = (int)((uint32_t*)c->pinned)[0];
    ALLOC(uint64_t, ckey, nrows);
    ALLOC(uint32_t, cval, nrows);
    ALLOC(uint64_t, ckey2, nrows);
    ALLOC(uint32_t, cval2, nrows);
    if (nrows > 0) {
      k_catalogue_keys<<<G1(H1)>>>(rows, keep, kscan, H1, ckey, cval);
      uint64_t* ph = nullptr;
      uint64_t* pl = ckey;
      uint32_t* pv = cval;
      CSO_TRY(radix_sort_128(&ph, &pl, &pv, nullptr, ckey2, cval2, nrows, bit_length_u64(hm.id_max), ws, st));
      uint32_t* row_w = nullptr;
      if (rows_w_out) {
        ALLOC(uint32_t, rw, nrows);
        row_w = rw;
        *rows_w_out = rw;
      }
      cso_radial* srad = nullptr;
      if (radial_out) {
        ALLOC(cso_radial, r2, nrows);
        srad = r2;
        *radial_out = r2;
      }
      k_catalogue_write<<<G1(nrows)>>>(rows, pv, nrows, hnuc, epos, sorted_rows, row_w, rad, srad);
      CSO_CUDA(cudaGetLastError());
    }
  }
  *rows_out = sorted_rows;
  *nrows_out = nrows;
#undef ALLOC
  return CSO_OK;
}

int pipeline_run(cso_ctx* c, const cso_input* in, const cso_params* p, cso_output* out) {
  cudaStream_t st = c->stream;
  const long long n = in->n;
  memset(c->stats, 0, sizeof(c->stats));
  c->stats[0] = n;
  const long long launches0 = g_cso_launches;
  c->nstages = 0;
  out->n_halos = 0;
  if (n == 0) return CSO_OK;
  int nc;
  CSO_TRY(cells_choose(p->b2, &nc));
  CSO_TRY(cells_check_dense(nc));
  const long long ncell = (long long)nc * nc * nc;
  const bool host_in = !in->on_device, host_out = !out->on_device;
  CSO_TRY(ctx_reserve(c, n, ncell, host_in || host_out));
  Workspace& ws = c->ws;
  Stages S{c, (c->flags & CSO_FLAG_TIMING) != 0};
  const int N = (int)n;

#define ALLOC(T, name, cnt)                              \
  T* name = ws.get<T>(cnt);                              \
  if (!name) {                                           \
    cso_set_error("workspace exhausted (%s)", #name);    \
    return CSO_ERR_BUDGET;                               \
  }

  // ---- inputs ----
  S.mark("h2d");
  const int32_t* pos = in->pos;
  const uint64_t* ids = in->ids;
  if (host_in) {
    ALLOC(int32_t, dpos, 3 * n);
    ALLOC(uint64_t, dids, n);
    CSO_CUDA(cudaMemcpyAsync(dpos, in->pos, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, st));
    CSO_CUDA(cudaMemcpyAsync(dids, in->ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
    pos = dpos;
    ids = dids;
  }
  ALLOC(Meta, meta, 1);
  CSO_CUDA(cudaMemsetAsync(meta, 0, sizeof(Meta), st));
  ws.err = &meta->timeout;

  // ---- bin ----
  S.mark("bin");
  ALLOC(uint32_t, start, ncell + 1);
  ALLOC(int4, spos, n);
  ALLOC(uint64_t, sid, n);
  CellGrid g = whole_box_grid(nc, start);
  ALLOC(uint32_t, inv, n);
  CSO_TRY(cells_bin(pos, ids, n, g, start, spos, sid, &meta->bad, ws, st, inv));

  // ---- density ----
  S.mark("density");
  ALLOC(long long, sigma, n);
  const bool count_pairs = (c->flags & CSO_FLAG_COUNT_PAIRS) != 0;
  CSO_TRY(cells_density(g, spos, N, (uint32_t)p->b2, p->include_self, sigma, count_pairs ? &meta->pairs : nullptr,
                        ws, st));

  // ---- fof ----
  S.mark("fof");
  ALLOC(int, parent, n);
  ALLOC(int, root, n);
  ALLOC(unsigned long long, minid, n);
  {
    size_t mark = ws.off;
    ALLOC(int, cell_root, n);  // per-cell tree summaries at each cell's first slot, transient
    CSO_TRY(cells_fof(g, spos, N, sigma, p->T_L0, (uint32_t)p->lfof2, sid, parent, root, minid, cell_root, ws, st));
    ws.off = mark;
  }

  // ---- outputs in input order ----
  uint64_t *ol0 = out->l0, *ol1 = out->l1, *ol2 = out->l2;
  int64_t* osig = out->sigma;
  if (host_out) {
    if (ol0) { ALLOC(uint64_t, t, n); ol0 = t; }
    if (ol1) { ALLOC(uint64_t, t, n); ol1 = t; }
    if (ol2) { ALLOC(uint64_t, t, n); ol2 = t; }
    if (osig) { ALLOC(int64_t, t, n); osig = t; }
  }
  if (ol1) k_fill_u64<<<G1(n)>>>(ol1, n, NONE);
  if (ol2) k_fill_u64<<<G1(n)>>>(ol2, n, NONE);
  // kernel sums and L0 labels are final here: write them in input order now,
  // and with host outputs copy them back on the copy stream while the group
  // stages run
  k_out_cells<<<G1(n)>>>(inv, N, sigma, root, minid, osig, ol0);
  CSO_CUDA(cudaGetLastError());
  const bool early_copy = host_out && (out->l0 || out->sigma);
  // every return from here on (errors included) leaves no copy in flight into
  // the caller's buffers
  struct CopyWait {
    cudaStream_t s;
    bool on;
    ~CopyWait() {
      if (on) cudaStreamSynchronize(s);
    }
  } copy_wait{c->copy, early_copy};
  if (early_copy) {
    CSO_CUDA(cudaEventRecord(c->out_ready, st));
    CSO_CUDA(cudaStreamWaitEvent(c->copy, c->out_ready, 0));
    if (out->l0) CSO_CUDA(cudaMemcpyAsync(out->l0, ol0, 8 * n, cudaMemcpyDeviceToHost, c->copy));
    if (out->sigma) CSO_CUDA(cudaMemcpyAsync(out->sigma, osig, 8 * n, cudaMemcpyDeviceToHost, c->copy));
    CSO_CUDA(cudaEventRecord(c->out_copied, c->copy));
  }

  GroupsIn gin{&g, spos, sigma, sid, root, minid, nullptr, N, 0};
  int nrows = 0;
  cso_halo* sorted_rows = nullptr;
  cso_radial* sorted_radial = nullptr;
  CSO_TRY(run_groups(c, p, gin, S, meta, ol1, ol2, &sorted_rows, &nrows, nullptr,
                     out->radial ? &sorted_radial : nullptr));
  if (count_pairs) {
    Meta hm2;
    CSO_CUDA(cudaMemcpyAsync(c->pinned, meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
    CSO_CUDA(cudaStreamSynchronize(st));
    memcpy(&hm2, c->pinned, sizeof(Meta));
    c->stats[6] = (int64_t)hm2.pairs;
  }
  S.mark("output");
  out->n_halos = nrows;
  c->stats[5] = nrows;
  const int ncopy = nrows <= out->halo_cap ? nrows : 0;
  if (ncopy > 0)
    CSO_CUDA(cudaMemcpyAsync(out->halos, sorted_rows, sizeof(cso_halo) * ncopy,
                             host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  if (ncopy > 0 && out->radial)
    CSO_CUDA(cudaMemcpyAsync(out->radial, sorted_radial, sizeof(cso_radial) * ncopy,
                             host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));

  // ---- d2h ----
  S.mark("d2h");
  if (host_out) {
    if (out->l1) CSO_CUDA(cudaMemcpyAsync(out->l1, ol1, 8 * n, cudaMemcpyDeviceToHost, st));
    if (out->l2) CSO_CUDA(cudaMemcpyAsync(out->l2, ol2, 8 * n, cudaMemcpyDeviceToHost, st));
  }
  if (early_copy) CSO_CUDA(cudaStreamWaitEvent(st, c->out_copied, 0));
  S.finish();
  CSO_CUDA(cudaMemcpyAsync(c->pinned, meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaStreamSynchronize(st));
  Meta hm;
  memcpy(&hm, c->pinned, sizeof(Meta));
  c->stats[7] = (int64_t)hm.work1;
  c->stats[8] = (int64_t)hm.work2;
  c->stats[9] = (int64_t)ws.peak;
  c->stats[10] = g_cso_launches - launches0;
#undef ALLOC
  if (hm.timeout) {
    cso_set_error("a bounded device wait gave up");
    return CSO_ERR_TIMEOUT;
  }
  if (nrows > out->halo_cap) {
    cso_set_error("catalogue has %d rows, halo_cap is %lld", nrows, (long long)out->halo_cap);
    return CSO_ERR_CAPACITY;
  }
  return CSO_OK;
}
