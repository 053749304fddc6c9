// The three steps of the path one at a time, for callers that distribute a
// box over several GPUs (the strict slab segmentation of Sec. 2.1) and
// exchange ghost particles and cross-boundary groups between the steps:
//
//   cso_density  kernel sums Sigma (Sec. 2.2.1, Eq. 1) of the first n_query
//                particles, with every given particle as a neighbour;
//   cso_fof      L0 groups (Sec. 2.2.1) of particles whose kernel sums the
//                caller supplies;
//   cso_levels   L1 and L2 (Sec. 2.2.2) inside caller-supplied L0 groups,
//                with labels and the catalogue.
//
// Each call bins its particles into the cell table like cso_find_groups and
// runs the same kernels; the outputs of cso_find_groups on a box equal those
// of the three calls chained on it.
#include <string.h>

#include "cells.cuh"
#include "compaso.cuh"
#include "pipeline.cuh"

namespace {

constexpr unsigned long long NONE = ~0ull;

#define G1(n) CL(cdiv((n), 256)), 256, 0, st

__global__ void k_sigma_out(const uint32_t* __restrict__ inv, long long n_query, const long long* __restrict__ ssig,
                            int64_t* __restrict__ sigma) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_query) sigma[i] = ssig[inv[i]];
}

// caller values in input order -> cell-sorted order
__global__ void k_to_sorted_i64(const int4* __restrict__ spos, int n, const int64_t* __restrict__ in,
                                long long* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = in[spos[s].w];
}

__global__ void k_label_keys(const int4* __restrict__ spos, int n, const uint64_t* __restrict__ l0,
                             uint32_t* __restrict__ flag) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) flag[s] = l0[spos[s].w] != NONE;
}

__global__ void k_label_compact(const int4* __restrict__ spos, int n, const uint64_t* __restrict__ l0,
                                const uint32_t* __restrict__ scan, uint64_t* __restrict__ key,
                                uint32_t* __restrict__ val) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint64_t lab = l0[spos[s].w];
  if (lab == NONE) return;
  key[scan[s]] = lab;
  val[scan[s]] = (uint32_t)s;
}

// root of every member: the first sorted index of its label's run; the
// group's L0 label is kept at the root
__global__ void k_label_roots(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, int m,
                              int* __restrict__ root, unsigned long long* __restrict__ minid) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  int first = k;
  // runs are short unless groups are big; the head of a run is found by
  // binary search for the first key equal to key[k]
  int lo = 0, hi = k;
  const uint64_t v = key[k];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (key[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  first = lo;
  const int r = (int)val[first];
  root[val[k]] = r;
  if (k == first) minid[r] = v;
}

__global__ void k_fill_i32(int* p, long long n, int v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_l0_out(const uint32_t* __restrict__ inv, int n, const int* __restrict__ root,
                         const unsigned long long* __restrict__ minid, uint64_t* __restrict__ l0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = root[inv[i]];
  l0[i] = r >= 0 ? minid[r] : NONE;
}

#define ALLOC(T, name, cnt)                              \
  T* name = ws.get<T>(cnt);                              \
  if (!name) {                                           \
    cso_set_error("workspace exhausted (%s)", #name);    \
    return CSO_ERR_BUDGET;                               \
  }

// Common set-up: derived parameters, the workspace, inputs on the device and
// the cell table; fills the sorted positions, ids and the slots of the input.
struct Binned {
  CellGrid g;
  int4* spos;
  uint64_t* sid;
  uint32_t* inv;
  Meta* meta;
};

int bin_request(cso_ctx* c, const int32_t* pos, const uint64_t* ids, long long n, const cso_params* p, bool host,
                size_t extra_per_particle, Binned& B, const int32_t** dpos_out) {
  int nc;
  CSO_TRY(cells_choose(p->b2, &nc));
  CSO_TRY(cells_check_dense(nc));
  const long long ncell = (long long)nc * nc * nc;
  CSO_TRY(ctx_reserve(c, n + (long long)(extra_per_particle * n / CSO_BYTES_PER_PARTICLE) + 1, ncell, host));
  Workspace& ws = c->ws;
  cudaStream_t st = c->stream;
  ALLOC(Meta, meta, 1);
  CSO_CUDA(cudaMemsetAsync(meta, 0, sizeof(Meta), st));
  ws.err = &meta->timeout;
  const int32_t* dpos = pos;
  const uint64_t* dids = ids;
  if (host) {
    ALLOC(int32_t, hp, 3 * n);
    CSO_CUDA(cudaMemcpyAsync(hp, pos, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, st));
    dpos = hp;
    if (ids) {
      ALLOC(uint64_t, hi, n);
      CSO_CUDA(cudaMemcpyAsync(hi, ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
      dids = hi;
    }
  }
  ALLOC(uint32_t, start, ncell + 1);
  ALLOC(int4, spos, n);
  ALLOC(uint64_t, sid, n);
  ALLOC(uint32_t, inv, n);
  if (!dids) {  // ids play no part in the kernel sums: the binning copies n unused words
    ALLOC(uint64_t, unused, n);
    dids = unused;
  }
  B.g = whole_box_grid(nc, start);
  B.spos = spos;
  B.sid = sid;
  B.inv = inv;
  B.meta = meta;
  *dpos_out = dpos;
  CSO_TRY(cells_bin(dpos, dids, n, B.g, start, spos, sid, &meta->bad, ws, st, inv));
  return CSO_OK;
}

int finish_request(cso_ctx* c, Meta* meta) {
  Meta hm;
  CSO_CUDA(cudaMemcpyAsync(c->pinned, meta, sizeof(Meta), cudaMemcpyDeviceToHost, c->stream));
  CSO_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(&hm, c->pinned, sizeof(Meta));
  if (hm.bad) {
    cso_set_error("positions outside [0, 2^21)");
    return CSO_ERR_ARG;
  }
  if (hm.timeout) {
    cso_set_error("a bounded device wait gave up");
    return CSO_ERR_TIMEOUT;
  }
  return CSO_OK;
}

int check_args(cso_ctx* c, const void* pos, long long n, const cso_params* pin, cso_params* p) {
  if (!c || !pin || n < 0 || (n > 0 && !pos)) {
    cso_set_error("null or negative argument");
    return CSO_ERR_ARG;
  }
  if (n >= (1ll << 31) - 1) {
    cso_set_error("n = %lld is too large for one request (< 2^31)", n);
    return CSO_ERR_ARG;
  }
  *p = *pin;
  CSO_TRY(cso_params_derive(p));
  CSO_CUDA(cudaSetDevice(c->device));
  return CSO_OK;
}

}  // namespace

extern "C" int cso_density(cso_ctx* c, const int32_t* pos, int64_t n, int64_t n_query, const cso_params* pin,
                           int64_t* sigma, int32_t on_device) {
  cso_params p;
  CSO_TRY(check_args(c, pos, n, pin, &p));
  if (n_query < 0 || n_query > n || (n_query > 0 && !sigma)) {
    cso_set_error("cso_density: need 0 <= n_query <= n and a sigma buffer");
    return CSO_ERR_ARG;
  }
  if (n == 0) return CSO_OK;
  const bool host = !on_device;
  Binned B;
  const int32_t* dpos;
  CSO_TRY(bin_request(c, pos, nullptr, n, &p, host, 16, B, &dpos));
  Workspace& ws = c->ws;
  cudaStream_t st = c->stream;
  ALLOC(long long, ssig, n);
  CSO_TRY(cells_density(B.g, B.spos, (int)n, (uint32_t)p.b2, p.include_self, ssig, nullptr, ws, st));
  int64_t* out = sigma;
  if (host) {
    ALLOC(int64_t, t, n_query);
    out = t;
  }
  if (n_query > 0) k_sigma_out<<<G1(n_query)>>>(B.inv, n_query, ssig, out);
  CSO_CUDA(cudaGetLastError());
  if (host && n_query > 0)
    CSO_CUDA(cudaMemcpyAsync(sigma, out, sizeof(int64_t) * n_query, cudaMemcpyDeviceToHost, st));
  return finish_request(c, B.meta);
}

extern "C" int cso_fof(cso_ctx* c, const int32_t* pos, const uint64_t* ids, const int64_t* sigma, int64_t n,
                       const cso_params* pin, uint64_t* l0, int32_t on_device) {
  cso_params p;
  CSO_TRY(check_args(c, pos, n, pin, &p));
  if (n > 0 && (!ids || !sigma || !l0)) {
    cso_set_error("cso_fof: ids, sigma and l0 are required");
    return CSO_ERR_ARG;
  }
  if (n == 0) return CSO_OK;
  const bool host = !on_device;
  Binned B;
  const int32_t* dpos;
  CSO_TRY(bin_request(c, pos, ids, n, &p, host, 64, B, &dpos));
  Workspace& ws = c->ws;
  cudaStream_t st = c->stream;
  const int64_t* dsig = sigma;
  if (host) {
    ALLOC(int64_t, t, n);
    CSO_CUDA(cudaMemcpyAsync(t, sigma, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
    dsig = t;
  }
  ALLOC(long long, ssig, n);
  k_to_sorted_i64<<<G1(n)>>>(B.spos, (int)n, dsig, ssig);
  ALLOC(int, parent, n);
  ALLOC(int, root, n);
  ALLOC(unsigned long long, minid, n);
  {
    size_t mark = ws.off;
    ALLOC(int, cell_root, n);
    CSO_TRY(cells_fof(B.g, B.spos, (int)n, ssig, p.T_L0, (uint32_t)p.lfof2, B.sid, parent, root, minid, cell_root, ws,
                      st));
    ws.off = mark;
  }
  uint64_t* out = l0;
  if (host) {
    ALLOC(uint64_t, t, n);
    out = t;
  }
  k_l0_out<<<G1(n)>>>(B.inv, (int)n, root, minid, out);
  CSO_CUDA(cudaGetLastError());
  if (host) CSO_CUDA(cudaMemcpyAsync(l0, out, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, st));
  return finish_request(c, B.meta);
}

extern "C" int cso_levels(cso_ctx* c, const int32_t* pos, const uint64_t* ids, const int64_t* sigma,
                          const uint64_t* l0, int64_t n, const cso_params* pin, cso_output* out) {
  cso_params p;
  CSO_TRY(check_args(c, pos, n, pin, &p));
  if (!out || (n > 0 && (!ids || !sigma || !l0)) || out->halo_cap < 0 || (out->halo_cap > 0 && !out->halos) ||
      out->radial) {
    cso_set_error("cso_levels: ids, sigma, l0 and an output block (no radial statistics) are required");
    return CSO_ERR_ARG;
  }
  out->n_halos = 0;
  if (n == 0) return CSO_OK;
  const bool host = !out->on_device;
  Binned B;
  const int32_t* dpos;
  CSO_TRY(bin_request(c, pos, ids, n, &p, host, 32, B, &dpos));
  Workspace& ws = c->ws;
  cudaStream_t st = c->stream;
  const int64_t* dsig = sigma;
  const uint64_t* dl0 = l0;
  if (host) {
    ALLOC(int64_t, t, n);
    CSO_CUDA(cudaMemcpyAsync(t, sigma, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
    dsig = t;
    ALLOC(uint64_t, t2, n);
    CSO_CUDA(cudaMemcpyAsync(t2, l0, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
    dl0 = t2;
  }
  ALLOC(long long, ssig, n);
  k_to_sorted_i64<<<G1(n)>>>(B.spos, (int)n, dsig, ssig);
  // groups from the caller's labels: members sorted by label, the first
  // member of each run is its root
  ALLOC(int, root, n);
  ALLOC(unsigned long long, minid, n);
  ALLOC(uint32_t, flag, n + 1);
  k_fill_i32<<<G1(n)>>>(root, n, -1);
  k_label_keys<<<G1(n)>>>(B.spos, (int)n, dl0, flag);
  CSO_TRY(scan_u32(flag, n, flag + n, ws, st));
  CSO_CUDA(cudaMemcpyAsync(c->pinned, flag + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaStreamSynchronize(st));
  const int m = (int)*(uint32_t*)c->pinned;
  if (m > 0) {
    size_t mark = ws.off;
    ALLOC(uint64_t, key, m);
    ALLOC(uint32_t, val, m);
    ALLOC(uint64_t, key2, m);
    ALLOC(uint32_t, val2, m);
    k_label_compact<<<G1(n)>>>(B.spos, (int)n, dl0, flag, key, val);
    uint64_t* ph = nullptr;
    uint64_t* pk = key;
    uint32_t* pv = val;
    CSO_TRY(radix_sort_128(&ph, &pk, &pv, nullptr, key2, val2, m, 64, ws, st));
    k_label_roots<<<G1(m)>>>(pk, pv, m, root, minid);
    CSO_CUDA(cudaGetLastError());
    ws.off = mark;
  }
  uint64_t *ol1 = out->l1, *ol2 = out->l2;
  if (host) {
    if (ol1) { ALLOC(uint64_t, t, n); ol1 = t; }
    if (ol2) { ALLOC(uint64_t, t, n); ol2 = t; }
  }
  if (ol1) CSO_CUDA(cudaMemsetAsync(ol1, 0xff, sizeof(uint64_t) * n, st));
  if (ol2) CSO_CUDA(cudaMemsetAsync(ol2, 0xff, sizeof(uint64_t) * n, st));
  Stages S{c, false};
  GroupsIn gin{&B.g, B.spos, ssig, B.sid, root, minid, nullptr, (int)n, 0};
  int nrows = 0;
  cso_halo* rows = nullptr;
  CSO_TRY(run_groups(c, &p, gin, S, B.meta, ol1, ol2, &rows, &nrows, nullptr));
  out->n_halos = nrows;
  const int ncopy = nrows <= out->halo_cap ? nrows : 0;
  if (ncopy > 0)
    CSO_CUDA(cudaMemcpyAsync(out->halos, rows, sizeof(cso_halo) * ncopy,
                             host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  if (host) {
    if (out->l1) CSO_CUDA(cudaMemcpyAsync(out->l1, ol1, 8 * n, cudaMemcpyDeviceToHost, st));
    if (out->l2) CSO_CUDA(cudaMemcpyAsync(out->l2, ol2, 8 * n, cudaMemcpyDeviceToHost, st));
  }
  CSO_TRY(finish_request(c, B.meta));
  if (nrows > out->halo_cap) {
    cso_set_error("catalogue has %d rows, halo_cap is %lld", nrows, (long long)out->halo_cap);
    return CSO_ERR_CAPACITY;
  }
  return CSO_OK;
}
