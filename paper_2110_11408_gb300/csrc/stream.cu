// Slab stream: one periodic box delivered as x-slabs in order, as the slabs
// of an N-body code's output (the strict slab segmentation of Sec. 2.1).
//
// The stream keeps on the device every particle that still matters: those
// without final labels and the ghost columns later densities need.  When a
// slab arrives:
//   * the kernel sums of the columns whose two neighbour columns have now
//     arrived are computed (Eq. 1 needs every particle within b);
//   * L0 groups are found among the particles with final kernel sums; a
//     group is closed when every member's neighbour columns have final sums
//     (no later particle can link to it), open otherwise;
//   * closed groups go through L1 and L2 (Sec. 2.2.2) and their members'
//     labels, and the non-dense particles' labels, are written straight into
//     the output buffers of the slabs they came from;
//   * labelled particles leave the device once both neighbour columns have
//     final sums.
// The periodic seam closes with the last slab.  A slab's ticket completes
// when all its particles have their labels; the labels equal those of the
// whole box processed at once.
#include <string.h>

#include <algorithm>

#include "cells.cuh"
#include "compaso.cuh"
#include "pipeline.cuh"
#include "stream.cuh"

namespace {

constexpr unsigned long long NONE = ~0ull;
constexpr uint8_t F_SIG = 1, F_LABEL = 2;

struct SlabPtrs {
  uint64_t* l0;
  uint64_t* l1;
  uint64_t* l2;
  int64_t* sigma;
  cso_halo* halos;
  long long halo_cap;
};

// the slab's positions and ids are already copied to the store at base
__global__ void k_append(int n, int base, uint32_t slab, int x_lo, int x_hi, const int32_t* __restrict__ rpos,
                         long long* __restrict__ rsig, uint8_t* __restrict__ rflag, uint32_t* __restrict__ rslab,
                         uint32_t* __restrict__ ridx, int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = base + i;
  const int x = rpos[3 * r], y = rpos[3 * r + 1], z = rpos[3 * r + 2];
  if (x < x_lo || x >= x_hi || (unsigned)y >= (unsigned)CSO_BOX || (unsigned)z >= (unsigned)CSO_BOX) atomicExch(bad, 1);
  rsig[r] = 0;
  rflag[r] = 0;
  rslab[r] = slab;
  ridx[r] = (uint32_t)i;
}

__global__ void k_col_hist(const int32_t* __restrict__ rpos, int n, int nc, unsigned* __restrict__ hist) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) atomicAdd(&hist[cell_coord(rpos[3 * r], nc)], 1u);
}

// kernel sums for the density pass: final ones from the store, the rest to be
// computed (masked in `todo`) or unknown
__global__ void k_window_sigma(const int4* __restrict__ spos, int n, CellGrid g, const long long* __restrict__ rsig,
                               const uint8_t* __restrict__ rflag, const uint8_t* __restrict__ col_new,
                               long long* __restrict__ sig, uint8_t* __restrict__ todo) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int w = spos[s].w;
  const int gcol = cell_coord((spos[s].x + g.x0) & (CSO_BOX - 1), g.nc);
  const bool fin = rflag[w] & F_SIG;
  todo[s] = !fin && col_new[gcol];
  sig[s] = fin ? rsig[w] : -1;
}

// store new sums; the sums FoF sees: unlabelled particles with final sums
__global__ void k_window_after_density(const int4* __restrict__ spos, int n, const uint8_t* __restrict__ todo,
                                       long long* __restrict__ sig, long long* __restrict__ rsig,
                                       uint8_t* __restrict__ rflag, long long* __restrict__ sig_fof) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int w = spos[s].w;
  if (todo[s]) {
    rsig[w] = sig[s];
    rflag[w] |= F_SIG;
  }
  const uint8_t f = rflag[w];
  sig_fof[s] = ((f & F_SIG) && !(f & F_LABEL)) ? sig[s] : -1;
}

// a group stays open while any member has a neighbour column without final sums
__global__ void k_open_groups(const int4* __restrict__ spos, int n, CellGrid g, const int* __restrict__ root,
                              const uint8_t* __restrict__ col_done, int* __restrict__ open) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int r = root[s];
  if (r < 0) return;
  const int gcol = cell_coord((spos[s].x + g.x0) & (CSO_BOX - 1), g.nc);
  if (!col_done[gcol]) open[r] = 1;
}

__global__ void k_select(const int* __restrict__ root, int n, const int* __restrict__ open,
                         uint8_t* __restrict__ select) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int r = root[s];
  select[s] = r >= 0 && !open[r];
}

// labels of closed-group members and of unlabelled non-dense particles with
// final sums, written into their slabs' outputs
__global__ void k_emit(const int4* __restrict__ spos, int n, const long long* __restrict__ sig_fof,
                       long long T_L0, const uint8_t* __restrict__ select, const int* __restrict__ root,
                       const unsigned long long* __restrict__ minid, const uint64_t* __restrict__ l1w,
                       const uint64_t* __restrict__ l2w, const long long* __restrict__ rsig,
                       uint8_t* __restrict__ rflag, const uint32_t* __restrict__ rslab,
                       const uint32_t* __restrict__ ridx, const SlabPtrs* __restrict__ slabs,
                       unsigned long long* __restrict__ done) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int w = spos[s].w;
  const uint8_t f = rflag[w];
  if (!(f & F_SIG) || (f & F_LABEL)) return;
  const bool dense = sig_fof[s] > T_L0;
  if (dense && !select[s]) return;  // member of an open group
  const SlabPtrs P = slabs[rslab[w]];
  const uint32_t i = ridx[w];
  if (P.sigma) P.sigma[i] = rsig[w];
  if (P.l0) P.l0[i] = dense ? minid[root[s]] : NONE;
  if (P.l1) P.l1[i] = dense ? l1w[w] : NONE;
  if (P.l2) P.l2[i] = dense ? l2w[w] : NONE;
  rflag[w] = f | F_LABEL;
  atomicAdd(&done[rslab[w]], 1ull);
}

__global__ void k_emit_rows(const cso_halo* __restrict__ rows, const uint32_t* __restrict__ row_w, int m,
                            const uint32_t* __restrict__ rslab, const SlabPtrs* __restrict__ slabs,
                            unsigned long long* __restrict__ nrows) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t sl = rslab[row_w[i]];
  const unsigned long long k = atomicAdd(&nrows[sl], 1ull);
  if ((long long)k < slabs[sl].halo_cap) slabs[sl].halos[k] = rows[i];
}

// keep unless labelled and no longer a ghost for a later density
__global__ void k_keep(const int32_t* __restrict__ rpos, int n, int nc, const uint8_t* __restrict__ rflag,
                       const uint8_t* __restrict__ col_fin, uint32_t* __restrict__ keep) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int c = cell_coord(rpos[3 * r], nc);
  const bool ghost_needed = !col_fin[(c + nc - 1) % nc] || !col_fin[(c + 1) % nc];
  keep[r] = !(rflag[r] & F_LABEL) || ghost_needed;
}

__global__ void k_compact_resident(const uint32_t* __restrict__ keep, const uint32_t* __restrict__ scan, int n,
                                   const int32_t* __restrict__ rpos, const uint64_t* __restrict__ rid,
                                   const long long* __restrict__ rsig, const uint8_t* __restrict__ rflag,
                                   const uint32_t* __restrict__ rslab, const uint32_t* __restrict__ ridx,
                                   int32_t* __restrict__ rpos2, uint64_t* __restrict__ rid2,
                                   long long* __restrict__ rsig2, uint8_t* __restrict__ rflag2,
                                   uint32_t* __restrict__ rslab2, uint32_t* __restrict__ ridx2) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || !keep[r]) return;
  const uint32_t d = scan[r];
  rpos2[3 * d] = rpos[3 * r];
  rpos2[3 * d + 1] = rpos[3 * r + 1];
  rpos2[3 * d + 2] = rpos[3 * r + 2];
  rid2[d] = rid[r];
  rsig2[d] = rsig[r];
  rflag2[d] = rflag[r];
  rslab2[d] = rslab[r];
  ridx2[d] = ridx[r];
}

#define G1(n) CL(cdiv((n), 256)), 256, 0, st

}  // namespace

// ---------------------------------------------------------------------------

void stream_release(StreamState* S) {
  if (!S) return;
  void* bufs[] = {S->rpos[0], S->rpos[1], S->rid[0], S->rid[1], S->rsig[0],  S->rsig[1],
                  S->rflag[0], S->rflag[1], S->rslab[0], S->rslab[1], S->ridx[0], S->ridx[1],
                  S->dslabs,  S->ddone,   S->dnrows, S->dhist,   S->dbad};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete S;
}

static int ensure_capacity(StreamState& S, long long need) {
  if (need <= S.cap) return CSO_OK;
  long long cap = std::max<long long>(need, S.cap * 3 / 2 + 1024);
  for (int k = 0; k < 2; ++k) {
    void *a = nullptr, *b = nullptr, *c = nullptr, *d = nullptr, *e = nullptr, *f = nullptr;
    CSO_CUDA(cudaMalloc(&a, sizeof(int32_t) * 3 * cap));
    CSO_CUDA(cudaMalloc(&b, sizeof(uint64_t) * cap));
    CSO_CUDA(cudaMalloc(&c, sizeof(long long) * cap));
    CSO_CUDA(cudaMalloc(&d, sizeof(uint8_t) * cap));
    CSO_CUDA(cudaMalloc(&e, sizeof(uint32_t) * cap));
    CSO_CUDA(cudaMalloc(&f, sizeof(uint32_t) * cap));
    if (k == S.cur && S.nr > 0) {  // keep the live copy
      CSO_CUDA(cudaMemcpy(a, S.rpos[k], sizeof(int32_t) * 3 * S.nr, cudaMemcpyDeviceToDevice));
      CSO_CUDA(cudaMemcpy(b, S.rid[k], sizeof(uint64_t) * S.nr, cudaMemcpyDeviceToDevice));
      CSO_CUDA(cudaMemcpy(c, S.rsig[k], sizeof(long long) * S.nr, cudaMemcpyDeviceToDevice));
      CSO_CUDA(cudaMemcpy(d, S.rflag[k], sizeof(uint8_t) * S.nr, cudaMemcpyDeviceToDevice));
      CSO_CUDA(cudaMemcpy(e, S.rslab[k], sizeof(uint32_t) * S.nr, cudaMemcpyDeviceToDevice));
      CSO_CUDA(cudaMemcpy(f, S.ridx[k], sizeof(uint32_t) * S.nr, cudaMemcpyDeviceToDevice));
    }
    void* old[] = {S.rpos[k], S.rid[k], S.rsig[k], S.rflag[k], S.rslab[k], S.ridx[k]};
    for (void* o : old)
      if (o) CSO_CUDA(cudaFree(o));
    S.rpos[k] = (int32_t*)a;
    S.rid[k] = (uint64_t*)b;
    S.rsig[k] = (long long*)c;
    S.rflag[k] = (uint8_t*)d;
    S.rslab[k] = (uint32_t*)e;
    S.ridx[k] = (uint32_t*)f;
  }
  S.cap = cap;
  return CSO_OK;
}

int stream_begin(StreamState** out, uint64_t id, const cso_params* p) {
  StreamState* S = new StreamState();
  S->id = id;
  S->p = *p;
  int rc = cso_params_derive(&S->p);
  if (rc == CSO_OK) rc = cells_choose(S->p.b2, &S->nc);
  if (rc != CSO_OK) {
    delete S;
    return rc;
  }
  S->col_fin.assign(S->nc, 0);
  *out = S;
  return CSO_OK;
}

// One slab of the stream on pipeline context c (its stream and workspace).
int stream_step(cso_ctx* c, StreamState& S, const cso_input* in, cso_output* out, ServedRequest* req) {
  cudaStream_t st = c->stream;
  const int nc = S.nc;
  const cso_params* p = &S.p;
  if (in->x_lo != S.x_received || in->x_hi <= in->x_lo || in->x_hi > CSO_BOX) {
    cso_set_error("slab [%d, %d) does not continue the stream at x = %lld", in->x_lo, in->x_hi,
                  (long long)S.x_received);
    return CSO_ERR_STATE;
  }
  if (!out->on_device) {
    cso_set_error("slab outputs must be device buffers");
    return CSO_ERR_ARG;
  }
  const int n_new = (int)in->n;
  const uint32_t slab = (uint32_t)S.slabs.size();
  S.slabs.push_back(StreamSlab{req, in->n, 0, *out, 0});

  // ---- append the slab's particles to the resident store ----
  CSO_CUDA(cudaStreamSynchronize(st));
  CSO_TRY(ensure_capacity(S, S.nr + n_new));
  if (!S.dhist) {
    CSO_CUDA(cudaMalloc((void**)&S.dhist, sizeof(unsigned) * nc));
    CSO_CUDA(cudaMalloc((void**)&S.dbad, sizeof(int)));
  }
  CSO_CUDA(cudaMemsetAsync(S.dbad, 0, sizeof(int), st));
  const int k = S.cur;
  if (n_new > 0) {
    const cudaMemcpyKind kind = in->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CSO_CUDA(cudaMemcpyAsync(S.rpos[k] + 3 * S.nr, in->pos, sizeof(int32_t) * 3 * n_new, kind, st));
    CSO_CUDA(cudaMemcpyAsync(S.rid[k] + S.nr, in->ids, sizeof(uint64_t) * n_new, kind, st));
    k_append<<<G1(n_new)>>>(n_new, (int)S.nr, slab, in->x_lo, in->x_hi, S.rpos[k], S.rsig[k], S.rflag[k],
                            S.rslab[k], S.ridx[k], S.dbad);
    CSO_CUDA(cudaGetLastError());
  }
  S.nr += n_new;
  S.x_received = in->x_hi;
  const bool last = in->x_hi == CSO_BOX;

  // ---- columns: arrived, final sums, and link-complete ----
  std::vector<uint8_t> recv(nc), fin(nc), done_col(nc), fresh(nc);
  for (int col = 0; col < nc; ++col) {
    const long long hi = col + 1 < nc ? (((long long)(col + 1) * CSO_BOX + nc - 1) / nc) : CSO_BOX;
    recv[col] = hi <= S.x_received;
  }
  for (int col = 0; col < nc; ++col)
    fin[col] = recv[(col + nc - 1) % nc] && recv[col] && recv[(col + 1) % nc];
  for (int col = 0; col < nc; ++col) {
    done_col[col] = fin[(col + nc - 1) % nc] && fin[col] && fin[(col + 1) % nc];
    fresh[col] = fin[col] && !S.col_fin[col];
  }

  // ---- window columns: those holding resident particles ----
  const int NR = (int)S.nr;
  CSO_CUDA(cudaMemsetAsync(S.dhist, 0, sizeof(unsigned) * nc, st));
  if (NR > 0) k_col_hist<<<G1(NR)>>>(S.rpos[k], NR, nc, S.dhist);
  std::vector<unsigned> h(nc);
  CSO_CUDA(cudaMemcpyAsync(h.data(), S.dhist, sizeof(unsigned) * nc, cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaMemcpyAsync(c->pinned, S.dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaStreamSynchronize(st));
  if (*(int*)c->pinned) {
    cso_set_error("slab particles outside the slab [%d, %d) or the box", in->x_lo, in->x_hi);
    S.failed = true;
    return CSO_ERR_ARG;
  }
  std::vector<int> cols;
  int gap_start = -1, best_gap = 0;
  {
    // the largest run of empty columns (circular) starts the window after it
    int run = 0, run_start = 0;
    for (int t = 0; t < 2 * nc; ++t) {
      const int col = t % nc;
      if (!h[col]) {
        if (run == 0) run_start = t;
        ++run;
        if (run > best_gap && run <= nc) {
          best_gap = run;
          gap_start = run_start;
        }
      } else {
        run = 0;
      }
    }
  }
  CellGrid g;
  std::vector<int> colmap(nc, -1);
  if (best_gap == 0) {
    g = whole_box_grid(nc, nullptr);
  } else {
    const int first = (gap_start + best_gap) % nc;
    for (int t = 0; t < nc; ++t) {
      const int col = (first + t) % nc;
      if (h[col]) {
        colmap[col] = (int)cols.size();
        cols.push_back(col);
      }
    }
    g = CellGrid{nc, (int)cols.size(), nullptr, nullptr, nullptr,
                 (int)(((long long)first * CSO_BOX + nc - 1) / nc)};
  }
  S.last_ncols = g.ncols;
  const long long ncell = (long long)g.ncols * nc * nc;
  if (ncell + 1 >= (1ll << 32)) {
    cso_set_error("slab window of %d columns of %d x %d cells exceeds 2^32 cells", g.ncols, nc, nc);
    S.failed = true;
    return CSO_ERR_BUDGET;
  }
  CSO_TRY(ctx_reserve(c, NR, ncell, false));
  Workspace& ws = c->ws;
#define ALLOC(T, name, cnt)                              \
  T* name = ws.get<T>(cnt);                              \
  if (!name) {                                           \
    cso_set_error("workspace exhausted (%s)", #name);    \
    return CSO_ERR_BUDGET;                               \
  }
  ALLOC(int, dcolmap, nc);
  ALLOC(int, dcols, nc);
  ALLOC(uint8_t, dfresh, nc);
  ALLOC(uint8_t, ddone, nc);
  ALLOC(uint8_t, dfin, nc);
  CSO_CUDA(cudaMemcpyAsync(dcolmap, colmap.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
  if (!cols.empty()) CSO_CUDA(cudaMemcpyAsync(dcols, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice, st));
  CSO_CUDA(cudaMemcpyAsync(dfresh, fresh.data(), nc, cudaMemcpyHostToDevice, st));
  CSO_CUDA(cudaMemcpyAsync(ddone, done_col.data(), nc, cudaMemcpyHostToDevice, st));
  CSO_CUDA(cudaMemcpyAsync(dfin, fin.data(), nc, cudaMemcpyHostToDevice, st));
  if (best_gap > 0) {
    g.colmap = dcolmap;
    g.cols = dcols;
  }
  ALLOC(uint32_t, start, ncell + 1);
  g.start = start;

  // slab output table (device) for every slab of the stream so far
  if ((long long)S.slabs.size() > S.slab_cap) {
    long long cap = std::max<long long>(64, (long long)S.slabs.size() * 2);
    void* a = nullptr;
    void* b = nullptr;
    void* d = nullptr;
    CSO_CUDA(cudaMalloc(&a, sizeof(SlabPtrs) * cap));
    CSO_CUDA(cudaMalloc(&b, sizeof(unsigned long long) * cap));
    CSO_CUDA(cudaMalloc(&d, sizeof(unsigned long long) * cap));
    CSO_CUDA(cudaMemsetAsync(b, 0, sizeof(unsigned long long) * cap, st));
    CSO_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * cap, st));
    if (S.slab_cap) {
      CSO_CUDA(cudaMemcpyAsync(b, S.ddone, sizeof(unsigned long long) * S.slab_cap, cudaMemcpyDeviceToDevice, st));
      CSO_CUDA(cudaMemcpyAsync(d, S.dnrows, sizeof(unsigned long long) * S.slab_cap, cudaMemcpyDeviceToDevice, st));
      CSO_CUDA(cudaStreamSynchronize(st));
      cudaFree(S.dslabs);
      cudaFree(S.ddone);
      cudaFree(S.dnrows);
    }
    S.dslabs = a;
    S.ddone = (unsigned long long*)b;
    S.dnrows = (unsigned long long*)d;
    S.slab_cap = cap;
  }
  {
    std::vector<SlabPtrs> tab(S.slabs.size());
    for (size_t i = 0; i < S.slabs.size(); ++i) {
      const cso_output& o = S.slabs[i].out;
      tab[i] = SlabPtrs{o.l0, o.l1, o.l2, o.sigma, o.halos, (long long)o.halo_cap};
    }
    CSO_CUDA(cudaMemcpyAsync(S.dslabs, tab.data(), sizeof(SlabPtrs) * tab.size(), cudaMemcpyHostToDevice, st));
  }

  if (NR > 0) {
    Stages SG{c, false};
    // ---- bin the resident particles into the window ----
    ALLOC(int4, spos, NR);
    ALLOC(uint64_t, sid, NR);
    ALLOC(Meta, meta, 1);
    // a window particle outside the window's columns sets meta->bad = 2
    CSO_CUDA(cudaMemsetAsync(meta, 0, sizeof(Meta), st));
    ws.err = &meta->timeout;
    CSO_TRY(cells_bin(S.rpos[k], S.rid[k], NR, g, start, spos, sid, &meta->bad, ws, st));

    // ---- kernel sums of the columns that became final ----
    ALLOC(long long, sig, NR);
    ALLOC(uint8_t, todo, NR);
    ALLOC(long long, sig_fof, NR);
    k_window_sigma<<<G1(NR)>>>(spos, NR, g, S.rsig[k], S.rflag[k], dfresh, sig, todo);
    CSO_TRY(cells_density(g, spos, NR, (uint32_t)p->b2, p->include_self, sig, nullptr, ws, st, todo));
    k_window_after_density<<<G1(NR)>>>(spos, NR, todo, sig, S.rsig[k], S.rflag[k], sig_fof);

    // ---- L0 among unlabelled particles with final sums; closed groups ----
    ALLOC(int, parent, NR);
    ALLOC(int, root, NR);
    ALLOC(unsigned long long, minid, NR);
    {
      size_t mark = ws.off;
      ALLOC(int, cell_root, NR);
      CSO_TRY(cells_fof(g, spos, NR, sig_fof, p->T_L0, (uint32_t)p->lfof2, sid, parent, root, minid, cell_root, ws, st));
      ws.off = mark;
    }
    ALLOC(int, open, NR);
    ALLOC(uint8_t, select, NR);
    CSO_CUDA(cudaMemsetAsync(open, 0, sizeof(int) * NR, st));
    k_open_groups<<<G1(NR)>>>(spos, NR, g, root, ddone, open);
    k_select<<<G1(NR)>>>(root, NR, open, select);

    // ---- L1 and L2 of the closed groups ----
    ALLOC(uint64_t, l1w, NR);
    ALLOC(uint64_t, l2w, NR);
    // members outside every L1 (L2) halo keep the no-group label
    CSO_CUDA(cudaMemsetAsync(l1w, 0xff, sizeof(uint64_t) * NR, st));
    CSO_CUDA(cudaMemsetAsync(l2w, 0xff, sizeof(uint64_t) * NR, st));
    GroupsIn gin{&g, spos, sig_fof, sid, root, minid, select, NR, g.x0};
    cso_halo* rows = nullptr;
    int nrows = 0;
    uint32_t* row_w = nullptr;
    CSO_TRY(run_groups(c, p, gin, SG, meta, l1w, l2w, &rows, &nrows, &row_w));

    // ---- labels and catalogue rows into the slabs' outputs ----
    k_emit<<<G1(NR)>>>(spos, NR, sig_fof, p->T_L0, select, root, minid, l1w, l2w, S.rsig[k], S.rflag[k],
                       S.rslab[k], S.ridx[k], (const SlabPtrs*)S.dslabs, S.ddone);
    if (nrows > 0)
      k_emit_rows<<<G1(nrows)>>>(rows, row_w, nrows, S.rslab[k], (const SlabPtrs*)S.dslabs, S.dnrows);
    CSO_CUDA(cudaGetLastError());

    // ---- drop what is labelled and no longer needed as a ghost ----
    ALLOC(uint32_t, keep, NR + 1);
    k_keep<<<G1(NR)>>>(S.rpos[k], NR, nc, S.rflag[k], dfin, keep);
    ALLOC(uint32_t, kscan, NR + 1);
    CSO_CUDA(cudaMemcpyAsync(kscan, keep, sizeof(uint32_t) * NR, cudaMemcpyDeviceToDevice, st));
    CSO_TRY(scan_u32(kscan, NR, kscan + NR, ws, st));
    const int o = 1 - k;
    k_compact_resident<<<G1(NR)>>>(keep, kscan, NR, S.rpos[k], S.rid[k], S.rsig[k], S.rflag[k], S.rslab[k],
                                   S.ridx[k], S.rpos[o], S.rid[o], S.rsig[o], S.rflag[o], S.rslab[o], S.ridx[o]);
    CSO_CUDA(cudaGetLastError());
    CSO_CUDA(cudaMemcpyAsync(c->pinned, kscan + NR, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CSO_CUDA(cudaMemcpyAsync((char*)c->pinned + 8, &meta->timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSO_CUDA(cudaStreamSynchronize(st));
    S.nr = *(uint32_t*)c->pinned;
    S.cur = o;
    if (*(int*)((char*)c->pinned + 8)) {
      cso_set_error("a bounded device wait gave up");
      S.failed = true;
      return CSO_ERR_TIMEOUT;
    }
  }
  S.col_fin = fin;

  // ---- completed slabs ----
  std::vector<unsigned long long> done(S.slabs.size()), nrow(S.slabs.size());
  CSO_CUDA(cudaMemcpyAsync(done.data(), S.ddone, sizeof(unsigned long long) * done.size(), cudaMemcpyDeviceToHost,
                           st));
  CSO_CUDA(cudaMemcpyAsync(nrow.data(), S.dnrows, sizeof(unsigned long long) * nrow.size(), cudaMemcpyDeviceToHost,
                           st));
  CSO_CUDA(cudaStreamSynchronize(st));
  for (size_t i = 0; i < S.slabs.size(); ++i) {
    StreamSlab& sl = S.slabs[i];
    sl.n_halos = (long long)nrow[i];
    if (!sl.completed && (long long)done[i] == sl.n) {
      sl.completed = true;
      sl.newly_completed = true;
    }
  }
  if (last) {
    for (auto& sl : S.slabs)
      if (!sl.completed) {
        cso_set_error("stream ended with %lld unlabelled particles", (long long)(sl.n - 0));
        return CSO_ERR_STATE;
      }
  }
#undef ALLOC
  return CSO_OK;
}
