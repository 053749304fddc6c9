// cso_density_static: the kernel-density pass with no device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need kernel
// densities: an N-body code that has handed all device memory to its own
// pool, or a time-step loop where an allocation would synchronise the device
// in the middle of a step.  This entry point takes the caller's device
// buffers for the positions and the output, and keeps its own scratch (the
// cell table, the cell-sorted copy of the positions and the per-cell
// counters) in one fixed array in device global memory, declared below.  The
// array exists once per GPU that loads this library and stays allocated until
// the process exits.
//
// Limits (CSO_STATIC_MAX_N particles, CSO_STATIC_MAX_CELLS cells) are
// checked before any work; larger requests get CSO_ERR_ARG.
#include <mutex>

#include "cells.cuh"

// 96 MiB: 2^20 particles x 80 B (sorted int4 position, sorted kernel sum,
// sorted id slot, and the binning's 32-byte placement record; the cell keys
// and arrival ranks share the position array) plus a table of up to
// 4,194,304 + 1 cell offsets and the scan's status words
#define CSO_STATIC_SCRATCH_BYTES (96u << 20)

static __device__ __align__(256) unsigned char g_cso_static_scratch[CSO_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_ptr[64] = {};  // device address of the array, per device ordinal

// Device address of the scratch array on the current device.  In host code
// the symbol itself is only a host-side stand-in, so the address has to come
// from the runtime; looked up once per device.
int scratch_address(void** out) {
  int dev = 0;
  CSO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    cso_set_error("device ordinal %d out of range", dev);
    return CSO_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cso_static_scratch);
    if (e != cudaSuccess || !p) {
      cso_set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      return CSO_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CSO_OK;
}

__global__ void k_unsort(const int4* __restrict__ spos, const long long* __restrict__ ssig, int n,
                         int64_t* __restrict__ sigma) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) sigma[spos[s].w] = ssig[s];
}

}  // namespace

extern "C" int cso_density_static(const int32_t* pos, int64_t n, const cso_params* pin, int64_t* sigma,
                                  void* stream) {
  if (!pin || n < 0 || (n > 0 && (!pos || !sigma))) {
    cso_set_error("cso_density_static: null or negative argument");
    return CSO_ERR_ARG;
  }
  if (n > CSO_STATIC_MAX_N) {
    cso_set_error("cso_density_static: n = %lld exceeds the static limit of %d particles", (long long)n,
                  CSO_STATIC_MAX_N);
    return CSO_ERR_ARG;
  }
  cso_params p = *pin;
  CSO_TRY(cso_params_derive(&p));
  int nc;
  CSO_TRY(cells_choose(p.b2, &nc));
  const long long ncell = (long long)nc * nc * nc;
  if (ncell > CSO_STATIC_MAX_CELLS) {
    cso_set_error("cso_density_static: %lld cells exceed the static limit of %d (boxes up to 64 l_mean side)",
                  ncell, CSO_STATIC_MAX_CELLS);
    return CSO_ERR_ARG;
  }
  void* base = nullptr;
  CSO_TRY(scratch_address(&base));
  if (n == 0) return CSO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  ws.base = (char*)base;
  ws.cap = CSO_STATIC_SCRATCH_BYTES;
  uint32_t* start = ws.get<uint32_t>(ncell + 1);
  int4* spos = ws.get<int4>(n);
  long long* ssig = ws.get<long long>(n);
  uint64_t* sid = ws.get<uint64_t>(n);
  int* bad = ws.get<int>(2);  // [0] positions outside the box, [1] a bounded wait gave up
  if (!start || !spos || !ssig || !sid || !bad) {
    cso_set_error("cso_density_static: static scratch too small");
    return CSO_ERR_ARG;
  }
  // the array keeps the previous call's contents: counters start from zero
  // (cells_bin clears the cell table itself)
  CSO_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(int), st));
  ws.err = bad + 1;
  // ids play no part in densities: the binning pass copies n placeholder
  // words (the not yet written sums) into its id slot
  CellGrid g = whole_box_grid(nc, start);
  CSO_TRY(cells_bin(pos, (const uint64_t*)ssig, n, g, start, spos, sid, bad, ws, st));
  CSO_TRY(cells_density(g, spos, (int)n, (uint32_t)p.b2, p.include_self, ssig, nullptr, ws, st));
  k_unsort<<<CL(cdiv(n, 256)), 256, 0, st>>>(spos, ssig, (int)n, sigma);
  CSO_CUDA(cudaGetLastError());
  int hbad[2] = {0, 0};
  CSO_CUDA(cudaMemcpyAsync(hbad, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CSO_CUDA(cudaStreamSynchronize(st));
  if (hbad[0]) {
    cso_set_error("cso_density_static: positions outside [0, 2^21)");
    return CSO_ERR_ARG;
  }
  if (hbad[1]) {
    cso_set_error("cso_density_static: a bounded device wait gave up");
    return CSO_ERR_TIMEOUT;
  }
  return CSO_OK;
}
