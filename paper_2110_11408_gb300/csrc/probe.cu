// Micro-benchmarks of the pipes the pair kernels run on, so that their
// rooflines are taken against measured rates rather than unit counts.
//
//   alu  : integer add and xor chains (the ALU pipe: IADD3 / LOP3 class)
//   imad : integer multiply-add chains (IMAD), a <- a * a + k
//   lds  : 128-bit shared-memory loads that every lane of a warp reads from
//          the same address (the broadcast the density and FoF tiles use)
//
// Every thread keeps eight independent chains, so the rate is bound by the
// pipe, not by the latency of one chain.  Results are written out so that no
// chain is dead code.
#include "cso_internal.cuh"

namespace {

constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(256) k_probe_alu(uint32_t k0, uint32_t k1, int iters, uint32_t* out) {
  uint32_t a[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = threadIdx.x * (c + 3) + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = (a[c] + k0) ^ k1;  // two lane-ops
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_imad(uint32_t k0, uint32_t k1, int iters, uint32_t* out) {
  uint32_t a[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = threadIdx.x * (c + 3) + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = a[c] * a[c] + k1;  // one lane-op (not foldable)
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_lds(int iters, uint32_t* out) {
  __shared__ int4 tile[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  tile[w][lane] = make_int4(lane, lane * 3, lane * 5, lane * 7);
  __syncwarp();
  uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 32; k += 4) {  // every lane reads the same element
      const int4 a = tile[w][(k + i) & 31], b = tile[w][(k + i + 1) & 31];
      const int4 c = tile[w][(k + i + 2) & 31], d = tile[w][(k + i + 3) & 31];
      s0 += (uint32_t)(a.x ^ a.w);
      s1 += (uint32_t)(b.y ^ b.z);
      s2 += (uint32_t)(c.x ^ c.z);
      s3 += (uint32_t)(d.y ^ d.w);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s0 ^ s1 ^ s2 ^ s3;
}

// device time (ms) of one launch, after one untimed launch
template <class F>
int time_launch(F launch, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  CSO_CUDA(cudaEventCreate(&e0));
  CSO_CUDA(cudaEventCreate(&e1));
  launch();
  CSO_CUDA(cudaGetLastError());
  CSO_CUDA(cudaEventRecord(e0, st));
  launch();
  CSO_CUDA(cudaEventRecord(e1, st));
  CSO_CUDA(cudaEventSynchronize(e1));
  CSO_CUDA(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return CSO_OK;
}

}  // namespace

extern "C" int cso_probe_peaks(int device, double* out, int n) {
  if (!out || n < 3) {
    cso_set_error("cso_probe_peaks needs room for 3 results");
    return CSO_ERR_ARG;
  }
  CSO_CUDA(cudaSetDevice(device));
  int sms = 0;
  CSO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int blocks = sms * 8, threads = 256, iters = 4096;
  uint32_t* buf = nullptr;
  CSO_CUDA(cudaMalloc((void**)&buf, sizeof(uint32_t) * blocks * threads));
  cudaStream_t st = nullptr;
  const double lanes = (double)blocks * threads;
  float ms = 0;
  int rc = time_launch([&] { k_probe_alu<<<blocks, threads, 0, st>>>(0x9e3779b9u, 0x85ebca6bu, iters, buf); }, st, &ms);
  if (rc == CSO_OK) out[0] = lanes * iters * 8 * PROBE_CHAINS * 2 / (ms * 1e-3) / 1e12;
  if (rc == CSO_OK)
    rc = time_launch([&] { k_probe_imad<<<blocks, threads, 0, st>>>(0x2545f491u, 0x9e3779b9u, iters, buf); }, st, &ms);
  if (rc == CSO_OK) out[1] = lanes * iters * 8 * PROBE_CHAINS / (ms * 1e-3) / 1e12;
  if (rc == CSO_OK) rc = time_launch([&] { k_probe_lds<<<blocks, threads, 0, st>>>(iters, buf); }, st, &ms);
  // bytes delivered to the lanes: 16 per lane per load
  if (rc == CSO_OK) out[2] = lanes * iters * 32 * 16.0 / (ms * 1e-3) / 1e12;
  cudaFree(buf);
  return rc;
}
