// Internal declarations of the CompaSO CUDA library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cso.h"

#define CSO_BOX (1 << 21)
#define CSO_HALF (1 << 20)

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
void cso_set_error(const char* fmt, ...);
#define CSO_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      cso_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return CSO_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)
#define CSO_CUDA_VOID(call) (void)(call)
#define CSO_TRY(expr)          \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != CSO_OK) return rc_; \
  } while (0)

static inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// streaming multiprocessors of the current device (read once per device)
int cso_sm_count();

// every kernel launch of the library passes its grid size through CL(), which
// counts the calling thread's launches for cso_last_stats
extern thread_local long long g_cso_launches;
template <class T>
static inline T CL(T grid) {
  ++g_cso_launches;
  return grid;
}

// ---------------------------------------------------------------------------
// workspace: bump allocator over one device buffer owned by the context
// ---------------------------------------------------------------------------
struct Workspace {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  size_t peak = 0;
  size_t need = 0;  // bytes requested during a sizing pass
  bool sizing = false;
  int* err = nullptr;  // device word set by a kernel whose bounded wait gave up (CSO_ERR_TIMEOUT)
  void* take(size_t bytes) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + bytes;
    if (off > peak) peak = off;
    if (sizing || off > cap) {
      need = off > need ? off : need;
      return nullptr;
    }
    return base + o;
  }
  template <class T>
  T* get(size_t count) {
    return (T*)take(sizeof(T) * (count ? count : 1));
  }
};

// ---------------------------------------------------------------------------
// primitives (scan_sort.cu)
// ---------------------------------------------------------------------------
// exclusive scan of n uint32 values in place; *total (device, may be null)
// receives the sum.  Scratch comes from ws.
int scan_u32(uint32_t* data, long long n, uint32_t* total, Workspace& ws, cudaStream_t st);

// Stable LSD radix sort of (key, val) pairs by the low `bits` bits of the
// 128-bit key (hi:lo).  Sorted output ends in (*khi, *klo, *val) which point
// to either the input or the alternate buffers.
int radix_sort_128(uint64_t** khi, uint64_t** klo, uint32_t** val, uint64_t* khi_alt, uint64_t* klo_alt,
                   uint32_t* val_alt, long long n, int bits, Workspace& ws, cudaStream_t st);

// Stable LSD radix sort of (key32, val) pairs by the low `bits` bits.
int radix_sort_32(uint32_t** key, uint32_t** val, uint32_t* key_alt, uint32_t* val_alt, long long n, int bits,
                  Workspace& ws, cudaStream_t st);

static inline int bit_length_u64(unsigned long long v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}
