// Shared host/device helpers of liblowrank: error plumbing, workspace arena,
// device status word, small warp utilities.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/lowrank.h"

namespace lr {

// ------------------------------------------------------------------ errors
struct Error {
  lr_status st;
  std::string msg;
};

#define LR_CHECK_CUDA(expr)                                                          \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw ::lr::Error{LR_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define LR_REQUIRE(cond, code, text)                         \
  do {                                                       \
    if (!(cond)) throw ::lr::Error{(code), std::string(text)}; \
  } while (0)

// Every kernel launch site of the library ends with LR_LAUNCH_CHECK(), which
// also counts the launch (reported by lr_kernel_launches).
extern std::atomic<uint64_t> g_kernel_launches;
#define LR_LAUNCH_CHECK()                                              \
  do {                                                                 \
    ::lr::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);   \
    LR_CHECK_CUDA(cudaGetLastError());                                 \
  } while (0)

// ------------------------------------------------------------- workspace
// Bump allocator over the caller's workspace.  With measure = true it only
// records the peak offset (used by lr_workspace_size to size a workspace by
// running the same allocation sequence without launching anything).
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  size_t peak = 0;
  bool measure = false;
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    size_t at = off;
    off += bytes;
    if (off > peak) peak = off;
    if (measure) return reinterpret_cast<T*>(uintptr_t(256) + at);  // never dereferenced
    if (off > cap) throw Error{LR_ERR_NOMEM, "workspace too small: need at least " + std::to_string(off) + " bytes"};
    return reinterpret_cast<T*>(base + at);
  }
};

// Restores the arena offset when a helper's temporaries go out of scope.
struct ArenaScope {
  Arena& a;
  size_t mark;
  explicit ArenaScope(Arena& ar) : a(ar), mark(ar.off) {}
  ~ArenaScope() { a.off = mark; }
};

// ---------------------------------------------------------- device status
// Device-side failures set the first nonzero code (atomicCAS keeps the first).
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

inline int ceil_div(int64_t a, int64_t b) { return int((a + b - 1) / b); }
// Grid (256-thread blocks) for an element-wise pass over a rows x cols
// column-major matrix: x strides over rows, y over columns, so a thread
// needs no division to find its element.
inline dim3 grid_2d(int64_t rows, int64_t cols) {
  const int64_t gx = (rows + 255) / 256;
  return dim3(unsigned(gx < 64 ? gx : 64), unsigned(cols < 1024 ? cols : 1024), 1);
}

// Device properties needed for grid sizing (cached per device).
struct DevInfo {
  int sms = 0;
  int max_smem_optin = 0;
};
DevInfo dev_info(int device);

}  // namespace lr
