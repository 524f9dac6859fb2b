// lr_sketch_range_static: the range view Y = A X without any allocation.
//
// Some callers cannot call cudaMalloc at all: a host program whose own pool
// allocator has reserved the device's memory, or one that cannot accept the
// device-wide synchronisation a cudaMalloc may imply.  Such callers cannot
// create an lr_handle (lr_create allocates a status word) or hand the library
// a workspace, so they cannot use lr_sketch.  This entry point serves them:
// the only scratch the range view needs -- the BF16 copy of the thin operand
// X that the tensor-core kernel reads through TMA, plus a status word -- lives
// in a file-scope __device__ array that the CUDA runtime reserves on a GPU
// when this code is loaded there (see below) and holds until the process
// exits.
//
// The array's host-side name is only a stand-in for the device symbol, so the
// device address is obtained once per device with cudaGetSymbolAddress (with
// that device current) and passed to the kernels.  The first call on a device
// performs that set-up, so make that first call before any stream capture
// begins.  Every call shares the one array: calls whose executions
// overlap on the GPU (different streams, or different host threads on the
// same device) race on it and must be serialised by the caller.  A later call
// overwrites what an earlier call left there; the status word is cleared at
// the start of every call and read back by lr_sketch_range_static_status.
//
// With lazy module loading (the CUDA default since 12.2) the array and this
// file's kernels are brought onto a device by the first call there, not when
// the library is loaded: that first call is where the runtime reserves the
// 4 MiB, so a caller whose pool later claims the device's memory makes it at
// start-up (or runs with CUDA_MODULE_LOADING=EAGER).
//
// For an F32 A the view runs on the SIMT GEMM (no scratch at all) and agrees
// with lr_sketch's 3xTF32 tensor-core view to within the view tolerance, not
// bit for bit; for a BF16 A it runs lr_sketch's own kernel.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace lr {
namespace {

// BF16 copy of X (ld = n rounded up to 8, ell columns) + status word.
constexpr size_t kStaticScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr size_t kStatusOffset = kStaticScratchBytes - 256;

static __device__ __align__(256) unsigned char g_sketch_scratch[kStaticScratchBytes];

struct DeviceScratch {
  std::once_flag once;
  void* ptr = nullptr;
  cudaError_t err = cudaSuccess;
};
DeviceScratch g_scratch[64];

void* scratch_for(int device) {
  LR_REQUIRE(device >= 0 && device < 64, LR_ERR_INVALID_ARG, "device index out of range");
  DeviceScratch& d = g_scratch[device];
  std::call_once(d.once, [&] {
    // the current device is `device` here (set by the caller below)
    d.err = cudaGetSymbolAddress(&d.ptr, g_sketch_scratch);
  });
  LR_REQUIRE(d.err == cudaSuccess && d.ptr != nullptr, LR_ERR_CUDA,
             std::string("cudaGetSymbolAddress(scratch) failed: ") + cudaGetErrorString(d.err));
  return d.ptr;
}

}  // namespace
}  // namespace lr

extern "C" lr_status lr_sketch_range_static(const lr_mat* A, const lr_mat* X, lr_mat* Y, void* stream) {
  using namespace lr;
  try {
    LR_REQUIRE(A && X && Y && A->data && X->data && Y->data, LR_ERR_INVALID_ARG, "NULL argument");
    LR_REQUIRE(A->dtype == LR_F32 || A->dtype == LR_BF16, LR_ERR_DTYPE, "A must be F32 or BF16");
    LR_REQUIRE(A->col_major == 0 && A->ld >= A->cols && A->rows >= 1 && A->cols >= 1, LR_ERR_SHAPE, "bad A");
    const size_t esz = A->dtype == LR_BF16 ? 2 : 4;
    LR_REQUIRE((reinterpret_cast<uintptr_t>(A->data) & 15) == 0 && (A->ld * int64_t(esz)) % 16 == 0,
               LR_ERR_ALIGNMENT, "A must be 16-byte aligned with a 16-byte row stride");
    LR_REQUIRE(X->dtype == LR_F32 && X->col_major == 1 && X->rows == A->cols && X->ld >= X->rows && X->cols >= 1,
               LR_ERR_SHAPE, "X must be F32 column-major n x ell");
    LR_REQUIRE(Y->dtype == LR_F32 && Y->col_major == 1 && Y->rows == A->rows && Y->cols == X->cols &&
                   Y->ld >= Y->rows,
               LR_ERR_SHAPE, "Y must be F32 column-major m x ell");
    const int64_t m = A->rows, n = A->cols, ell = X->cols;
    LR_REQUIRE(ell <= 256, LR_ERR_UNSUPPORTED, "ell must be <= 256");
    const int64_t ldx = (n + 7) / 8 * 8;
    if (A->dtype == LR_BF16) {
      LR_REQUIRE(size_t(ldx) * size_t(ell) * 2 <= kStatusOffset, LR_ERR_UNSUPPORTED,
                 "n x ell too large for the 4 MiB static scratch (BF16 copy of X needs ceil8(n) * ell * 2 bytes)");
    }
    int device = 0;
    LR_CHECK_CUDA(cudaGetDevice(&device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(scratch_for(device));
    int* status = reinterpret_cast<int*>(base + kStatusOffset);
    LR_CHECK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    float* y = static_cast<float*>(Y->data);
    zero_f32(y, m, ell, Y->ld, s);  // partial tiles are added into Y
    if (A->dtype == LR_BF16) {
      auto* xb = reinterpret_cast<__nv_bfloat16*>(base);
      f32_to_bf16(static_cast<const float*>(X->data), X->ld, xb, nullptr, ldx, n, ell, s);
      ViewBf16Args a;
      a.device = device;
      a.mode = 0;
      a.A = static_cast<const __nv_bfloat16*>(A->data);
      a.lda = A->ld;
      a.row0 = 0;
      a.rows = m;
      a.n = n;
      a.B = xb;
      a.ldb = ldx;
      a.ell = int(ell);
      a.out = y;
      a.ldo = Y->ld;
      a.status = status;
      view_bf16(a, s);
    } else {
      GemmArgs g;
      g.mode = GEMM_ATOMIC_F32;
      g.M = m; g.N = ell; g.K = n; g.ta = true;
      g.A = static_cast<const float*>(A->data); g.lda = A->ld;
      g.B = static_cast<const float*>(X->data); g.ldb = X->ld;
      g.C = y; g.ldc = Y->ld;
      g.split_k = split_for(m, ell, n, dev_info(device).sms);
      sgemm(g, s);
    }
    return LR_OK;
  } catch (const Error& e) {
    return e.st;
  }
}

extern "C" lr_status lr_sketch_range_static_status(void* stream, int* device_status) {
  using namespace lr;
  try {
    LR_REQUIRE(device_status, LR_ERR_INVALID_ARG, "device_status is NULL");
    int device = 0;
    LR_CHECK_CUDA(cudaGetDevice(&device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char* base = static_cast<const char*>(scratch_for(device));
    int v = 0;
    LR_CHECK_CUDA(cudaMemcpyAsync(&v, base + kStatusOffset, sizeof(int), cudaMemcpyDeviceToHost, s));
    LR_CHECK_CUDA(cudaStreamSynchronize(s));
    *device_status = v;
    return LR_OK;
  } catch (const Error& e) {
    return e.st;
  }
}
