// Gradient step that allocates nothing: the split-K partial sums of the
// A-pass live in a fixed array in the library's own device memory instead of
// a cudaMallocAsync buffer.
//
// This is for callers that cannot allocate device memory at the time they
// call: code inside an allocator callback or a custom memory pool that must
// not recurse into the allocator, code that may only allocate at start-up,
// or processes whose memory budget is fixed up front.  The array (1.25 MiB)
// is reserved on every GPU where the library's device code is loaded and is
// held until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Nothing in it needs to start at zero: each launch writes every
// partial row it later reads.  Calls whose kernels overlap on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
//
// The device address of the array is looked up on the first call on each
// device and cached for the life of the process; a cudaDeviceReset of that
// device invalidates it (the module, and with it the array, is reloaded at a
// new address), so the entry point must not be called after such a reset.
#include <cfloat>
#include <mutex>

#include "internal.h"

namespace mihs {
namespace {

constexpr int kNoAllocMaxPartials = 160;   // ≥ one partial per SM on GB300 (152)
constexpr size_t kNoAllocFloats = (size_t)kNoAllocMaxPartials * kMaxD;  // 1.25 MiB

static __device__ __align__(256) float g_gradient_scratch[kNoAllocFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (the host-side name of a __device__ variable is not a device address).
int scratch_for_current_device(float** out) {
  int dev = 0;
  MIHS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("mihs_gradient_noalloc: device ordinal %d beyond %d", dev, kMaxDevices);
    return MIHS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_gradient_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error("mihs_gradient_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return MIHS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MIHS_OK;
}

}  // namespace
}  // namespace mihs

using namespace mihs;

extern "C" int mihs_gradient_noalloc(const float* A, int64_t n, int64_t d, int64_t lda,
                                     const float* b, const float* x, double lambda, float* g,
                                     void* stream) {
  set_error("");
  MIHS_ARG(A != nullptr && b != nullptr && x != nullptr && g != nullptr,
           "mihs_gradient_noalloc: null pointer");
  MIHS_ARG(d >= 1 && d <= kMaxD, "mihs_gradient_noalloc: d=%lld outside [1, %d]", (long long)d, kMaxD);
  MIHS_ARG(n >= 1 && n < (1LL << 31), "mihs_gradient_noalloc: n=%lld outside [1, 2^31)", (long long)n);
  MIHS_ARG(lda >= d && lda % 4 == 0, "mihs_gradient_noalloc: lda=%lld must be >= d and a multiple of 4",
           (long long)lda);
  MIHS_ARG((reinterpret_cast<uintptr_t>(A) & 15u) == 0,
           "mihs_gradient_noalloc: matrix pointer must be 16-byte aligned");
  MIHS_ARG(lambda >= 0.0 && lambda <= (double)FLT_MAX,
           "mihs_gradient_noalloc: lambda must be in [0, FLT_MAX] (the kernel computes in fp32)");
  const int P = apass_num_partials(n, d);
  const size_t need = (size_t)P * (size_t)apass_dpad(d);
  if (need > kNoAllocFloats) {
    set_error("mihs_gradient_noalloc: needs %zu floats of scratch (%d partial rows x %lld), "
              "more than the fixed %zu", need, P, (long long)apass_dpad(d), kNoAllocFloats);
    return MIHS_ERR_UNSUPPORTED;
  }
  float* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = launch_apass_partial(A, n, d, lda, b, x, scratch, nullptr, s);
  if (rc) return rc;
  return launch_apass_finalize(scratch, P, d, x, (float)lambda, g, nullptr, s);
}
