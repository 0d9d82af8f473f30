// Host → device copy by the SMs (mihs_copy_to_device).  On a GPU joined to
// its CPU by a coherent link (NVLink-C2C on Grace systems) kernels can load
// pinned host memory directly; with enough 16-byte loads in flight per SM
// this moves data faster than one copy engine, and a few SMs suffice, so the
// copy can run beside compute on other streams.  Anything the kernel cannot
// take (pageable or unaligned memory) goes to cudaMemcpyAsync.
#include <cstdlib>

#include "internal.h"

namespace mihs {
namespace {

constexpr int kCopyThreads = 512;
constexpr int kCopyUnroll = 8;  // 16-byte loads in flight per thread

__global__ void __launch_bounds__(kCopyThreads) h2d_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                           size_t n16) {
  const size_t chunk = (size_t)kCopyThreads * kCopyUnroll;
  for (size_t base = (size_t)blockIdx.x * chunk + threadIdx.x; base < n16; base += (size_t)gridDim.x * chunk) {
    uint4 v[kCopyUnroll];
#pragma unroll
    for (int k = 0; k < kCopyUnroll; ++k) {
      const size_t i = base + (size_t)k * kCopyThreads;
      if (i < n16) v[k] = __ldg(src + i);
    }
#pragma unroll
    for (int k = 0; k < kCopyUnroll; ++k) {
      const size_t i = base + (size_t)k * kCopyThreads;
      if (i < n16) __stcs(dst + i, v[k]);
    }
  }
}

int copy_blocks() {
  const char* e = std::getenv("MIHS_H2D_BLOCKS");
  const int v = e != nullptr ? std::atoi(e) : 0;
  return v > 0 ? v : num_sms();
}

}  // namespace
}  // namespace mihs

using namespace mihs;

int mihs_copy_to_device(void* dst, const void* src, int64_t bytes, void* stream) {
  set_error("");
  MIHS_ARG(bytes >= 0, "mihs_copy_to_device: bytes %lld < 0", (long long)bytes);
  if (bytes == 0) return MIHS_OK;
  MIHS_ARG(dst != nullptr && src != nullptr, "mihs_copy_to_device: null pointer");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaPointerAttributes as = {}, ad = {};
  MIHS_CUDA_TRY(cudaPointerGetAttributes(&as, src));
  MIHS_CUDA_TRY(cudaPointerGetAttributes(&ad, dst));
  MIHS_ARG(ad.type == cudaMemoryTypeDevice || ad.type == cudaMemoryTypeManaged,
           "mihs_copy_to_device: dst is not device memory");
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0;
  const void* dsrc = as.type == cudaMemoryTypeHost ? as.devicePointer : nullptr;
  if (dsrc == nullptr || !aligned || dsrc != src) {
    MIHS_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDefault, s));
    return MIHS_OK;
  }
  const size_t n16 = (size_t)bytes / 16, tail = (size_t)bytes % 16;
  if (n16 > 0) {
    const size_t chunk = (size_t)kCopyThreads * kCopyUnroll;
    size_t grid = (n16 + chunk - 1) / chunk;
    if (grid > (size_t)copy_blocks()) grid = (size_t)copy_blocks();
    h2d_kernel<<<(unsigned)grid, kCopyThreads, 0, s>>>(static_cast<const uint4*>(dsrc), static_cast<uint4*>(dst), n16);
    MIHS_CHECK_LAUNCH();
    count_launch();
  }
  if (tail > 0)
    MIHS_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(dst) + n16 * 16, static_cast<const char*>(src) + n16 * 16, tail,
                                  cudaMemcpyDefault, s));
  return MIHS_OK;
}

int mihs_copy_to_device_dma(void* dst, const void* src, int64_t bytes, void* stream) {
  set_error("");
  MIHS_ARG(bytes >= 0, "mihs_copy_to_device_dma: bytes %lld < 0", (long long)bytes);
  if (bytes == 0) return MIHS_OK;
  MIHS_ARG(dst != nullptr && src != nullptr, "mihs_copy_to_device_dma: null pointer");
  cudaPointerAttributes ad = {};
  MIHS_CUDA_TRY(cudaPointerGetAttributes(&ad, dst));
  MIHS_ARG(ad.type == cudaMemoryTypeDevice || ad.type == cudaMemoryTypeManaged,
           "mihs_copy_to_device_dma: dst is not device memory");
  MIHS_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDefault, static_cast<cudaStream_t>(stream)));
  return MIHS_OK;
}
