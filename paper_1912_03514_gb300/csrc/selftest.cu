// Failure-detection self-test (mihs_selftest_wait): the library's bounded
// waits, run on conditions that nothing satisfies with a short limit, must
// return and report a timeout instead of hanging.  Uses the same helpers as
// the production kernels (mbar_wait, grid_barrier); nothing here faults.
#include "common.cuh"
#include "grid_sync.cuh"

namespace mihs {
namespace {

// An mbarrier initialised for one arrival that never comes; thread 0 waits
// on its first phase.
__global__ void selftest_mbar_kernel(uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  const bool ok = mbar_wait(&bar, 0u, limit_ns);
  *status = ok ? MIHS_OK : MIHS_ERR_TIMEOUT;
}

// Two blocks share a zeroed barrier word; block 1 leaves without arriving,
// so block 0's wait for the last arrival cannot end before its limit.
__global__ void selftest_grid_kernel(unsigned int* word, uint64_t limit_ns, int* status) {
  __shared__ int s_ok;
  if (blockIdx.x != 0) return;
  GridBarrier gb = {};
  if (threadIdx.x == 0) grid_barrier_init(gb, word);
  const bool ok = grid_barrier(gb, &s_ok, limit_ns);
  if (threadIdx.x == 0) *status = ok ? MIHS_OK : MIHS_ERR_TIMEOUT;
}

// Launches the chosen wait on buf ([0] status, [1] barrier word) and reads
// the status back.
int run_wait(int which, int64_t limit_ns, int* buf, int* host, cudaStream_t s) {
  MIHS_CUDA_TRY(cudaMemsetAsync(buf, 0xff, sizeof(int), s));  // status −1 until the kernel writes it
  MIHS_CUDA_TRY(cudaMemsetAsync(buf + 1, 0, sizeof(int), s));
  if (which == 0) {
    selftest_mbar_kernel<<<1, 32, 0, s>>>((uint64_t)limit_ns, buf);
  } else {
    selftest_grid_kernel<<<2, 32, 0, s>>>(reinterpret_cast<unsigned int*>(buf + 1), (uint64_t)limit_ns, buf);
  }
  MIHS_CHECK_LAUNCH();
  count_launch();
  MIHS_CUDA_TRY(cudaMemcpyAsync(host, buf, sizeof(int), cudaMemcpyDeviceToHost, s));
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  return MIHS_OK;
}

}  // namespace
}  // namespace mihs

using namespace mihs;

int mihs_selftest_wait(int which, int64_t limit_ns, int* status, void* stream) {
  set_error("");
  MIHS_ARG(which == 0 || which == 1, "mihs_selftest_wait: unknown wait %d", which);
  MIHS_ARG(limit_ns >= 1000000 && limit_ns <= 10000000000ll, "mihs_selftest_wait: limit %lld ns out of range",
           (long long)limit_ns);
  MIHS_ARG(status != nullptr, "mihs_selftest_wait: null status");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* buf = nullptr;  // [0] status, [1] barrier word
  const cudaError_t e = cudaMalloc(&buf, 2 * sizeof(int));
  if (e != cudaSuccess) {
    set_error("mihs_selftest_wait: cudaMalloc: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
  }
  int host = -1;
  const int rc = run_wait(which, limit_ns, buf, &host, s);
  cudaFree(buf);
  if (rc == MIHS_OK) *status = host;
  return rc;
}
