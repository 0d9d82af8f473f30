// Shared device helpers and host plumbing of libmihs.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <string>

#include "../../include/mihs.h"

namespace mihs {

// ---------------------------------------------------------------- host side
// Last error message of this host thread (mihs_last_error()).
void set_error(const char* fmt, ...);
// Counts kernel launches for mihs_launch_count().
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int num_sms();                // SM count of the current device (cached per device)

#define MIHS_CUDA_TRY(expr)                                                        \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      ::mihs::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,               \
                        cudaGetErrorString(_e));                                   \
      return _e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;       \
    }                                                                              \
  } while (0)

#define MIHS_CHECK_LAUNCH()                                                        \
  do {                                                                             \
    cudaError_t _e = cudaGetLastError();                                           \
    if (_e != cudaSuccess) {                                                       \
      ::mihs::set_error("%s:%d: kernel launch: %s", __FILE__, __LINE__,           \
                        cudaGetErrorString(_e));                                   \
      return MIHS_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

#define MIHS_ARG(cond, ...)                                                        \
  do {                                                                             \
    if (!(cond)) {                                                                 \
      ::mihs::set_error(__VA_ARGS__);                                              \
      return MIHS_ERR_INVALID_ARG;                                                 \
    }                                                                              \
  } while (0)

constexpr int kMaxD = 2048;

inline int64_t round_up(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

// Control block of one solve, in device memory (written by the kernels).
struct SolveCtl {
  int done;          // 1 once the solve has stopped: later kernels return at once
  int outer;         // momentum steps taken
  int inner_total;   // AAb passes summed
  int status;        // MIHS_OK / MIHS_NOT_CONVERGED / MIHS_ERR_NUMERIC
  int max_outer;
  int gnorm0_known;  // ‖Aᵀb‖ already in gnorm0
  float tol;         // stop when ‖g‖ ≤ tol·‖Aᵀb‖
  float gnorm0;      // ‖Aᵀb‖
  float gnorm;       // ‖g‖ of the current x
  int phase;         // refinement solves: 0 = plain fp32 gradient, 1 = compensated
  float switch_tol;  // switch to phase 1 once ‖g‖ ≤ switch_tol·‖Aᵀb‖ ...
  float gmin;        // ... or once ‖g‖ has set no new minimum (gmin) for
  int stall;         //     three steps (stall counts them)
  // Refinement (phase 1): a compensated refresh fixes g(x_ref); the steps
  // after it take g(x) = g(x_ref) − H(x − x_ref) from an fp32 pass.
  int corr;          // corrections enabled (cleared when a cycle gains < 4×)
  int refresh;       // the next gradient is a compensated refresh
  int since;         // correction steps since the last refresh
  float gref;        // ‖g‖ at the last refresh
};

// Bookkeeping of one outer step of a refinement solve, by the one thread
// that writes the control block, once the step's ‖g‖ (θ₁) is known; phase,
// refresh and corr are the control block's values when the step began.
//   phase 0: plain fp32 steps until ‖g‖ ≤ switch_tol·g0 or no new minimum
//            for three steps (the fp32 floor), then phase 1 with a refresh.
//   phase 1, corrections on: after a refresh, fp32 corrections until ‖g‖
//            has set no new minimum for two steps (the correction's own
//            rounding floor, ∝ ‖x − x_ref‖; the heavy ball's residual is not
//            monotone), reaches the tolerance (only a refresh may stop the
//            solve) or 10 steps; corrections are turned off for good once a
//            whole cycle gained less than 4×.  gmin / stall track the cycle.
__device__ __forceinline__ void refine_step_update(SolveCtl* c, int phase, int refresh, int corr, float theta1,
                                                   float g0, float tol, float switch_tol) {
  if (phase == 0) {
    const float gmin = c->gmin;
    const int stall = theta1 < gmin ? 0 : c->stall + 1;
    if (theta1 < gmin) c->gmin = theta1;
    c->stall = stall;
    if (theta1 <= switch_tol * g0 || stall >= 3) {
      c->phase = 1;
      c->refresh = 1;
    }
  } else if (corr) {
    if (refresh) {
      const int on = (c->gref < 3.0e38f && theta1 > 0.25f * c->gref) ? 0 : 1;
      c->corr = on;
      c->gref = theta1;
      c->since = 0;
      c->gmin = theta1;
      c->stall = 0;
      c->refresh = on ? 0 : 1;
    } else {
      const int since = c->since + 1;
      c->since = since;
      const float gmin = c->gmin;
      const int stall = theta1 < gmin ? 0 : c->stall + 1;
      if (theta1 < gmin) c->gmin = theta1;
      c->stall = stall;
      if ((tol > 0.f && theta1 <= tol * g0) || stall >= 2 || since >= 10) c->refresh = 1;
    }
  }
}

// Which gradient a step of a refinement solve computes: 0 the plain fp32
// pass (phase 0), 1 a compensated refresh, 2 an fp32 correction from the
// last refresh.  Kernels launched with gate k run only when this is k.
__host__ __device__ inline int ctl_gate(const SolveCtl* c) {
  return c->phase == 0 ? 0 : (c->refresh ? 1 : 2);
}

// ------------------------------------------------------------- device side
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0,c1,c2,c3) → (hi(M1·c2)⊕c1⊕k0, lo(M1·c2), hi(M0·c0)⊕c3⊕k1, lo(M0·c0)),
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Box–Muller on 24-bit uniforms: u1 = (⌊a/2⁸⌋+1)·2⁻²⁴ ∈ (0,1] and
// u2 = ⌊b/2⁸⌋·2⁻²⁴ ∈ [0,1) are exact in fp32; r = √(−2 ln u1),
// (z0, z1) = (r cos 2πu2, r sin 2πu2).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
  const float u1 = (float)((a >> 8) + 1u) * 0x1p-24f;
  const float u2 = (float)(b >> 8) * 0x1p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

enum : uint32_t { kTagGaussian = 0, kTagCountSketch = 1, kTagSrhtSigns = 2, kTagSrhtRows = 3, kTagHutchinson = 4 };

}  // namespace mihs

// ------------------------------------------------- async copies and mbarriers
namespace mihs {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the async proxy (bulk copies).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most
// `limit_ns` nanoseconds of wall time; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0 && global_timer_ns() - t0 > limit_ns) return false;
  }
}

// Bulk global → shared copy (16-byte aligned addresses, size a multiple of
// 16) that signals `bar` with its byte count on completion.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy ones (bulk copies, TMA, tensor core reads).
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tiled 2D TMA load of the box at column x, row y of `map` into shared memory
// (x·element size a multiple of 16 bytes); completes on `bar` with the box's
// full byte count, out-of-bounds elements filled with zeros.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Named barrier over `nthreads` threads (a multiple of 32).
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: far beyond any legitimate wait

}  // namespace mihs
