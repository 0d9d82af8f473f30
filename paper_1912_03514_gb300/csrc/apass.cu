// Gradient step of Algorithm 1:  g = Aᵀ(b − Ax) − λx.
//
// One streaming pass over A (the only O(nd) work per iteration, "4nd + 3d" in
// Algorithm 1).  Each row's residual r_i = b_i − A_i·x is formed and r_i·A_i
// accumulated as soon as the row arrives, so A is read exactly once and no
// grid-wide synchronisation happens inside the pass (the paper's point that
// M-IHS needs no inner products in the outer loop).  Each block owns a
// contiguous row range; its warps' partial d-vectors are summed in smem and
// written as one split-K partial.  A second small kernel sums the partials in
// a fixed order (deterministic result) and subtracts λx.
#include <cstdlib>

#include "internal.h"

namespace mihs {

namespace {

constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;  // + one producer warp
constexpr size_t kRingBudget = 180 * 1024;

// Library-wide device error word (a bounded wait that ran out), read and
// cleared by mihs_device_status().
__device__ int g_apass_error = 0;

// One block per SM streams a contiguous row range of A through a ring of
// shared-memory stages: a producer lane issues bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on a "full" mbarrier) up to
// `stages` stages ahead; eight consumer warps each take RW rows of a stage,
// form r_i = b_i − A_i·x with a warp all-reduce and accumulate r_i·A_i into
// registers (lane ℓ owns columns 4ℓ + 128c), then release the stage on its
// "empty" mbarrier.  Bytes in flight per SM are set by the ring (up to
// ~180 KB), not by registers.
template <int CH, int RW>
__global__ void __launch_bounds__(kThreads, 1)
apass_partial_kernel(const float* __restrict__ A, int n, int d, long long lda,
                     const float* __restrict__ b, const float* __restrict__ x,
                     float* __restrict__ partials, int dpad, int rows_per_cta, int stages,
                     SolveCtl* __restrict__ ctl, int gate) {
  constexpr int NC = kConsumerWarps, R = NC * RW;
  constexpr bool XS = CH > 8;  // wide rows: keep x in smem instead of registers
  if (ctl != nullptr && (ctl->done || (gate >= 0 && ctl_gate(ctl) != gate))) return;  // uniform
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)stages * R * dpad);
  uint64_t* empty = full + stages;
  float* xsm = reinterpret_cast<float*>(empty + stages);  // CH·128 floats when XS
  __shared__ int issued;  // stages the producer has issued (for the abort path)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min((long long)n, r0 + rows_per_cta);
  const int nst = r1 > r0 ? (int)((r1 - r0 + R - 1) / R) : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
    }
    issued = 0;
    fence_mbar_init();
  }
  if (XS)
    for (int j = threadIdx.x; j < CH * 128; j += kThreads) xsm[j] = (x != nullptr && j < d) ? x[j] : 0.f;
  __syncthreads();

  if (warp == NC) {  // ---------------------------------------------- producer
    if (lane == 0) {
      const uint32_t row_bytes = (uint32_t)dpad * 4u;
      const bool contiguous = lda == (long long)dpad;
      for (int it = 0; it < nst; ++it) {
        const int s = it % stages;
        const uint32_t ph = (uint32_t)(it / stages) & 1u;
        if (it >= stages && !mbar_wait(&empty[s], ph ^ 1u, kWaitLimitNs)) {
          atomicExch(&g_apass_error, MIHS_ERR_TIMEOUT);
          break;
        }
        const long long row0 = r0 + (long long)it * R;
        const int rows = (int)min((long long)R, r1 - row0);
        float* dst = ring + (size_t)s * R * dpad;
        mbar_arrive_expect_tx(&full[s], (uint32_t)rows * row_bytes);
        if (contiguous) {
          bulk_copy_g2s(dst, A + row0 * lda, (uint32_t)rows * row_bytes, &full[s]);
        } else {
          for (int r = 0; r < rows; ++r)
            bulk_copy_g2s(dst + (size_t)r * dpad, A + (row0 + r) * lda, row_bytes, &full[s]);
        }
        *(volatile int*)&issued = it + 1;
      }
    }
    return;
  }

  // ---------------------------------------------------------------- consumers
  float4 xr[XS ? 1 : CH], acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (XS) continue;
    const int col = 4 * lane + 128 * c;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x != nullptr && col < d) {
      v.x = x[col];
      if (col + 1 < d) v.y = x[col + 1];
      if (col + 2 < d) v.z = x[col + 2];
      if (col + 3 < d) v.w = x[col + 3];
    }
    xr[XS ? 0 : c] = v;
  }
  const float4* xs4 = reinterpret_cast<const float4*>(xsm);
  int consumed = 0;
  for (int it = 0; it < nst; ++it) {
    const int s = it % stages;
    const uint32_t ph = (uint32_t)(it / stages) & 1u;
    const long long rw0 = r0 + (long long)it * R + (long long)warp * RW;
    float bv[RW];
#pragma unroll
    for (int k = 0; k < RW; ++k) bv[k] = (b != nullptr && rw0 + k < r1) ? __ldg(b + rw0 + k) : 0.f;
    if (!mbar_wait(&full[s], ph, kWaitLimitNs)) {
      atomicExch(&g_apass_error, MIHS_ERR_TIMEOUT);
      break;
    }
    const float* rows = ring + ((size_t)s * R + (size_t)warp * RW) * dpad;
#pragma unroll
    for (int k = 0; k < RW; ++k) {
      if (rw0 + k >= r1) break;  // uniform across the warp
      const float4* row4 = reinterpret_cast<const float4*>(rows + (size_t)k * dpad);
      float4 a[CH];
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int col = 4 * lane + 128 * c;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (col < d) {
          t = row4[lane + 32 * c];
          if (col + 4 > d) {  // ragged last float4: the copied padding may hold anything
            if (col + 1 >= d) t.y = 0.f;
            if (col + 2 >= d) t.z = 0.f;
            t.w = 0.f;
          }
        }
        a[c] = t;
        const float4 xv = XS ? xs4[lane + 32 * c] : xr[XS ? 0 : c];
        s0 = fmaf(t.x, xv.x, s0);
        s1 = fmaf(t.y, xv.y, s1);
        s2 = fmaf(t.z, xv.z, s2);
        s3 = fmaf(t.w, xv.w, s3);
      }
      const float r = bv[k] - warp_sum((s0 + s1) + (s2 + s3));
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        acc[c].x = fmaf(r, a[c].x, acc[c].x);
        acc[c].y = fmaf(r, a[c].y, acc[c].y);
        acc[c].z = fmaf(r, a[c].z, acc[c].z);
        acc[c].w = fmaf(r, a[c].w, acc[c].w);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    consumed = it + 1;
  }
  if (consumed < nst && warp == 0 && lane == 0) {
    // Aborted: let the copies already issued land before the block exits.
    const int iss = *(volatile int*)&issued;
    for (int it = consumed; it < iss; ++it)
      if (!mbar_wait(&full[it % stages], (uint32_t)(it / stages) & 1u, kWaitLimitNs)) break;
  }
  if (consumed < nst && ctl != nullptr && warp == 0 && lane == 0) {
    ctl->status = MIHS_ERR_TIMEOUT;
    ctl->done = 1;
  }
  named_sync(1, NC * 32);  // every consumer is done with the ring
  float* wpart = ring;     // reuse stage memory: NC × dpad warp partials
  float4* wp4 = reinterpret_cast<float4*>(wpart + (size_t)warp * dpad);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = 4 * lane + 128 * c;
    if (col < dpad) wp4[lane + 32 * c] = acc[c];
  }
  named_sync(1, NC * 32);
  float* out = partials + (size_t)blockIdx.x * dpad;
  for (int j = threadIdx.x; j < dpad; j += NC * 32) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < NC; ++w) t += wpart[(size_t)w * dpad + j];
    out[j] = t;
  }
}

// g[j] = Σ_p partials[p][j] − λ x[j]; 32 columns × 8 partial groups per block.
__global__ void __launch_bounds__(256)
apass_finalize_kernel(const float* __restrict__ partials, int P, int d, int dpad,
                      const float* __restrict__ x, float lambda, const float* __restrict__ rhs,
                      float* __restrict__ g, const SolveCtl* __restrict__ ctl, int gate,
                      const double* __restrict__ base64) {
  if (ctl != nullptr && (ctl->done || (gate >= 0 && ctl_gate(ctl) != gate))) return;
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < d) {
    for (int p = grp; p < P; p += 8) s += partials[(size_t)p * dpad + j];
  }
  red[grp][lane] = s;
  __syncthreads();
  if (grp == 0 && j < d) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    if (rhs != nullptr) t += rhs[j];
    t -= (x != nullptr ? lambda * x[j] : 0.f);
    g[j] = base64 != nullptr ? (float)(base64[j] + (double)t) : t;
  }
}

struct ApassKernel {
  const void* fn;
  int rows_per_stage;
};

template <int CH, int RW>
ApassKernel make_kernel() {
  return ApassKernel{reinterpret_cast<const void*>(&apass_partial_kernel<CH, RW>),
                     kConsumerWarps * RW};
}

ApassKernel pick(int64_t d) {
  const int ch = (int)((d + 127) / 128);
  if (ch <= 1) return make_kernel<1, 8>();
  if (ch <= 2) return make_kernel<2, 4>();
  if (ch <= 4) return make_kernel<4, 2>();
  if (ch <= 8) return make_kernel<8, 1>();
  if (ch <= 12) return make_kernel<12, 1>();
  return make_kernel<16, 1>();
}

}  // namespace

int apass_num_partials(int64_t n, int64_t d) {
  const ApassKernel k = pick(d);
  const int64_t by_rows = (n + k.rows_per_stage - 1) / k.rows_per_stage;
  // One block per SM; MIHS_APASS_BLOCKS caps the grid (leaving SMs free for
  // the inner solves of concurrent solves on other streams).
  static const int cap = [] {
    const char* e = std::getenv("MIHS_APASS_BLOCKS");
    return e != nullptr ? std::atoi(e) : 0;
  }();
  int64_t P = num_sms();
  if (cap > 0 && cap < P) P = cap;
  if (P > by_rows) P = by_rows;
  return (int)(P < 1 ? 1 : P);
}

int launch_apass_partial(const float* A, int64_t n, int64_t d, int64_t lda, const float* b,
                         const float* x, float* partials, SolveCtl* ctl, cudaStream_t s, int gate) {
  const ApassKernel k = pick(d);
  const int P = apass_num_partials(n, d);
  const int64_t dpad = apass_dpad(d);
  const int R = k.rows_per_stage;
  const int rows_per_cta = (int)round_up((n + P - 1) / P, R);
  const size_t stage_bytes = (size_t)R * dpad * sizeof(float);
  int stages = (int)(kRingBudget / stage_bytes);
  stages = stages < 2 ? 2 : (stages > 8 ? 8 : stages);
  const size_t smem = (size_t)stages * stage_bytes + 2 * sizeof(uint64_t) * stages +
                      (size_t)((d + 127) / 128) * 128 * sizeof(float);
  MIHS_CUDA_TRY(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int n32 = (int)n, d32 = (int)d, dp32 = (int)dpad;
  long long lda64 = lda;
  void* args[] = {(void*)&A, &n32, &d32, &lda64, (void*)&b, (void*)&x,
                  (void*)&partials, &dp32, (void*)&rows_per_cta, &stages, (void*)&ctl, &gate};
  // refinement corrections (gate 2) are timed apart from plain gradients
  const int timer = gate == 2 ? kTimerApassCorr : kTimerApass;
  timing_begin(timer, s);
  MIHS_CUDA_TRY(cudaLaunchKernel(k.fn, dim3(P), dim3(kThreads), args, smem, s));
  timing_end(timer, s);
  count_launch();
  return MIHS_OK;
}

int apass_device_error(int* code) {
  int v = 0, zero = 0;
  MIHS_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_apass_error, sizeof(int)));
  if (v != 0) MIHS_CUDA_TRY(cudaMemcpyToSymbol(g_apass_error, &zero, sizeof(int)));
  *code = v;
  return MIHS_OK;
}

int launch_apass_finalize(const float* partials, int P, int64_t d, const float* x,
                          float lambda, float* g, const SolveCtl* ctl, cudaStream_t s, int gate,
                          const float* rhs, const double* base64) {
  const int64_t dpad = apass_dpad(d);
  apass_finalize_kernel<<<(unsigned)((d + 31) / 32), 256, 0, s>>>(partials, P, (int)d, (int)dpad,
                                                                   x, lambda, rhs, g, ctl, gate, base64);
  MIHS_CHECK_LAUNCH();
  count_launch();
  return MIHS_OK;
}

}  // namespace mihs
