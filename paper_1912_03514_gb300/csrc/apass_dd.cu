// Compensated gradient for the refinement solve:  g = Aᵀ(b − Ax) − λx with
// x in fp64 and the sums carried in double-float (an unevaluated pair of
// fp32 numbers hi + lo):
//   * products by TwoProduct (p = a·x_hi, e = fma(a, x_hi, −p) exactly, plus
//     a·x_lo), sums by TwoSum (Knuth; Ogita, Rump & Oishi, "Accurate sum and
//     dot product", SIAM J. Sci. Comput. 2005), so the row residual and the
//     column sums keep about twice the fp32 precision;
//   * the split-K partials are pairs, summed in fp64 by the finalize kernel,
//     which also subtracts λx in fp64.
// The stream of A is the same as the plain A-pass (bulk-copy ring, one read
// of A); the extra fp32 arithmetic (11 operations per element and phase)
// runs as packed .f32x2 instructions, two independent chains at a time.  This is the accuracy-critical step of M-IHS:
// the iteration's fixed point is where this gradient vanishes, while the
// sketch and AAb_Solver only precondition.
#include "internal.h"

namespace mihs {

namespace {

// Seven consumer warps and the producer: 256 threads, so that each thread may
// hold 255 registers with one block per SM (rows wider than 1024: the
// double-float column accumulators need 8 registers per float4 column
// group), or 128 with two (rows up to 1024 wide).  Two blocks per SM keep 14
// consumer warps on the schedulers: the pass is bound by the latency of its
// dependent TwoSum chains (one block of eight consumer warps left each
// scheduler without an eligible warp 45% of the time; two blocks of nine
// warps get only 96 registers and spill).
template <int CH>
struct DdCfg {
  static constexpr int NC = 7;
  static constexpr int kThreads = (NC + 1) * 32;
  static constexpr int kBlocksPerSm = CH > 8 ? 1 : 2;
  static constexpr size_t kRingBudget = CH > 8 ? 150 * 1024 : 96 * 1024;
};

__device__ int g_apass_dd_error = 0;

struct DF {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// (s.hi + s.lo) += v (+ ve): compensated accumulation of a value with its error.
__device__ __forceinline__ void df_add(DF& s, float v, float ve) {
  float t, e;
  two_sum(s.hi, v, t, e);
  s.hi = t;
  s.lo += e + ve;
}

// a·(x_hi + x_lo) as (p, e) with p + e exact up to a·x_lo's rounding.
__device__ __forceinline__ void df_prod(float a, float xh, float xl, float& p, float& e) {
  p = a * xh;
  e = fmaf(a, xh, -p);
  e = fmaf(a, xl, e);
}

// Packed pairs of fp32 (PTX .f32x2, sm_100 and later): one instruction does
// the same IEEE round-to-nearest operation on both halves, so two
// independent double-float chains advance per instruction.
typedef unsigned long long P2;
__device__ __forceinline__ P2 p2_add(P2 a, P2 b) {
  P2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ P2 p2_sub(P2 a, P2 b) {
  P2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ P2 p2_mul(P2 a, P2 b) {
  P2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ P2 p2_fma(P2 a, P2 b, P2 c) {
  P2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ P2 p2_pack(float x, float y) {
  P2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(x), "f"(y));
  return d;
}
__device__ __forceinline__ float2 p2_unpack(P2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

struct DF2 {  // two double-float values, hi halves and lo halves packed
  P2 hi, lo;
};

// (s.hi + s.lo) += a·(yh + yl) for both halves, given nyh = −yh: the
// product's rounded part is p = −fl(a·nyh) (rounding is symmetric), its
// error fma(a, yh, −p) + a·yl (TwoProduct), the sum by TwoSum(s.hi, p) with
// its error and the product's added to s.lo — the same operations and
// roundings, half by half, as df_prod followed by df_add.
__device__ __forceinline__ void df2_madd(DF2& s, P2 a, P2 yh, P2 nyh, P2 yl) {
  const P2 pn = p2_mul(a, nyh);                    // −p
  P2 e = p2_fma(a, yh, pn);                        // a·yh − p, exact
  e = p2_fma(a, yl, e);
  const P2 t = p2_sub(s.hi, pn);                   // s.hi + p
  const P2 z = p2_sub(t, s.hi);
  const P2 e2 = p2_sub(p2_sub(s.hi, p2_sub(t, z)), p2_add(pn, z));  // (s.hi − (t − z)) + (p − z)
  s.hi = t;
  s.lo = p2_add(s.lo, p2_add(e2, e));
}

__device__ __forceinline__ DF df_shfl_xor_sum(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, v.hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, v.lo, o);
    float t, e;
    two_sum(v.hi, oh, t, e);
    v.hi = t;
    v.lo = v.lo + ol + e;
  }
  return v;
}

template <int CH, bool RAGGED>
__global__ void __launch_bounds__(DdCfg<CH>::kThreads, DdCfg<CH>::kBlocksPerSm)
apass_dd_kernel(const float* __restrict__ A, int n, int d, long long lda, const float* __restrict__ b,
                const double* __restrict__ x, float2* __restrict__ partials, int dpad, int rows_per_cta,
                int stages, SolveCtl* __restrict__ ctl, int gate) {
  constexpr int NC = DdCfg<CH>::NC, R = NC;
  constexpr int kThreads = DdCfg<CH>::kThreads;
  if (ctl != nullptr && (ctl->done || (gate >= 0 && ctl_gate(ctl) != gate))) return;  // uniform
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)stages * R * dpad);
  uint64_t* empty = full + stages;
  float* xh = reinterpret_cast<float*>(empty + stages);  // CH·128 each: x_hi, x_lo, −x_hi
  float* xl = xh + CH * 128;
  float* nxh = xl + CH * 128;
  __shared__ int issued;
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
  for (int j = threadIdx.x; j < CH * 128; j += kThreads) {
    const double xv = (x != nullptr && j < d) ? x[j] : 0.0;
    const float h = (float)xv;
    xh[j] = h;
    xl[j] = (float)(xv - (double)h);
    nxh[j] = -h;
  }
  __syncthreads();

  if (warp == NC) {  // producer
    if (lane == 0) {
      const uint32_t row_bytes = (uint32_t)dpad * 4u;
      const bool contiguous = lda == (long long)dpad;
      for (int it = 0; it < nst; ++it) {
        const int s = it % stages;
        const uint32_t ph = (uint32_t)(it / stages) & 1u;
        if (it >= stages && !mbar_wait(&empty[s], ph ^ 1u, kWaitLimitNs)) {
          atomicExch(&g_apass_dd_error, MIHS_ERR_TIMEOUT);
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

  // Column accumulators: group c's components (x, y) and (z, w), packed.
  DF2 acc[CH][2];
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int q = 0; q < 2; ++q) acc[c][q] = DF2{0ull, 0ull};
  int consumed = 0;
  for (int it = 0; it < nst; ++it) {
    const int s = it % stages;
    const uint32_t ph = (uint32_t)(it / stages) & 1u;
    const long long row = r0 + (long long)it * R + warp;
    const float bi = (b != nullptr && row < r1) ? __ldg(b + row) : 0.f;
    if (!mbar_wait(&full[s], ph, kWaitLimitNs)) {
      atomicExch(&g_apass_dd_error, MIHS_ERR_TIMEOUT);
      break;
    }
    if (row < r1) {  // uniform across the warp
      const float4* row4 = reinterpret_cast<const float4*>(ring + ((size_t)s * R + warp) * dpad);
      // Column group c of the row; the ragged last float4 is masked because the
      // copied padding may hold anything.  Read twice (dot, then accumulate)
      // instead of being kept in registers.
      auto chunk = [&](int c) {
        if (!RAGGED) return row4[lane + 32 * c];  // d = 128·CH: no ragged group
        const int col = 4 * lane + 128 * c;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (col < d) {
          t = row4[lane + 32 * c];
          if (col + 4 > d) {
            if (col + 1 >= d) t.y = 0.f;
            if (col + 2 >= d) t.z = 0.f;
            t.w = 0.f;
          }
        }
        return t;
      };
      // Four independent double-float chains (one per float4 component, two
      // per packed instruction) so that consecutive TwoSums do not wait on
      // each other.
      DF2 sxy = {0ull, 0ull}, szw = {0ull, 0ull};
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int col = 4 * lane + 128 * c;
        const float4 t = chunk(c);
        const ulonglong2 h2 = *reinterpret_cast<const ulonglong2*>(xh + col);
        const ulonglong2 l2 = *reinterpret_cast<const ulonglong2*>(xl + col);
        const ulonglong2 n2 = *reinterpret_cast<const ulonglong2*>(nxh + col);
        df2_madd(sxy, p2_pack(t.x, t.y), h2.x, n2.x, l2.x);
        df2_madd(szw, p2_pack(t.z, t.w), h2.y, n2.y, l2.y);
      }
      const float2 xyh = p2_unpack(sxy.hi), xyl = p2_unpack(sxy.lo);
      const float2 zwh = p2_unpack(szw.hi), zwl = p2_unpack(szw.lo);
      DF sx = {xyh.x, xyl.x}, sz = {zwh.x, zwl.x};
      df_add(sx, xyh.y, xyl.y);
      df_add(sz, zwh.y, zwl.y);
      df_add(sx, sz.hi, sz.lo);
      DF sum = sx;
      sum = df_shfl_xor_sum(sum);
      // r = b − (sum.hi + sum.lo), renormalised to a double-float pair
      float rh, re;
      two_sum(bi, -sum.hi, rh, re);
      float r_hi, r_lo;
      two_sum(rh, re - sum.lo, r_hi, r_lo);
      const P2 rh2 = p2_pack(r_hi, r_hi), nrh2 = p2_pack(-r_hi, -r_hi), rl2 = p2_pack(r_lo, r_lo);
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const float4 t = chunk(c);
        df2_madd(acc[c][0], p2_pack(t.x, t.y), rh2, nrh2, rl2);
        df2_madd(acc[c][1], p2_pack(t.z, t.w), rh2, nrh2, rl2);
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
    if (ctl != nullptr) {
      ctl->status = MIHS_ERR_TIMEOUT;
      ctl->done = 1;
    }
  }
  named_sync(1, NC * 32);  // every consumer is done with the ring
  // Per-warp pairs into the ring memory, then a fixed-order fp64 sum per column.
  float2* wpart = reinterpret_cast<float2*>(ring);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = 4 * lane + 128 * c;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2 h = p2_unpack(acc[c][q].hi), l = p2_unpack(acc[c][q].lo);
      if (col + 2 * q < dpad) wpart[(size_t)warp * dpad + col + 2 * q] = make_float2(h.x, l.x);
      if (col + 2 * q + 1 < dpad) wpart[(size_t)warp * dpad + col + 2 * q + 1] = make_float2(h.y, l.y);
    }
  }
  named_sync(1, NC * 32);
  float2* out = partials + (size_t)blockIdx.x * dpad;
  for (int j = threadIdx.x; j < dpad; j += NC * 32) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NC; ++w) {
      const float2 v = wpart[(size_t)w * dpad + j];
      t += (double)v.x + (double)v.y;
    }
    const float hi = (float)t;
    out[j] = make_float2(hi, (float)(t - (double)hi));
  }
}

// g[j] = Σ_p (hi + lo) − λ·x[j] in fp64 (fixed order); also an fp32 copy.
__global__ void __launch_bounds__(256)
apass_dd_finalize_kernel(const float2* __restrict__ partials, int P, int d, int dpad,
                         const double* __restrict__ x, double lambda, double* __restrict__ g64,
                         float* __restrict__ g32, const SolveCtl* __restrict__ ctl, int gate,
                         const float* __restrict__ rhs, double* __restrict__ xref) {
  if (ctl != nullptr && (ctl->done || (gate >= 0 && ctl_gate(ctl) != gate))) return;
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (j < d)
    for (int p = grp; p < P; p += 8) {
      const float2 v = partials[(size_t)p * dpad + j];
      s += (double)v.x + (double)v.y;
    }
  red[grp][lane] = s;
  __syncthreads();
  if (grp == 0 && j < d) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    if (rhs != nullptr) t += (double)rhs[j];
    if (x != nullptr) t -= lambda * x[j];
    if (g64 != nullptr) g64[j] = t;
    if (g32 != nullptr) g32[j] = (float)t;
    if (xref != nullptr) xref[j] = x[j];  // the point this gradient was taken at
  }
}

struct DdKernel {
  const void* fn;
  int chunks;
  int nc;  // consumer warps = rows per stage
  int blocks_per_sm;
  size_t ring_budget;
};

template <int CH>
DdKernel make_dd(bool ragged) {
  using C = DdCfg<CH>;
  const void* fn = ragged ? reinterpret_cast<const void*>(&apass_dd_kernel<CH, true>)
                          : reinterpret_cast<const void*>(&apass_dd_kernel<CH, false>);
  return DdKernel{fn, CH, C::NC, C::kBlocksPerSm, C::kRingBudget};
}

DdKernel pick_dd(int64_t d) {
  const int ch = (int)((d + 127) / 128);
  if (ch <= 1) return make_dd<1>(d != 128);
  if (ch <= 2) return make_dd<2>(d != 256);
  if (ch <= 4) return make_dd<4>(d != 512);
  if (ch <= 8) return make_dd<8>(d != 1024);
  if (ch <= 12) return make_dd<12>(d != 1536);
  return make_dd<16>(d != 2048);
}

}  // namespace

int apass_dd_num_partials(int64_t n, int64_t d) {
  const DdKernel k = pick_dd(d);
  const int nc = k.nc;
  const int64_t by_rows = (n + nc - 1) / nc;
  int64_t P = (int64_t)num_sms() * k.blocks_per_sm;
  if (P > by_rows) P = by_rows;
  return (int)(P < 1 ? 1 : P);
}

int launch_apass_dd(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const double* x,
                    float2* partials, SolveCtl* ctl, cudaStream_t s, int gate) {
  const DdKernel k = pick_dd(d);
  const int P = apass_dd_num_partials(n, d);
  const int64_t dpad = apass_dpad(d);
  const int R = k.nc;
  const int rows_per_cta = (int)round_up((n + P - 1) / P, R);
  const size_t stage_bytes = (size_t)R * dpad * sizeof(float);
  int stages = (int)(k.ring_budget / stage_bytes);
  stages = stages < 2 ? 2 : (stages > 8 ? 8 : stages);
  // The ring must also hold the NC × dpad float2 warp pairs at the end.
  while ((size_t)stages * stage_bytes < (size_t)k.nc * dpad * sizeof(float2)) ++stages;
  const size_t smem = (size_t)stages * stage_bytes + 2 * sizeof(uint64_t) * stages +
                      3 * (size_t)k.chunks * 128 * sizeof(float);
  MIHS_CUDA_TRY(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int n32 = (int)n, d32 = (int)d, dp32 = (int)dpad;
  long long lda64 = lda;
  void* args[] = {(void*)&A, &n32, &d32, &lda64, (void*)&b, (void*)&x,
                  (void*)&partials, &dp32, (void*)&rows_per_cta, &stages, (void*)&ctl, &gate};
  timing_begin(kTimerApassDd, s);
  MIHS_CUDA_TRY(cudaLaunchKernel(k.fn, dim3(P), dim3((k.nc + 1) * 32), args, smem, s));
  timing_end(kTimerApassDd, s);
  count_launch();
  return MIHS_OK;
}

int launch_apass_dd_finalize(const float2* partials, int P, int64_t d, const double* x, double lambda,
                             double* g64, float* g32, const SolveCtl* ctl, cudaStream_t s, int gate,
                             const float* rhs, double* xref) {
  apass_dd_finalize_kernel<<<(unsigned)((d + 31) / 32), 256, 0, s>>>(partials, P, (int)d, (int)apass_dpad(d), x,
                                                                     lambda, g64, g32, ctl, gate, rhs, xref);
  MIHS_CHECK_LAUNCH();
  count_launch();
  return MIHS_OK;
}

int apass_dd_device_error(int* code) {
  int v = 0, zero = 0;
  MIHS_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_apass_dd_error, sizeof(int)));
  if (v != 0) MIHS_CUDA_TRY(cudaMemcpyToSymbol(g_apass_dd_error, &zero, sizeof(int)));
  *code = v;
  return MIHS_OK;
}

}  // namespace mihs
