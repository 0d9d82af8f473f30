// Gradient step of Algorithm 1:  g = Aᵀ(b − Ax) − λx.
//
// One streaming pass over A (the only O(nd) work per iteration, "4nd + 3d" in
// Algorithm 1).  Each warp takes whole rows: lane ℓ holds columns 4ℓ + 128c
// of the row as float4, the row residual r_i = b_i − A_i·x is a warp
// all-reduce, and r_i·A_i is accumulated into the lane's registers at once,
// so A is read exactly once and no grid-wide synchronisation happens inside
// the pass (the paper's point that M-IHS needs no inner products in the outer
// loop).  Each block owns a contiguous row range; its warps' partial d-vectors
// are summed in smem and written as one split-K partial.  A second small
// kernel sums the partials in a fixed order (deterministic result) and
// subtracts λx.
#include "internal.h"

namespace mihs {

namespace {

template <int CH>
__device__ __forceinline__ void load_row(float4 (&v)[CH], const float* __restrict__ A,
                                         long long row, long long lda, int d, int lane) {
  const float4* p = reinterpret_cast<const float4*>(A + row * lda);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = 4 * lane + 128 * c;
    if (col < d) {
      float4 t = __ldcs(p + lane + 32 * c);
      if (col + 4 > d) {  // ragged last float4: zero the columns ≥ d
        if (col + 1 >= d) t.y = 0.f;
        if (col + 2 >= d) t.z = 0.f;
        t.w = 0.f;
      }
      v[c] = t;
    } else {
      v[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

template <int CH, int RPI, int NT>
__global__ void __launch_bounds__(NT, 1)
apass_partial_kernel(const float* __restrict__ A, int n, int d, long long lda,
                     const float* __restrict__ b, const float* __restrict__ x,
                     float* __restrict__ partials, int dpad, int rows_per_cta,
                     const SolveCtl* __restrict__ ctl) {
  if (ctl != nullptr && ctl->done) return;  // same value for every block
  constexpr int NW = NT / 32;
  extern __shared__ float4 smem4[];
  float* xs = reinterpret_cast<float*>(smem4);  // x, CH·128 floats, zero padded
  float* wpart = xs + CH * 128;                 // NW × dpad warp partials
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = tid; j < CH * 128; j += NT) xs[j] = (x != nullptr && j < d) ? x[j] : 0.f;
  __syncthreads();

  float4 acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);

  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min((long long)n, r0 + rows_per_cta);
  const float4* xs4 = reinterpret_cast<const float4*>(xs);

  // Software pipeline: the next RPI rows are in flight while the current RPI
  // rows are reduced.
  float4 cur[RPI][CH];
  float bcur[RPI];
  long long row = r0 + (long long)warp * RPI;
#pragma unroll
  for (int k = 0; k < RPI; ++k) {
    if (row + k < r1) {
      load_row<CH>(cur[k], A, row + k, lda, d, lane);
      bcur[k] = __ldg(b + row + k);
    } else {
#pragma unroll
      for (int c = 0; c < CH; ++c) cur[k][c] = make_float4(0.f, 0.f, 0.f, 0.f);
      bcur[k] = 0.f;
    }
  }
  for (; row < r1; row += (long long)NW * RPI) {
    const long long nrow = row + (long long)NW * RPI;
    float4 nxt[RPI][CH];
    float bnxt[RPI];
#pragma unroll
    for (int k = 0; k < RPI; ++k) {
      if (nrow + k < r1) {
        load_row<CH>(nxt[k], A, nrow + k, lda, d, lane);
        bnxt[k] = __ldg(b + nrow + k);
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c) nxt[k][c] = make_float4(0.f, 0.f, 0.f, 0.f);
        bnxt[k] = 0.f;
      }
    }
    float dot[RPI];
#pragma unroll
    for (int k = 0; k < RPI; ++k) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const float4 xv = xs4[lane + 32 * c];
        s = fmaf(cur[k][c].x, xv.x, s);
        s = fmaf(cur[k][c].y, xv.y, s);
        s = fmaf(cur[k][c].z, xv.z, s);
        s = fmaf(cur[k][c].w, xv.w, s);
      }
      dot[k] = s;
    }
#pragma unroll
    for (int k = 0; k < RPI; ++k) dot[k] = warp_sum(dot[k]);
#pragma unroll
    for (int k = 0; k < RPI; ++k) {
      const float r = bcur[k] - dot[k];  // rows past r1 carry zeros: r·0 = 0
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        acc[c].x = fmaf(r, cur[k][c].x, acc[c].x);
        acc[c].y = fmaf(r, cur[k][c].y, acc[c].y);
        acc[c].z = fmaf(r, cur[k][c].z, acc[c].z);
        acc[c].w = fmaf(r, cur[k][c].w, acc[c].w);
      }
    }
#pragma unroll
    for (int k = 0; k < RPI; ++k) {
      bcur[k] = bnxt[k];
#pragma unroll
      for (int c = 0; c < CH; ++c) cur[k][c] = nxt[k][c];
    }
  }

  float4* wp4 = reinterpret_cast<float4*>(wpart + (size_t)warp * dpad);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = 4 * lane + 128 * c;
    if (col < dpad) wp4[lane + 32 * c] = acc[c];
  }
  __syncthreads();
  float* out = partials + (size_t)blockIdx.x * dpad;
  for (int j = tid; j < dpad; j += NT) {
    float s = 0.f;
#pragma unroll 4
    for (int w = 0; w < NW; ++w) s += wpart[(size_t)w * dpad + j];
    out[j] = s;
  }
}

// g[j] = Σ_p partials[p][j] − λ x[j]; 32 columns × 8 partial groups per block.
__global__ void __launch_bounds__(256)
apass_finalize_kernel(const float* __restrict__ partials, int P, int d, int dpad,
                      const float* __restrict__ x, float lambda, float* __restrict__ g,
                      const SolveCtl* __restrict__ ctl) {
  if (ctl != nullptr && ctl->done) return;
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
    g[j] = t - (x != nullptr ? lambda * x[j] : 0.f);
  }
}

struct ApassKernel {
  const void* fn;
  int chunks;
  int threads;
  int rows_per_step;  // rows a block advances per warp step (NW·RPI)
};

template <int CH, int RPI, int NT>
ApassKernel make_kernel() {
  return ApassKernel{reinterpret_cast<const void*>(&apass_partial_kernel<CH, RPI, NT>), CH, NT,
                     (NT / 32) * RPI};
}

ApassKernel pick(int64_t d) {
  const int ch = (int)((d + 127) / 128);
  if (ch <= 1) return make_kernel<1, 8, 512>();
  if (ch <= 2) return make_kernel<2, 4, 512>();
  if (ch <= 4) return make_kernel<4, 2, 512>();
  if (ch <= 8) return make_kernel<8, 1, 512>();
  if (ch <= 12) return make_kernel<12, 1, 256>();
  return make_kernel<16, 1, 256>();
}

}  // namespace

int apass_num_partials(int64_t n, int64_t d) {
  const ApassKernel k = pick(d);
  const int64_t by_rows = (n + k.rows_per_step - 1) / k.rows_per_step;  // ≥ one step of rows
  int64_t P = num_sms();
  if (P > by_rows) P = by_rows;
  return (int)(P < 1 ? 1 : P);
}

int launch_apass_partial(const float* A, int64_t n, int64_t d, int64_t lda, const float* b,
                         const float* x, float* partials, const SolveCtl* ctl,
                         cudaStream_t s) {
  const ApassKernel k = pick(d);
  const int P = apass_num_partials(n, d);
  const int64_t dpad = apass_dpad(d);
  const int rows_per_cta = (int)((n + P - 1) / P);
  const size_t smem = ((size_t)k.chunks * 128 + (size_t)(k.threads / 32) * dpad) * sizeof(float);
  MIHS_CUDA_TRY(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  int n32 = (int)n, d32 = (int)d, dp32 = (int)dpad;
  long long lda64 = lda;
  void* args[] = {(void*)&A, &n32, &d32, &lda64, (void*)&b, (void*)&x,
                  (void*)&partials, &dp32, (void*)&rows_per_cta, (void*)&ctl};
  timing_begin(kTimerApass, s);
  MIHS_CUDA_TRY(cudaLaunchKernel(k.fn, dim3(P), dim3(k.threads), args, smem, s));
  timing_end(kTimerApass, s);
  count_launch();
  return MIHS_OK;
}

int launch_apass_finalize(const float* partials, int P, int64_t d, const float* x,
                          float lambda, float* g, const SolveCtl* ctl, cudaStream_t s) {
  const int64_t dpad = apass_dpad(d);
  apass_finalize_kernel<<<(unsigned)((d + 31) / 32), 256, 0, s>>>(partials, P, (int)d, (int)dpad,
                                                                   x, lambda, g, ctl);
  MIHS_CHECK_LAUNCH();
  count_launch();
  return MIHS_OK;
}

}  // namespace mihs
