// Gradients of the ridge solution x(A, b, λ) = (AᵀA + λI)⁻¹Aᵀb with respect
// to its inputs, given the adjoint v = (AᵀA + λI)⁻¹ ḡ of an upstream gradient
// ḡ = ∂L/∂x.  Differentiating H x = Aᵀb (H = AᵀA + λI) gives
//   dx = H⁻¹(dAᵀ r − Aᵀ dA x + Aᵀ db − dλ x),  r = b − Ax,
// so dL = ḡᵀdx = rᵀdA v − (Av)ᵀdA x + (Av)ᵀdb − (xᵀv) dλ, i.e.
//   ∂L/∂A = r vᵀ − (Av) xᵀ,  ∂L/∂b = Av,  ∂L/∂λ = −xᵀv.
// (The paper does not differentiate the solve; this is the standard adjoint
// of a linear system with a symmetric matrix, so the same M-IHS solver with
// the same sketch computes v.)
//
// One pass over A: each warp takes whole rows, forms r_i = b_i − A_i·x and
// q_i = A_i·v with warp reductions, and writes the row A-gradient
// r_i v − q_i x and db_i = q_i.  The pass reads A once and writes dA once:
// 8·n·d + 8·n bytes, HBM-bound.
#include "internal.h"

namespace mihs {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// dλ = −Σ_j x_j v_j, accumulated in fp64 in a fixed order (one block).
__global__ void __launch_bounds__(kThreads) neg_dot_kernel(const float* __restrict__ x,
                                                           const float* __restrict__ v, int d,
                                                           double* __restrict__ out) {
  __shared__ double red[kWarps];
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += kThreads) s += (double)x[j] * (double)v[j];
  s = warp_sum_f64(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += red[w];
    *out = -t;
  }
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// Vector path: d, lda, ldda multiples of 4 and 16-byte aligned rows.  Lane
// `l` holds columns 4(32c + l) … 4(32c + l) + 3 of chunk c < CH, CH =
// ⌈d/128⌉; x and v live in registers (CH ≤ 4) or shared memory (CH ≥ 8:
// held in registers they cap the CTA count per SM and, measured at 2²⁰×1024,
// the pass ran at 0.57 of HBM bandwidth instead of 0.97).  RW rows per warp
// iteration give each warp RW·CH independent 16-byte loads in flight.
template <int CH, int RW>
__global__ void __launch_bounds__(kThreads)
    backward_rows_vec_kernel(const float* __restrict__ A, long long n, int d, long long lda,
                             const float* __restrict__ b, const float* __restrict__ x,
                             const float* __restrict__ v, float* __restrict__ dA, long long ldda,
                             float* __restrict__ db) {
  constexpr bool XS = CH >= 8;
  __shared__ float4 xs4[XS ? CH * 32 : 1], vs4[XS ? CH * 32 : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d4 = d >> 2;
  float4 xr[XS ? 1 : CH], vr[XS ? 1 : CH];
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (XS) {
    for (int i = threadIdx.x; i < CH * 32; i += kThreads) {
      xs4[i] = i < d4 ? x4[i] : z4;
      vs4[i] = i < d4 ? v4[i] : z4;
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int c = 0; c < (XS ? 1 : CH); ++c) {
      const int i = c * 32 + lane;
      xr[c] = i < d4 ? x4[i] : z4;
      vr[c] = i < d4 ? v4[i] : z4;
    }
  }
  const long long nw = (long long)gridDim.x * kWarps;
  for (long long r0 = ((long long)blockIdx.x * kWarps + warp) * RW; r0 < n; r0 += nw * RW) {
    float4 a[RW][CH];
#pragma unroll
    for (int k = 0; k < RW; ++k) {
      const long long row = r0 + k;
      const float4* Ar = reinterpret_cast<const float4*>(A + (row < n ? row : 0) * lda);
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int i = c * 32 + lane;
        a[k][c] = (row < n && i < d4) ? __ldg(Ar + i) : z4;
      }
    }
    float rr[RW], qq[RW];
#pragma unroll
    for (int k = 0; k < RW; ++k) {
      float sx0 = 0.f, sx1 = 0.f, sv0 = 0.f, sv1 = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const float4 xc = XS ? xs4[c * 32 + lane] : xr[XS ? 0 : c];
        const float4 vc = XS ? vs4[c * 32 + lane] : vr[XS ? 0 : c];
        if (c & 1) {
          sx1 += dot4(a[k][c], xc);
          sv1 += dot4(a[k][c], vc);
        } else {
          sx0 += dot4(a[k][c], xc);
          sv0 += dot4(a[k][c], vc);
        }
      }
      const long long row = r0 + k;
      const float bi = (row < n && b != nullptr) ? __ldg(b + row) : 0.f;
      rr[k] = bi - warp_sum(sx0 + sx1);
      qq[k] = warp_sum(sv0 + sv1);
    }
#pragma unroll
    for (int k = 0; k < RW; ++k) {
      const long long row = r0 + k;
      if (row >= n) break;
      if (db != nullptr && lane == 0) db[row] = qq[k];
      if (dA == nullptr) continue;
      float4* Dr = reinterpret_cast<float4*>(dA + row * ldda);
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int i = c * 32 + lane;
        if (i < d4) {
          const float4 xc = XS ? xs4[i] : xr[XS ? 0 : c];
          const float4 vc = XS ? vs4[i] : vr[XS ? 0 : c];
          float4 o;
          o.x = fmaf(rr[k], vc.x, -qq[k] * xc.x);
          o.y = fmaf(rr[k], vc.y, -qq[k] * xc.y);
          o.z = fmaf(rr[k], vc.z, -qq[k] * xc.z);
          o.w = fmaf(rr[k], vc.w, -qq[k] * xc.w);
          __stcs(Dr + i, o);  // streamed: dA is written once and not re-read here
        }
      }
    }
  }
}

// Any d, lda, ldda: x and v in shared memory, two sweeps over each row (the
// second one hits L1/L2).
__global__ void __launch_bounds__(kThreads)
    backward_rows_kernel(const float* __restrict__ A, long long n, int d, long long lda,
                         const float* __restrict__ b, const float* __restrict__ x,
                         const float* __restrict__ v, float* __restrict__ dA, long long ldda,
                         float* __restrict__ db) {
  __shared__ float xs[kMaxD], vs[kMaxD];
  for (int j = threadIdx.x; j < d; j += kThreads) {
    xs[j] = x[j];
    vs[j] = v[j];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long nw = (long long)gridDim.x * kWarps;
  for (long long row = (long long)blockIdx.x * kWarps + warp; row < n; row += nw) {
    const float* Ar = A + row * lda;
    float sx = 0.f, sv = 0.f;
    for (int j = lane; j < d; j += 32) {
      const float aij = __ldg(Ar + j);
      sx = fmaf(aij, xs[j], sx);
      sv = fmaf(aij, vs[j], sv);
    }
    const float r = (b != nullptr ? __ldg(b + row) : 0.f) - warp_sum(sx);
    const float q = warp_sum(sv);
    if (db != nullptr && lane == 0) db[row] = q;
    if (dA != nullptr) {
      float* Dr = dA + row * ldda;
      for (int j = lane; j < d; j += 32) Dr[j] = fmaf(r, vs[j], -q * xs[j]);
    }
  }
}

template <typename K>
int launch_rows(K kernel, long long n, const void* const* args, cudaStream_t s) {
  int per_sm = 0;
  MIHS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const long long want = (n + kWarps - 1) / kWarps;
  long long grid = (long long)num_sms() * per_sm;
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  MIHS_CUDA_TRY(cudaLaunchKernel((const void*)kernel, dim3((unsigned)grid), dim3(kThreads),
                                 const_cast<void**>(args), 0, s));
  count_launch();
  return MIHS_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

int launch_backward_grads(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const float* x,
                          const float* v, float* dA, int64_t ldda, float* db, double* dlambda, cudaStream_t s) {
  if (dlambda != nullptr) {
    neg_dot_kernel<<<1, kThreads, 0, s>>>(x, v, (int)d, dlambda);
    MIHS_CHECK_LAUNCH();
    count_launch();
  }
  if ((dA == nullptr && db == nullptr) || n == 0) return MIHS_OK;
  long long n_ = n, lda_ = lda, ldda_ = dA != nullptr ? ldda : 0;
  int d_ = (int)d;
  const void* args[] = {&A, &n_, &d_, &lda_, &b, &x, &v, &dA, &ldda_, &db};
  const bool vec = d % 4 == 0 && lda % 4 == 0 && aligned16(A) && aligned16(x) && aligned16(v) &&
                   (dA == nullptr || (ldda % 4 == 0 && aligned16(dA)));
  const int ch = (int)((d + 127) / 128);
  timing_begin(kTimerBackward, s);
  int rc;
  if (!vec) rc = launch_rows(backward_rows_kernel, n, args, s);
  else if (ch <= 1) rc = launch_rows(backward_rows_vec_kernel<1, 4>, n, args, s);
  else if (ch <= 2) rc = launch_rows(backward_rows_vec_kernel<2, 4>, n, args, s);
  else if (ch <= 4) rc = launch_rows(backward_rows_vec_kernel<4, 2>, n, args, s);
  else if (ch <= 8) rc = launch_rows(backward_rows_vec_kernel<8, 2>, n, args, s);
  else rc = launch_rows(backward_rows_vec_kernel<16, 1>, n, args, s);
  timing_end(kTimerBackward, s);
  return rc;
}

}  // namespace mihs
