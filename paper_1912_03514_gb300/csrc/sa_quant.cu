// Quantised storage of the sketch SA for AAb_Solver: bf16 (round to nearest
// even), or fp8 e4m3 with one fp32 scale per 128 × 128 tile,
//   scale_t = max_{(i,j) ∈ t} |SA_ij| / 448   (1 for an all-zero tile),
//   q_ij    = e4m3(SA_ij / scale_t)           (round to nearest even, saturating),
// decoded as q_ij · scale_t.  Rows have a pitch of ldq elements (a multiple of
// 16, so that every row starts on a 16-byte boundary); columns d … ldq − 1
// are stored as zero.  The sketch only preconditions the iteration (its fixed
// point is where the exact gradient vanishes, Section 3.1), so a coarser SA
// changes the rate, not the solution.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "internal.h"

namespace mihs {

namespace {

constexpr int kTile = 128;

__global__ void quant_bf16_kernel(const float* __restrict__ SA, int m, int d, long long ldsa,
                                  __nv_bfloat16* __restrict__ out, long long ldq) {
  const long long total = (long long)m * ldq;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / ldq, j = e - i * ldq;
    const float v = j < d ? SA[i * ldsa + j] : 0.f;
    out[e] = __float2bfloat16_rn(v);
  }
}

// One block per 128 × 128 tile: the largest magnitude, then the scale.
__global__ void tile_scale_kernel(const float* __restrict__ SA, int m, int d, long long ldsa,
                                  float* __restrict__ scales, int ntc) {
  const int tr = blockIdx.y, tc = blockIdx.x;
  __shared__ float red[32];
  float mx = 0.f;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int i = tr * kTile + e / kTile, j = tc * kTile + e % kTile;
    if (i < m && j < d) mx = fmaxf(mx, fabsf(SA[(long long)i * ldsa + j]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    scales[tr * ntc + tc] = t > 0.f ? t / 448.0f : 1.0f;
  }
}

__global__ void quant_fp8_kernel(const float* __restrict__ SA, int m, int d, long long ldsa,
                                 const float* __restrict__ scales, int ntc, __nv_fp8_e4m3* __restrict__ out,
                                 long long ldq) {
  const long long total = (long long)m * ldq;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / ldq, j = e - i * ldq;
    __nv_fp8_e4m3 q;
    if (j < d) {
      q.__x = __nv_cvt_float_to_fp8(SA[i * ldsa + j] / scales[(size_t)(i / kTile) * ntc + j / kTile],
                                    __NV_SATFINITE, __NV_E4M3);
    } else {
      q.__x = 0;
    }
    out[e] = q;
  }
}

// Σ (decoded q − SA)² over the block's elements (a fixed range per block),
// each element's error formed in fp32 exactly as the AAb kernels decode it and
// squared and summed in fp64: one partial per block.
template <typename TQ>
__global__ void quant_err_kernel(const float* __restrict__ SA, int m, int d, long long ldsa, const TQ* __restrict__ q,
                                 long long ldq, const float* __restrict__ scales, int ntc,
                                 double* __restrict__ partial) {
  const long long total = (long long)m * d;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long e0 = (long long)blockIdx.x * per, e1 = e0 + per < total ? e0 + per : total;
  double acc = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const long long i = e / d, j = e - i * d;
    float dec;
    if constexpr (sizeof(TQ) == 2) {
      dec = __bfloat162float(q[i * ldq + j]);
    } else {
      const __half_raw h = __nv_cvt_fp8_to_halfraw(q[i * ldq + j].__x, __NV_E4M3);
      dec = __half2float(__half(h)) * scales[(size_t)(i / kTile) * ntc + j / kTile];
    }
    const double err = (double)dec - (double)SA[i * ldsa + j];
    acc = fma(err, err, acc);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void quant_err_sum_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < n; ++b) t += partial[b];
    *out = t;
  }
}

}  // namespace

int launch_quant_error(const float* SA, int64_t m, int64_t d, int64_t ldsa, int prec, const void* q, int64_t ldq,
                       const float* scales, double* scratch, double* err_out, cudaStream_t s) {
  if (m == 0) {
    MIHS_CUDA_TRY(cudaMemsetAsync(err_out, 0, sizeof(double), s));
    return MIHS_OK;
  }
  const int ntc = (int)((round_up(d, 4) + kTile - 1) / kTile);
  if (prec == MIHS_SA_BF16)
    quant_err_kernel<__nv_bfloat16><<<kQuantErrBlocks, 256, 0, s>>>(
        SA, (int)m, (int)d, ldsa, static_cast<const __nv_bfloat16*>(q), ldq, scales, ntc, scratch);
  else
    quant_err_kernel<__nv_fp8_e4m3><<<kQuantErrBlocks, 256, 0, s>>>(
        SA, (int)m, (int)d, ldsa, static_cast<const __nv_fp8_e4m3*>(q), ldq, scales, ntc, scratch);
  MIHS_CHECK_LAUNCH();
  quant_err_sum_kernel<<<1, 32, 0, s>>>(scratch, kQuantErrBlocks, err_out);
  MIHS_CHECK_LAUNCH();
  count_launch(2);
  return MIHS_OK;
}

int64_t sa_quant_ld(int64_t d) { return round_up(d, 16); }
int64_t sa_scale_count(int64_t m, int64_t d) {
  return ((m + kTile - 1) / kTile) * ((round_up(d, 4) + kTile - 1) / kTile);
}

int launch_quantize_sa(const float* SA, int64_t m, int64_t d, int64_t ldsa, int prec, void* out, int64_t ldq,
                       float* scales, cudaStream_t s) {
  if (m == 0) return MIHS_OK;
  const int threads = 256;
  const long long blocks = (m * ldq + threads - 1) / threads;
  const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
  if (prec == MIHS_SA_BF16) {
    quant_bf16_kernel<<<grid, threads, 0, s>>>(SA, (int)m, (int)d, ldsa, static_cast<__nv_bfloat16*>(out), ldq);
    MIHS_CHECK_LAUNCH();
    count_launch();
    return MIHS_OK;
  }
  if (prec == MIHS_SA_FP8E4M3) {
    const int ntr = (int)((m + kTile - 1) / kTile), ntc = (int)((round_up(d, 4) + kTile - 1) / kTile);
    if (ntr > 65535) {
      set_error("quantize_sa: m=%lld too large for fp8 tiles", (long long)m);
      return MIHS_ERR_UNSUPPORTED;
    }
    tile_scale_kernel<<<dim3(ntc, ntr), 256, 0, s>>>(SA, (int)m, (int)d, ldsa, scales, ntc);
    MIHS_CHECK_LAUNCH();
    quant_fp8_kernel<<<grid, threads, 0, s>>>(SA, (int)m, (int)d, ldsa, scales, ntc,
                                              static_cast<__nv_fp8_e4m3*>(out), ldq);
    MIHS_CHECK_LAUNCH();
    count_launch(2);
    return MIHS_OK;
  }
  set_error("quantize_sa: unknown precision %d", prec);
  return MIHS_ERR_INVALID_ARG;
}

}  // namespace mihs
