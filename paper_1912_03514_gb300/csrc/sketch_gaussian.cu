// Gaussian sketch (Lemma 3, case iv):  SA = S·A with S_ij ~ N(0, 1/m).
//
// S is never stored: the tile of S a block needs is regenerated from the
// Philox4x32-10 counter (⌊j/4⌋, i, 0, 0) and a Box–Muller transform right
// before it is used, so the only HBM traffic is one read of A (split-K over
// the n rows) plus the small m×d partial sums.  This file holds the fp32 SIMT
// version (64×128 output tile, k-step 16), used when the tensor-core version
// (sketch_gaussian_tc.cu) is unavailable or MIHS_GAUSSIAN_SIMT is set.
#include <cmath>
#include <cstdlib>

#include "internal.h"

namespace mihs {

namespace {

constexpr int TM = 64, TN = 128, TK = 16, kThreads = 256;

__global__ void __launch_bounds__(kThreads)
gauss_simt_kernel(const float* __restrict__ A, int n, int d, long long lda, int m,
                  uint32_t k0, uint32_t k1, int rows_per_split,
                  float* __restrict__ part, int dp) {
  __shared__ __align__(16) float Ss[TK][TM + 4];  // S tile, k-major
  __shared__ __align__(16) float As[TK][TN];
  const int tid = threadIdx.x;
  const int n0 = blockIdx.x * TN;      // first column of A / SA
  const int i0 = blockIdx.y * TM;      // first row of S / SA
  const int kb = blockIdx.z * rows_per_split;
  const int ke = min(n, kb + rows_per_split);
  const int ti = tid >> 4, tj = tid & 15;
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  for (int kk = kb; kk < ke; kk += TK) {
    {  // S tile: thread → (row i, counter group q): 4 normals
      const int i = tid >> 2, q = tid & 3;
      const int gi = i0 + i;
      const int j0 = kk + 4 * q;
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (gi < m && j0 < ke) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(j0 >> 2), (uint32_t)gi, kTagGaussian, 0u), k0, k1);
        const float2 za = box_muller(w.x, w.y);
        const float2 zb = box_muller(w.z, w.w);
        z[0] = za.x; z[1] = za.y; z[2] = zb.x; z[3] = zb.y;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (j0 + e >= ke) z[e] = 0.f;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) Ss[4 * q + e][i] = z[e];
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {  // A tile: 16 rows × 128 columns
      const int idx = tid + r * kThreads;
      const int k = idx >> 5, c4 = idx & 31;
      const int row = kk + k, col = n0 + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < ke && col < d) {
        const float* src = A + (long long)row * lda + col;
        if (col + 4 <= d) {
          v = __ldcs(reinterpret_cast<const float4*>(src));
        } else {
          v.x = src[0];
          if (col + 1 < d) v.y = src[1];
          if (col + 2 < d) v.z = src[2];
        }
      }
      *reinterpret_cast<float4*>(&As[k][4 * c4]) = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      const float4 sa = *reinterpret_cast<const float4*>(&Ss[k][4 * ti]);
      const float4 b0 = *reinterpret_cast<const float4*>(&As[k][4 * tj]);
      const float4 b1 = *reinterpret_cast<const float4*>(&As[k][64 + 4 * tj]);
      const float s4[4] = {sa.x, sa.y, sa.z, sa.w};
      const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(s4[a], bb[b], acc[a][b]);
    }
    __syncthreads();
  }
  float* out = part + (size_t)blockIdx.z * m * dp;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + 4 * ti + a;
    if (gi >= m) continue;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int c = n0 + (b < 4 ? 4 * tj + b : 64 + 4 * tj + (b - 4));
      if (c < d) out[(size_t)gi * dp + c] = acc[a][b];
    }
  }
}

// SA[i][c] = scale · Σ_z part[z][i][c] (fixed order).
__global__ void gauss_reduce_kernel(const float* __restrict__ part, int KS, int m, int d, int dp,
                                    float scale, float* __restrict__ SA, long long ldsa) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * d) return;
  const int i = (int)(idx / d), c = (int)(idx - (long long)i * d);
  float s = 0.f;
  for (int z = 0; z < KS; ++z) s += part[((size_t)z * m + i) * dp + c];
  SA[(long long)i * ldsa + c] = s * scale;
}

}  // namespace

int sketch_gaussian(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed,
                    float* SA, int64_t ldsa, cudaStream_t s) {
  // Tensor-core path by default; MIHS_GAUSSIAN_SIMT selects this fp32 SIMT path.
  static const bool force_simt = std::getenv("MIHS_GAUSSIAN_SIMT") != nullptr;
  if (!force_simt && gaussian_tc_available()) return sketch_gaussian_tc(A, n, d, lda, m, seed, SA, ldsa, s);
  const int tn = (int)((d + TN - 1) / TN), tm = (int)((m + TM - 1) / TM);
  const int64_t ksteps = (n + TK - 1) / TK;
  int64_t KS = (2LL * num_sms() + (int64_t)tn * tm - 1) / ((int64_t)tn * tm);
  if (KS < 1) KS = 1;
  if (KS > ksteps) KS = ksteps;
  if (KS > 65535) KS = 65535;
  const int rows_per_split = (int)(((n + KS - 1) / KS + TK - 1) / TK * TK);
  KS = (n + rows_per_split - 1) / rows_per_split;
  const int dp = (int)round_up(d, 4);
  StreamScratch scratch;
  int rc = scratch.alloc(sizeof(float) * (size_t)KS * m * dp, s);
  if (rc) return rc;
  float* part = static_cast<float*>(scratch.p);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  gauss_simt_kernel<<<dim3(tn, tm, (unsigned)KS), kThreads, 0, s>>>(A, (int)n, (int)d, lda, (int)m,
                                                                    k0, k1, rows_per_split, part, dp);
  MIHS_CHECK_LAUNCH();
  const long long tot = (long long)m * d;
  gauss_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      part, (int)KS, (int)m, (int)d, dp, (float)(1.0 / std::sqrt((double)m)), SA, ldsa);
  MIHS_CHECK_LAUNCH();
  count_launch(2);
  return MIHS_OK;
}

}  // namespace mihs
