// Statistical dimension estimate (Algorithm 4, inexact Hutchinson trace
// estimator):  sd ≈ d − (λ/T)·Σ_ℓ ⟨v^ℓ, z^ℓ⟩,  z^ℓ = AAb_Solver(SA, v^ℓ, λ, ε_tr),
// with Rademacher probes v^ℓ.  Each probe is one AAb_Solver cluster launch on
// the sketched matrix plus a fixed-order dot product.
#include "internal.h"

namespace mihs {

namespace {

// v_j = +1 if w0 of Philox counter (j, ℓ, 4, 0) is even, else −1.
__global__ void rademacher_kernel(int d, int ell, uint32_t k0, uint32_t k1, float* __restrict__ v) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)ell, kTagHutchinson, 0u), k0, k1);
  v[j] = (w.x & 1u) ? -1.f : 1.f;
}

// tau += λ·⟨v, z⟩ (one block, fixed order, fp64 accumulation of fp32 products).
__global__ void __launch_bounds__(256) hutch_dot_kernel(const float* __restrict__ v, const float* __restrict__ z,
                                                        int d, double lambda, double* __restrict__ tau) {
  __shared__ double red[256];
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += 256) s += (double)v[j] * (double)z[j];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 256; ++i) t += red[i];
    *tau += lambda * t;
  }
}

}  // namespace

int estimate_sd(const float* SA, int64_t m, int64_t d, int64_t ldsa, double lambda, int T, double eps_tr,
                uint64_t seed, double* sd_out, cudaStream_t s) {
  StreamScratch scratch;
  int rc = scratch.alloc(sizeof(double) + 2 * sizeof(float) * (size_t)round_up(d, 4), s);
  if (rc) return rc;
  double* tau = static_cast<double*>(scratch.p);
  float* v = reinterpret_cast<float*>(tau + 1);
  float* z = v + round_up(d, 4);
  MIHS_CUDA_TRY(cudaMemsetAsync(tau, 0, sizeof(double), s));
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int ell = 0; ell < T; ++ell) {
    rademacher_kernel<<<(unsigned)((d + 255) / 256), 256, 0, s>>>((int)d, ell, k0, k1, v);
    MIHS_CHECK_LAUNCH();
    AabLaunch a = {};
    a.SA = SA;
    a.m = (int)m;
    a.d = (int)d;
    a.ldsa = ldsa;
    a.g = v;
    a.lambda = (float)lambda;
    a.eps = (float)eps_tr;
    a.max_passes = (int)(m < d ? m : d);
    a.delta = z;
    rc = launch_aab(a, s);
    if (rc) return rc;
    hutch_dot_kernel<<<1, 256, 0, s>>>(v, z, (int)d, lambda, tau);
    MIHS_CHECK_LAUNCH();
    count_launch(2);
  }
  double host_tau = 0.0;
  MIHS_CUDA_TRY(cudaMemcpyAsync(&host_tau, tau, sizeof(double), cudaMemcpyDeviceToHost, s));
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  *sd_out = (double)d - host_tau / (double)T;
  return MIHS_OK;
}

}  // namespace mihs
