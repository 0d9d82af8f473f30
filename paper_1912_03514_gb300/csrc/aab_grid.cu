// AAb_Solver (Algorithm 5, Section 3.6) fused with the heavy ball and stop
// test of Algorithm 1, for one λ, as a grid of one block per SM: the form for
// sketches too large for the shared memory of one thread-block cluster
// (16 SMs × ≈ 200 KB; e.g. SA of 3076 × 2048 fp32 is 25 MB).
//
// Block b keeps rows [b·R, b·R + R) of SA in its shared memory for the whole
// launch, so every pass reads SA from shared memory on all SMs instead of
// streaming it from L2 through one cluster.  The recursion is the one of the
// cluster kernel (aab_kernel.cuh) with the cluster's DSMEM exchanges replaced
// by global partials and grid-wide barriers:
//   sweep     w = SA_b·v − θp_b, ρ²_b = ‖w‖², U_b = SA_bᵀw     (own rows)
//   barrier A ρ² = Σ_b ρ²_b; block b sums U over blocks on its column slice,
//             z = U/ρ − ρv there, θ²_b = ‖z_slice‖², z → global Z
//   barrier B θ² = Σ_b θ²_b; v = Z/θ (every block reads all of Z)
// Every sum over blocks runs in a fixed order, so all blocks compute the same
// scalars and take the same branches.  The grid barrier is a counter in
// global memory whose top bit flips once all blocks have arrived
// (grid_sync.cuh); each wait is bounded and a wait that runs out stops the
// solve with MIHS_ERR_TIMEOUT instead of hanging.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "aab_kernel.cuh"
#include "grid_sync.cuh"

namespace mihs {

namespace {

using namespace aabk;

__device__ int g_aab_grid_error = 0;

struct AabGridParams {
  const void* SA;
  int m, d, dp;
  long long ldsa;
  int sa_pitch;        // shared-memory row pitch (elements of TS)
  const float* sa_scale;
  int scale_ld;
  int R, Rpad;         // rows per block
  int cs;              // owned column slice (multiple of 4)
  int sa_vec;          // rows 16-byte aligned: staged by bulk copies
  const float* g;
  float lambda, eps;
  int max_passes;
  float* delta;
  int* passes;
  float alpha, beta;
  float* x;
  float* x_prev;
  double* x64;
  double* x_prev64;
  float* x32_shadow;
  double alpha64, beta64;
  SolveCtl* ctl;
  float* hist;
  unsigned long long cond;
  // global scratch
  float* Upart;        // G × dp
  float* rho2;         // G
  float* theta2;       // G
  float* Z;            // dp
  unsigned int* bar;   // grid barrier word (0 between launches)
};

// Σ_b part[b] over the G blocks in a fixed order (lane l takes b ≡ l mod 32,
// then a butterfly): the same value in every block.  Called by one warp.
// All loads are issued before the first add (one L2 round trip for G ≤ 256).
__device__ __forceinline__ float sum_over_blocks(const float* part, int G) {
  const int lane = threadIdx.x & 31;
  float t = 0.f;
  for (int b0 = lane; b0 < G; b0 += 8 * 32) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int b = b0 + 32 * k;
      v[k] = b < G ? __ldcg(part + b) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) t += v[k];
  }
  return warp_sum(t);
}

// Σ_{b ≡ q (mod step), b < G} col[b·stride] in order of b, with up to 16
// loads in flight before the first add.
__device__ __forceinline__ float strided_sum(const float* col, size_t stride, int q, int step, int G) {
  float t = 0.f;
  for (int b0 = q; b0 < G; b0 += 16 * step) {
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int b = b0 + step * k;
      v[k] = b < G ? __ldcg(col + (size_t)b * stride) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) t += v[k];
  }
  return t;
}

// One sweep over the block's rows (SA in shared memory): the row dots
// w_i = SA_i·v − θp_i with their ρ² share, then the column sums U = SA_bᵀw
// with each thread owning its columns, stored straight to this block's row
// of the global partials; the warps' ρ² shares are summed in order.
template <int CH, typename TS>
__device__ __forceinline__ void grid_sweep_store(const TS* sa, int pitch, int nr, int d, int dp, const float* v,
                                                 const float* p, float theta, float* w, const float* scales,
                                                 int sld, int r0, float* red, float* tmp, float* out,
                                                 float* out_rho2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float rsq = row_dots<CH, TS>(sa, pitch, nr, v, p, theta, w, dp, scales, sld, r0);
  if (lane == 0) red[warp] = rsq;
  __syncthreads();  // w complete
  col_sums<CH, TS>(sa, pitch, nr, dp, w, scales, sld, r0, tmp, out);
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) t += red[q];
    __stcg(out_rho2, t);
  }
}

struct GridSmem {
  size_t v, buf, p, w, dvs, xss, red, scal, sa;  // byte offsets
  size_t total;
};

__host__ __device__ inline GridSmem grid_smem_layout(int dp, int Rpad, int cs, int R, int pitch, int elem) {
  GridSmem L;
  L.v = 0;
  L.buf = L.v + sizeof(float) * (size_t)dp;
  // max(4·dp, 4·kThreads) floats: the row groups' partial column sums of a
  // sweep (ng·dp ≤ 4·kThreads when ng > 1) and the column-slice reduction
  // (nsub subsets × cs columns ≤ kThreads)
  L.p = L.buf + sizeof(float) * (size_t)(dp > kThreads ? 4 * dp : 4 * kThreads);
  L.w = L.p + sizeof(float) * (size_t)Rpad;
  L.dvs = L.w + sizeof(float) * (size_t)Rpad;
  L.xss = L.dvs + sizeof(float) * (size_t)cs;
  L.red = L.xss + sizeof(float) * (size_t)cs;
  L.scal = L.red + sizeof(float) * kWarps;
  L.sa = L.scal + 64;  // 8 scalar slots, the staging mbarrier, padding (16-byte aligned)
  L.total = L.sa + (size_t)R * pitch * elem;
  return L;
}

template <int CH, typename TS>
__global__ void __launch_bounds__(kThreads, 1) aab_grid_kernel(const AabGridParams P) {
  const int blk = blockIdx.x, G = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int d = P.d, dp = P.dp;
  extern __shared__ float4 smem4[];
  char* base = reinterpret_cast<char*>(smem4);
  const GridSmem L = grid_smem_layout(dp, P.Rpad, P.cs, P.R, P.sa_pitch, (int)sizeof(TS));
  float* v = reinterpret_cast<float*>(base + L.v);
  float* buf = reinterpret_cast<float*>(base + L.buf);
  float* p = reinterpret_cast<float*>(base + L.p);
  float* w = reinterpret_cast<float*>(base + L.w);
  float* dvs = reinterpret_cast<float*>(base + L.dvs);
  float* xss = reinterpret_cast<float*>(base + L.xss);
  float* red = reinterpret_cast<float*>(base + L.red);
  float* scal = reinterpret_cast<float*>(base + L.scal);
  uint64_t* stage_bar = reinterpret_cast<uint64_t*>(base + L.scal + 32);
  int* s_ok = reinterpret_cast<int*>(base + L.scal + 48);
  TS* sa = reinterpret_cast<TS*>(base + L.sa);
  const TS* SAg = static_cast<const TS*>(P.SA);
  SolveCtl* ctl = P.ctl;

  // Control block: every block reads it before the first grid barrier; block
  // 0 writes it only after that barrier.
  int done = 0, outer = 0, max_outer = 0, g0known = 0, phase = 1, refresh = 1, corr = 0;
  float tol = 0.f, gnorm0 = 0.f, switch_tol = 0.f;
  if (ctl != nullptr) {
    done = ctl->done;
    outer = ctl->outer;
    max_outer = ctl->max_outer;
    g0known = ctl->gnorm0_known;
    tol = ctl->tol;
    gnorm0 = ctl->gnorm0;
    phase = ctl->phase;
    switch_tol = ctl->switch_tol;
    refresh = ctl->refresh;
    corr = ctl->corr;
  }
  if (done) {  // the same in every block: nothing has written it in this launch
    if (P.cond != 0ull && blk == 0 && tid == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
    return;
  }

  GridBarrier gbar{P.bar, 0u};
  if (tid == 0) grid_barrier_init(gbar, P.bar);  // before this block's first arrival
  const int r0 = blk * P.R;
  const int nr = max(0, min(P.m, r0 + P.R) - r0);
  const int c0 = blk * P.cs;
  const int c1 = min(dp, c0 + P.cs);
  const int ncol = max(0, c1 - c0);
  const uint32_t row_bytes = (uint32_t)P.sa_pitch * (uint32_t)sizeof(TS);
  // SA rows of this block: by bulk copies when the rows are 16-byte aligned
  // (sa_pitch elements of each row, sa_pitch ≤ ldsa; fp32 columns ≥ d are
  // masked when read), counted on one mbarrier; otherwise (fp32 only) by
  // plain masked loads.
  const bool bulk = P.sa_vec != 0;
  if (tid == 0) {
    mbar_init(stage_bar, 1);
    fence_mbar_init();
    if (bulk && nr > 0) {
      mbar_arrive_expect_tx(stage_bar, (uint32_t)nr * row_bytes);
      for (int i = 0; i < nr; ++i)
        bulk_copy_g2s(sa + (size_t)i * P.sa_pitch, SAg + (long long)(r0 + i) * P.ldsa, row_bytes, stage_bar);
    } else {
      mbar_arrive(stage_bar);
    }
  }
  if constexpr (sizeof(TS) == 4) {
    if (!bulk) {
      for (int i = 0; i < nr; ++i) {
        const float* src = reinterpret_cast<const float*>(SAg) + (long long)(r0 + i) * P.ldsa;
        for (int j = 4 * tid; j < dp; j += 4 * kThreads)
          *reinterpret_cast<float4*>(reinterpret_cast<float*>(sa) + (size_t)i * P.sa_pitch + j) =
              load4_masked(src, j, d, false);
      }
    }
  }

  // θ₁ v = g (identical in every block: same data, same summation order)
  float gsq = 0.f;
  for (int j = tid; j < dp; j += kThreads) {
    const float gj = j < d ? P.g[j] : 0.f;
    v[j] = gj;
    gsq = fmaf(gj, gj, gsq);
  }
  for (int i = tid; i < P.Rpad; i += kThreads) p[i] = 0.f;
  for (int j = tid; j < P.cs; j += kThreads) {
    dvs[j] = 0.f;
    xss[j] = 0.f;
  }
  const float theta1 = sqrtf(block_sum(gsq, red));
  bool alive = grid_barrier(gbar, s_ok);  // every block has read the control block
  // Every thread waits for its rows (also on the exits below, so that no copy
  // is still landing when the block exits).
  if (!mbar_wait(stage_bar, 0u, kWaitLimitNs)) alive = false;
  __syncthreads();
  if constexpr (sizeof(TS) == 4) {
    // Bulk-copied fp32 rows carry the caller's padding in columns [d, dp):
    // zero them, so that the sweeps read every column without a mask.
    if (bulk && d < dp && alive) {
      const int pad = dp - d;
      for (int e = tid; e < nr * pad; e += kThreads) {
        const int i = e / pad;
        reinterpret_cast<float*>(sa)[(size_t)i * P.sa_pitch + d + (e - i * pad)] = 0.f;
      }
      __syncthreads();
    }
  }
  if (!alive) {
    if (tid == 0) {
      atomicExch(&g_aab_grid_error, MIHS_ERR_TIMEOUT);
      if (ctl != nullptr) {
        ctl->status = MIHS_ERR_TIMEOUT;
        ctl->done = 1;
      }
      if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
    }
    return;
  }

  if (ctl != nullptr) {  // stop test of Algorithm 1 on ‖g‖ = θ₁
    const float g0 = g0known ? gnorm0 : theta1;
    if (P.hist != nullptr && blk == 0 && tid == 0 && outer < kHistCap) P.hist[outer] = theta1;
    const bool bad = !(theta1 <= 3.0e38f);
    // A refinement correction's gradient is approximate: it never stops the
    // solve; nor does a refinement solve's plain fp32 gradient (phase 0), whose
    // rounding floor lies above the tolerances refinement is asked for (it
    // can round to zero near the solution): only a compensated one certifies.
    const bool correction = phase == 1 && corr && !refresh;
    const bool conv = tol > 0.f && theta1 <= tol * g0 && !correction && phase != 0;
    const bool capped = outer >= max_outer;
    if (blk == 0 && tid == 0) refine_step_update(ctl, phase, refresh, corr, theta1, g0, tol, switch_tol);
    if (bad || conv || capped) {
      if (blk == 0 && tid == 0) {
        ctl->gnorm = theta1;
        ctl->gnorm0 = g0;
        ctl->gnorm0_known = 1;
        ctl->status = bad ? MIHS_ERR_NUMERIC : (conv ? MIHS_OK : MIHS_NOT_CONVERGED);
        ctl->done = 1;
        if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
      }
      return;
    }
  }

  int k = 0;
  if (theta1 > 0.f) {
    const float inv_theta1 = 1.0f / theta1;
    for (int j = tid; j < dp; j += kThreads) v[j] *= inv_theta1;
    __syncthreads();
    // First sweep: w = SA v (p = 0), its ρ² share and U = SAᵀw (ρp = w; the
    // normalisation by ρ is deferred so that one barrier publishes both).
    grid_sweep_store<CH, TS>(sa, P.sa_pitch, nr, d, dp, v, p, 0.f, w, P.sa_scale, P.scale_ld, r0, red, buf,
                             P.Upart + (size_t)blk * dp, P.rho2 + blk);
    alive = grid_barrier(gbar, s_ok);  // (A) ρ² and U partials
    const float lam = P.lambda;
    float rho = 0.f, rhobar = 0.f, c = 0.f, s = 0.f, phi = 0.f, theta = 0.f;
    float t = __int_as_float(0x7f800000);  // +inf
    const int nsub = P.cs >= kThreads ? 1 : kThreads / P.cs;
    bool first = true;
    while (alive) {
      // ---- after barrier A: U summed over blocks on the owned slice (nsub
      // subsets of blocks per column) and, in warp 0, ρ² — both loads issued
      // before either is waited for.
      float rv[8];  // warp 0: the ρ² partials, loads issued before the slice's (G ≤ 256)
      if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) rv[k] = lane + 32 * k < G ? __ldcg(P.rho2 + lane + 32 * k) : 0.f;
      }
      if (P.cs < kThreads) {
        const int jj = tid % P.cs, q = tid / P.cs;
        if (q < nsub && jj < ncol) buf[q * P.cs + jj] = strided_sum(P.Upart + c0 + jj, (size_t)dp, q, nsub, G);
      }
      if (warp == 0) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += rv[k];
        t = warp_sum(t);
        if (lane == 0) scal[2] = t;
      }
      __syncthreads();
      rho = sqrtf(scal[2]);
      if (first) {
        rhobar = sqrtf(rho * rho + lam);
        c = rho / rhobar;
        s = sqrtf(lam) / rhobar;
        phi = theta1 / rhobar;
        const float inv = 1.0f / rhobar;
        for (int jj = tid; jj < ncol; jj += kThreads) {
          dvs[jj] = v[c0 + jj] * inv;
          xss[jj] = phi * dvs[jj];
        }
        first = false;
      } else {
        // Eldén's rotation of √λ, the φ recursion and the forward substitution
        const float lambar = sqrtf(lam + (s * theta) * (s * theta));
        const float thetabar = c * theta;
        rhobar = sqrtf(rho * rho + lambar * lambar);
        const float inv_rhobar = 1.0f / rhobar;
        c = rho * inv_rhobar;
        s = lambar * inv_rhobar;
        phi = -phi * thetabar * inv_rhobar;
        for (int jj = tid; jj < ncol; jj += kThreads) {
          const float dn = (v[c0 + jj] - thetabar * dvs[jj]) * inv_rhobar;
          dvs[jj] = dn;
          xss[jj] = fmaf(phi, dn, xss[jj]);
        }
        t = fabsf(phi * rhobar) / theta1;
        ++k;
      }
      if (rho > 0.f) {
        const float inv = 1.0f / rho;
        for (int i = tid; i < nr; i += kThreads) p[i] = w[i] * inv;
      }
      if (!(t >= P.eps && k < P.max_passes && rho > 0.f)) break;  // the same in every block
      // ---- θ v := SAᵀp − ρ v on the owned slice, with SAᵀp = (Σ_b U_b)/ρ
      const float inv_rho = 1.0f / rho;
      float zpart = 0.f;
      for (int jj = tid; jj < ncol; jj += kThreads) {
        float u = 0.f;
        if (P.cs < kThreads) {
          for (int q = 0; q < nsub; ++q) u += buf[q * P.cs + jj];
        } else {
          u = strided_sum(P.Upart + c0 + jj, (size_t)dp, 0, 1, G);
        }
        const int j = c0 + jj;
        const float z = j < d ? u * inv_rho - rho * v[j] : 0.f;
        __stcg(P.Z + j, z);
        zpart = fmaf(z, z, zpart);
      }
      zpart = block_sum(zpart, red);
      if (tid == 0) __stcg(P.theta2 + blk, zpart);
      alive = grid_barrier(gbar, s_ok);  // (B) slices of θv and θ² partials
      if (!alive) break;
      // ---- after barrier B: θ² (warp 0) and all of Z, loads issued together
      float4 zr[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int j4 = tid + r * kThreads;
        zr[r] = 4 * j4 < dp ? __ldcg(reinterpret_cast<const float4*>(P.Z) + j4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (warp == 0) {
        const float t2 = sum_over_blocks(P.theta2, G);
        if (lane == 0) scal[3] = t2;
      }
      __syncthreads();
      theta = sqrtf(scal[3]);
      if (!(theta > 0.f)) break;  // invariant subspace: the same decision everywhere
      const float inv_theta = 1.0f / theta;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int j4 = tid + r * kThreads;
        if (4 * j4 < dp)
          reinterpret_cast<float4*>(v)[j4] =
              make_float4(zr[r].x * inv_theta, zr[r].y * inv_theta, zr[r].z * inv_theta, zr[r].w * inv_theta);
      }
      __syncthreads();
      // ---- ρ p := SA v − θ p (unnormalised in w until ρ is known), ρ², SAᵀw
      grid_sweep_store<CH, TS>(sa, P.sa_pitch, nr, d, dp, v, p, theta, w, P.sa_scale, P.scale_ld, r0, red, buf,
                               P.Upart + (size_t)blk * dp, P.rho2 + blk);
      alive = grid_barrier(gbar, s_ok);  // (A)
    }
  }
  if (!alive) {
    if (tid == 0) {
      atomicExch(&g_aab_grid_error, MIHS_ERR_TIMEOUT);
      if (ctl != nullptr) {
        ctl->status = MIHS_ERR_TIMEOUT;
        ctl->done = 1;
      }
      if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
    }
    return;
  }
  __syncthreads();

  // Outputs on the owned column slice: Δ and the heavy ball.
  for (int jj = tid; jj < ncol; jj += kThreads) {
    const int j = c0 + jj;
    if (j >= d) continue;
    const float dj = xss[jj];
    if (P.delta != nullptr) P.delta[j] = dj;
    if (P.x != nullptr) {
      const float xj = P.x[j], xp = P.x_prev[j];
      P.x[j] = xj + P.alpha * dj + P.beta * (xj - xp);
      P.x_prev[j] = xj;
    }
    if (P.x64 != nullptr) {
      const double xj = P.x64[j], xp = P.x_prev64[j];
      const double xn = xj + P.alpha64 * (double)dj + P.beta64 * (xj - xp);
      P.x64[j] = xn;
      P.x_prev64[j] = xj;
      if (P.x32_shadow != nullptr) P.x32_shadow[j] = (float)xn;
    }
  }
  if (blk == 0 && tid == 0) {
    if (P.passes != nullptr) *P.passes = k;
    if (ctl != nullptr) {
      ctl->outer = outer + 1;
      ctl->inner_total += k;
      ctl->gnorm = theta1;
      if (!g0known) {
        ctl->gnorm0 = theta1;
        ctl->gnorm0_known = 1;
      }
    }
  }
}

using GridFn = void (*)(const AabGridParams);

template <typename TS>
GridFn grid_kernel_for(int dp) {
  const int ch = (dp + 127) / 128;
  if (ch <= 2) return aab_grid_kernel<2, TS>;
  if (ch <= 4) return aab_grid_kernel<4, TS>;
  if (ch <= 8) return aab_grid_kernel<8, TS>;
  return aab_grid_kernel<16, TS>;
}

GridFn grid_kernel(int dp, int sa_type) {
  if (sa_type == MIHS_SA_BF16) return grid_kernel_for<__nv_bfloat16>(dp);
  if (sa_type == MIHS_SA_FP8E4M3) return grid_kernel_for<__nv_fp8_e4m3>(dp);
  return grid_kernel_for<float>(dp);
}

size_t elem_size(int sa_type) { return sa_type == MIHS_SA_BF16 ? 2 : (sa_type == MIHS_SA_FP8E4M3 ? 1 : 4); }

struct GridPlan {
  int G = 0, R = 0, Rpad = 0, cs = 0, pitch = 0;
  size_t smem = 0;
};

// Rows per block so that SA is spread over `blocks` blocks (0: one per SM),
// raised to the fewest blocks whose row slices fit in shared memory, and the
// launch that holds it; G = 0 when SA does not fit even one block per SM.
GridPlan plan_grid(int m, int dp, int sa_type, int blocks) {
  GridPlan gp;
  const int nsm = num_sms();
  int want = nsm;
  if (blocks > 0) {
    want = blocks;
  } else if (const char* e = std::getenv("MIHS_AAB_GRID_BLOCKS")) {
    const int v = std::atoi(e);
    if (v > 0) want = v;
  }
  if (want > nsm) want = nsm;
  const int pitch = sa_type == MIHS_SA_FP32 ? dp : (int)round_up(dp, 16);
  for (;; want = std::min(nsm, want + (want < 8 ? 1 : want / 8))) {
    const int R = (m + want - 1) / want;
    const int G = (m + R - 1) / R;
    if (G > 256) return gp;  // the kernel sums block partials with one load per lane and 8 per warp
    const int cs = (int)round_up((dp + G - 1) / G, 4);
    const GridSmem L = grid_smem_layout(dp, (int)round_up(R, 4), cs, R, pitch, (int)elem_size(sa_type));
    if (L.total > kSmemBudget + 16 * 1024) {
      if (want >= nsm) return gp;
      continue;
    }
    gp.G = G;
    gp.R = R;
    gp.Rpad = (int)round_up(R, 4);
    gp.cs = cs;
    gp.pitch = pitch;
    gp.smem = L.total;
    return gp;
  }
}

std::mutex g_grid_mu;

}  // namespace

size_t aab_grid_ws_bytes(int d) {
  const size_t dp = (size_t)round_up(d, 4);
  const size_t G4 = (size_t)round_up(num_sms(), 4);
  return kAabGridBarBytes + sizeof(float) * (G4 * dp + 2 * G4 + dp);
}

int aab_grid_device_error(int* code) {
  int v = 0, z = 0;
  MIHS_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_aab_grid_error, sizeof(int)));
  if (v != 0) MIHS_CUDA_TRY(cudaMemcpyToSymbol(g_aab_grid_error, &z, sizeof(int)));
  *code = v;
  return MIHS_OK;
}

int launch_aab_grid(const AabLaunch& a, void* ws, cudaStream_t s) {
  if (a.path || ws == nullptr) return MIHS_ERR_UNSUPPORTED;
  const int dp = (int)round_up(a.d, 4);
  // Quantised rows are bulk-copied (launch_aab has checked their 16-byte
  // alignment and pitch); fp32 rows when 16-byte aligned.
  const bool vec = (reinterpret_cast<uintptr_t>(a.SA) & 15u) == 0 &&
                   (a.sa_type != MIHS_SA_FP32 || a.ldsa % 4 == 0);
  if (a.sa_type != MIHS_SA_FP32 && (!vec || a.ldsa < round_up(dp, 16))) return MIHS_ERR_UNSUPPORTED;
  const GridPlan gp = plan_grid(a.m, dp, a.sa_type, a.grid_blocks);
  if (gp.G == 0) return MIHS_ERR_UNSUPPORTED;
  const GridFn fn = grid_kernel(dp, a.sa_type);
  {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    MIHS_CUDA_TRY(cudaFuncSetAttribute((void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gp.smem));
  }
  int per_sm = 0;
  MIHS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, gp.smem));
  if (per_sm < 1 || gp.G > per_sm * num_sms()) return MIHS_ERR_UNSUPPORTED;  // all blocks resident
  AabGridParams P = {};
  P.SA = a.SA;
  P.m = a.m;
  P.d = a.d;
  P.dp = dp;
  P.ldsa = a.ldsa;
  P.sa_pitch = gp.pitch;
  P.sa_scale = a.sa_type == MIHS_SA_FP8E4M3 ? a.sa_scale : nullptr;
  P.scale_ld = (dp + 127) / 128;
  P.R = gp.R;
  P.Rpad = gp.Rpad;
  P.cs = gp.cs;
  P.sa_vec = vec ? 1 : 0;
  P.g = a.g;
  P.lambda = a.lambda;
  P.eps = a.eps;
  P.max_passes = a.max_passes;
  P.delta = a.delta;
  P.passes = a.passes;
  P.alpha = a.alpha;
  P.beta = a.beta;
  P.x = a.x;
  P.x_prev = a.x_prev;
  P.x64 = a.x64;
  P.x_prev64 = a.x_prev64;
  P.x32_shadow = a.x32_shadow;
  P.alpha64 = a.alpha64;
  P.beta64 = a.beta64;
  P.ctl = a.ctl;
  P.hist = a.hist;
  P.cond = a.cond;
  const size_t G4 = (size_t)round_up(num_sms(), 4);
  P.bar = static_cast<unsigned int*>(ws);
  float* f = reinterpret_cast<float*>(static_cast<char*>(ws) + kAabGridBarBytes);
  P.Upart = f;
  P.rho2 = f + G4 * dp;
  P.theta2 = P.rho2 + G4;
  P.Z = P.theta2 + G4;  // 16-byte aligned (float4 reads)
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(gp.G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = gp.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  timing_begin(kTimerAab, s);
  MIHS_CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, P));
  timing_end(kTimerAab, s);
  count_launch();
  return MIHS_OK;
}

}  // namespace mihs
