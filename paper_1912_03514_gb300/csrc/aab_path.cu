// AAb_Solver (Algorithm 5, Section 3.6) for every λ of a path at once, fused
// with the stop test and heavy ball of Algorithm 1, for sketches too large
// for one cluster's shared memory (m = 4·sd(λ_min) makes SA up to ~17 MB).
//
// SA does not depend on λ, so the 16 bidiagonalisations (one per λ, each
// with its own v, p, scalars and stop) share every read of SA: one pass is
//   W = SA·V − P·diag(θ)   (m × 16)       U = SAᵀ·W   (d × 16)
// a register-tiled FP32 contraction like the path gradient pass.  The grid
// is cooperative (one block per SM, all resident): block c keeps rows
// [c·R, c·R + R) of SA in its shared memory for the whole launch; U is
// summed over blocks through global partials, each block reducing its own
// column slice; norms are summed over blocks in a fixed order so that every
// block computes the same scalars and takes the same branches.  Two grid
// barriers per pass (the deferred normalisation of p by ρ lets the ρ²
// partials travel with the U partials, as in the single-λ kernel).
#include <cooperative_groups.h>

#include <mutex>

#include "grid_sync.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace mihs {

namespace {

constexpr int kPL = 16;             // λ per launch
constexpr int kAThreads = 256;      // 8 warps
constexpr int kAWarps = kAThreads / 32;
constexpr size_t kAabPathSmemBudget = 220 * 1024;
constexpr size_t kBarFloats = 64;   // 256 bytes of the scratch hold the grid barrier word

__device__ int g_aab_path_error = 0;

struct AabPathParams {
  const float* SA;
  int m, d, dp;
  long long ldsa;
  int rows_per_block;  // R
  int pitch;           // dp + 4 (bank-conflict-free phase-1 reads)
  int cols_per_block;  // owned column slice (multiple of 4)
  const float* G;      // λ-major gradients, pitch dp
  float* X;            // λ-major iterates, pitch ldx
  long long ldx;
  float* Xprev;        // pitch dp
  SolveCtl* ctl;       // kPL control blocks
  PathScalars ps;
  float eps;
  int max_passes;
  int* path_ndone;
  int* path_all_done;
  unsigned long long cond;
  // global scratch
  float* Upart;        // blocks × kPL × dp
  float* rho2part;     // blocks × kPL
  float* theta2part;   // blocks × kPL
  float* Z;            // kPL × dp
  unsigned int* bar;   // grid barrier word (zero before the path solve)
};

struct AabPathSmem {
  size_t sa, v, p, w, rpart, dvs, xss, red;  // float offsets
  size_t total;                              // floats
};

__host__ __device__ inline AabPathSmem aab_path_layout(int R, int pitch, int dp, int cs) {
  AabPathSmem L;
  const size_t Rp = (size_t)((R + 15) / 16) * 16;  // phase 1 reads rows in groups of 16
  L.sa = 0;
  L.v = L.sa + Rp * pitch;
  L.p = L.v + (size_t)kPL * dp;
  L.w = L.p + Rp * kPL;
  L.rpart = L.w + Rp * kPL;
  L.dvs = L.rpart + (size_t)kAWarps * 16 * kPL;
  L.xss = L.dvs + (size_t)kPL * cs;
  L.red = L.xss + (size_t)kPL * cs;
  const size_t nred = (size_t)kPL * cs > 256 ? (size_t)kPL * cs : 256;
  L.total = L.red + nred;
  return L;
}

// Phase 1 for 16 rows starting at `row0` (< R): out[i][l] = SA_i·V_l over the
// block's rows, summed over the 32 K-groups (lane bits 3–4, then warps).
// The sums land in `dots` (16 × kPL); rows ≥ nr read stale data and are
// ignored by the caller.
__device__ __forceinline__ void rows16_dots(const float* sa, int pitch, int row0, const float* v, int dp, int d,
                                            float* rpart, float* dots) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kg = warp * 4 + (lane >> 3), rl = lane & 7;
  float acc[2][kPL];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int l = 0; l < kPL; ++l) acc[q][l] = 0.f;
  for (int c = 4 * kg; c < dp; c += 128) {
    float4 a0 = *reinterpret_cast<const float4*>(sa + (size_t)(row0 + rl) * pitch + c);
    float4 a1 = *reinterpret_cast<const float4*>(sa + (size_t)(row0 + rl + 8) * pitch + c);
    if (c + 4 > d) {
      if (c + 1 >= d) a0.y = a1.y = 0.f;
      if (c + 2 >= d) a0.z = a1.z = 0.f;
      a0.w = a1.w = 0.f;
    }
#pragma unroll
    for (int l = 0; l < kPL; ++l) {
      const float4 xv = *reinterpret_cast<const float4*>(v + (size_t)l * dp + c);
      acc[0][l] = fmaf(a0.x, xv.x, fmaf(a0.y, xv.y, fmaf(a0.z, xv.z, fmaf(a0.w, xv.w, acc[0][l]))));
      acc[1][l] = fmaf(a1.x, xv.x, fmaf(a1.y, xv.y, fmaf(a1.z, xv.z, fmaf(a1.w, xv.w, acc[1][l]))));
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int l = 0; l < kPL; ++l) {
      float t = acc[q][l];
      t += __shfl_xor_sync(0xffffffffu, t, 8);
      t += __shfl_xor_sync(0xffffffffu, t, 16);
      acc[q][l] = t;
    }
  if ((lane >> 3) == 0)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int l = 0; l < kPL; ++l) rpart[((size_t)warp * 16 + rl + 8 * q) * kPL + l] = acc[q][l];
  __syncthreads();
  {
    const int row = tid >> 4, l = tid & (kPL - 1);
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kAWarps; ++w) t += rpart[((size_t)w * 16 + row) * kPL + l];
    dots[row * kPL + l] = t;
  }
  __syncthreads();
}


// out[l] = Σ_b part[b][l] over the grid's blocks, in a fixed order that is the
// same in every block: 16 interleaved groups of blocks, then the groups.
// Latency-bound (the partials were written by other SMs moments ago), so the
// loads are spread over all threads and unrolled.
__device__ __forceinline__ void sum_over_blocks16(const float* part, int nblk, float* red, float* out) {
  const int tid = threadIdx.x, l = tid & (kPL - 1), q = tid >> 4;
  float t = 0.f;
  for (int b0 = q; b0 < nblk; b0 += 16 * 16) {  // every load of a batch before the first add
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int b = b0 + 16 * k;
      v[k] = b < nblk ? __ldcg(part + (size_t)b * kPL + l) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) t += v[k];
  }
  red[q * kPL + l] = t;
  __syncthreads();
  if (tid < kPL) {
    float u = 0.f;
#pragma unroll
    for (int g = 0; g < 16; ++g) u += red[g * kPL + tid];
    out[tid] = u;
  }
  __syncthreads();
}

// One sweep over the block's rows: W = SA·V − P·diag(θ) (rows ≥ nr give 0),
// per-λ ρ² partial → rho2part[blk], U = SAᵀW (this block's rows, split into
// rsub row subsets for narrow SA) → Upart[blk].
__device__ void path_sweep(const AabPathParams& P, const float* sa, int nr, const float* v, const float* p,
                           const float* theta, float* w, float* rpart, float* red) {
  const int tid = threadIdx.x, blk = blockIdx.x;
  const int dp = P.dp, d = P.d, pitch = P.pitch;
  const int Rp = ((P.rows_per_block + 15) / 16) * 16;
  float rsq = 0.f;  // thread (row, l) → its l's partial over the chunks
  for (int row0 = 0; row0 < Rp; row0 += 16) {
    rows16_dots(sa, pitch, row0, v, dp, d, rpart, w + (size_t)row0 * kPL);
    const int row = row0 + (tid >> 4), l = tid & (kPL - 1);
    float wv = 0.f;
    if (row < nr) wv = w[(size_t)row * kPL + l] - theta[l] * p[(size_t)row * kPL + l];
    w[(size_t)row * kPL + l] = wv;
    rsq = fmaf(wv, wv, rsq);
  }
  red[tid] = rsq;  // red has ≥ 256 floats
  __syncthreads();
  if (tid < kPL) {
    float t = 0.f;
    for (int q = 0; q < 16; ++q) t += red[q * kPL + tid];
    P.rho2part[(size_t)blk * kPL + tid] = t;
  }
  __syncthreads();  // every row of w written
  // phase 2: thread (cg, rs) accumulates 4 columns × 16 λ over rows rs, rs + rsub, …
  const int ngroups = dp >> 2;
  const int rsub = ngroups >= kAThreads ? 1 : kAThreads / ngroups;
  const int cgi = tid % ngroups, rs = tid / ngroups;
  if (rs < rsub) {
    float acc[4][kPL];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int l = 0; l < kPL; ++l) acc[q][l] = 0.f;
    for (int row = rs; row < nr; row += rsub) {
      const float4 a = *reinterpret_cast<const float4*>(sa + (size_t)row * pitch + 4 * cgi);
      const float4* wr = reinterpret_cast<const float4*>(w + (size_t)row * kPL);
#pragma unroll
      for (int l4 = 0; l4 < kPL / 4; ++l4) {
        const float4 r4 = wr[l4];
        const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc[0][4 * l4 + k] = fmaf(a.x, rv[k], acc[0][4 * l4 + k]);
          acc[1][4 * l4 + k] = fmaf(a.y, rv[k], acc[1][4 * l4 + k]);
          acc[2][4 * l4 + k] = fmaf(a.z, rv[k], acc[2][4 * l4 + k]);
          acc[3][4 * l4 + k] = fmaf(a.w, rv[k], acc[3][4 * l4 + k]);
        }
      }
    }
    const size_t upp = (size_t)rsub * dp;
#pragma unroll
    for (int l = 0; l < kPL; ++l)
      *reinterpret_cast<float4*>(P.Upart + ((size_t)blk * kPL + l) * upp + (size_t)rs * dp + 4 * cgi) =
          make_float4(acc[0][l], acc[1][l], acc[2][l], acc[3][l]);
  }
}

__global__ void __launch_bounds__(kAThreads, 1) aab_path_kernel(const AabPathParams P) {
  cg::grid_group grid = cg::this_grid();
  if (!grid.is_valid()) {
    // Not launched cooperatively (grid barriers unavailable): stop every λ
    // with an error instead of waiting at a barrier, and end the loop.
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicExch(&g_aab_path_error, MIHS_ERR_UNSUPPORTED);
      for (int l = 0; l < P.ps.nl; ++l) {
        P.ctl[l].status = MIHS_ERR_UNSUPPORTED;
        P.ctl[l].done = 1;
      }
      *P.path_all_done = 1;
      if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
    }
    return;
  }
  extern __shared__ __align__(16) float sm[];
  const int blk = blockIdx.x, nblk = gridDim.x, tid = threadIdx.x;
  __shared__ int s_ok;
  GridBarrier gbar{P.bar, 0u};
  if (tid == 0) grid_barrier_init(gbar, P.bar);  // before this block's first arrival
  bool alive = true;
  const int d = P.d, dp = P.dp, R = P.rows_per_block, pitch = P.pitch, cs = P.cols_per_block;
  const AabPathSmem L = aab_path_layout(R, pitch, dp, cs);
  float* sa = sm + L.sa;
  float* v = sm + L.v;
  float* p = sm + L.p;
  float* w = sm + L.w;
  float* rpart = sm + L.rpart;
  float* dvs = sm + L.dvs;
  float* xss = sm + L.xss;
  float* red = sm + L.red;  // ≥ 256 floats (rpart spills into it: sized together)
  __shared__ float s_theta1[kPL], s_rho[kPL], s_rhobar[kPL], s_c[kPL], s_s[kPL], s_phi[kPL], s_theta[kPL],
      s_t[kPL], s_g0[kPL];
  __shared__ int s_k[kPL], s_act[kPL], s_run[kPL], s_stop[kPL];
  __shared__ int s_any;
  __shared__ float s_sum[kPL];
  const int nl = P.ps.nl;
  const int r0 = blk * R;
  const int nr = max(0, min(P.m, r0 + R) - r0);
  const int Rp = ((R + 15) / 16) * 16;
  const int c0 = blk * cs, c1 = min(dp, c0 + cs), ncol = max(0, c1 - c0);

  // SA rows of this block (zero beyond nr), V = g, P = 0.
  {
    const int q4 = dp >> 2;
#pragma unroll 4
    for (int e = tid; e < Rp * q4; e += kAThreads) {
      const int i = e / q4, j = 4 * (e - i * q4);
      *reinterpret_cast<float4*>(sa + (size_t)i * pitch + j) =
          i < nr ? __ldg(reinterpret_cast<const float4*>(P.SA + (long long)(r0 + i) * P.ldsa + j))
                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll 4
    for (int e = tid; e < kPL * q4; e += kAThreads) {
      const int l = e / q4, j = 4 * (e - l * q4);
      float4 g4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (l < nl) {
        g4 = __ldg(reinterpret_cast<const float4*>(P.G + (size_t)l * dp + j));
        if (j + 1 >= d) g4.y = 0.f;  // columns ≥ d are zero
        if (j + 2 >= d) g4.z = 0.f;
        if (j + 3 >= d) g4.w = 0.f;
      }
      *reinterpret_cast<float4*>(v + (size_t)l * dp + j) = g4;
    }
  }
  for (int i = tid; i < Rp * kPL; i += kAThreads) p[i] = 0.f;
  __syncthreads();
  {  // θ₁ = ‖g_l‖: 16 column interleaves per λ, summed in a fixed order
    const int l = tid & (kPL - 1), part = tid >> 4;
    float t = 0.f;
    for (int j = part; j < dp; j += 16) t = fmaf(v[(size_t)l * dp + j], v[(size_t)l * dp + j], t);
    red[part * kPL + l] = t;
  }
  __syncthreads();
  if (tid < kPL) {
    const int l = tid;
    float t = 0.f;
    for (int q = 0; q < 16; ++q) t += red[q * kPL + l];
    const float theta1 = sqrtf(t);
    int run = 0, stop = 0;
    float g0 = theta1;
    if (l < nl) {
      const SolveCtl c = P.ctl[l];
      if (!c.done) {
        g0 = c.gnorm0_known ? c.gnorm0 : theta1;
        const bool bad = !(theta1 <= 3.0e38f);
        const bool conv = c.tol > 0.f && theta1 <= c.tol * g0;
        const bool capped = c.outer >= c.max_outer;
        if (bad || conv || capped) stop = bad ? 3 : (conv ? 1 : 2);
        else run = 1;
      }
    }
    s_theta1[l] = theta1;
    s_g0[l] = g0;
    s_run[l] = run;
    s_stop[l] = stop;
    s_act[l] = run && theta1 > 0.f;
    s_k[l] = 0;
    s_theta[l] = 0.f;
    s_t[l] = __int_as_float(0x7f800000);
  }
  __syncthreads();
  if (tid == 0) {
    int any = 0;
    for (int l = 0; l < kPL; ++l) any |= s_act[l];
    s_any = any;
  }
  __syncthreads();
  const bool work = s_any != 0;  // the same in every block
  if (work) {
    for (int i = tid; i < kPL * dp; i += kAThreads) {
      const int l = i / dp;
      v[i] = s_act[l] ? v[i] / s_theta1[l] : 0.f;
    }
    __syncthreads();
    path_sweep(P, sa, nr, v, p, s_theta, w, rpart, red);
    alive = grid_barrier(gbar, &s_ok);  // (A) ρ² and U partials of the first sweep
    if (alive) {
    sum_over_blocks16(P.rho2part, nblk, red, s_sum);
    if (tid < kPL) {
      const int l = tid;
      const float rho = sqrtf(s_sum[l]), lam = P.ps.lam[l];
      const float rhobar = sqrtf(rho * rho + lam);
      s_rho[l] = rho;
      s_rhobar[l] = rhobar;
      s_c[l] = rho / rhobar;
      s_s[l] = sqrtf(lam) / rhobar;
      s_phi[l] = s_theta1[l] / rhobar;
    }
    __syncthreads();
    for (int i = tid; i < kPL * cs; i += kAThreads) {
      const int l = i / cs, j = c0 + (i - l * cs);
      const float dn = (j < c1 && s_act[l]) ? v[(size_t)l * dp + j] / s_rhobar[l] : 0.f;
      dvs[i] = dn;
      xss[i] = s_act[l] ? s_phi[l] * dn : 0.f;
    }
    for (int i = tid; i < nr * kPL; i += kAThreads) {
      const int l = i & (kPL - 1);
      p[i] = (s_act[l] && s_rho[l] > 0.f) ? w[i] / s_rho[l] : 0.f;
    }
    __syncthreads();
    for (;;) {
      if (tid < kPL) {
        const int l = tid;
        s_act[l] = s_act[l] && s_t[l] >= P.eps && s_k[l] < P.max_passes && s_rho[l] > 0.f;
      }
      __syncthreads();
      if (tid == 0) {
        int any = 0;
        for (int l = 0; l < kPL; ++l) any |= s_act[l];
        s_any = any;
      }
      __syncthreads();
      if (!s_any) break;  // same decision in every block
      // (B) θv = SAᵀp − ρv on the owned column slice: U summed over blocks
      // and row subsets in a fixed order.
      {
        const int ngroups = dp >> 2;
        const int rsub = ngroups >= kAThreads ? 1 : kAThreads / ngroups;
        const size_t upp = (size_t)rsub * dp;
        const int npairs = ncol * kPL;
        const int nq = ncol >> 2;               // float4 groups of the owned slice
        const int nitems = nq * kPL;            // (λ, float4 group)
        const int ngrp = nitems > 0 ? max(1, min(kAThreads / nitems, 8)) : 1;
        float* zsum = rpart;  // ngrp × npairs ≤ 8 × 256 floats
        for (int idx = tid; idx < nitems * ngrp; idx += kAThreads) {
          const int item = idx % nitems, grp = idx / nitems;
          const int l = item / nq, j = c0 + 4 * (item - l * nq);
          float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
          // written by other blocks in this launch: read through L2, not L1;
          // the (block, row subset) pairs in order, eight loads issued per batch
          const int nb = nblk > grp ? (nblk - grp + ngrp - 1) / ngrp : 0;
          const int ne = nb * rsub;
          for (int e0 = 0; e0 < ne; e0 += 8) {
            float4 u4[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int e = e0 + k;
              const int b = grp + (e / rsub) * ngrp, q = e % rsub;
              u4[k] = e < ne ? __ldcg(reinterpret_cast<const float4*>(P.Upart + ((size_t)b * kPL + l) * upp +
                                                                      (size_t)q * dp + j))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              t.x += u4[k].x;
              t.y += u4[k].y;
              t.z += u4[k].z;
              t.w += u4[k].w;
            }
          }
          float* zs = zsum + (size_t)grp * npairs + l * ncol + (j - c0);
          zs[0] = t.x;
          zs[1] = t.y;
          zs[2] = t.z;
          zs[3] = t.w;
        }
        __syncthreads();
        const int nparts = ngrp;
        for (int pair = tid; pair < npairs; pair += kAThreads) {
          const int l = pair / ncol, j = c0 + (pair - l * ncol);
          float u = 0.f;
          for (int q = 0; q < nparts; ++q) u += zsum[q * npairs + pair];
          const float z = (s_act[l] && j < d) ? u / s_rho[l] - s_rho[l] * v[(size_t)l * dp + j] : 0.f;
          P.Z[(size_t)l * dp + j] = z;
          red[pair] = z * z;  // npairs ≤ red's size
        }
        __syncthreads();
        if (tid < kPL) {
          float t = 0.f;
          for (int jj = 0; jj < ncol; ++jj) t += red[tid * ncol + jj];
          P.theta2part[(size_t)blk * kPL + tid] = t;
        }
      }
      alive = grid_barrier(gbar, &s_ok);  // (B) Z slices and θ² partials visible
      if (!alive) break;
      sum_over_blocks16(P.theta2part, nblk, red, s_sum);
      if (tid < kPL) {
        const int l = tid;
        const float theta = sqrtf(s_sum[l]);
        s_theta[l] = theta;
        if (!(theta > 0.f)) s_act[l] = 0;  // invariant subspace reached for this λ
      }
      __syncthreads();
      {
        const int n4 = kPL * dp / 4;
#pragma unroll 4
        for (int i4 = tid; i4 < n4; i4 += kAThreads) {
          const int l = (4 * i4) / dp;
          float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          if (s_act[l]) {
            z = __ldcg(reinterpret_cast<const float4*>(P.Z) + i4);
            const float inv = 1.0f / s_theta[l];
            z.x *= inv;
            z.y *= inv;
            z.z *= inv;
            z.w *= inv;
          }
          reinterpret_cast<float4*>(v)[i4] = z;
        }
      }
      if (tid < kPL && !s_act[tid]) s_theta[tid] = 0.f;
      __syncthreads();
      // (A) ρp = SAv − θp, its ρ² and SAᵀ(ρp) in one sweep
      path_sweep(P, sa, nr, v, p, s_theta, w, rpart, red);
      alive = grid_barrier(gbar, &s_ok);  // (A)
      if (!alive) break;
      sum_over_blocks16(P.rho2part, nblk, red, s_sum);
      if (tid < kPL) {
        const int l = tid;
        if (s_act[l]) {
          const float rho = sqrtf(s_sum[l]), lam = P.ps.lam[l], theta = s_theta[l];
          // Eldén's rotation of √λ, the φ recursion and the forward substitution
          const float lambar = sqrtf(lam + (s_s[l] * theta) * (s_s[l] * theta));
          const float thetabar = s_c[l] * theta;
          const float rhobar = sqrtf(rho * rho + lambar * lambar);
          const float inv_rhobar = 1.0f / rhobar;
          s_c[l] = rho * inv_rhobar;
          s_s[l] = lambar * inv_rhobar;
          s_phi[l] = -s_phi[l] * thetabar * inv_rhobar;
          s_rho[l] = rho;
          s_rhobar[l] = rhobar;
          s_theta[l] = thetabar;  // θ̄ for the slice update below; θ is rebuilt next pass
          s_t[l] = fabsf(s_phi[l] * rhobar) / s_theta1[l];
          s_k[l] += 1;
        }
      }
      __syncthreads();
      for (int i = tid; i < kPL * cs; i += kAThreads) {
        const int l = i / cs, j = c0 + (i - l * cs);
        if (s_act[l] && j < c1) {
          const float dn = (v[(size_t)l * dp + j] - s_theta[l] * dvs[i]) / s_rhobar[l];
          dvs[i] = dn;
          xss[i] = fmaf(s_phi[l], dn, xss[i]);
        }
      }
      for (int i = tid; i < nr * kPL; i += kAThreads) {
        const int l = i & (kPL - 1);
        if (s_act[l]) p[i] = s_rho[l] > 0.f ? w[i] / s_rho[l] : 0.f;
      }
      __syncthreads();
      if (tid < kPL) s_theta[tid] = 0.f;  // unused until rebuilt
      __syncthreads();
    }
    }  // alive after the first sweep
  }
  // every block has read the control blocks before block 0 writes them
  if (alive) alive = grid_barrier(gbar, &s_ok);
  if (!alive) {
    // A grid barrier ran out: stop every λ of the path with an error.
    if (tid == 0) {
      atomicExch(&g_aab_path_error, MIHS_ERR_TIMEOUT);
      for (int l = 0; l < P.ps.nl; ++l) {
        P.ctl[l].status = MIHS_ERR_TIMEOUT;
        P.ctl[l].done = 1;
      }
      *P.path_all_done = 1;
      if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
    }
    return;
  }
  // Heavy ball on the owned slice for every λ that took this step.
  for (int i = tid; i < kPL * cs; i += kAThreads) {
    const int l = i / cs, j = c0 + (i - l * cs);
    if (l < nl && s_run[l] && j < c1 && j < d) {
      float* xl = P.X + (long long)l * P.ldx;
      float* xp = P.Xprev + (size_t)l * dp;
      const float xj = xl[j], xo = xp[j];
      xl[j] = xj + P.ps.alpha[l] * xss[i] + P.ps.beta[l] * (xj - xo);
      xp[j] = xj;
    }
  }
  if (blk == 0 && tid < kPL) {
    const int l = tid;
    if (l < nl) {
      SolveCtl* c = P.ctl + l;
      if (s_run[l]) {
        c->outer += 1;
        c->inner_total += s_k[l];
        c->gnorm = s_theta1[l];
        if (!c->gnorm0_known) {
          c->gnorm0 = s_theta1[l];
          c->gnorm0_known = 1;
        }
      } else if (s_stop[l]) {
        c->gnorm = s_theta1[l];
        c->gnorm0 = s_g0[l];
        c->gnorm0_known = 1;
        c->status = s_stop[l] == 3 ? MIHS_ERR_NUMERIC : (s_stop[l] == 1 ? MIHS_OK : MIHS_NOT_CONVERGED);
        c->done = 1;
        if (atomicAdd(P.path_ndone, 1) + 1 == nl) {  // the last λ of the path to stop
          *P.path_all_done = 1;
          if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
        }
      }
    }
  }
}

}  // namespace

int aab_path_device_error(int* code) {
  int v = 0, z = 0;
  MIHS_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_aab_path_error, sizeof(int)));
  MIHS_CUDA_TRY(cudaMemcpyToSymbol(g_aab_path_error, &z, sizeof(int)));
  *code = v;
  return MIHS_OK;
}

size_t aab_path_ws_floats(int dp) {
  const size_t G = (size_t)num_sms();
  return kBarFloats + G * kPL * 1024 + 2 * G * kPL + (size_t)kPL * dp;
}

int launch_aab_path(const AabLaunch& a, float* ws, cudaStream_t s) {
  const int dp = (int)round_up(a.d, 4);
  if (!a.path || a.d > 1024 || a.x64 != nullptr || ws == nullptr || a.sa_type != MIHS_SA_FP32)
    return MIHS_ERR_UNSUPPORTED;
  const int nsm = num_sms();
  // rows per block: a multiple of 16 with at most one block per SM
  int R = (int)round_up((a.m + nsm - 1) / nsm, 16);
  const int G = (a.m + R - 1) / R;
  const int cs = (int)round_up((dp + G - 1) / G, 4);
  if (cs * kPL > kAWarps * 16 * kPL) return MIHS_ERR_UNSUPPORTED;  // owned slice must fit the reduce buffer
  const int pitch = dp + 4;
  const AabPathSmem L = aab_path_layout(R, pitch, dp, cs);
  const size_t smem = L.total * sizeof(float);
  if (smem > kAabPathSmemBudget) return MIHS_ERR_UNSUPPORTED;
  if ((a.ldsa % 4) != 0 || (reinterpret_cast<uintptr_t>(a.SA) & 15u) != 0) return MIHS_ERR_UNSUPPORTED;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    MIHS_CUDA_TRY(cudaFuncSetAttribute(aab_path_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int per_sm = 0;
  MIHS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aab_path_kernel, kAThreads, smem));
  if (per_sm < 1 || G > per_sm * nsm) return MIHS_ERR_UNSUPPORTED;  // all blocks must be resident
  AabPathParams P = {};
  P.SA = static_cast<const float*>(a.SA);
  P.m = a.m;
  P.d = a.d;
  P.dp = dp;
  P.ldsa = a.ldsa;
  P.rows_per_block = R;
  P.pitch = pitch;
  P.cols_per_block = cs;
  P.G = a.g;
  P.X = a.x;
  P.ldx = a.path_ldx;
  P.Xprev = a.x_prev;
  P.ctl = a.ctl;
  P.ps = a.ps;
  P.eps = a.eps;
  P.max_passes = a.max_passes;
  P.path_ndone = a.path_ndone;
  P.path_all_done = a.path_all_done;
  P.cond = a.cond;
  const size_t Gmax = (size_t)nsm;
  P.bar = reinterpret_cast<unsigned int*>(ws);  // first kBarFloats floats: the barrier word
  ws += kBarFloats;
  P.Upart = ws;
  P.rho2part = ws + Gmax * kPL * 1024;
  P.theta2part = P.rho2part + Gmax * kPL;
  P.Z = P.theta2part + Gmax * kPL;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kAThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  timing_begin(kTimerAab, s);
  MIHS_CUDA_TRY(cudaLaunchKernelEx(&cfg, aab_path_kernel, P));
  timing_end(kTimerAab, s);
  count_launch();
  return MIHS_OK;
}

}  // namespace mihs
