// AAb_Solver (Algorithm 5, Section 3.6) on the sketched matrix SA, fused with
// the heavy-ball step of Eq. mihs1 and the stop test of Algorithm 1.
//
// The solver is latency-bound: each loop pass is one product with SAᵀ, one
// with SA and two norms, all of which every later step depends on.  It runs
// as ONE thread-block cluster (up to 16 blocks on 16 SMs):
//   * SA is split by rows; block `rank` keeps rows [rank·R, rank·R + R) in
//     its shared memory for the whole solve (m·d·4/CL bytes per block), so
//     both products read SA from shared memory, not from L2.
//   * SA·v needs the full d-vector v in every block (replicated); SAᵀp gives a
//     partial d-vector per block, summed by a reduce-scatter over distributed
//     shared memory (block r owns a slice of the columns), and the new v is
//     all-gathered the same way.  ‖·‖² partials are exchanged through DSMEM.
//   * Two cluster barriers per pass: the normalisation of p by ρ is deferred
//     so that the ρ² partials and the next SAᵀw partials travel together.
//     Scalars (θ, ρ, c, s, φ, t) are recomputed identically in every thread
//     from partials summed in a fixed order, so all blocks take the same
//     branch and the result is deterministic.
// The d-vectors of the recursion (v, d, x) are replicated per block (O(d)
// work, negligible next to the O(md/CL) products).
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"

namespace mihs {
namespace aabk {

namespace cg = cooperative_groups;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr size_t kSmemBudget = 210 * 1024;

struct AabParams {
  const void* SA;      // element type: the kernel's TS (float, bf16 or fp8 e4m3)
  int m, d, dp;        // dp = d rounded up to 4
  long long ldsa;
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
  int rpc;             // rows per block
  int rpc_pad;         // rpc rounded up to 4
  int cols_per;        // column slice per block (a power of two ≥ 4)
  int cols_log2;
  int sa_in_smem;
  int sa_vec;          // SA rows may be read as float4 (ldsa % 4 == 0, 16-byte aligned)
  int sa_pitch;        // row pitch (elements of TS) of SA rows kept in shared memory
  const float* sa_scale;  // fp8: one scale per 128 × 128 tile, row-major, scale_ld tiles per tile row
  int scale_ld;
  int path;            // λ-path mode: cluster row blockIdx.y solves λ_y
  PathScalars ps;
  long long path_ldg, path_ldx;
  int* path_ndone;
  int* path_all_done;
};

// Deterministic block-wide sum; every thread returns the same value.
__device__ __forceinline__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t += red[w];
  __syncthreads();
  return t;
}

__device__ __forceinline__ float4 load4_masked(const float* row, int j, int d, bool vec = true) {
  // j is a multiple of 4 and j < dp; columns ≥ d read as zero.
  if (vec && j + 4 <= d) return *reinterpret_cast<const float4*>(row + j);
  if (j + 4 <= d) return make_float4(row[j], row[j + 1], row[j + 2], row[j + 3]);
  float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
  if (j < d) t.x = row[j];
  if (j + 1 < d) t.y = row[j + 1];
  if (j + 2 < d) t.z = row[j + 2];
  return t;
}

// Four consecutive elements of a stored SA row (j a multiple of 4, j < dp),
// decoded to fp32 and multiplied by the tile's scale (fp8); columns ≥ d are
// zero in the quantised layouts, masked in the fp32 one.
template <typename TS>
__device__ __forceinline__ float4 load_sa4(const TS* row, int j, int d, bool vec, float scale);

template <>
__device__ __forceinline__ float4 load_sa4<float>(const float* row, int j, int d, bool vec, float) {
  return load4_masked(row, j, d, vec);
}

template <>
__device__ __forceinline__ float4 load_sa4<__nv_bfloat16>(const __nv_bfloat16* row, int j, int, bool, float) {
  const uint2 raw = *reinterpret_cast<const uint2*>(row + j);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
  return make_float4(a.x, a.y, b.x, b.y);
}

template <>
__device__ __forceinline__ float4 load_sa4<__nv_fp8_e4m3>(const __nv_fp8_e4m3* row, int j, int, bool, float scale) {
  const uint32_t raw = *reinterpret_cast<const uint32_t*>(row + j);
  __nv_fp8x4_e4m3 q;
  q.__x = raw;
  const float4 f = static_cast<float4>(q);
  return make_float4(f.x * scale, f.y * scale, f.z * scale, f.w * scale);
}

// Σ over the cluster of one scalar slot: lane r loads rank r's value, then a
// fixed butterfly sums them (identical wherever it is computed).
template <int CL>
__device__ __forceinline__ float cluster_scalar_sum(const float* my_rank_scal, int slot) {
  const int lane = threadIdx.x & 31;
  float v = lane < CL ? my_rank_scal[slot] : 0.f;
  return warp_sum(v);
}

// Fused sweep over the block's rows of SA (each row read once per pass):
//   w_i = SA_i·v − θ·p_i            (warp all-reduce of the row dot)
//   u  += SA_iᵀ·w_i                 (lane ℓ accumulates columns 4ℓ + 128c)
//   ρ²_part += w_i²
// Warp `warp` takes rows warp, warp + 8, …; v and u live in registers (CH
// float4 per lane), the per-warp u partials are written to `wpart`.
template <int CH, typename TS>
__device__ __forceinline__ float fused_sweep(const TS* SAc, long long ldc, int nr, int d,
                                             const float* v, const float* p, float theta,
                                             float* w, float* wpart, int dp, bool vec,
                                             const float* scales, int sld, int r0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 vr[CH], ur[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int j = 4 * lane + 128 * c;
    vr[c] = j < dp ? *reinterpret_cast<const float4*>(v + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    ur[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float rsq = 0.f;
  int i = warp;
  if constexpr (CH <= 8) {
    // Two rows per step (i and i + kWarps): independent loads, dots and
    // shuffle trees in flight together (the sweep is latency-bound).
    for (; i + kWarps < nr; i += 2 * kWarps) {
      const TS* row0 = SAc + (long long)i * ldc;
      const TS* row1 = row0 + (long long)kWarps * ldc;
      const float* srow0 = scales != nullptr ? scales + (size_t)((r0 + i) >> 7) * sld : nullptr;
      const float* srow1 = scales != nullptr ? scales + (size_t)((r0 + i + kWarps) >> 7) * sld : nullptr;
      float4 a[CH], b[CH];
      float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int j = 4 * lane + 128 * c;
        a[c] = j < dp ? load_sa4<TS>(row0, j, d, vec, srow0 != nullptr ? srow0[c] : 1.f)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
        b[c] = j < dp ? load_sa4<TS>(row1, j, d, vec, srow1 != nullptr ? srow1[c] : 1.f)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
        s0 = fmaf(a[c].x, vr[c].x, s0);
        s1 = fmaf(a[c].y, vr[c].y, s1);
        s0 = fmaf(a[c].z, vr[c].z, s0);
        s1 = fmaf(a[c].w, vr[c].w, s1);
        t0 = fmaf(b[c].x, vr[c].x, t0);
        t1 = fmaf(b[c].y, vr[c].y, t1);
        t0 = fmaf(b[c].z, vr[c].z, t0);
        t1 = fmaf(b[c].w, vr[c].w, t1);
      }
      float sa_ = s0 + s1, sb_ = t0 + t1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sa_ += __shfl_xor_sync(0xffffffffu, sa_, o);
        sb_ += __shfl_xor_sync(0xffffffffu, sb_, o);
      }
      const float wa = sa_ - theta * p[i], wb = sb_ - theta * p[i + kWarps];
      rsq = fmaf(wa, wa, rsq);
      rsq = fmaf(wb, wb, rsq);
      if (lane == 0) {
        w[i] = wa;
        w[i + kWarps] = wb;
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        ur[c].x = fmaf(b[c].x, wb, fmaf(a[c].x, wa, ur[c].x));
        ur[c].y = fmaf(b[c].y, wb, fmaf(a[c].y, wa, ur[c].y));
        ur[c].z = fmaf(b[c].z, wb, fmaf(a[c].z, wa, ur[c].z));
        ur[c].w = fmaf(b[c].w, wb, fmaf(a[c].w, wa, ur[c].w));
      }
    }
  }
  for (; i < nr; i += kWarps) {
    const TS* row = SAc + (long long)i * ldc;
    const float* srow = scales != nullptr ? scales + (size_t)((r0 + i) >> 7) * sld : nullptr;
    float4 a[CH];
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j = 4 * lane + 128 * c;
      a[c] = j < dp ? load_sa4<TS>(row, j, d, vec, srow != nullptr ? srow[c] : 1.f)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
      s0 = fmaf(a[c].x, vr[c].x, s0);
      s1 = fmaf(a[c].y, vr[c].y, s1);
      s0 = fmaf(a[c].z, vr[c].z, s0);
      s1 = fmaf(a[c].w, vr[c].w, s1);
    }
    const float wi = warp_sum(s0 + s1) - theta * p[i];
    rsq = fmaf(wi, wi, rsq);
    if (lane == 0) w[i] = wi;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      ur[c].x = fmaf(a[c].x, wi, ur[c].x);
      ur[c].y = fmaf(a[c].y, wi, ur[c].y);
      ur[c].z = fmaf(a[c].z, wi, ur[c].z);
      ur[c].w = fmaf(a[c].w, wi, ur[c].w);
    }
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int j = 4 * lane + 128 * c;
    if (j < dp) *reinterpret_cast<float4*>(wpart + (size_t)warp * dp + j) = ur[c];
  }
  return rsq;  // this warp's share of ρ² (same in all lanes)
}

// Split sweep over SA rows held in shared memory (each row read twice per
// pass, with no dependency between a row's dot and its update).  Rows sit at
// `sa` with a pitch of `sp` elements; the columns in [d, dp) are zero there
// (masked when staged, or zero in the quantised layouts), so every load is an
// unmasked 16-byte (fp32), 8-byte (bf16) or 4-byte (fp8) read.

// Four consecutive decoded elements of a row held in shared memory.
template <typename TS>
__device__ __forceinline__ float4 ld_sa_row4(const TS* row, int j, float scale);
template <>
__device__ __forceinline__ float4 ld_sa_row4<float>(const float* row, int j, float) {
  return *reinterpret_cast<const float4*>(row + j);
}
template <>
__device__ __forceinline__ float4 ld_sa_row4<__nv_bfloat16>(const __nv_bfloat16* row, int j, float s) {
  return load_sa4<__nv_bfloat16>(row, j, 0, true, s);
}
template <>
__device__ __forceinline__ float4 ld_sa_row4<__nv_fp8_e4m3>(const __nv_fp8_e4m3* row, int j, float s) {
  return load_sa4<__nv_fp8_e4m3>(row, j, 0, true, s);
}

// Phase 1, row dots: w_i = SA_i·v − θ·p_i for the block's rows.  Warp `warp`
// takes rows warp, warp + kWarps, …: four at a time (independent loads,
// chains and shuffle trees) while four remain, then one at a time.  A lane's
// column groups j = 4·lane + 128·c at or past dp read the group dp − 4 with
// v = 0.  Lane 0 stores w_i.  Returns the warp's share of ρ² = Σ w_i² (rows in
// a fixed order; the same in all lanes).
template <int CH, typename TS>
__device__ __forceinline__ float row_dots(const TS* sa, int sp, int nr, const float* v, const float* p, float theta,
                                          float* w, int dp, const float* scales, int sld, int r0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 vr[CH];
  int jc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int j = 4 * lane + 128 * c;
    jc[c] = j < dp ? j : dp - 4;
    vr[c] = j < dp ? *reinterpret_cast<const float4*>(v + j) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float rsq = 0.f;
  int i = warp;
  for (; i + 3 * kWarps < nr; i += 4 * kWarps) {
    float s0[4], s1[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      s0[r] = 0.f;
      s1[r] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int ii = i + r * kWarps;
        const float sc = scales != nullptr ? scales[(size_t)((r0 + ii) >> 7) * sld + (jc[c] >> 7)] : 1.f;
        const float4 a = ld_sa_row4<TS>(sa + (size_t)ii * sp, jc[c], sc);
        s0[r] = fmaf(a.x, vr[c].x, s0[r]);
        s1[r] = fmaf(a.y, vr[c].y, s1[r]);
        s0[r] = fmaf(a.z, vr[c].z, s0[r]);
        s1[r] = fmaf(a.w, vr[c].w, s1[r]);
      }
    }
    float t[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) t[r] = s0[r] + s1[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int r = 0; r < 4; ++r) t[r] += __shfl_xor_sync(0xffffffffu, t[r], o);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int ii = i + r * kWarps;
      const float wi = t[r] - theta * p[ii];
      rsq = fmaf(wi, wi, rsq);
      if (lane == 0) w[ii] = wi;
    }
  }
  for (; i < nr; i += kWarps) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const float sc = scales != nullptr ? scales[(size_t)((r0 + i) >> 7) * sld + (jc[c] >> 7)] : 1.f;
      const float4 a = ld_sa_row4<TS>(sa + (size_t)i * sp, jc[c], sc);
      s0 = fmaf(a.x, vr[c].x, s0);
      s1 = fmaf(a.y, vr[c].y, s1);
      s0 = fmaf(a.z, vr[c].z, s0);
      s1 = fmaf(a.w, vr[c].w, s1);
    }
    const float wi = warp_sum(s0 + s1) - theta * p[i];
    rsq = fmaf(wi, wi, rsq);
    if (lane == 0) w[i] = wi;
  }
  return rsq;
}

// Phase 2, column sums: u_j = Σ_i SA_ij·w_i over the block's rows.  The
// dp/4 column groups (16 bytes) are spread over the threads: with at least
// kThreads groups, thread t owns groups t + kThreads·c over all rows; with
// fewer, the threads form ng = kThreads/⌈groups⌉₃₂ row groups, group g
// summing rows ≡ g (mod ng), and the ng partials are added in order of g
// through `tmp` (ng·dp floats).  Each thread keeps four accumulators (rows
// four apart, each in row order) added as (u0 + u1) + (u2 + u3).  w_i is a
// shared-memory broadcast.  Writes u to out[0, dp) (shared or global memory);
// synchronises the block when ng > 1.
template <int CH, typename TS>
__device__ __forceinline__ void col_sums(const TS* sa, int sp, int nr, int dp, const float* w, const float* scales,
                                         int sld, int r0, float* tmp, float* out) {
  constexpr int CC = (CH * 128 + 4 * kThreads - 1) / (4 * kThreads);
  const int t = threadIdx.x;
  const int groups = dp >> 2;
  const int tg = groups >= kThreads ? kThreads : ((groups + 31) & ~31);
  const int ng = kThreads / tg;
  const int g = t / tg, jg = t - g * tg;
  const bool active = g < ng && jg < groups;
  float4 u[CC];
  if (active) {
    float4 acc[4][CC];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < CC; ++c) acc[r][c] = make_float4(0.f, 0.f, 0.f, 0.f);
    int jj[CC];
#pragma unroll
    for (int c = 0; c < CC; ++c) {
      const int q = jg + kThreads * c;
      jj[c] = 4 * (q < groups ? q : groups - 1);  // a group past the end: a valid load, never stored
    }
    int i = g;
    const int step = ng;
    for (; i + 3 * step < nr; i += 4 * step) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int ii = i + r * step;
        const float wi = w[ii];
        const TS* row = sa + (size_t)ii * sp;
#pragma unroll
        for (int c = 0; c < CC; ++c) {
          const float sc = scales != nullptr ? scales[(size_t)((r0 + ii) >> 7) * sld + (jj[c] >> 7)] : 1.f;
          const float4 a = ld_sa_row4<TS>(row, jj[c], sc);
          acc[r][c].x = fmaf(a.x, wi, acc[r][c].x);
          acc[r][c].y = fmaf(a.y, wi, acc[r][c].y);
          acc[r][c].z = fmaf(a.z, wi, acc[r][c].z);
          acc[r][c].w = fmaf(a.w, wi, acc[r][c].w);
        }
      }
    }
    for (int r = 0; i < nr; i += step, ++r) {  // the last < 4 rows of this group
      const float wi = w[i];
      const TS* row = sa + (size_t)i * sp;
#pragma unroll
      for (int c = 0; c < CC; ++c) {
        const float sc = scales != nullptr ? scales[(size_t)((r0 + i) >> 7) * sld + (jj[c] >> 7)] : 1.f;
        const float4 a = ld_sa_row4<TS>(row, jj[c], sc);
        // rows i, i + step, i + 2·step go to accumulators 0, 1, 2
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (r == q) {
            acc[q][c].x = fmaf(a.x, wi, acc[q][c].x);
            acc[q][c].y = fmaf(a.y, wi, acc[q][c].y);
            acc[q][c].z = fmaf(a.z, wi, acc[q][c].z);
            acc[q][c].w = fmaf(a.w, wi, acc[q][c].w);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CC; ++c) {
      u[c].x = (acc[0][c].x + acc[1][c].x) + (acc[2][c].x + acc[3][c].x);
      u[c].y = (acc[0][c].y + acc[1][c].y) + (acc[2][c].y + acc[3][c].y);
      u[c].z = (acc[0][c].z + acc[1][c].z) + (acc[2][c].z + acc[3][c].z);
      u[c].w = (acc[0][c].w + acc[1][c].w) + (acc[2][c].w + acc[3][c].w);
    }
  }
  if (ng == 1) {
    if (active) {
#pragma unroll
      for (int c = 0; c < CC; ++c) {
        const int q = jg + kThreads * c;
        if (q < groups) *reinterpret_cast<float4*>(out + 4 * q) = u[c];
      }
    }
    return;
  }
  if (active) *reinterpret_cast<float4*>(tmp + (size_t)g * dp + 4 * jg) = u[0];
  __syncthreads();
  for (int q = t; q < groups; q += kThreads) {
    float4 sacc = *reinterpret_cast<const float4*>(tmp + 4 * q);
    for (int gg = 1; gg < ng; ++gg) {
      const float4 b = *reinterpret_cast<const float4*>(tmp + (size_t)gg * dp + 4 * q);
      sacc.x += b.x;
      sacc.y += b.y;
      sacc.z += b.z;
      sacc.w += b.w;
    }
    *reinterpret_cast<float4*>(out + 4 * q) = sacc;
  }
}

template <int CL, int CH, typename TS>
__global__ void __launch_bounds__(kThreads, 1) aab_cluster_kernel(const AabParams P) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int d = P.d, dp = P.dp;
  // λ-path mode: the clusters of grid row blockIdx.y solve λ_y with their own
  // g, x, x⁻ and control block; the path's stop counter ends the graph loop
  // once every λ has stopped.
  const int li = P.path ? (int)blockIdx.y : 0;
  const float* g_in = P.g + (long long)li * P.path_ldg;
  SolveCtl* ctl_ = P.ctl != nullptr ? P.ctl + li : nullptr;
  float* x_ = P.x != nullptr ? P.x + (long long)li * P.path_ldx : nullptr;
  float* xprev_ = P.x_prev != nullptr ? P.x_prev + (long long)li * P.path_ldg : nullptr;
  float* delta_ = P.path ? nullptr : P.delta;
  int* passes_ = P.path ? nullptr : P.passes;
  float* hist_ = P.path ? nullptr : P.hist;
  const float lam_ = P.path ? P.ps.lam[li] : P.lambda;
  const float alpha_ = P.path ? P.ps.alpha[li] : P.alpha;
  const float beta_ = P.path ? P.ps.beta[li] : P.beta;

  extern __shared__ float4 smem4[];
  float* v = reinterpret_cast<float*>(smem4);  // replicated d-vectors
  float* dv = v + dp;
  float* xs = dv + dp;
  float* up = xs + dp;      // this block's SAᵀw (read remotely)
  float* zsl = up + dp;     // this block's slice of θv (read remotely)
  float* wpart = zsl + dp;  // kWarps × dp per-warp partials of SAᵀw
  float* p = wpart + (size_t)kWarps * dp;  // own rows
  float* w = p + P.rpc_pad;
  float* red = w + P.rpc_pad;  // kWarps floats
  float* scal = red + kWarps;  // [0] θ² partial, [1] ρ² partial (read remotely), [2] broadcast
  uint64_t* stage_bar = reinterpret_cast<uint64_t*>(scal + 6);  // 8-byte aligned slot
  TS* sa = reinterpret_cast<TS*>(scal + 8);  // SA rows (when kept in smem), pitch P.sa_pitch
  const TS* SAg = static_cast<const TS*>(P.SA);

  // Solve-mode control block: read everything before the first barrier; only
  // rank 0 writes it, after the last barrier.
  int done = 0, outer = 0, max_outer = 0, g0known = 0, phase = 1, refresh = 1, corr = 0;
  float tol = 0.f, gnorm0 = 0.f, switch_tol = 0.f;
  if (ctl_ != nullptr) {
    done = ctl_->done;
    outer = ctl_->outer;
    max_outer = ctl_->max_outer;
    g0known = ctl_->gnorm0_known;
    tol = ctl_->tol;
    gnorm0 = ctl_->gnorm0;
    phase = ctl_->phase;
    switch_tol = ctl_->switch_tol;
    refresh = ctl_->refresh;
    corr = ctl_->corr;
  }
  cluster.sync();  // every block is running before any DSMEM access
  if (done) {
    // Already stopped: make sure a device-side loop around this kernel ends.
    if (P.cond != 0ull && !P.path && rank == 0 && tid == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
    return;
  }
  const float* lane_scal = cluster.map_shared_rank(scal, lane % CL);

  const int r0 = rank * P.rpc;
  const int nr = max(0, min(P.m, r0 + P.rpc) - r0);
  const TS* SAc;
  long long ldc;
  bool staged_async = false;
  const int sp = P.sa_pitch;
  const uint32_t row_bytes = (uint32_t)sp * (uint32_t)sizeof(TS);
  if (P.sa_in_smem && P.sa_vec && (sizeof(TS) != 4 || d == dp) && row_bytes % 16u == 0 && nr > 0) {
    // Whole rows by bulk asynchronous copies, counted in bytes on one mbarrier.
    if (tid == 0) {
      mbar_init(stage_bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(stage_bar, (uint32_t)nr * row_bytes);
      for (int i = 0; i < nr; ++i)
        bulk_copy_g2s(sa + (size_t)i * sp, SAg + (long long)(r0 + i) * P.ldsa, row_bytes, stage_bar);
    }
    staged_async = true;
    SAc = sa;
    ldc = sp;
  } else if (P.sa_in_smem) {
    // fp32 rows, masked beyond d (quantised rows are always bulk-copied)
    for (int i = 0; i < nr; ++i) {
      const float* src = reinterpret_cast<const float*>(SAg) + (long long)(r0 + i) * P.ldsa;
      for (int j = 4 * tid; j < dp; j += 4 * kThreads)
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(sa) + (size_t)i * sp + j) =
            load4_masked(src, j, d, P.sa_vec != 0);
    }
    SAc = sa;
    ldc = sp;
  } else {
    SAc = SAg + (long long)r0 * P.ldsa;
    ldc = P.ldsa;
  }

  // θ₁ v = g
  float gsq = 0.f;
  for (int j = tid; j < dp; j += kThreads) {
    const float gj = j < d ? g_in[j] : 0.f;
    v[j] = gj;
    gsq = fmaf(gj, gj, gsq);
    xs[j] = 0.f;
    dv[j] = 0.f;
  }
  for (int i = tid; i < P.rpc_pad; i += kThreads) p[i] = 0.f;
  const float theta1 = sqrtf(block_sum(gsq, red));
  if (staged_async) {
    // Every thread waits for the rows (also on the early-exit paths below, so
    // that no copy is still landing when the block exits).
    if (!mbar_wait(stage_bar, 0u, kWaitLimitNs) && tid == 0 && ctl_ != nullptr) {
      ctl_->status = MIHS_ERR_TIMEOUT;
      ctl_->done = 1;
    }
  }

  if (ctl_ != nullptr) {  // stop test of Algorithm 1 on ‖g‖ = θ₁
    const float g0 = g0known ? gnorm0 : theta1;
    if (hist_ != nullptr && rank == 0 && tid == 0 && outer < kHistCap) hist_[outer] = theta1;
    const bool bad = !(theta1 <= 3.0e38f);
    // A refinement correction's gradient is approximate: it never stops the
    // solve; nor does a refinement solve's plain fp32 gradient (phase 0), whose
    // rounding floor lies above the tolerances refinement is asked for (it
    // can round to zero near the solution): only a compensated one certifies.
    const bool correction = phase == 1 && corr && !refresh;
    const bool conv = tol > 0.f && theta1 <= tol * g0 && !correction && phase != 0;
    const bool capped = outer >= max_outer;
    if (rank == 0 && tid == 0) refine_step_update(ctl_, phase, refresh, corr, theta1, g0, tol, switch_tol);
    if (bad || conv || capped) {
      if (rank == 0 && tid == 0) {
        ctl_->gnorm = theta1;
        ctl_->gnorm0 = g0;
        ctl_->gnorm0_known = 1;
        ctl_->status = bad ? MIHS_ERR_NUMERIC : (conv ? MIHS_OK : MIHS_NOT_CONVERGED);
        ctl_->done = 1;
        if (P.path) {
          if (atomicAdd(P.path_ndone, 1) + 1 == P.ps.nl) {  // the last λ of the path to stop
            *P.path_all_done = 1;
            if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
          }
        } else if (P.cond != 0ull) {
          cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
        }
      }
      return;  // no DSMEM access has happened since the barrier
    }
  }

  int k = 0;
  const int c0 = rank * P.cols_per;
  const int c1 = min(dp, c0 + P.cols_per);
  const int ncol = max(0, c1 - c0);
  const bool split = P.sa_in_smem != 0;
  // One sweep: w = SA·v − θp (own rows), this block's SAᵀw in `up` and its
  // ρ² share in scal[1].  With SA in shared memory, row dots then column
  // sums; streaming SA from L2, the fused sweep that reads each row once.
  auto sweep = [&](float theta_) {
    if (split) {
      const float rsq = row_dots<CH, TS>(sa, sp, nr, v, p, theta_, w, dp, P.sa_scale, P.scale_ld, r0);
      if (lane == 0) red[warp] = rsq;
      __syncthreads();  // w complete
      col_sums<CH, TS>(sa, sp, nr, dp, w, P.sa_scale, P.scale_ld, r0, wpart, up);
    } else {
      const float rsq = fused_sweep<CH, TS>(SAc, ldc, nr, d, v, p, theta_, w, wpart, dp, P.sa_vec != 0,
                                            P.sa_scale, P.scale_ld, r0);
      if (lane == 0) red[warp] = rsq;
      __syncthreads();
      for (int j = tid; j < dp; j += kThreads) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) t += wpart[(size_t)q * dp + j];
        up[j] = t;
      }
    }
    if (tid == 0) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) t += red[q];
      scal[1] = t;
    }
  };
  if (theta1 > 0.f) {
    const float inv_theta1 = 1.0f / theta1;
    for (int j = tid; j < dp; j += kThreads) v[j] *= inv_theta1;
    __syncthreads();
    // First sweep: w = SA v (p = 0), ρ² share and SAᵀw (ρ p = w; the
    // normalisation by ρ is deferred so that one barrier publishes both).
    sweep(0.f);
    const float lam = lam_;
    float rho = 0.f, rhobar = 0.f, c = 0.f, s = 0.f, phi = 0.f, theta = 0.f;
    float t = __int_as_float(0x7f800000);  // +inf
    const int q4 = P.cols_per >> 2;        // float4 groups in a column slice
    float* ubuf = wpart;                   // CL × cols_per: the ranks' SAᵀw on this block's slice
    bool first = true;
    for (;;) {
      cluster.sync();  // (A) ρ² partials and SAᵀw partials visible
      // ρ² (warp 0) and every rank's SAᵀw on this block's column slice, all
      // loads issued together (one DSMEM round trip).
      for (int e = tid; e < CL * q4; e += kThreads) {
        const int r = e / q4, q = e - r * q4;
        const int j = c0 + 4 * q;
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < dp) val = *reinterpret_cast<const float4*>(cluster.map_shared_rank(up, r) + j);
        *reinterpret_cast<float4*>(ubuf + (size_t)r * P.cols_per + 4 * q) = val;
      }
      if (warp == 0) {
        const float r2 = cluster_scalar_sum<CL>(lane_scal, 1);
        if (lane == 0) scal[2] = r2;
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
          dv[c0 + jj] = v[c0 + jj] * inv;
          xs[c0 + jj] = phi * dv[c0 + jj];
        }
        first = false;
      } else {
        // Eldén's rotation of √λ into the bidiagonal, then the φ recursion
        // and the forward-substitution update (Section 3.6), on the slice.
        const float lambar = sqrtf(lam + (s * theta) * (s * theta));
        const float thetabar = c * theta;
        rhobar = sqrtf(rho * rho + lambar * lambar);
        const float inv_rhobar = 1.0f / rhobar;
        c = rho * inv_rhobar;
        s = lambar * inv_rhobar;
        phi = -phi * thetabar * inv_rhobar;
        for (int jj = tid; jj < ncol; jj += kThreads) {
          const int j = c0 + jj;
          const float dn = (v[j] - thetabar * dv[j]) * inv_rhobar;
          dv[j] = dn;
          xs[j] = fmaf(phi, dn, xs[j]);
        }
        t = fabsf(phi * rhobar) / theta1;
        ++k;
      }
      if (rho > 0.f) {
        const float inv = 1.0f / rho;
        for (int i = tid; i < nr; i += kThreads) p[i] = w[i] * inv;
      }
      if (!(t >= P.eps && k < P.max_passes && rho > 0.f)) break;  // the same in every block
      // θ v := SAᵀp − ρ v on the slice, SAᵀp = (Σ_ranks SAᵀw)/ρ (ranks in order)
      const float inv_rho = 1.0f / rho;
      float zpart = 0.f;
      for (int jj = tid; jj < ncol; jj += kThreads) {
        float us = 0.f;
#pragma unroll
        for (int r = 0; r < CL; ++r) us += ubuf[(size_t)r * P.cols_per + jj];
        const int j = c0 + jj;
        const float z = j < d ? us * inv_rho - rho * v[j] : 0.f;
        zsl[j] = z;
        zpart = fmaf(z, z, zpart);
      }
      zpart = block_sum(zpart, red);
      if (tid == 0) scal[0] = zpart;
      cluster.sync();  // (B) slices of θv and θ² partials visible
      // θ² (warp 0) and all of θv from the slices' owners, loads issued together
      constexpr int CV = (CH * 128 + 4 * kThreads - 1) / (4 * kThreads);
      float4 zr[CV];
#pragma unroll
      for (int cc = 0; cc < CV; ++cc) {
        const int j = 4 * tid + 4 * kThreads * cc;
        zr[cc] = j < dp ? *reinterpret_cast<const float4*>(cluster.map_shared_rank(zsl, j >> P.cols_log2) + j)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (warp == 0) {
        const float t2 = cluster_scalar_sum<CL>(lane_scal, 0);
        if (lane == 0) scal[2] = t2;
      }
      __syncthreads();
      theta = sqrtf(scal[2]);
      if (!(theta > 0.f)) break;  // invariant subspace: same decision everywhere
      const float inv_theta = 1.0f / theta;
#pragma unroll
      for (int cc = 0; cc < CV; ++cc) {
        const int j = 4 * tid + 4 * kThreads * cc;
        if (j < dp)
          *reinterpret_cast<float4*>(v + j) =
              make_float4(zr[cc].x * inv_theta, zr[cc].y * inv_theta, zr[cc].z * inv_theta, zr[cc].w * inv_theta);
      }
      __syncthreads();
      // ρ p := SA v − θ p (kept unnormalised in w until ρ is known), its ρ²
      // share and SAᵀw.
      sweep(theta);
    }
  }
  __syncthreads();

  // Outputs: each block writes its column slice.
  {
    const int e1 = min(d, c0 + P.cols_per);
    for (int j = c0 + tid; j < e1; j += kThreads) {
      const float dj = xs[j];
      if (delta_ != nullptr) delta_[j] = dj;
      if (x_ != nullptr) {
        const float xj = x_[j], xp = xprev_[j];
        x_[j] = xj + alpha_ * dj + beta_ * (xj - xp);
        xprev_[j] = xj;
      }
      if (P.x64 != nullptr) {
        const double xj = P.x64[j], xp = P.x_prev64[j];
        const double xn = xj + P.alpha64 * (double)dj + P.beta64 * (xj - xp);
        P.x64[j] = xn;
        P.x_prev64[j] = xj;
        if (P.x32_shadow != nullptr) P.x32_shadow[j] = (float)xn;
      }
    }
  }
  if (rank == 0 && tid == 0) {
    if (passes_ != nullptr) *passes_ = k;
    if (ctl_ != nullptr) {
      ctl_->outer = outer + 1;
      ctl_->inner_total += k;
      ctl_->gnorm = theta1;
      if (!g0known) {
        ctl_->gnorm0 = theta1;
        ctl_->gnorm0_known = 1;
      }
    }
  }
  cluster.sync();  // keep this block's shared memory alive for remote readers
}


using AabKernelFn = void (*)(const AabParams);

// Kernel for a cluster size and a padded width dp (CH float4 per lane), per
// storage type of SA (each instantiated in its own translation unit).
AabKernelFn kernel_for_f32(int cl, int dp);
AabKernelFn kernel_for_bf16(int cl, int dp);
AabKernelFn kernel_for_fp8(int cl, int dp);

template <int CL, typename TS>
AabKernelFn kernel_for_ch(int ch) {
  if (ch <= 2) return aab_cluster_kernel<CL, 2, TS>;
  if (ch <= 4) return aab_cluster_kernel<CL, 4, TS>;
  if (ch <= 8) return aab_cluster_kernel<CL, 8, TS>;
  return aab_cluster_kernel<CL, 16, TS>;
}

template <typename TS>
AabKernelFn kernel_for_type(int cl, int dp) {
  const int ch = (dp + 127) / 128;
  switch (cl) {
    case 1: return kernel_for_ch<1, TS>(ch);
    case 2: return kernel_for_ch<2, TS>(ch);
    case 4: return kernel_for_ch<4, TS>(ch);
    case 8: return kernel_for_ch<8, TS>(ch);
    default: return kernel_for_ch<16, TS>(ch);
  }
}

}  // namespace aabk
}  // namespace mihs
