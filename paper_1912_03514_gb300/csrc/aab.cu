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
#include <cooperative_groups.h>

#include <cstdlib>
#include <map>
#include <mutex>

#include "internal.h"

namespace cg = cooperative_groups;

namespace mihs {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr size_t kSmemBudget = 200 * 1024;

struct AabParams {
  const float* SA;
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
  SolveCtl* ctl;
  float* hist;
  unsigned long long cond;
  int rpc;             // rows per block
  int rpc_pad;         // rpc rounded up to 4
  int cols_per;        // column slice per block (a power of two ≥ 4)
  int cols_log2;
  int sa_in_smem;
  int sa_vec;          // SA rows may be read as float4 (ldsa % 4 == 0, 16-byte aligned)
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

// out[i] = SAc[i,:]·v for the block's rows.  Warp w takes rows w, w+16, …,
// four at a time, so each chunk of v read from smem feeds four rows.
__device__ __forceinline__ void rows_dot4(const float* SAc, long long ldc, int nr, int d, int dp,
                                          const float* v, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = warp; i0 < nr; i0 += 4 * kWarps) {
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    const float* rows[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) rows[q] = SAc + (long long)min(i0 + q * kWarps, nr - 1) * ldc;
#pragma unroll 2
    for (int j = 4 * lane; j < dp; j += 128) {
      const float4 b = *reinterpret_cast<const float4*>(v + j);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 a = load4_masked(rows[q], j, d);
        s[q] = fmaf(a.x, b.x, s[q]);
        s[q] = fmaf(a.y, b.y, s[q]);
        s[q] = fmaf(a.z, b.z, s[q]);
        s[q] = fmaf(a.w, b.w, s[q]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + q * kWarps < nr) out[i0 + q * kWarps] = s[q];
    }
  }
}

// u_h[j] = Σ_{i in half h} SAc[i][j]·w[i]: threads [256h, 256h+256) take row
// half h, one float4 column group each (the two halves are summed later, in
// a fixed order, by the reduce-scatter).
__device__ __forceinline__ void cols_dot_halves(const float* SAc, long long ldc, int nr, int d,
                                                int dp, const float* w, float* u0, float* u1) {
  const int h = threadIdx.x >> 8, t = threadIdx.x & 255;
  const int half = (nr + 1) >> 1;
  const int ib = h * half, ie = min(nr, ib + half);
  float* u = h ? u1 : u0;
  for (int j = 4 * t; j < dp; j += 1024) {
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    int i = ib;
#pragma unroll 2
    for (; i + 2 <= ie; i += 2) {
      const float4 r0 = load4_masked(SAc + (long long)i * ldc, j, d);
      const float4 r1 = load4_masked(SAc + (long long)(i + 1) * ldc, j, d);
      const float w0 = w[i], w1 = w[i + 1];
      a0.x = fmaf(r0.x, w0, a0.x); a0.y = fmaf(r0.y, w0, a0.y);
      a0.z = fmaf(r0.z, w0, a0.z); a0.w = fmaf(r0.w, w0, a0.w);
      a1.x = fmaf(r1.x, w1, a1.x); a1.y = fmaf(r1.y, w1, a1.y);
      a1.z = fmaf(r1.z, w1, a1.z); a1.w = fmaf(r1.w, w1, a1.w);
    }
    if (i < ie) {
      const float4 r0 = load4_masked(SAc + (long long)i * ldc, j, d);
      const float w0 = w[i];
      a0.x = fmaf(r0.x, w0, a0.x); a0.y = fmaf(r0.y, w0, a0.y);
      a0.z = fmaf(r0.z, w0, a0.z); a0.w = fmaf(r0.w, w0, a0.w);
    }
    *reinterpret_cast<float4*>(u + j) = make_float4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
  }
}

// Σ over the cluster of one scalar slot: lane r of every warp loads rank r's
// value, then a fixed butterfly sums them (identical in every thread and
// every block).
template <int CL>
__device__ __forceinline__ float cluster_scalar_sum(const float* my_rank_scal, int slot) {
  const int lane = threadIdx.x & 31;
  float v = lane < CL ? my_rank_scal[slot] : 0.f;
  return warp_sum(v);
}

template <int CL>
__global__ void __launch_bounds__(kThreads, 1) aab_cluster_kernel(const AabParams P) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31;
  const int d = P.d, dp = P.dp;

  extern __shared__ float4 smem4[];
  float* v = reinterpret_cast<float*>(smem4);  // replicated d-vectors
  float* dv = v + dp;
  float* xs = dv + dp;
  float* up0 = xs + dp;     // this block's partial SAᵀw, row half 0 (read remotely)
  float* up1 = up0 + dp;    // row half 1 (read remotely)
  float* zsl = up1 + dp;    // this block's slice of θv (read remotely)
  float* p = zsl + dp;      // own rows
  float* w = p + P.rpc_pad;
  float* red = w + P.rpc_pad;  // kWarps floats
  float* scal = red + kWarps;  // [0] θ² partial, [1] ρ² partial (read remotely)
  uint64_t* stage_bar = reinterpret_cast<uint64_t*>(scal + 6);  // 8-byte aligned slot
  float* sa = scal + 8;        // SA rows (when kept in smem)

  // Solve-mode control block: read everything before the first barrier; only
  // rank 0 writes it, after the last barrier.
  int done = 0, outer = 0, max_outer = 0, g0known = 0;
  float tol = 0.f, gnorm0 = 0.f;
  if (P.ctl != nullptr) {
    done = P.ctl->done;
    outer = P.ctl->outer;
    max_outer = P.ctl->max_outer;
    g0known = P.ctl->gnorm0_known;
    tol = P.ctl->tol;
    gnorm0 = P.ctl->gnorm0;
  }
  cluster.sync();  // every block is running before any DSMEM access
  if (done) {
    // Already stopped: make sure a device-side loop around this kernel ends.
    if (P.cond != 0ull && rank == 0 && tid == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
    return;
  }
  const float* lane_scal = cluster.map_shared_rank(scal, lane % CL);

  const int r0 = rank * P.rpc;
  const int nr = max(0, min(P.m, r0 + P.rpc) - r0);
  const float* SAc;
  long long ldc;
  bool staged_async = false;
  if (P.sa_in_smem && P.sa_vec && d == dp && nr > 0) {
    // Whole rows by bulk asynchronous copies, counted in bytes on one mbarrier.
    if (tid == 0) {
      mbar_init(stage_bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(stage_bar, (uint32_t)nr * (uint32_t)dp * 4u);
      for (int i = 0; i < nr; ++i)
        bulk_copy_g2s(sa + (size_t)i * dp, P.SA + (long long)(r0 + i) * P.ldsa, (uint32_t)dp * 4u, stage_bar);
    }
    staged_async = true;
    SAc = sa;
    ldc = dp;
  } else if (P.sa_in_smem) {
    const int q = dp / 4;
    for (int i = 0; i < nr; ++i) {
      const float* src = P.SA + (long long)(r0 + i) * P.ldsa;
      for (int j = 4 * tid; j < dp; j += 4 * kThreads)
        *reinterpret_cast<float4*>(sa + (size_t)i * dp + j) = load4_masked(src, j, d, P.sa_vec != 0);
    }
    (void)q;
    SAc = sa;
    ldc = dp;
  } else {
    SAc = P.SA + (long long)r0 * P.ldsa;
    ldc = P.ldsa;
  }

  // θ₁ v = g
  float gsq = 0.f;
  for (int j = tid; j < dp; j += kThreads) {
    const float gj = j < d ? P.g[j] : 0.f;
    v[j] = gj;
    gsq = fmaf(gj, gj, gsq);
    xs[j] = 0.f;
    dv[j] = 0.f;
  }
  const float theta1 = sqrtf(block_sum(gsq, red));
  if (staged_async) {
    // Every thread waits for the rows (also on the early-exit paths below, so
    // that no copy is still landing when the block exits).
    if (!mbar_wait(stage_bar, 0u, kWaitLimitNs) && tid == 0 && P.ctl != nullptr) {
      P.ctl->status = MIHS_ERR_TIMEOUT;
      P.ctl->done = 1;
    }
  }

  if (P.ctl != nullptr) {  // stop test of Algorithm 1 on ‖g‖ = θ₁
    const float g0 = g0known ? gnorm0 : theta1;
    if (P.hist != nullptr && rank == 0 && tid == 0 && outer < kHistCap) P.hist[outer] = theta1;
    const bool bad = !(theta1 <= 3.0e38f);
    const bool conv = tol > 0.f && theta1 <= tol * g0;
    const bool capped = outer >= max_outer;
    if (bad || conv || capped) {
      if (rank == 0 && tid == 0) {
        P.ctl->gnorm = theta1;
        P.ctl->gnorm0 = g0;
        P.ctl->gnorm0_known = 1;
        P.ctl->status = bad ? MIHS_ERR_NUMERIC : (conv ? MIHS_OK : MIHS_NOT_CONVERGED);
        P.ctl->done = 1;
        if (P.cond != 0ull) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
      }
      return;  // no DSMEM access has happened since the barrier
    }
  }

  int k = 0;
  const int c0 = rank * P.cols_per;
  const int c1 = min(dp, c0 + P.cols_per);
  if (theta1 > 0.f) {
    const float inv_theta1 = 1.0f / theta1;
    for (int j = tid; j < dp; j += kThreads) v[j] *= inv_theta1;
    __syncthreads();
    // ρ p = SA v.  The normalisation by ρ is deferred: the block also forms
    // SAᵀw for the next product before the cluster learns ρ, so one barrier
    // publishes both the ρ² partials and the SAᵀw partials.
    rows_dot4(SAc, ldc, nr, d, dp, v, w);
    __syncthreads();
    float part = 0.f;
    for (int i = tid; i < nr; i += kThreads) part = fmaf(w[i], w[i], part);
    part = block_sum(part, red);
    if (tid == 0) scal[1] = part;
    cols_dot_halves(SAc, ldc, nr, d, dp, w, up0, up1);
    cluster.sync();  // (A) ρ² partials and SAᵀw partials visible
    float rho = sqrtf(cluster_scalar_sum<CL>(lane_scal, 1));

    const float lam = P.lambda;
    float rhobar = sqrtf(rho * rho + lam);
    float c = rho / rhobar;
    float s = sqrtf(lam) / rhobar;
    float phi = theta1 / rhobar;
    {
      const float inv = 1.0f / rhobar;
      for (int j = tid; j < dp; j += kThreads) {
        dv[j] = v[j] * inv;
        xs[j] = phi * dv[j];
      }
    }
    float t = __int_as_float(0x7f800000);  // +inf
    if (rho > 0.f) {
      const float inv = 1.0f / rho;
      for (int i = tid; i < nr; i += kThreads) p[i] = w[i] * inv;
    }

    while (t >= P.eps && k < P.max_passes && rho > 0.f) {
      // θ v := SAᵀ p − ρ v  with SAᵀp = (Σ_ranks SAᵀw)/ρ on this block's column slice
      const float inv_rho = 1.0f / rho;
      float zpart = 0.f;
      for (int j = c0 + tid; j < c1; j += kThreads) {
        float u0[CL], u1[CL];
#pragma unroll
        for (int r = 0; r < CL; ++r) {
          u0[r] = cluster.map_shared_rank(up0, r)[j];
          u1[r] = cluster.map_shared_rank(up1, r)[j];
        }
        float us = 0.f;
#pragma unroll
        for (int r = 0; r < CL; ++r) us += u0[r] + u1[r];
        const float z = j < d ? us * inv_rho - rho * v[j] : 0.f;
        zsl[j] = z;
        zpart = fmaf(z, z, zpart);
      }
      zpart = block_sum(zpart, red);
      if (tid == 0) scal[0] = zpart;
      cluster.sync();  // (B) slices of θv and θ² partials visible
      const float theta = sqrtf(cluster_scalar_sum<CL>(lane_scal, 0));
      if (!(theta > 0.f)) break;  // invariant subspace: same decision everywhere
      const float inv_theta = 1.0f / theta;
      for (int j = tid; j < dp; j += kThreads)
        v[j] = cluster.map_shared_rank(zsl, j >> P.cols_log2)[j] * inv_theta;
      __syncthreads();
      // ρ p := SA v − θ p (kept unnormalised in w until ρ is known)
      rows_dot4(SAc, ldc, nr, d, dp, v, w);
      __syncthreads();
      part = 0.f;
      for (int i = tid; i < nr; i += kThreads) {
        const float wi = w[i] - theta * p[i];
        w[i] = wi;
        part = fmaf(wi, wi, part);
      }
      part = block_sum(part, red);  // also orders the w updates before the next product
      if (tid == 0) scal[1] = part;
      cols_dot_halves(SAc, ldc, nr, d, dp, w, up0, up1);
      cluster.sync();  // (A) ρ² partials and SAᵀw partials visible
      rho = sqrtf(cluster_scalar_sum<CL>(lane_scal, 1));
      // Eldén's rotation of √λ into the bidiagonal, then the φ recursion and
      // the forward-substitution update (Section 3.6).
      const float lambar = sqrtf(lam + (s * theta) * (s * theta));
      const float thetabar = c * theta;
      rhobar = sqrtf(rho * rho + lambar * lambar);
      const float inv_rhobar = 1.0f / rhobar;
      c = rho * inv_rhobar;
      s = lambar * inv_rhobar;
      phi = -phi * thetabar * inv_rhobar;
      for (int j = tid; j < dp; j += kThreads) {
        const float dn = (v[j] - thetabar * dv[j]) * inv_rhobar;
        dv[j] = dn;
        xs[j] = fmaf(phi, dn, xs[j]);
      }
      t = fabsf(phi * rhobar) / theta1;
      ++k;
      if (rho > 0.f) {
        const float inv = 1.0f / rho;
        for (int i = tid; i < nr; i += kThreads) p[i] = w[i] * inv;
      }
      __syncthreads();
    }
  }

  // Outputs: each block writes its column slice.
  {
    const int e1 = min(d, c0 + P.cols_per);
    for (int j = c0 + tid; j < e1; j += kThreads) {
      const float dj = xs[j];
      if (P.delta != nullptr) P.delta[j] = dj;
      if (P.x != nullptr) {
        const float xj = P.x[j], xp = P.x_prev[j];
        P.x[j] = xj + P.alpha * dj + P.beta * (xj - xp);
        P.x_prev[j] = xj;
      }
    }
  }
  if (rank == 0 && tid == 0) {
    if (P.passes != nullptr) *P.passes = k;
    if (P.ctl != nullptr) {
      P.ctl->outer = outer + 1;
      P.ctl->inner_total += k;
      P.ctl->gnorm = theta1;
      if (!g0known) {
        P.ctl->gnorm0 = theta1;
        P.ctl->gnorm0_known = 1;
      }
    }
  }
  cluster.sync();  // keep this block's shared memory alive for remote readers
}

using AabKernelFn = void (*)(const AabParams);

AabKernelFn kernel_for(int cl) {
  switch (cl) {
    case 1: return aab_cluster_kernel<1>;
    case 2: return aab_cluster_kernel<2>;
    case 4: return aab_cluster_kernel<4>;
    case 8: return aab_cluster_kernel<8>;
    default: return aab_cluster_kernel<16>;
  }
}

struct ClusterPlan {
  int cl;
  int in_smem;
  size_t smem;
};

size_t smem_bytes(int m, int dp, int cl, bool in_smem) {
  const int rpc = (m + cl - 1) / cl;
  const int rpc_pad = (int)round_up(rpc, 4);
  size_t base = (size_t)(6 * dp + 2 * rpc_pad + kWarps + 8) * sizeof(float);
  if (in_smem) base += (size_t)rpc * dp * sizeof(float);
  return base;
}

bool cluster_fits(int cl, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)kernel_for(cl), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

ClusterPlan plan_cluster_uncached(int m, int dp) {
  static bool attr_set = false;
  if (!attr_set) {
    for (int cl : {1, 2, 4, 8, 16}) {
      cudaFuncSetAttribute((void*)kernel_for(cl), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaFuncSetAttribute((void*)kernel_for(cl), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kSmemBudget + 16 * 1024);
    }
    attr_set = true;
  }
  int forced = 0;
  if (const char* e = std::getenv("MIHS_AAB_CLUSTER")) forced = std::atoi(e);
  const int sizes[] = {1, 2, 4, 8, 16};
  // Smallest cluster whose row slices of SA fit in shared memory.
  for (int cl : sizes) {
    if (forced > 0 && cl != forced) continue;
    if (cl > m && cl > 1) break;
    const size_t sm = smem_bytes(m, dp, cl, true);
    if (sm <= kSmemBudget && cluster_fits(cl, sm)) return {cl, 1, sm};
  }
  // Otherwise the largest launchable cluster reading SA from global memory (L2).
  for (int i = 4; i >= 0; --i) {
    const int cl = sizes[i];
    if (forced > 0 && cl != forced) continue;
    if (cl > m && cl > 1) continue;
    const size_t sm = smem_bytes(m, dp, cl, false);
    if (sm <= kSmemBudget && cluster_fits(cl, sm)) return {cl, 0, sm};
  }
  return {0, 0, 0};
}

std::mutex g_plan_mu;
std::map<std::pair<int, int>, ClusterPlan> g_plans;  // (m, dp) → plan (current device)

ClusterPlan plan_cluster(int m, int dp) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find({m, dp});
  if (it != g_plans.end()) return it->second;
  const ClusterPlan cp = plan_cluster_uncached(m, dp);
  g_plans[{m, dp}] = cp;
  return cp;
}

}  // namespace

void aab_prepare(int m, int d) { (void)plan_cluster(m, (int)round_up(d, 4)); }

int launch_aab(const AabLaunch& a, cudaStream_t s) {
  AabParams P = {};
  P.SA = a.SA;
  P.m = a.m;
  P.d = a.d;
  P.dp = (int)round_up(a.d, 4);
  P.ldsa = a.ldsa;
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
  P.ctl = a.ctl;
  P.cond = a.cond;
  P.hist = a.hist;
  const ClusterPlan cp = plan_cluster(a.m, P.dp);
  if (cp.cl == 0) {
    set_error("aab: no thread-block cluster fits for m=%d d=%d", a.m, a.d);
    return MIHS_ERR_UNSUPPORTED;
  }
  P.rpc = (a.m + cp.cl - 1) / cp.cl;
  P.rpc_pad = (int)round_up(P.rpc, 4);
  {
    int cp2 = 4, lg = 2;
    while ((int64_t)cp2 * cp.cl < P.dp) { cp2 <<= 1; ++lg; }
    P.cols_per = cp2;
    P.cols_log2 = lg;
  }
  P.sa_in_smem = cp.in_smem;
  P.sa_vec = (a.ldsa % 4 == 0 && (reinterpret_cast<uintptr_t>(a.SA) & 15u) == 0) ? 1 : 0;
  if (!P.sa_in_smem && !P.sa_vec) {
    set_error("aab: SA of %d×%d does not fit in shared memory; its rows must then be 16-byte "
              "aligned (ldsa %% 4 == 0)", a.m, a.d);
    return MIHS_ERR_INVALID_ARG;
  }

  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cp.cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cp.cl);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = cp.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  timing_begin(kTimerAab, s);
  MIHS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel_for(cp.cl), P));
  timing_end(kTimerAab, s);
  count_launch();
  return MIHS_OK;
}

}  // namespace mihs
