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
//   * Three cluster barriers per pass; scalars (θ, ρ, c, s, φ, t) are
//     recomputed identically in every thread from partials summed in a fixed
//     order, so all blocks take the same branch and the result is
//     deterministic.
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

constexpr int kThreads = 256;
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
  unsigned long long cond;
  int rpc;             // rows per block
  int rpc_pad;         // rpc rounded up to 4
  int cols_per;        // column slice per block (multiple of 4)
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

// out[i] = SAc[i,:]·v for the block's rows (one warp per row).
__device__ __forceinline__ void rows_dot(const float* SAc, long long ldc, int nr, int d, int dp,
                                         const float* v, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < nr; i += kWarps) {
    const float* row = SAc + (long long)i * ldc;
    float s = 0.f;
    for (int j = 4 * lane; j < dp; j += 128) {
      const float4 a = load4_masked(row, j, d);
      const float4 b = *reinterpret_cast<const float4*>(v + j);
      s = fmaf(a.x, b.x, s);
      s = fmaf(a.y, b.y, s);
      s = fmaf(a.z, b.z, s);
      s = fmaf(a.w, b.w, s);
    }
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
  }
}

// u[j] = Σ_i SAc[i][j]·p[i] over the block's rows (one float4 column group per thread).
__device__ __forceinline__ void cols_dot(const float* SAc, long long ldc, int nr, int d, int dp,
                                         const float* p, float* u) {
  for (int j = 4 * threadIdx.x; j < dp; j += 4 * kThreads) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < nr; ++i) {
      const float4 a = load4_masked(SAc + (long long)i * ldc, j, d);
      const float pi = p[i];
      acc.x = fmaf(a.x, pi, acc.x);
      acc.y = fmaf(a.y, pi, acc.y);
      acc.z = fmaf(a.z, pi, acc.z);
      acc.w = fmaf(a.w, pi, acc.w);
    }
    *reinterpret_cast<float4*>(u + j) = acc;
  }
}

__global__ void __launch_bounds__(kThreads, 1) aab_cluster_kernel(const AabParams P) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CL = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  const int d = P.d, dp = P.dp;

  extern __shared__ float4 smem4[];
  float* v = reinterpret_cast<float*>(smem4);  // replicated d-vectors
  float* dv = v + dp;
  float* xs = dv + dp;
  float* upart = xs + dp;   // this block's partial SAᵀp (read remotely)
  float* zsl = upart + dp;  // this block's slice of θv (read remotely)
  float* p = zsl + dp;      // own rows
  float* w = p + P.rpc_pad;
  float* red = w + P.rpc_pad;  // 8 floats
  float* scal = red + 8;       // [0] θ² partial, [1] ρ² partial (read remotely)
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

  const int r0 = rank * P.rpc;
  const int nr = max(0, min(P.m, r0 + P.rpc) - r0);
  const float* SAc;
  long long ldc;
  if (P.sa_in_smem) {
    const int q = dp / 4;
    for (int idx = tid; idx < nr * q; idx += kThreads) {
      const int i = idx / q, j = 4 * (idx - i * q);
      *reinterpret_cast<float4*>(sa + (size_t)i * dp + j) =
          load4_masked(P.SA + (long long)(r0 + i) * P.ldsa, j, d, P.sa_vec != 0);
    }
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

  if (P.ctl != nullptr) {  // stop test of Algorithm 1 on ‖g‖ = θ₁
    const float g0 = g0known ? gnorm0 : theta1;
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
  if (theta1 > 0.f) {
    for (int j = tid; j < dp; j += kThreads) v[j] = v[j] / theta1;
    __syncthreads();
    // ρ p = SA v
    rows_dot(SAc, ldc, nr, d, dp, v, w);
    __syncthreads();
    float part = 0.f;
    for (int i = tid; i < nr; i += kThreads) part = fmaf(w[i], w[i], part);
    part = block_sum(part, red);
    if (tid == 0) scal[1] = part;
    cluster.sync();
    float rsq = 0.f;
    for (int r = 0; r < CL; ++r) rsq += cluster.map_shared_rank(scal, r)[1];
    float rho = sqrtf(rsq);
    for (int i = tid; i < nr; i += kThreads) p[i] = w[i] / rho;

    const float lam = P.lambda;
    float rhobar = sqrtf(rho * rho + lam);
    float c = rho / rhobar;
    float s = sqrtf(lam) / rhobar;
    float phi = theta1 / rhobar;
    for (int j = tid; j < dp; j += kThreads) {
      dv[j] = v[j] / rhobar;
      xs[j] = phi * dv[j];
    }
    float t = __int_as_float(0x7f800000);  // +inf
    __syncthreads();

    const int c0 = rank * P.cols_per;
    const int c1 = min(dp, c0 + P.cols_per);
    while (t >= P.eps && k < P.max_passes && rho > 0.f) {
      // θ v := SAᵀ p − ρ v
      cols_dot(SAc, ldc, nr, d, dp, p, upart);
      cluster.sync();  // (1) partial SAᵀp visible
      float zpart = 0.f;
      for (int j = c0 + tid; j < c1; j += kThreads) {
        float u = 0.f;
        for (int r = 0; r < CL; ++r) u += cluster.map_shared_rank(upart, r)[j];
        const float z = j < d ? u - rho * v[j] : 0.f;
        zsl[j] = z;
        zpart = fmaf(z, z, zpart);
      }
      zpart = block_sum(zpart, red);
      if (tid == 0) scal[0] = zpart;
      cluster.sync();  // (2) slices of θv and θ² partials visible
      float tsq = 0.f;
      for (int r = 0; r < CL; ++r) tsq += cluster.map_shared_rank(scal, r)[0];
      const float theta = sqrtf(tsq);
      if (!(theta > 0.f)) break;  // invariant subspace: same decision everywhere
      for (int j = tid; j < dp; j += kThreads) {
        const int owner = j / P.cols_per;
        v[j] = cluster.map_shared_rank(zsl, owner)[j] / theta;
      }
      __syncthreads();
      // ρ p := SA v − θ p
      rows_dot(SAc, ldc, nr, d, dp, v, w);
      __syncthreads();
      part = 0.f;
      for (int i = tid; i < nr; i += kThreads) {
        const float wi = w[i] - theta * p[i];
        w[i] = wi;
        part = fmaf(wi, wi, part);
      }
      part = block_sum(part, red);
      if (tid == 0) scal[1] = part;
      cluster.sync();  // (3) ρ² partials visible
      rsq = 0.f;
      for (int r = 0; r < CL; ++r) rsq += cluster.map_shared_rank(scal, r)[1];
      rho = sqrtf(rsq);
      // Eldén's rotation of √λ into the bidiagonal, then the φ recursion and
      // the forward-substitution update (Section 3.6).
      const float lambar = sqrtf(lam + (s * theta) * (s * theta));
      const float thetabar = c * theta;
      rhobar = sqrtf(rho * rho + lambar * lambar);
      c = rho / rhobar;
      s = lambar / rhobar;
      phi = -phi * thetabar / rhobar;
      for (int j = tid; j < dp; j += kThreads) {
        const float dn = (v[j] - thetabar * dv[j]) / rhobar;
        dv[j] = dn;
        xs[j] = fmaf(phi, dn, xs[j]);
      }
      t = fabsf(phi * rhobar) / theta1;
      ++k;
      if (rho > 0.f)
        for (int i = tid; i < nr; i += kThreads) p[i] = w[i] / rho;
      __syncthreads();
    }
  }

  // Outputs: each block writes its column slice.
  {
    const int c0 = rank * P.cols_per;
    const int c1 = min(d, c0 + P.cols_per);
    for (int j = c0 + tid; j < c1; j += kThreads) {
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

struct ClusterPlan {
  int cl;
  int in_smem;
  size_t smem;
};

size_t smem_bytes(int m, int dp, int cl, bool in_smem) {
  const int rpc = (m + cl - 1) / cl;
  const int rpc_pad = (int)round_up(rpc, 4);
  size_t base = (size_t)(5 * dp + 2 * rpc_pad + 16) * sizeof(float);
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
  if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)aab_cluster_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

ClusterPlan plan_cluster_uncached(int m, int dp) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute((void*)aab_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute((void*)aab_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmemBudget + 16 * 1024);
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
  const ClusterPlan cp = plan_cluster(a.m, P.dp);
  if (cp.cl == 0) {
    set_error("aab: no thread-block cluster fits for m=%d d=%d", a.m, a.d);
    return MIHS_ERR_UNSUPPORTED;
  }
  P.rpc = (a.m + cp.cl - 1) / cp.cl;
  P.rpc_pad = (int)round_up(P.rpc, 4);
  P.cols_per = (int)round_up((P.dp + cp.cl - 1) / cp.cl, 4);
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
  MIHS_CUDA_TRY(cudaLaunchKernelEx(&cfg, aab_cluster_kernel, P));
  timing_end(kTimerAab, s);
  count_launch();
  return MIHS_OK;
}

}  // namespace mihs
