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
// work, negligible next to the O(md/CL) products).  When SA is too large for
// the shared memory of 16 blocks, launch_aab hands a single-λ solve that has
// scratch to the grid form (aab_grid.cu); otherwise the cluster's blocks
// read their rows of SA from global memory (L2) on every pass.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "aab_kernel.cuh"

namespace mihs {

using namespace aabk;

AabKernelFn aabk::kernel_for_f32(int cl, int dp) { return kernel_for_type<float>(cl, dp); }

namespace {

AabKernelFn kernel_for(int cl, int dp, int sa_type) {
  if (sa_type == MIHS_SA_BF16) return kernel_for_bf16(cl, dp);
  if (sa_type == MIHS_SA_FP8E4M3) return kernel_for_fp8(cl, dp);
  return kernel_for_f32(cl, dp);
}

struct ClusterPlan {
  int cl;
  int in_smem;
  size_t smem;
};

size_t elem_bytes(int sa_type) { return sa_type == MIHS_SA_BF16 ? 2 : (sa_type == MIHS_SA_FP8E4M3 ? 1 : 4); }

// Shared-memory row pitch (elements) of SA kept in shared memory: dp for
// fp32, the 16-element-aligned storage pitch for the quantised types.
int smem_pitch(int dp, int sa_type) { return sa_type == MIHS_SA_FP32 ? dp : (int)round_up(dp, 16); }

size_t smem_bytes(int m, int dp, int cl, bool in_smem, int sa_type) {
  const int rpc = (m + cl - 1) / cl;
  const int rpc_pad = (int)round_up(rpc, 4);
  size_t base = (size_t)((5 + kWarps) * dp + 2 * rpc_pad + kWarps + 8) * sizeof(float);
  if (in_smem) base += (size_t)rpc * smem_pitch(dp, sa_type) * elem_bytes(sa_type);
  return base;
}

bool cluster_fits(int cl, int dp, size_t smem, int sa_type) {
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
  if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)kernel_for(cl, dp, sa_type), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

ClusterPlan plan_cluster_uncached(int m, int dp, int sa_type) {
  static bool attr_set = false;
  if (!attr_set) {
    for (int t : {MIHS_SA_FP32, MIHS_SA_BF16, MIHS_SA_FP8E4M3})
      for (int cl : {1, 2, 4, 8, 16})
        for (int w : {256, 512, 1024, 2048}) {
          cudaFuncSetAttribute((void*)kernel_for(cl, w, t), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
          cudaFuncSetAttribute((void*)kernel_for(cl, w, t), cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    const size_t sm = smem_bytes(m, dp, cl, true, sa_type);
    if (sm <= kSmemBudget && cluster_fits(cl, dp, sm, sa_type)) return {cl, 1, sm};
  }
  // Otherwise the largest launchable cluster reading SA from global memory (L2).
  for (int i = 4; i >= 0; --i) {
    const int cl = sizes[i];
    if (forced > 0 && cl != forced) continue;
    if (cl > m && cl > 1) continue;
    const size_t sm = smem_bytes(m, dp, cl, false, sa_type);
    if (sm <= kSmemBudget && cluster_fits(cl, dp, sm, sa_type)) return {cl, 0, sm};
  }
  return {0, 0, 0};
}

std::mutex g_plan_mu;
std::map<std::tuple<int, int, int>, ClusterPlan> g_plans;  // (m, dp, SA type) → plan (current device)

ClusterPlan plan_cluster(int m, int dp, int sa_type) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find({m, dp, sa_type});
  if (it != g_plans.end()) return it->second;
  const ClusterPlan cp = plan_cluster_uncached(m, dp, sa_type);
  g_plans[{m, dp, sa_type}] = cp;
  return cp;
}

}  // namespace

void aab_prepare(int m, int d, int sa_type) { (void)plan_cluster(m, (int)round_up(d, 4), sa_type); }

bool aab_grid_wanted(int m, int d, int sa_type, int form) {
  if (form == MIHS_AAB_GRID) return true;
  if (form == MIHS_AAB_CLUSTER) return false;
  if (const char* e = std::getenv("MIHS_AAB_FORM")) {
    if (std::strcmp(e, "grid") == 0) return true;
    if (std::strcmp(e, "cluster") == 0) return false;
  }
  return plan_cluster(m, (int)round_up(d, 4), sa_type).in_smem == 0;
}

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
  P.x64 = a.x64;
  P.x_prev64 = a.x_prev64;
  P.x32_shadow = a.x32_shadow;
  P.alpha64 = a.alpha64;
  P.beta64 = a.beta64;
  P.ctl = a.ctl;
  P.cond = a.cond;
  P.hist = a.hist;
  P.path = a.path;
  P.ps = a.ps;
  P.path_ldg = a.path_ldg;
  P.path_ldx = a.path_ldx;
  P.path_ndone = a.path_ndone;
  P.path_all_done = a.path_all_done;
  if (a.path && (a.ps.nl < 1 || a.ps.nl > 16 || a.x64 != nullptr)) {
    set_error("aab: path mode needs 1..16 λ and an fp32 iterate");
    return MIHS_ERR_INVALID_ARG;
  }
  if (a.sa_type != MIHS_SA_FP32 && (a.ldsa % 16 != 0 || (reinterpret_cast<uintptr_t>(a.SA) & 15u) != 0 ||
                                    (a.sa_type == MIHS_SA_FP8E4M3 && a.sa_scale == nullptr))) {
    set_error("aab: quantised SA needs 16-byte aligned rows (ldsa %% 16 == 0) and fp8 tile scales");
    return MIHS_ERR_INVALID_ARG;
  }
  P.sa_scale = a.sa_type == MIHS_SA_FP8E4M3 ? a.sa_scale : nullptr;
  P.scale_ld = (int)((round_up(a.d, 4) + 127) / 128);
  if (!a.path && a.grid_ws != nullptr && aab_grid_wanted(a.m, a.d, a.sa_type, a.aab_form)) {
    // SA does not fit one cluster's shared memory (or the caller asked for
    // the grid form): spread it over the SMs.
    const int rc = launch_aab_grid(a, a.grid_ws, s);
    if (rc != MIHS_ERR_UNSUPPORTED) return rc;
  }
  const ClusterPlan cp = plan_cluster(a.m, P.dp, a.sa_type);
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
  P.sa_pitch = smem_pitch(P.dp, a.sa_type);
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
  cfg.gridDim = dim3(cp.cl, a.path ? a.ps.nl : 1);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = cp.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  timing_begin(kTimerAab, s);
  MIHS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel_for(cp.cl, P.dp, a.sa_type), P));
  timing_end(kTimerAab, s);
  count_launch();
  return MIHS_OK;
}

}  // namespace mihs
