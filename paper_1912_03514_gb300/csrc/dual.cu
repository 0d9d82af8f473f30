// Dual M-IHS (Algorithm 2, Section 2) for n ≤ d: the M-IHS iteration on the
// dual problem ν* = argmin ½‖Aᵀν‖² + (λ/2)‖ν‖² − ⟨b, ν⟩ (Eq. intro_dual), with
// the sketch taken along the d coordinates (S·Aᵀ, m × n) and the primal
// solution recovered as x = Aᵀν (Eq. dual_relation).  Per step:
//   u = Aᵀν            one pass over A: blocks own a column slice × row split,
//                      the splits' partials summed in order
//   g = b − A·u − λν   one pass over A, one block per row
//   Δν = AAb_Solver(SAᵀ, g, λ, ε_sub), ν⁺ = ν + αΔν + β(ν − ν⁻)   (aab.cu)
// all inside a CUDA graph WHILE loop that the AAb kernel ends.
#include <cfloat>
#include <cmath>
#include <cstdlib>

#include <utility>
#include <vector>

#include "internal.h"

using namespace mihs;

namespace {

constexpr int kT = 256;

__device__ __forceinline__ float block_sum256(float v, float* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < kT / 32; ++w) t += red[w];
  return t;
}

// At[j][i] = A[i][j] through a padded 32 × 32 shared-memory tile.
__global__ void transpose_kernel(const float* __restrict__ A, int n, int d, long long lda, float* __restrict__ At,
                                 long long ldt) {
  __shared__ float tile[32][33];
  const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < d) ? A[(long long)i * lda + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (j < d && i < n) At[(long long)j * ldt + i] = tile[threadIdx.x][r];
  }
}

// Partial u over a row split: part[z][j] = Σ_{i in split z} ν_i A[i][j].  A
// thread owns 4 consecutive columns (one float4 per row, coalesced across the
// warp) and walks its split's rows in order, eight rows of loads in flight.
constexpr int kAtnuRows = 256;  // rows per split

__global__ void __launch_bounds__(kT) atnu_partial_kernel(const float* __restrict__ A, int n, int d, long long lda,
                                                          const float* __restrict__ nu, float* __restrict__ part,
                                                          long long ldp, const SolveCtl* __restrict__ ctl) {
  if (ctl != nullptr && ctl->done) return;
  __shared__ float nus[kAtnuRows];
  const int i0 = blockIdx.y * kAtnuRows, i1 = min(n, i0 + kAtnuRows);
  for (int i = i0 + threadIdx.x; i < i1; i += kT) nus[i - i0] = nu[i];
  __syncthreads();
  const long long c = ((long long)blockIdx.x * kT + threadIdx.x) * 4;
  if (c >= d) return;
  float* out = part + (long long)blockIdx.y * ldp + c;
  if (c + 4 <= d) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const float* col = A + c;
    int i = i0;
    for (; i + 8 <= i1; i += 8) {
      float4 a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = __ldg(reinterpret_cast<const float4*>(col + (long long)(i + k) * lda));
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float s = nus[i + k - i0];
        acc.x = fmaf(s, a[k].x, acc.x);
        acc.y = fmaf(s, a[k].y, acc.y);
        acc.z = fmaf(s, a[k].z, acc.z);
        acc.w = fmaf(s, a[k].w, acc.w);
      }
    }
    for (; i < i1; ++i) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(col + (long long)i * lda));
      const float s = nus[i - i0];
      acc.x = fmaf(s, a.x, acc.x);
      acc.y = fmaf(s, a.y, acc.y);
      acc.z = fmaf(s, a.z, acc.z);
      acc.w = fmaf(s, a.w, acc.w);
    }
    *reinterpret_cast<float4*>(out) = acc;
  } else {
    float t[3] = {0.f, 0.f, 0.f};
    for (int i = i0; i < i1; ++i)
      for (int k = 0; k < 3 && c + k < d; ++k) t[k] = fmaf(nus[i - i0], A[(long long)i * lda + c + k], t[k]);
    for (int k = 0; k < 3 && c + k < d; ++k) out[k] = t[k];
  }
}

// u[j] = Σ_z part[z][j] in split order.
__global__ void atnu_reduce_kernel(const float* __restrict__ part, int nsplit, long long ldp, int d,
                                   float* __restrict__ u, const SolveCtl* __restrict__ ctl) {
  if (ctl != nullptr && ctl->done) return;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  float t = 0.f;
  for (int z = 0; z < nsplit; ++z) t += part[(long long)z * ldp + j];
  u[j] = t;
}

// g_i = b_i − A_i·u − λν_i for kRowsPerBlock rows per block (each load of u
// serves them all), fixed-order block sums.
constexpr int kResidRows = 4;

__global__ void __launch_bounds__(kT) dual_resid_kernel(const float* __restrict__ A, int n, int d, long long lda,
                                                        const float* __restrict__ u, const float* __restrict__ b,
                                                        const float* __restrict__ nu, float lam,
                                                        float* __restrict__ g, const SolveCtl* __restrict__ ctl) {
  if (ctl != nullptr && ctl->done) return;
  __shared__ float red[kResidRows][kT / 32];
  const int i0 = blockIdx.x * kResidRows;
  const int d4 = d >> 2;
  float s0[kResidRows], s1[kResidRows];
#pragma unroll
  for (int r = 0; r < kResidRows; ++r) s0[r] = s1[r] = 0.f;
  const float* rows[kResidRows];
#pragma unroll
  for (int r = 0; r < kResidRows; ++r) rows[r] = A + (long long)min(i0 + r, n - 1) * lda;
  for (int k = threadIdx.x; k < d4; k += kT) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(u) + k);
#pragma unroll
    for (int r = 0; r < kResidRows; ++r) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(rows[r]) + k);
      s0[r] = fmaf(a.x, v.x, fmaf(a.z, v.z, s0[r]));
      s1[r] = fmaf(a.y, v.y, fmaf(a.w, v.w, s1[r]));
    }
  }
  for (int j = 4 * d4 + threadIdx.x; j < d; j += kT) {
#pragma unroll
    for (int r = 0; r < kResidRows; ++r) s0[r] = fmaf(rows[r][j], u[j], s0[r]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kResidRows; ++r) {
    const float t = warp_sum(s0[r] + s1[r]);
    if (lane == 0) red[r][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < kResidRows) {
    const int r = threadIdx.x, i = i0 + r;
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) t += red[r][w];
    if (i < n) g[i] = b[i] - t - (nu != nullptr ? lam * nu[i] : 0.f);
  }
}

__global__ void dual_ctl_init_kernel(SolveCtl* ctl, int max_outer, float tol) {
  SolveCtl c = {};
  c.max_outer = max_outer;
  c.tol = tol;
  c.status = MIHS_OK;
  c.phase = 1;
  c.gmin = 3.0e38f;
  *ctl = c;
}

__global__ void dual_gnorm0_kernel(SolveCtl* ctl, const float* b, int n) {
  __shared__ float red[kT / 32];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += kT) s = fmaf(b[i], b[i], s);
  const float t = block_sum256(s, red);
  if (threadIdx.x == 0) {
    ctl->gnorm0 = sqrtf(t);
    ctl->gnorm0_known = 1;
  }
}

int atnu_num_splits(int64_t n) { return (int)((n + kAtnuRows - 1) / kAtnuRows); }

// u = Aᵀν through row-split partials `part` (atnu_num_splits(n) × round_up(d, 4) floats).
int launch_atnu(const float* A, int64_t n, int64_t d, int64_t lda, const float* nu, float* u, float* part,
                const SolveCtl* ctl, cudaStream_t s) {
  const int ns = atnu_num_splits(n);
  const long long ldp = round_up(d, 4);
  const unsigned cblocks = (unsigned)((d + 4 * kT - 1) / (4 * kT));
  atnu_partial_kernel<<<dim3(cblocks, (unsigned)ns), kT, 0, s>>>(A, (int)n, (int)d, lda, nu, part, ldp, ctl);
  MIHS_CHECK_LAUNCH();
  atnu_reduce_kernel<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(part, ns, ldp, (int)d, u, ctl);
  MIHS_CHECK_LAUNCH();
  count_launch(2);
  return MIHS_OK;
}

int launch_dual_resid(const float* A, int64_t n, int64_t d, int64_t lda, const float* u, const float* b,
                      const float* nu, float lam, float* g, const SolveCtl* ctl, cudaStream_t s) {
  dual_resid_kernel<<<(unsigned)((n + kResidRows - 1) / kResidRows), kT, 0, s>>>(A, (int)n, (int)d, lda, u, b, nu,
                                                                                 lam, g, ctl);
  MIHS_CHECK_LAUNCH();
  count_launch();
  return MIHS_OK;
}

int check_dual(const float* A, int64_t n, int64_t d, int64_t lda, const char* who) {
  MIHS_ARG(A != nullptr, "%s: null A", who);
  MIHS_ARG(n >= 1 && n <= kMaxD, "%s: n=%lld must be in [1, %d] (the dual inner dimension)", who, (long long)n,
           kMaxD);
  MIHS_ARG(d >= n && d < (1ll << 31), "%s: the dual form needs n <= d (n=%lld, d=%lld)", who, (long long)n,
           (long long)d);
  MIHS_ARG(lda >= d && lda % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0,
           "%s: lda=%lld must be >= d, a multiple of 4, rows 16-byte aligned", who, (long long)lda);
  return MIHS_OK;
}

}  // namespace

struct mihs_dual_s {
  int64_t n, d, m, np;
  int family;
  uint64_t seed;
  float* SAt = nullptr;   // m × np
  float* u = nullptr;     // d
  float* upart = nullptr; // atnu_num_splits(n) × round_up(d, 4): row-split partials of Aᵀν
  float* g = nullptr;     // np
  float* nu_prev = nullptr;  // np
  void* grid_ws = nullptr;   // scratch of the grid form of AAb_Solver (first solve that needs it)
  SolveCtl* ctl = nullptr;
  SolveCtl* ctl_host = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // Replaced executables, destroyed with the handle (or all at once past 64):
  // cudaGraphExecDestroy holds the host until the work in flight finishes.
  std::vector<std::pair<cudaGraphExec_t, cudaGraph_t>> retired;
  bool graph_failed = false;
  struct Key {
    const float* A; int64_t lda; const float* b; float* nu; double lam, alpha, beta; float eps; int max_passes;
    bool operator==(const Key& o) const {
      return A == o.A && lda == o.lda && b == o.b && nu == o.nu && lam == o.lam && alpha == o.alpha &&
             beta == o.beta && eps == o.eps && max_passes == o.max_passes;
    }
  } key = {};
};

namespace {

int dual_sketch_into(mihs_dual_t dk, const float* A, int64_t lda, uint64_t seed, cudaStream_t s) {
  // Aᵀ (d × np, zero columns n … np − 1), then the family's sketch of its rows.
  StreamScratch at;
  int rc = at.alloc(sizeof(float) * (size_t)dk->d * dk->np, s);
  if (rc) return rc;
  float* At = static_cast<float*>(at.p);
  MIHS_CUDA_TRY(cudaMemsetAsync(At, 0, sizeof(float) * (size_t)dk->d * dk->np, s));
  transpose_kernel<<<dim3((unsigned)((dk->d + 31) / 32), (unsigned)((dk->n + 31) / 32)), dim3(32, 8), 0, s>>>(
      A, (int)dk->n, (int)dk->d, lda, At, dk->np);
  MIHS_CHECK_LAUNCH();
  count_launch();
  rc = mihs_sketch_apply(At, dk->d, dk->n, dk->np, dk->family, dk->m, seed, dk->SAt, dk->np, s);
  if (rc) return rc;
  dk->seed = seed;
  return MIHS_OK;
}

// One step of Algorithm 2 (both gradient passes and the AAb + heavy ball).
int dual_step(mihs_dual_t dk, const mihs_dual_s::Key& k, const AabLaunch& a, cudaStream_t s) {
  int rc = launch_atnu(k.A, dk->n, dk->d, k.lda, k.nu, dk->u, dk->upart, dk->ctl, s);
  if (!rc) rc = launch_dual_resid(k.A, dk->n, dk->d, k.lda, dk->u, k.b, k.nu, (float)k.lam, dk->g, dk->ctl, s);
  if (!rc) rc = launch_aab(a, s);
  return rc;
}

void drop_dual_graph(mihs_dual_t dk) {
  if (dk->exec) cudaGraphExecDestroy(dk->exec);
  if (dk->graph) cudaGraphDestroy(dk->graph);
  dk->exec = nullptr;
  dk->graph = nullptr;
}

void free_dual_retired(mihs_dual_t dk) {
  for (auto& r : dk->retired) {
    cudaGraphExecDestroy(r.first);
    cudaGraphDestroy(r.second);
  }
  dk->retired.clear();
}

int build_dual_graph(mihs_dual_t dk, const mihs_dual_s::Key& key, const AabLaunch& proto) {
  if (dk->exec != nullptr) {  // retire the replaced executable rather than wait for the GPU
    if (dk->retired.size() >= 64) free_dual_retired(dk);
    dk->retired.push_back({dk->exec, dk->graph});
    dk->exec = nullptr;
    dk->graph = nullptr;
  }
  drop_dual_graph(dk);
  if (!dk->cap) MIHS_CUDA_TRY(cudaStreamCreateWithFlags(&dk->cap, cudaStreamNonBlocking));
  MIHS_CUDA_TRY(cudaGraphCreate(&dk->graph, 0));
  cudaGraphConditionalHandle h;
  MIHS_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, dk->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  MIHS_CUDA_TRY(cudaGraphAddNode(&node, dk->graph, nullptr, nullptr, 0, &np));
  aab_prepare((int)dk->m, (int)dk->n);
  MIHS_CUDA_TRY(cudaStreamBeginCaptureToGraph(dk->cap, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
  AabLaunch a = proto;
  a.cond = (unsigned long long)h;
  const int rc = dual_step(dk, key, a, dk->cap);
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(dk->cap, &out);
  if (rc) return rc;
  if (e != cudaSuccess) {
    set_error("dual graph capture: %s", cudaGetErrorString(e));
    return MIHS_ERR_CUDA;
  }
  MIHS_CUDA_TRY(cudaGraphInstantiate(&dk->exec, dk->graph, 0));
  dk->key = key;
  return MIHS_OK;
}

}  // namespace

extern "C" {

int mihs_dual_sketch(const float* A, int64_t n, int64_t d, int64_t lda, int family, int64_t m, uint64_t seed,
                     void* stream, mihs_dual_t* out) {
  set_error("");
  MIHS_ARG(out != nullptr, "mihs_dual_sketch: null out");
  *out = nullptr;
  int rc = check_dual(A, n, d, lda, "mihs_dual_sketch");
  if (rc) return rc;
  MIHS_ARG(family >= MIHS_GAUSSIAN && family <= MIHS_SRHT, "mihs_dual_sketch: unknown family %d", family);
  MIHS_ARG(m >= 1 && m <= d, "mihs_dual_sketch: m=%lld must be in [1, d]", (long long)m);
  mihs_dual_t dk = new (std::nothrow) mihs_dual_s();
  if (dk == nullptr) {
    set_error("mihs_dual_sketch: out of host memory");
    return MIHS_ERR_OOM;
  }
  dk->n = n;
  dk->d = d;
  dk->m = m;
  dk->np = round_up(n, 4);
  dk->family = family;
  char* p = nullptr;
  const size_t fl = (size_t)m * dk->np + (size_t)round_up(d, 4) + 2 * (size_t)dk->np +
                    (size_t)atnu_num_splits(n) * (size_t)round_up(d, 4);
  cudaError_t e = cudaMalloc(&p, fl * sizeof(float) + sizeof(SolveCtl));
  if (e == cudaSuccess) e = cudaMallocHost(&dk->ctl_host, sizeof(SolveCtl));
  if (e != cudaSuccess) {
    if (p) cudaFree(p);
    delete dk;
    set_error("mihs_dual_sketch: allocation: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
  }
  dk->SAt = reinterpret_cast<float*>(p);
  dk->u = dk->SAt + (size_t)m * dk->np;
  dk->g = dk->u + round_up(d, 4);
  dk->nu_prev = dk->g + dk->np;
  dk->upart = dk->nu_prev + dk->np;
  dk->ctl = reinterpret_cast<SolveCtl*>(dk->upart + (size_t)atnu_num_splits(n) * (size_t)round_up(d, 4));
  rc = dual_sketch_into(dk, A, lda, seed, static_cast<cudaStream_t>(stream));
  if (rc) {
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));  // nothing of this handle still in flight
    cudaFree(dk->SAt);
    cudaFreeHost(dk->ctl_host);
    delete dk;
    return rc;
  }
  *out = dk;
  return MIHS_OK;
}

int mihs_dual_resketch(mihs_dual_t dk, const float* A, int64_t lda, uint64_t seed, void* stream) {
  set_error("");
  MIHS_ARG(dk != nullptr, "mihs_dual_resketch: null handle");
  const int rc = check_dual(A, dk->n, dk->d, lda, "mihs_dual_resketch");
  if (rc) return rc;
  return dual_sketch_into(dk, A, lda, seed, static_cast<cudaStream_t>(stream));
}

int mihs_dual_copy(mihs_dual_t dk, float* dst, int64_t ldd, void* stream) {
  set_error("");
  MIHS_ARG(dk != nullptr && dst != nullptr && ldd >= dk->n, "mihs_dual_copy: bad argument");
  MIHS_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)ldd * sizeof(float), dk->SAt, (size_t)dk->np * sizeof(float),
                                  (size_t)dk->n * sizeof(float), (size_t)dk->m, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream)));
  return MIHS_OK;
}

int mihs_dual_destroy(mihs_dual_t dk) {
  if (dk == nullptr) return MIHS_OK;
  cudaDeviceSynchronize();
  drop_dual_graph(dk);
  free_dual_retired(dk);
  if (dk->cap) cudaStreamDestroy(dk->cap);
  if (dk->grid_ws) cudaFree(dk->grid_ws);
  cudaFree(dk->SAt);
  cudaFreeHost(dk->ctl_host);
  delete dk;
  return MIHS_OK;
}

int mihs_gradient_dual(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const float* nu,
                       double lambda, float* g, void* stream) {
  set_error("");
  int rc = check_dual(A, n, d, lda, "mihs_gradient_dual");
  if (rc) return rc;
  MIHS_ARG(b != nullptr && nu != nullptr && g != nullptr, "mihs_gradient_dual: null vector");
  MIHS_ARG(lambda >= 0.0 && lambda <= (double)FLT_MAX, "mihs_gradient_dual: lambda must be in [0, FLT_MAX]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch us;
  rc = us.alloc(sizeof(float) * (size_t)round_up(d, 4) * (size_t)(1 + atnu_num_splits(n)), s);
  if (rc) return rc;
  float* u = static_cast<float*>(us.p);
  rc = launch_atnu(A, n, d, lda, nu, u, u + round_up(d, 4), nullptr, s);
  if (rc) return rc;
  return launch_dual_resid(A, n, d, lda, u, b, nu, (float)lambda, g, nullptr, s);
}

int mihs_dual_recover(const float* A, int64_t n, int64_t d, int64_t lda, const float* nu, float* x, void* stream) {
  set_error("");
  const int rc = check_dual(A, n, d, lda, "mihs_dual_recover");
  if (rc) return rc;
  MIHS_ARG(nu != nullptr && x != nullptr, "mihs_dual_recover: null vector");
  MIHS_ARG((reinterpret_cast<uintptr_t>(x) & 15u) == 0, "mihs_dual_recover: x must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch ps;
  const int prc = ps.alloc(sizeof(float) * (size_t)round_up(d, 4) * (size_t)atnu_num_splits(n), s);
  if (prc) return prc;
  return launch_atnu(A, n, d, lda, nu, x, static_cast<float*>(ps.p), nullptr, s);
}

int mihs_solve_dual(mihs_dual_t dk, const float* A, int64_t lda, const float* b, double lambda,
                    const mihs_opts* opts, float* x, float* nu, mihs_info* info, void* stream) {
  set_error("");
  MIHS_ARG(dk != nullptr && opts != nullptr, "mihs_solve_dual: null handle or opts");
  int rc = check_dual(A, dk->n, dk->d, lda, "mihs_solve_dual");
  if (rc) return rc;
  MIHS_ARG(b != nullptr && nu != nullptr, "mihs_solve_dual: null b or nu");
  MIHS_ARG(x == nullptr || (reinterpret_cast<uintptr_t>(x) & 15u) == 0, "mihs_solve_dual: x must be 16-byte aligned");
  MIHS_ARG(lambda > 0.0 && lambda <= (double)FLT_MAX, "mihs_solve_dual: lambda must be in (0, FLT_MAX]");
  MIHS_ARG(opts->sd < (double)dk->m, "mihs_solve_dual: sd=%g must be < m", opts->sd);
  MIHS_ARG(opts->max_outer >= 0 && opts->max_outer < (1 << 24), "mihs_solve_dual: bad max_outer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = dk->n;
  double sd = opts->sd;
  if (!(sd > 0.0)) {  // Algorithm 4 on SAᵀ (T = 2, ε_tr = 0.5), capped below m
    rc = estimate_sd(dk->SAt, dk->m, n, dk->np, lambda, 2, 0.5, dk->seed ^ 0x4855544348ull, &sd, s);
    if (rc) return rc;
    if (!(sd > 0.0)) sd = 1.0;
    if (sd > 0.95 * (double)dk->m) sd = 0.95 * (double)dk->m;
  }
  const double beta = sd / (double)dk->m;  // Corollary 3
  const double alpha = (1.0 - beta) * (1.0 - beta);
  dual_ctl_init_kernel<<<1, 1, 0, s>>>(dk->ctl, opts->max_outer, (float)opts->tol);
  MIHS_CHECK_LAUNCH();
  count_launch();
  if (opts->warm_start) {
    dual_gnorm0_kernel<<<1, kT, 0, s>>>(dk->ctl, b, (int)n);  // ‖g(0)‖ = ‖b‖
    MIHS_CHECK_LAUNCH();
    count_launch();
  } else {
    MIHS_CUDA_TRY(cudaMemsetAsync(nu, 0, sizeof(float) * (size_t)n, s));
  }
  MIHS_CUDA_TRY(cudaMemcpyAsync(dk->nu_prev, nu, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  AabLaunch a = {};
  a.SA = dk->SAt;
  a.m = (int)dk->m;
  a.d = (int)n;
  a.ldsa = dk->np;
  a.g = dk->g;
  a.lambda = (float)lambda;
  a.eps = (float)opts->eps_sub;
  {
    const int64_t mn = dk->m < n ? dk->m : n;
    a.max_passes = (int)(opts->max_inner > 0 && opts->max_inner < mn ? opts->max_inner : mn);
  }
  a.alpha = (float)alpha;
  a.beta = (float)beta;
  a.x = nu;
  a.x_prev = dk->nu_prev;
  a.ctl = dk->ctl;
  if (aab_grid_wanted(a.m, a.d, MIHS_SA_FP32)) {  // SAᵀ too large for one cluster: the grid form
    if (dk->grid_ws == nullptr) {
      const size_t bytes = aab_grid_ws_bytes(a.d);
      const cudaError_t e = cudaMalloc(&dk->grid_ws, bytes);
      if (e != cudaSuccess) {
        dk->grid_ws = nullptr;
        set_error("mihs_solve_dual: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
      }
    }
    MIHS_CUDA_TRY(cudaMemsetAsync(dk->grid_ws, 0, kAabGridBarBytes, s));
    a.grid_ws = dk->grid_ws;
  }
  const mihs_dual_s::Key key = {A, lda, b, nu, lambda, alpha, beta, a.eps, a.max_passes};
  bool graph_ran = false;
  if (!timing_on() && !dk->graph_failed && std::getenv("MIHS_NO_GRAPH") == nullptr) {
    if (!(dk->exec && dk->key == key)) {
      if (build_dual_graph(dk, key, a) != MIHS_OK) {
        drop_dual_graph(dk);
        dk->graph_failed = true;
        cudaGetLastError();
      }
    }
    if (dk->exec) {
      MIHS_CUDA_TRY(cudaGraphLaunch(dk->exec, s));
      graph_ran = true;
    }
  }
  if (!graph_ran) {
    const bool poll = timing_on();
    for (int it = 0; it <= opts->max_outer; ++it) {
      rc = dual_step(dk, key, a, s);
      if (rc) return rc;
      if (poll) {
        MIHS_CUDA_TRY(cudaMemcpyAsync(dk->ctl_host, dk->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
        MIHS_CUDA_TRY(cudaStreamSynchronize(s));
        if (dk->ctl_host->done) break;
      }
    }
  }
  if (x != nullptr) {  // x = Aᵀν (Eq. dual_relation)
    rc = launch_atnu(A, n, dk->d, lda, nu, x, dk->upart, nullptr, s);
    if (rc) return rc;
  }
  if (info == nullptr) return MIHS_OK;
  MIHS_CUDA_TRY(cudaMemcpyAsync(dk->ctl_host, dk->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  const SolveCtl& c = *dk->ctl_host;
  info->outer_iters = c.outer;
  info->inner_iters_total = c.inner_total;
  info->rel_resid = c.gnorm0 > 0.f ? (double)c.gnorm / (double)c.gnorm0 : 0.0;
  info->status = c.done ? c.status : MIHS_NOT_CONVERGED;
  if (graph_ran) count_launch(4ull * (uint64_t)(c.outer + 1));
  return info->status;
}

}  // extern "C"
