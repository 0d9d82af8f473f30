// C ABI of libmihs: argument checks, handles and the host side of Algorithm 1.
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "internal.h"

namespace mihs {

std::atomic<uint64_t> g_launches{0};

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int num_sms() {
  static std::mutex mu;
  static std::vector<int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
  if (cache[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

namespace {

struct Timing {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> ev[kNumTimers];  // (start, stop) pairs
  size_t used[kNumTimers] = {};
};
Timing& timing_state() {
  static Timing* t = new Timing();  // never destroyed: events outlive static teardown
  return *t;
}

}  // namespace

bool timing_on() { return timing_state().on; }

void timing_begin(int which, cudaStream_t s) {
  Timing& t = timing_state();
  if (!t.on) return;
  std::lock_guard<std::mutex> lk(t.mu);
  const size_t i = t.used[which];
  while (t.ev[which].size() < 2 * i + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    t.ev[which].push_back(e);
  }
  cudaEventRecord(t.ev[which][2 * i], s);
}

void timing_end(int which, cudaStream_t s) {
  Timing& t = timing_state();
  if (!t.on) return;
  std::lock_guard<std::mutex> lk(t.mu);
  const size_t i = t.used[which];
  if (t.ev[which].size() < 2 * i + 2) return;
  cudaEventRecord(t.ev[which][2 * i + 1], s);
  t.used[which] = i + 1;
}

namespace {

__global__ void ctl_init_kernel(SolveCtl* ctl, int max_outer, float tol, int phase, float switch_tol, int corr) {
  SolveCtl c = {};
  c.max_outer = max_outer;
  c.tol = tol;
  c.status = MIHS_OK;
  c.phase = phase;
  c.switch_tol = switch_tol;
  c.gmin = 3.0e38f;
  c.stall = 0;
  c.corr = corr;
  c.refresh = 1;
  c.since = 0;
  c.gref = 3.0e38f;
  *ctl = c;
}

// δ = x − x_ref in fp32 for the correction step of a refinement solve.
__global__ void refine_delta_kernel(const double* __restrict__ x, const double* __restrict__ xref,
                                    float* __restrict__ delta, int d, const SolveCtl* __restrict__ ctl) {
  if (ctl->done || ctl_gate(ctl) != 2) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < d) delta[j] = (float)(x[j] - xref[j]);
}

// λ-path control blocks: one per λ (plain solves), the stop counter cleared.
__global__ void path_init_kernel(SolveCtl* ctl, int* cnt, int nl, int max_outer, float tol) {
  const int l = threadIdx.x;
  if (l < nl) {
    SolveCtl c = {};
    c.max_outer = max_outer;
    c.tol = tol;
    c.status = MIHS_OK;
    c.phase = 1;
    c.gmin = 3.0e38f;
    ctl[l] = c;
  }
  if (l == 0) {
    cnt[0] = 0;
    cnt[1] = 0;
  }
}

// ‖g‖ (g = Aᵀb) as the path's common relative-residual denominator.
__global__ void path_set_gnorm0_kernel(SolveCtl* ctl, int nl, const float* g, int d) {
  __shared__ float red[32];
  float s = 0.f;
  for (int j = threadIdx.x; j < d; j += blockDim.x) s = fmaf(g[j], g[j], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    for (int l = 0; l < nl; ++l) {
      ctl[l].gnorm0 = sqrtf(t);
      ctl[l].gnorm0_known = 1;
    }
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < d) b[j] = (float)a[j];
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, int d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < d) b[j] = (double)a[j];
}

// ‖g‖ for the warm-start reference norm ‖Aᵀb‖ (one block, fixed order).
__global__ void ctl_set_gnorm0_kernel(SolveCtl* ctl, const float* g, int d) {
  __shared__ float red[32];
  float s = 0.f;
  for (int j = threadIdx.x; j < d; j += blockDim.x) s = fmaf(g[j], g[j], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    ctl->gnorm0 = sqrtf(t);
    ctl->gnorm0_known = 1;
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_matrix(const float* A, int64_t n, int64_t d, int64_t lda, const char* what) {
  MIHS_ARG(A != nullptr, "%s: null matrix", what);
  MIHS_ARG(d >= 1 && d <= kMaxD, "%s: d=%lld outside [1, %d]", what, (long long)d, kMaxD);
  MIHS_ARG(n >= 1 && n < (1LL << 31), "%s: n=%lld outside [1, 2^31)", what, (long long)n);
  MIHS_ARG(lda >= d && lda % 4 == 0, "%s: lda=%lld must be >= d and a multiple of 4", what,
           (long long)lda);
  MIHS_ARG(aligned16(A), "%s: matrix pointer must be 16-byte aligned", what);
  return MIHS_OK;
}

}  // namespace
}  // namespace mihs

using namespace mihs;

struct mihs_sketch_s {
  int device;
  int64_t n, d, m, dp;
  int family;
  uint64_t seed;
  int P;              // split-K partials of the A-pass
  float* SA;          // m × dp
  int sa_prec = MIHS_SA_FP32;  // storage of SA inside AAb_Solver
  void* SAq = nullptr;         // quantised SA (m × ldq) when sa_prec != fp32
  float* sa_scales = nullptr;  // fp8 tile scales
  int64_t ldq = 0;
  double* sa_qerr_dev = nullptr;  // kQuantErrBlocks partials + ‖SA_q − SA‖_F²
  double sa_qerr = 0.0;           // host copy of ‖SA_q − SA‖_F² for the current SA_q
  float* partials;    // P × dp
  float* g;           // dp
  float* x_prev;      // dp
  float* hist;        // kHistCap: ‖g‖ per gradient step of the last solve
  // Refinement workspace (allocated on first refined solve): double-float
  // partials of the compensated A-pass and the fp64 previous iterate.
  float2* dd_partials = nullptr;
  double* x_prev64 = nullptr;
  float* x32_shadow = nullptr;
  float* bw32 = nullptr;  // 2·dp: fp32 roundings of x and v for refined backward solves
  double* gref64 = nullptr;  // dp: the compensated gradient at the last refresh
  double* xref64 = nullptr;  // dp: the point it was taken at
  float* delta32 = nullptr;  // dp: x − x_ref for the fp32 correction pass
  int P_dd = 0;
  double last_sd = 0; // sd estimated by the last solve that was given sd ≤ 0
  SolveCtl* ctl;
  SolveCtl* ctl_host; // pinned
  // Device-side outer loop: a CUDA graph holding one conditional WHILE node
  // whose body is (A-pass, partial-sum reduce, AAb + heavy ball); the AAb
  // kernel clears the condition when the stop test fires.  Up to
  // kGraphWays graphs per kind of solve (plain, refinement, adjoint), keyed
  // by the solve's pointers and scalars and replaced least recently used, so
  // that a caller alternating between input buffers (a copy of the next
  // problem landing while this one solves) or refining several λ relaunches
  // instead of rebuilding.  A replaced executable is retired, not destroyed:
  // cudaGraphExecDestroy holds the host until the work in flight has
  // finished (measured: 17.6 ms behind one solve, 2.6 ms behind another even
  // when the destroyed graph's own launch had ended), which serialises every
  // stream.  Retired executables are freed with the handle, or all at once
  // when more than kMaxRetired have gathered.
  cudaStream_t cap = nullptr;
  struct Key {
    const float* A; int64_t lda; const float* b; void* x;
    double lam, alpha, beta; float eps; int max_passes;
    const float* rhs;  // adjoint solves: g = rhs − AᵀAx − λx (b null)
    int sa_prec;       // storage of SA read by AAb_Solver
    int aab_form, aab_blocks;
    bool operator==(const Key& o) const {
      return A == o.A && lda == o.lda && b == o.b && x == o.x && rhs == o.rhs && sa_prec == o.sa_prec &&
             aab_form == o.aab_form && aab_blocks == o.aab_blocks &&
             lam == o.lam &&
             alpha == o.alpha && beta == o.beta && eps == o.eps && max_passes == o.max_passes;
    }
  };
  static constexpr int kGraphWays = 8;
  static constexpr size_t kMaxRetired = 64;
  struct GraphSlot {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Key key = {};
    uint64_t used = 0;  // launch tick of the last use (0: empty)
  } slots[4][kGraphWays];      // kind = (refined ? 1 : 0) + (adjoint ? 2 : 0)
  std::vector<std::pair<cudaGraphExec_t, cudaGraph_t>> retired;  // replaced, not yet destroyed
  bool graph_failed[4] = {};   // capture failed once: host-driven steps for that kind from then on
  uint64_t graph_tick = 0;
  // λ-path workspace (allocated on the first path solve): split-K partials
  // (P_path × 16 × dp), G and X⁻ (16 × dp each), 16 control blocks and the
  // path's stop counter / flag.
  void* aab_grid_ws = nullptr;   // global scratch of the single-λ grid AAb kernel (first solve that needs it)
  int aab_form = MIHS_AAB_AUTO;  // form of AAb_Solver in single-λ solves (mihs_sketch_set_aab)
  int aab_grid_blocks = 0;
  float* path_partials = nullptr;
  float* path_aab_ws = nullptr;  // global scratch of the cooperative multi-λ AAb kernel
  float* path_g = nullptr;
  float* path_xprev = nullptr;
  SolveCtl* path_ctl = nullptr;
  int* path_cnt = nullptr;  // [0] λ stopped, [1] all stopped
  SolveCtl* path_ctl_host = nullptr;  // pinned, path_ctl_cap entries (one per λ of the last path)
  int path_ctl_cap = 0;
  int P_path = 0;
  struct PathKey {
    const float* A; int64_t lda; const float* b; float* X; int64_t ldx;
    PathScalars ps; float eps; int max_passes; int sa_prec;
    bool operator==(const PathKey& o) const {
      return A == o.A && lda == o.lda && b == o.b && X == o.X && ldx == o.ldx && eps == o.eps &&
             sa_prec == o.sa_prec &&
             max_passes == o.max_passes && std::memcmp(&ps, &o.ps, sizeof(ps)) == 0;
    }
  };
  cudaGraph_t path_graph = nullptr;
  cudaGraphExec_t path_exec = nullptr;
  PathKey path_key = {};
  bool path_graph_failed = false;
  // Refinement of chosen λ of a path (mihs_refine_batched): the fp64 iterate
  // of the refined solve and pinned host copies of its control blocks.
  double* ref_x64 = nullptr;
  SolveCtl* ref_ctl_host = nullptr;
  int ref_ctl_cap = 0;
};

namespace {

// The SA that AAb_Solver reads: fp32, or the quantised copy.
void set_sa(AabLaunch& a, const mihs_sketch_s* sk) {
  if (sk->sa_prec != MIHS_SA_FP32 && sk->SAq != nullptr) {
    a.SA = sk->SAq;
    a.sa_type = sk->sa_prec;
    a.sa_scale = sk->sa_scales;
    a.ldsa = sk->ldq;
  } else {
    a.SA = sk->SA;
    a.sa_type = MIHS_SA_FP32;
    a.ldsa = sk->dp;
  }
}

// The grid form of AAb_Solver (SA too large for one cluster's shared memory,
// or asked for by mihs_sketch_set_aab) needs global scratch: the handle's,
// allocated on first use; its barrier word is zeroed on the solve's stream
// before every solve.
int use_grid_ws(mihs_sketch_s* sk, AabLaunch& a, cudaStream_t s) {
  a.aab_form = sk->aab_form;
  a.grid_blocks = sk->aab_grid_blocks;
  if (!aab_grid_wanted(a.m, a.d, a.sa_type, a.aab_form)) return MIHS_OK;
  if (sk->aab_grid_ws == nullptr) {
    const size_t bytes = aab_grid_ws_bytes(a.d);
    cudaError_t e = cudaMalloc(&sk->aab_grid_ws, bytes);
    if (e != cudaSuccess) {
      sk->aab_grid_ws = nullptr;
      set_error("AAb grid scratch: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
    }
  }
  MIHS_CUDA_TRY(cudaMemsetAsync(sk->aab_grid_ws, 0, kAabGridBarBytes, s));
  a.grid_ws = sk->aab_grid_ws;
  return MIHS_OK;
}

// Row-level calls take the grid form's scratch from the stream-ordered pool.
int use_grid_scratch(AabLaunch& a, StreamScratch& ws, cudaStream_t s) {
  if (!aab_grid_wanted(a.m, a.d, a.sa_type)) return MIHS_OK;
  int rc = ws.alloc(aab_grid_ws_bytes(a.d), s);
  if (rc) return rc;
  MIHS_CUDA_TRY(cudaMemsetAsync(ws.p, 0, kAabGridBarBytes, s));
  a.grid_ws = ws.p;
  return MIHS_OK;
}

void drop_graph(mihs_sketch_s::GraphSlot& gs) {
  if (gs.exec) cudaGraphExecDestroy(gs.exec);
  if (gs.graph) cudaGraphDestroy(gs.graph);
  gs.exec = nullptr;
  gs.graph = nullptr;
}

// Destroys every retired executable (this waits for the work in flight).
void free_retired(mihs_sketch_s* sk) {
  for (auto& r : sk->retired) {
    cudaGraphExecDestroy(r.first);
    cudaGraphDestroy(r.second);
  }
  sk->retired.clear();
}

// Moves a graph out of the way it occupies into the retired list.
void retire_graph(mihs_sketch_s* sk, cudaGraphExec_t& exec, cudaGraph_t& graph) {
  if (exec != nullptr) {
    if (sk->retired.size() >= mihs_sketch_s::kMaxRetired) free_retired(sk);
    sk->retired.push_back({exec, graph});
  } else if (graph != nullptr) {
    cudaGraphDestroy(graph);  // never instantiated: nothing can be running it
  }
  exec = nullptr;
  graph = nullptr;
}

// One outer step of Algorithm 1 (gradient, partial-sum reduce, AAb_Solver +
// heavy ball), plain fp32 or compensated (refinement).
// In a refinement solve both gradient variants are launched, each gated on
// ctl->phase (plain fp32 while it is 0, compensated once it is 1), unless
// `phase` names the one the host knows to be current.
int launch_step(mihs_sketch_s* sk, const mihs_sketch_s::Key& key, const AabLaunch& a, bool refined,
                cudaStream_t s, int phase = -1) {
  int rc = MIHS_OK;
  if (refined) {
    // gate 0: plain fp32 pass at the fp32 shadow of x (phase 0)
    if (phase < 0 || phase == 0) {
      rc = launch_apass_partial(key.A, sk->n, sk->d, key.lda, key.b, sk->x32_shadow, sk->partials, sk->ctl, s, 0);
      if (!rc) rc = launch_apass_finalize(sk->partials, sk->P, sk->d, sk->x32_shadow, (float)key.lam, sk->g,
                                          sk->ctl, s, 0, key.rhs);
    }
    // gate 1: compensated refresh at x, kept with x as (g_ref, x_ref)
    if (!rc && (phase < 0 || phase == 1)) {
      const double* x64 = static_cast<const double*>(key.x);
      rc = launch_apass_dd(key.A, sk->n, sk->d, key.lda, key.b, x64, sk->dd_partials, sk->ctl, s, 1);
      if (!rc) rc = launch_apass_dd_finalize(sk->dd_partials, sk->P_dd, sk->d, x64, key.lam, sk->gref64, sk->g,
                                             sk->ctl, s, 1, key.rhs, sk->xref64);
    }
    // gate 2: g = g_ref − H(x − x_ref), H·δ by the fp32 pass with b = 0
    if (!rc && (phase < 0 || phase == 2)) {
      refine_delta_kernel<<<(unsigned)((sk->d + 255) / 256), 256, 0, s>>>(
          static_cast<const double*>(key.x), sk->xref64, sk->delta32, (int)sk->d, sk->ctl);
      MIHS_CHECK_LAUNCH();
      count_launch();
      rc = launch_apass_partial(key.A, sk->n, sk->d, key.lda, nullptr, sk->delta32, sk->partials, sk->ctl, s, 2);
      if (!rc) rc = launch_apass_finalize(sk->partials, sk->P, sk->d, sk->delta32, (float)key.lam, sk->g,
                                          sk->ctl, s, 2, nullptr, sk->gref64);
    }
  } else {
    rc = launch_apass_partial(key.A, sk->n, sk->d, key.lda, key.b, static_cast<const float*>(key.x),
                              sk->partials, sk->ctl, s);
    if (!rc) rc = launch_apass_finalize(sk->partials, sk->P, sk->d, static_cast<const float*>(key.x),
                                        (float)key.lam, sk->g, sk->ctl, s, -1, key.rhs);
  }
  if (!rc) rc = launch_aab(a, s);
  return rc;
}

// Captures `body(cond, stream)` into the body graph of a conditional WHILE
// node.  Returns MIHS_OK or an error (the caller then falls back to
// host-driven iterations).
template <typename Body>
int build_while_graph(mihs_sketch_s* sk, int m, int d, cudaGraph_t& graph, cudaGraphExec_t& exec, Body body) {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  if (!sk->cap) MIHS_CUDA_TRY(cudaStreamCreateWithFlags(&sk->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  MIHS_CUDA_TRY(cudaGraphCreate(&g, 0));
  graph = g;
  cudaGraphConditionalHandle h;
  MIHS_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  MIHS_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  aab_prepare(m, d, sk->sa_prec);
  MIHS_CUDA_TRY(cudaStreamBeginCaptureToGraph(sk->cap, bodyg, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
  int rc = body((unsigned long long)h, sk->cap);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(sk->cap, &out);
  if (rc) return rc;
  if (e != cudaSuccess) {
    set_error("graph capture: %s", cudaGetErrorString(e));
    return MIHS_ERR_CUDA;
  }
  MIHS_CUDA_TRY(cudaGraphInstantiate(&exec, g, 0));
  return MIHS_OK;
}

int build_graph(mihs_sketch_s* sk, const mihs_sketch_s::Key& key, const AabLaunch& proto, bool refined,
                mihs_sketch_s::GraphSlot& gs) {
  const int rc = build_while_graph(sk, (int)sk->m, (int)sk->d, gs.graph, gs.exec,
                                   [&](unsigned long long cond, cudaStream_t cs) {
                                     AabLaunch a = proto;
                                     a.cond = cond;
                                     return launch_step(sk, key, a, refined, cs);
                                   });
  if (rc == MIHS_OK) gs.key = key;
  return rc;
}

// Whether a path solve on this handle takes the all-λ grid form of
// AAb_Solver (opt-in, MIHS_PATH_AAB=grid).  Measured on the batched workload
// (64 matrices × 16 λ, SA up to 16 MB) the one-cluster-per-λ form is twice as
// fast even where SA does not fit a cluster's shared memory: each λ stops on
// its own, clusters of different problems run concurrently on four streams,
// while the grid form keeps every λ until the slowest stops and must not run
// beside another grid.
bool path_uses_grid(const mihs_sketch_s* sk) {
  const char* e = std::getenv("MIHS_PATH_AAB");
  return e != nullptr && std::strcmp(e, "grid") == 0 && sk->sa_prec == MIHS_SA_FP32 && sk->d <= 1024;
}

// One outer step of Algorithm 1 for every λ of a path: the shared gradient
// pass, its reduce, and one AAb_Solver cluster per λ (+ heavy ball).
int launch_path_step(mihs_sketch_s* sk, const mihs_sketch_s::PathKey& k, const AabLaunch& a, cudaStream_t s) {
  const int* all_done = sk->path_cnt + 1;
  int rc = launch_apass_path(k.A, sk->n, sk->d, k.lda, k.b, k.X, k.ldx, k.ps.nl, sk->path_partials, all_done, s);
  if (!rc) rc = launch_apass_path_finalize(sk->path_partials, sk->P_path, sk->d, k.X, k.ldx, k.ps, sk->path_g,
                                           sk->dp, all_done, s);
  if (rc) return rc;
  // One thread-block cluster per λ, or (opt-in) all λ in one cooperative
  // grid with SA spread over the SMs' shared memory.
  if (path_uses_grid(sk)) {
    rc = launch_aab_path(a, sk->path_aab_ws, s);
    if (rc != MIHS_ERR_UNSUPPORTED) return rc;
  }
  return launch_aab(a, s);
}

}  // namespace

extern "C" {

const char* mihs_strerror(int code) {
  switch (code) {
    case MIHS_OK: return "ok";
    case MIHS_NOT_CONVERGED: return "not converged within max_outer";
    case MIHS_ERR_INVALID_ARG: return "invalid argument";
    case MIHS_ERR_CUDA: return "CUDA error";
    case MIHS_ERR_OOM: return "out of device memory";
    case MIHS_ERR_TIMEOUT: return "device wait timed out";
    case MIHS_ERR_NUMERIC: return "non-finite value encountered";
    case MIHS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

const char* mihs_last_error(void) { return g_err; }

uint64_t mihs_launch_count(void) { return g_launches.load(); }

int mihs_device_status(int* code) {
  set_error("");
  MIHS_ARG(code != nullptr, "mihs_device_status: null code");
  int a = 0, g = 0, dd = 0, pa = 0, ab = 0;
  int rc = apass_device_error(&a);
  if (rc) return rc;
  rc = gauss_tc_device_error(&g);
  if (rc) return rc;
  rc = apass_dd_device_error(&dd);
  if (rc) return rc;
  rc = apass_path_device_error(&pa);
  if (rc) return rc;
  rc = aab_path_device_error(&ab);
  if (rc) return rc;
  int gr = 0;
  rc = aab_grid_device_error(&gr);
  if (rc) return rc;
  int sr = 0;
  rc = srht_device_error(&sr);
  if (rc) return rc;
  *code = a ? a : (g ? g : (dd ? dd : (pa ? pa : (ab ? ab : (gr ? gr : sr)))));
  return MIHS_OK;
}

mihs_opts mihs_default_opts(void) {
  mihs_opts o;
  o.tol = 1e-6;
  o.max_outer = 100;
  o.eps_sub = 0.1;
  o.max_inner = 0;
  o.sd = 0.0;
  o.warm_start = 0;
  return o;
}

int mihs_sketch_apply(const float* A, int64_t n, int64_t d, int64_t lda, int family, int64_t m,
                      uint64_t seed, float* SA, int64_t ldsa, void* stream) {
  set_error("");
  int rc = check_matrix(A, n, d, lda, "mihs_sketch_apply");
  if (rc) return rc;
  MIHS_ARG(SA != nullptr, "mihs_sketch_apply: null SA");
  MIHS_ARG(m >= 1 && m <= n, "mihs_sketch_apply: m=%lld outside [1, n]", (long long)m);
  MIHS_ARG(ldsa >= d, "mihs_sketch_apply: ldsa < d");
  MIHS_ARG(family >= MIHS_GAUSSIAN && family <= MIHS_SRHT, "mihs_sketch_apply: unknown family %d",
           family);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  timing_begin(kTimerSketch, s);
  switch (family) {
    case MIHS_GAUSSIAN: rc = sketch_gaussian(A, n, d, lda, m, seed, SA, ldsa, s); break;
    case MIHS_COUNTSKETCH: rc = sketch_countsketch(A, n, d, lda, m, seed, SA, ldsa, s); break;
    default: rc = sketch_srht(A, n, d, lda, m, seed, SA, ldsa, s); break;
  }
  timing_end(kTimerSketch, s);
  return rc;
}

static int gaussian_lowp(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed, float* SA,
                         int64_t ldsa, void* stream, int prec, const char* who) {
  set_error("");
  int rc = check_matrix(A, n, d, lda, who);
  if (rc) return rc;
  MIHS_ARG(SA != nullptr, "%s: null SA", who);
  MIHS_ARG(m >= 1 && m <= n, "%s: m=%lld outside [1, n]", who, (long long)m);
  MIHS_ARG(ldsa >= d, "%s: ldsa < d", who);
  if (!gaussian_tc_available()) {
    set_error("%s: the tensor-core sketch is unavailable (no cuTensorMapEncodeTiled)", who);
    return MIHS_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  timing_begin(kTimerSketch, s);
  rc = sketch_gaussian_tc(A, n, d, lda, m, seed, SA, ldsa, s, prec);
  timing_end(kTimerSketch, s);
  return rc;
}

int mihs_sketch_gaussian_bf16(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed,
                              float* SA, int64_t ldsa, void* stream) {
  return gaussian_lowp(A, n, d, lda, m, seed, SA, ldsa, stream, 1, "mihs_sketch_gaussian_bf16");
}

int mihs_sketch_gaussian_fp8(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed,
                             float* SA, int64_t ldsa, void* stream) {
  return gaussian_lowp(A, n, d, lda, m, seed, SA, ldsa, stream, 2, "mihs_sketch_gaussian_fp8");
}

int mihs_timing(int on) {
  Timing& t = timing_state();
  std::lock_guard<std::mutex> lk(t.mu);
  t.on = on != 0;
  for (int w = 0; w < kNumTimers; ++w) t.used[w] = 0;
  return MIHS_OK;
}

int mihs_timing_read(int which, double* total_ms, int64_t* count) {
  set_error("");
  MIHS_ARG(which >= 0 && which < kNumTimers, "mihs_timing_read: bad timer %d", which);
  MIHS_ARG(total_ms != nullptr && count != nullptr, "mihs_timing_read: null output");
  Timing& t = timing_state();
  std::lock_guard<std::mutex> lk(t.mu);
  double tot = 0.0;
  for (size_t i = 0; i < t.used[which]; ++i) {
    MIHS_CUDA_TRY(cudaEventSynchronize(t.ev[which][2 * i + 1]));
    float ms = 0.f;
    MIHS_CUDA_TRY(cudaEventElapsedTime(&ms, t.ev[which][2 * i], t.ev[which][2 * i + 1]));
    tot += ms;
  }
  *total_ms = tot;
  *count = (int64_t)t.used[which];
  return MIHS_OK;
}

int mihs_gradient(const float* A, int64_t n, int64_t d, int64_t lda, const float* b,
                  const float* x, double lambda, float* g, void* stream) {
  set_error("");
  int rc = check_matrix(A, n, d, lda, "mihs_gradient");
  if (rc) return rc;
  MIHS_ARG(b != nullptr && x != nullptr && g != nullptr, "mihs_gradient: null vector");
  MIHS_ARG(lambda >= 0.0 && lambda <= (double)FLT_MAX, "mihs_gradient: lambda must be in [0, FLT_MAX]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = apass_num_partials(n, d);
  StreamScratch scratch;
  rc = scratch.alloc(sizeof(float) * (size_t)P * apass_dpad(d), s);
  if (rc) return rc;
  float* part = static_cast<float*>(scratch.p);
  rc = launch_apass_partial(A, n, d, lda, b, x, part, nullptr, s);
  if (rc) return rc;
  return launch_apass_finalize(part, P, d, x, (float)lambda, g, nullptr, s);
}

static int aab_common(const float* SA, int64_t m, int64_t d, int64_t ldsa, const float* g,
                      double lambda, double eps_sub, int max_inner, const char* who) {
  MIHS_ARG(SA != nullptr && g != nullptr, "%s: null pointer", who);
  MIHS_ARG(m >= 1 && m < (1LL << 31), "%s: m=%lld out of range", who, (long long)m);
  MIHS_ARG(d >= 1 && d <= kMaxD, "%s: d=%lld outside [1, %d]", who, (long long)d, kMaxD);
  MIHS_ARG(ldsa >= d, "%s: ldsa must be >= d", who);
  MIHS_ARG(lambda > 0.0 && lambda <= (double)FLT_MAX, "%s: lambda must be in (0, FLT_MAX]", who);
  MIHS_ARG(eps_sub >= 0.0, "%s: eps_sub must be >= 0", who);
  (void)max_inner;
  return MIHS_OK;
}

static int cap_passes(int64_t m, int64_t d, int max_inner) {
  const int64_t mn = m < d ? m : d;
  return (int)(max_inner > 0 && max_inner < mn ? max_inner : mn);
}

int mihs_quantize_sa(const float* SA, int64_t m, int64_t d, int64_t ldsa, int sa_prec, void* out, int64_t ldq,
                     float* scales, void* stream) {
  set_error("");
  MIHS_ARG(SA != nullptr && out != nullptr, "mihs_quantize_sa: null SA or out");
  MIHS_ARG(m >= 1 && d >= 1 && d <= kMaxD && ldsa >= d, "mihs_quantize_sa: bad shape");
  MIHS_ARG(sa_prec == MIHS_SA_BF16 || sa_prec == MIHS_SA_FP8E4M3, "mihs_quantize_sa: precision must be bf16 or fp8");
  MIHS_ARG(ldq >= d && ldq % 16 == 0, "mihs_quantize_sa: ldq must be >= d and a multiple of 16");
  MIHS_ARG(sa_prec != MIHS_SA_FP8E4M3 || scales != nullptr, "mihs_quantize_sa: fp8 needs a scale array");
  return launch_quantize_sa(SA, m, d, ldsa, sa_prec, out, ldq, scales, static_cast<cudaStream_t>(stream));
}

int mihs_aab_solve_q(const void* SAq, int sa_prec, const float* scales, int64_t m, int64_t d, int64_t ldq,
                     const float* g, double lambda, double eps_sub, int max_inner, float* delta, int* passes,
                     void* stream) {
  set_error("");
  MIHS_ARG(sa_prec == MIHS_SA_BF16 || sa_prec == MIHS_SA_FP8E4M3, "mihs_aab_solve_q: precision must be bf16 or fp8");
  MIHS_ARG(SAq != nullptr && g != nullptr && delta != nullptr, "mihs_aab_solve_q: null argument");
  MIHS_ARG(m >= 1 && d >= 1 && d <= kMaxD && ldq >= d && ldq % 16 == 0, "mihs_aab_solve_q: bad shape");
  MIHS_ARG(lambda > 0.0 && lambda <= (double)FLT_MAX && eps_sub >= 0.0, "mihs_aab_solve_q: bad lambda or eps");
  AabLaunch a = {};
  a.SA = SAq;
  a.sa_type = sa_prec;
  a.sa_scale = scales;
  a.m = (int)m;
  a.d = (int)d;
  a.ldsa = ldq;
  a.g = g;
  a.lambda = (float)lambda;
  a.eps = (float)eps_sub;
  a.max_passes = cap_passes(m, d, max_inner);
  a.delta = delta;
  a.passes = passes;
  StreamScratch ws;
  int rc = use_grid_scratch(a, ws, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return launch_aab(a, static_cast<cudaStream_t>(stream));
}

int mihs_aab_solve(const float* SA, int64_t m, int64_t d, int64_t ldsa, const float* g,
                   double lambda, double eps_sub, int max_inner, float* delta, int* passes,
                   void* stream) {
  set_error("");
  int rc = aab_common(SA, m, d, ldsa, g, lambda, eps_sub, max_inner, "mihs_aab_solve");
  if (rc) return rc;
  MIHS_ARG(delta != nullptr, "mihs_aab_solve: null delta");
  AabLaunch a = {};
  a.SA = SA;
  a.m = (int)m;
  a.d = (int)d;
  a.ldsa = ldsa;
  a.g = g;
  a.lambda = (float)lambda;
  a.eps = (float)eps_sub;
  a.max_passes = cap_passes(m, d, max_inner);
  a.delta = delta;
  a.passes = passes;
  StreamScratch ws;
  rc = use_grid_scratch(a, ws, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return launch_aab(a, static_cast<cudaStream_t>(stream));
}

int mihs_aab_heavy_ball(const float* SA, int64_t m, int64_t d, int64_t ldsa, const float* g,
                        double lambda, double eps_sub, int max_inner, double alpha, double beta,
                        float* x, float* x_prev, int* passes, void* stream) {
  set_error("");
  int rc = aab_common(SA, m, d, ldsa, g, lambda, eps_sub, max_inner, "mihs_aab_heavy_ball");
  if (rc) return rc;
  MIHS_ARG(x != nullptr && x_prev != nullptr, "mihs_aab_heavy_ball: null x or x_prev");
  AabLaunch a = {};
  a.SA = SA;
  a.m = (int)m;
  a.d = (int)d;
  a.ldsa = ldsa;
  a.g = g;
  a.lambda = (float)lambda;
  a.eps = (float)eps_sub;
  a.max_passes = cap_passes(m, d, max_inner);
  a.passes = passes;
  a.alpha = (float)alpha;
  a.beta = (float)beta;
  a.x = x;
  a.x_prev = x_prev;
  StreamScratch ws;
  rc = use_grid_scratch(a, ws, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return launch_aab(a, static_cast<cudaStream_t>(stream));
}

int mihs_estimate_sd(const float* SA, int64_t m, int64_t d, int64_t ldsa, double lambda, int T,
                     double eps_tr, uint64_t seed, double* sd_out, void* stream) {
  set_error("");
  int rc = aab_common(SA, m, d, ldsa, SA, lambda, eps_tr, 0, "mihs_estimate_sd");
  if (rc) return rc;
  MIHS_ARG(T >= 1 && T <= 1024, "mihs_estimate_sd: T=%d outside [1, 1024]", T);
  MIHS_ARG(sd_out != nullptr, "mihs_estimate_sd: null sd_out");
  return estimate_sd(SA, m, d, ldsa, lambda, T, eps_tr, seed, sd_out, static_cast<cudaStream_t>(stream));
}

int mihs_sketch(const float* A, int64_t n, int64_t d, int64_t lda, int family, int64_t m,
                uint64_t seed, void* stream, mihs_sketch_t* out) {
  set_error("");
  MIHS_ARG(out != nullptr, "mihs_sketch: null out");
  *out = nullptr;
  int rc = check_matrix(A, n, d, lda, "mihs_sketch");
  if (rc) return rc;
  MIHS_ARG(m >= 1 && m <= n, "mihs_sketch: m=%lld outside [1, n]", (long long)m);
  MIHS_ARG(family >= MIHS_GAUSSIAN && family <= MIHS_SRHT, "mihs_sketch: unknown family %d", family);
  mihs_sketch_s* h = new (std::nothrow) mihs_sketch_s();
  if (!h) return MIHS_ERR_OOM;
  const cudaError_t ed = cudaGetDevice(&h->device);
  if (ed != cudaSuccess) {
    delete h;
    set_error("mihs_sketch: cudaGetDevice: %s", cudaGetErrorString(ed));
    return MIHS_ERR_CUDA;
  }
  h->n = n;
  h->d = d;
  h->m = m;
  h->dp = apass_dpad(d);
  h->family = family;
  h->seed = seed;
  h->P = apass_num_partials(n, d);
  const size_t bytes = sizeof(float) * ((size_t)m * h->dp + (size_t)h->P * h->dp + 2 * h->dp + kHistCap) +
                       sizeof(SolveCtl) + 256;
  char* base = nullptr;
  cudaError_t e = cudaMalloc(&base, bytes);
  if (e != cudaSuccess) {
    delete h;
    set_error("mihs_sketch: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
  }
  h->SA = reinterpret_cast<float*>(base);
  h->partials = h->SA + (size_t)m * h->dp;
  h->g = h->partials + (size_t)h->P * h->dp;
  h->x_prev = h->g + h->dp;
  h->hist = h->x_prev + h->dp;
  h->ctl = reinterpret_cast<SolveCtl*>(round_up(reinterpret_cast<uintptr_t>(h->hist + kHistCap), 64));
  e = cudaMallocHost(&h->ctl_host, sizeof(SolveCtl));
  if (e != cudaSuccess) {
    cudaFree(base);
    delete h;
    set_error("mihs_sketch: cudaMallocHost: %s", cudaGetErrorString(e));
    return MIHS_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  e = h->dp != d ? cudaMemsetAsync(h->SA, 0, sizeof(float) * (size_t)m * h->dp, s) : cudaSuccess;
  if (e != cudaSuccess) {
    set_error("mihs_sketch: cudaMemsetAsync: %s", cudaGetErrorString(e));
    rc = MIHS_ERR_CUDA;
  } else {
    rc = mihs_sketch_apply(A, n, d, lda, family, m, seed, h->SA, h->dp, stream);
  }
  if (rc) {
    cudaStreamSynchronize(s);
    cudaFreeHost(h->ctl_host);
    cudaFree(base);
    delete h;
    return rc;
  }
  *out = h;
  return MIHS_OK;
}

// Quantises the handle's SA into SA_q and reads ‖SA_q − SA‖_F² back to the
// host (synchronises the stream) for the guard of quantised solves.
static int quantize_handle(mihs_sketch_t sk, cudaStream_t s) {
  int rc = launch_quantize_sa(sk->SA, sk->m, sk->d, sk->dp, sk->sa_prec, sk->SAq, sk->ldq, sk->sa_scales, s);
  if (rc) return rc;
  rc = launch_quant_error(sk->SA, sk->m, sk->d, sk->dp, sk->sa_prec, sk->SAq, sk->ldq, sk->sa_scales,
                          sk->sa_qerr_dev, sk->sa_qerr_dev + kQuantErrBlocks, s);
  if (rc) return rc;
  MIHS_CUDA_TRY(cudaMemcpyAsync(&sk->sa_qerr, sk->sa_qerr_dev + kQuantErrBlocks, sizeof(double),
                                cudaMemcpyDeviceToHost, s));
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  return MIHS_OK;
}

// Solves on a quantised SA are refused where the rounding E = SA_q − SA can
// no longer be trusted to leave a preconditioner: the sketched Hessian stays
// within a factor 2 of the exact one (SA_qᵀSA_q + λI ⪰ ½(SAᵀSA + λI)) when
// ‖E‖₂² ≤ λ/2, and beyond that the spectrum of (SA_qᵀSA_q + λI)⁻¹(AᵀA + λI)
// can leave the region where the heavy ball of Theorem 1 converges (fp8 e4m3
// at κ(AᵀA + λI) ≈ 1e6 puts its largest eigenvalue near 8, past the
// 2(1 + β)/α ≈ 4.4 of β = 1/4).
static int check_quantised(const mihs_sketch_s* sk, double lambda, const char* who) {
  if (sk->sa_prec == MIHS_SA_FP32 || sk->SAq == nullptr) return MIHS_OK;
  const double est = quant_spectral_estimate(sk->sa_qerr, sk->m, sk->d);
  if (est <= 0.5 * lambda) return MIHS_OK;
  set_error("%s: SA stored in %s has an estimated rounding ||SA_q - SA||_2^2 = %.3g = %.3g lambda > lambda/2 "
            "(lambda = %g): at this lambda the quantised sketch no longer preconditions Algorithm 1; store SA "
            "in a wider format (bf16 or fp32)", who, sk->sa_prec == MIHS_SA_BF16 ? "bf16" : "fp8 e4m3", est,
            est / lambda, lambda);
  return MIHS_ERR_UNSUPPORTED;
}

int mihs_resketch(mihs_sketch_t sk, const float* A, int64_t lda, uint64_t seed, void* stream) {
  set_error("");
  MIHS_ARG(sk != nullptr, "mihs_resketch: null handle");
  int rc = check_matrix(A, sk->n, sk->d, lda, "mihs_resketch");
  if (rc) return rc;
  sk->seed = seed;
  // A handle whose SA is stored quantised forms a Gaussian S·A from operands
  // of that precision too (bf16, or fp8 e4m3 with A scaled; fp32
  // accumulation): the sketch only preconditions.
  if (sk->family == MIHS_GAUSSIAN && sk->sa_prec == MIHS_SA_BF16)
    rc = mihs_sketch_gaussian_bf16(A, sk->n, sk->d, lda, sk->m, seed, sk->SA, sk->dp, stream);
  else if (sk->family == MIHS_GAUSSIAN && sk->sa_prec == MIHS_SA_FP8E4M3)
    rc = mihs_sketch_gaussian_fp8(A, sk->n, sk->d, lda, sk->m, seed, sk->SA, sk->dp, stream);
  else
    rc = mihs_sketch_apply(A, sk->n, sk->d, lda, sk->family, sk->m, seed, sk->SA, sk->dp, stream);
  if (rc || sk->sa_prec == MIHS_SA_FP32) return rc;
  return quantize_handle(sk, static_cast<cudaStream_t>(stream));
}

int mihs_sketch_set_precision(mihs_sketch_t sk, int sa_prec, void* stream) {
  set_error("");
  MIHS_ARG(sk != nullptr, "mihs_sketch_set_precision: null handle");
  MIHS_ARG(sa_prec == MIHS_SA_FP32 || sa_prec == MIHS_SA_BF16 || sa_prec == MIHS_SA_FP8E4M3,
           "mihs_sketch_set_precision: unknown precision %d", sa_prec);
  if (sa_prec != MIHS_SA_FP32 && sk->SAq == nullptr) {
    sk->ldq = sa_quant_ld(sk->d);
    const size_t qbytes = round_up((int64_t)sk->m * sk->ldq, 256);  // ≤ 1 byte/element more than fp8 needs
    const size_t sbytes = round_up(sizeof(float) * (size_t)sa_scale_count(sk->m, sk->d), 256);
    const size_t bytes = 2 * qbytes + sbytes + sizeof(double) * (kQuantErrBlocks + 1);
    char* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      set_error("mihs_sketch_set_precision: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
    }
    sk->SAq = p;
    sk->sa_scales = reinterpret_cast<float*>(p + 2 * qbytes);
    sk->sa_qerr_dev = reinterpret_cast<double*>(p + 2 * qbytes + sbytes);
  }
  sk->sa_prec = sa_prec;
  if (sa_prec == MIHS_SA_FP32) return MIHS_OK;
  return quantize_handle(sk, static_cast<cudaStream_t>(stream));
}

int mihs_sketch_set_aab(mihs_sketch_t sk, int form, int grid_blocks) {
  set_error("");
  MIHS_ARG(sk != nullptr, "mihs_sketch_set_aab: null handle");
  MIHS_ARG(form == MIHS_AAB_AUTO || form == MIHS_AAB_CLUSTER || form == MIHS_AAB_GRID,
           "mihs_sketch_set_aab: unknown form %d", form);
  MIHS_ARG(grid_blocks >= 0, "mihs_sketch_set_aab: grid_blocks %d < 0", grid_blocks);
  sk->aab_form = form;
  sk->aab_grid_blocks = form == MIHS_AAB_GRID ? grid_blocks : 0;
  return MIHS_OK;
}

int mihs_sketch_info(mihs_sketch_t sk, const float** SA, int64_t* m, int64_t* d, int64_t* n,
                     int* family) {
  MIHS_ARG(sk != nullptr, "mihs_sketch_info: null handle");
  if (SA) *SA = sk->SA;
  if (m) *m = sk->m;
  if (d) *d = sk->d;
  if (n) *n = sk->n;
  if (family) *family = sk->family;
  return MIHS_OK;
}

int mihs_solve_history(mihs_sketch_t sk, float* host_out, int cap, int* count) {
  set_error("");
  MIHS_ARG(sk != nullptr && host_out != nullptr && count != nullptr && cap >= 0,
           "mihs_solve_history: bad argument");
  MIHS_CUDA_TRY(cudaDeviceSynchronize());
  SolveCtl c;
  MIHS_CUDA_TRY(cudaMemcpy(&c, sk->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost));
  int k = c.outer + 1;
  if (k > kHistCap) k = kHistCap;
  if (k > cap) k = cap;
  if (k > 0) MIHS_CUDA_TRY(cudaMemcpy(host_out, sk->hist, sizeof(float) * (size_t)k, cudaMemcpyDeviceToHost));
  for (int i = 0; i < k; ++i) host_out[i] = c.gnorm0 > 0.f ? host_out[i] / c.gnorm0 : 0.f;
  *count = k;
  return MIHS_OK;
}

int mihs_sketch_copy(mihs_sketch_t sk, float* dst, int64_t ldd, void* stream) {
  set_error("");
  MIHS_ARG(sk != nullptr && dst != nullptr, "mihs_sketch_copy: null argument");
  MIHS_ARG(ldd >= sk->d, "mihs_sketch_copy: ldd < d");
  MIHS_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(float) * (size_t)ldd, sk->SA, sizeof(float) * (size_t)sk->dp,
                                  sizeof(float) * (size_t)sk->d, (size_t)sk->m, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream)));
  return MIHS_OK;
}

int mihs_sketch_destroy(mihs_sketch_t sk) {
  if (sk == nullptr) return MIHS_OK;
  cudaDeviceSynchronize();
  for (auto& kind : sk->slots)
    for (auto& gs : kind) drop_graph(gs);
  free_retired(sk);
  if (sk->path_exec) cudaGraphExecDestroy(sk->path_exec);
  if (sk->path_graph) cudaGraphDestroy(sk->path_graph);
  if (sk->cap) cudaStreamDestroy(sk->cap);
  if (sk->dd_partials) cudaFree(sk->dd_partials);
  if (sk->aab_grid_ws) cudaFree(sk->aab_grid_ws);
  if (sk->path_partials) cudaFree(sk->path_partials);
  if (sk->SAq) cudaFree(sk->SAq);
  if (sk->path_ctl_host) cudaFreeHost(sk->path_ctl_host);
  if (sk->ref_x64) cudaFree(sk->ref_x64);
  if (sk->ref_ctl_host) cudaFreeHost(sk->ref_ctl_host);
  cudaFreeHost(sk->ctl_host);
  cudaFree(sk->SA);
  delete sk;
  return MIHS_OK;
}

// Algorithm 1 on H x = Aᵀb + rhs (rhs null for the ridge problem itself; b
// null and rhs = ḡ for the adjoint solve H v = ḡ).
static int solve_impl(mihs_sketch_t sk, const float* A, int64_t lda, const float* b, double lambda,
                      const mihs_opts* opts, void* xv, bool refined, mihs_info* info, void* stream,
                      const float* rhs = nullptr) {
  MIHS_ARG(sk != nullptr && opts != nullptr, "mihs_solve: null handle or opts");
  int rc = check_matrix(A, sk->n, sk->d, lda, "mihs_solve");
  if (rc) return rc;
  MIHS_ARG((b != nullptr || rhs != nullptr) && xv != nullptr, "mihs_solve: null b or x");
  MIHS_ARG(lambda > 0.0 && lambda <= (double)FLT_MAX, "mihs_solve: lambda must be in (0, FLT_MAX]");
  MIHS_ARG(opts->sd < (double)sk->m, "mihs_solve: sd=%g must be < m=%lld", opts->sd, (long long)sk->m);
  MIHS_ARG(opts->max_outer >= 0 && opts->max_outer < (1 << 24), "mihs_solve: bad max_outer");
  MIHS_ARG(opts->eps_sub >= 0.0, "mihs_solve: eps_sub must be >= 0");
  rc = check_quantised(sk, lambda, "mihs_solve");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = sk->n, d = sk->d;
  if (refined && sk->dd_partials == nullptr) {
    sk->P_dd = apass_dd_num_partials(n, d);
    char* p = nullptr;
    const size_t bytes = sizeof(float2) * (size_t)sk->P_dd * sk->dp + 3 * sizeof(double) * (size_t)sk->dp +
                         4 * sizeof(float) * (size_t)sk->dp;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      set_error("mihs_solve_refined: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
    }
    sk->dd_partials = reinterpret_cast<float2*>(p);
    sk->x_prev64 = reinterpret_cast<double*>(p + sizeof(float2) * (size_t)sk->P_dd * sk->dp);
    sk->gref64 = sk->x_prev64 + sk->dp;
    sk->xref64 = sk->gref64 + sk->dp;
    sk->x32_shadow = reinterpret_cast<float*>(sk->xref64 + sk->dp);
    sk->bw32 = sk->x32_shadow + sk->dp;
    sk->delta32 = sk->bw32 + 2 * sk->dp;
  }
  // sd ≤ 0: estimate it from SA (Algorithm 4 with the paper's T = 2,
  // ε_tr = 0.5); an over-estimate only slows the rate (Remark after
  // Corollary 3), so the estimate is capped below m.
  double sd = opts->sd;
  if (!(sd > 0.0)) {
    rc = estimate_sd(sk->SA, sk->m, sk->d, sk->dp, lambda, 2, 0.5, sk->seed ^ 0x4855544348ull, &sd, s);
    if (rc) return rc;
    const double cap = 0.95 * (double)sk->m;
    if (!(sd > 0.0)) sd = 1.0;
    if (sd > cap) sd = cap;
    sk->last_sd = sd;
  }
  // Corollary 3: β = sd/m, α = (1 − β)².
  const double beta = sd / (double)sk->m;
  const double alpha = (1.0 - beta) * (1.0 - beta);
  const size_t xbytes = (refined ? sizeof(double) : sizeof(float)) * (size_t)d;

  // Refinement solves start with plain fp32 gradients and switch to the
  // compensated pass once the relative residual is below 1e-7 or stops
  // improving (the fp32 floor); plain solves never switch.
  const float switch_tol = refined ? 1e-7f : 0.f;
  // Refinement corrections (fp32 passes between compensated refreshes) are on
  // unless MIHS_REFINE_CORR=0.
  static const bool corr_on = [] {
    const char* e = std::getenv("MIHS_REFINE_CORR");
    return e == nullptr || std::strcmp(e, "0") != 0;
  }();
  ctl_init_kernel<<<1, 1, 0, s>>>(sk->ctl, opts->max_outer, (float)opts->tol, refined ? 0 : 1, switch_tol,
                                  refined && corr_on ? 1 : 0);
  MIHS_CHECK_LAUNCH();
  count_launch();
  if (opts->warm_start) {
    // ‖g(0)‖ (= ‖Aᵀb‖ for the ridge problem) for the relative residual.
    rc = launch_apass_partial(A, n, d, lda, b, nullptr, sk->partials, nullptr, s);
    if (rc) return rc;
    rc = launch_apass_finalize(sk->partials, sk->P, d, nullptr, 0.f, sk->g, nullptr, s, -1, rhs);
    if (rc) return rc;
    ctl_set_gnorm0_kernel<<<1, 256, 0, s>>>(sk->ctl, sk->g, (int)d);
    MIHS_CHECK_LAUNCH();
    count_launch();
  } else {
    MIHS_CUDA_TRY(cudaMemsetAsync(xv, 0, xbytes, s));
  }
  MIHS_CUDA_TRY(cudaMemcpyAsync(refined ? (void*)sk->x_prev64 : (void*)sk->x_prev, xv, xbytes,
                                cudaMemcpyDeviceToDevice, s));
  if (refined) {
    f64_to_f32_kernel<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(static_cast<const double*>(xv), sk->x32_shadow,
                                                                 (int)d);
    MIHS_CHECK_LAUNCH();
    count_launch();
  }

  AabLaunch a = {};
  set_sa(a, sk);
  a.m = (int)sk->m;
  a.d = (int)d;
  a.g = sk->g;
  a.lambda = (float)lambda;
  a.eps = (float)opts->eps_sub;
  a.max_passes = cap_passes(sk->m, d, opts->max_inner);
  if (refined) {
    a.x64 = static_cast<double*>(xv);
    a.x_prev64 = sk->x_prev64;
    a.x32_shadow = sk->x32_shadow;
    a.alpha64 = alpha;
    a.beta64 = beta;
  } else {
    a.alpha = (float)alpha;
    a.beta = (float)beta;
    a.x = static_cast<float*>(xv);
    a.x_prev = sk->x_prev;
  }
  a.ctl = sk->ctl;
  a.hist = sk->hist;
  rc = use_grid_ws(sk, a, s);
  if (rc) return rc;
  // Algorithm 1: up to max_outer momentum steps, each after a gradient.
  const mihs_sketch_s::Key key = {A,         lda,         b,          xv,           lambda,
                                  alpha,     beta,        a.eps,      a.max_passes, rhs,
                                  sk->sa_prec, sk->aab_form, sk->aab_grid_blocks};
  bool graph_ran = false;
  const int kind = (refined ? 1 : 0) + (rhs != nullptr ? 2 : 0);
  if (!timing_on() && !sk->graph_failed[kind] && std::getenv("MIHS_NO_GRAPH") == nullptr) {
    mihs_sketch_s::GraphSlot* ways = sk->slots[kind];
    mihs_sketch_s::GraphSlot* gs = nullptr;
    for (int w = 0; w < mihs_sketch_s::kGraphWays && gs == nullptr; ++w)
      if (ways[w].exec && ways[w].key == key) gs = &ways[w];
    if (gs == nullptr) {  // an empty way, else the least recently used one
      gs = &ways[0];
      for (int w = 1; w < mihs_sketch_s::kGraphWays; ++w)
        if (ways[w].used < gs->used) gs = &ways[w];
      retire_graph(sk, gs->exec, gs->graph);
      gs->used = 0;
      if (build_graph(sk, key, a, refined, *gs) != MIHS_OK) {
        retire_graph(sk, gs->exec, gs->graph);
        gs->used = 0;
        sk->graph_failed[kind] = true;  // keep the message; use host-driven steps from now on
        cudaGetLastError();
      }
    }
    if (gs->exec) {
      MIHS_CUDA_TRY(cudaGraphLaunch(gs->exec, s));
      gs->used = ++sk->graph_tick;
      graph_ran = true;
    }
  }
  if (!graph_ran) {
    // Host-driven steps; the kernels return at once after the stop test has
    // fired (ctl->done).  With per-kernel timing on, the control block is
    // read back after every step so that only working launches are timed.
    const bool poll = timing_on();
    int phase = poll && refined ? 0 : -1;  // the gate of the next step, when the host knows it
    for (int it = 0; it <= opts->max_outer; ++it) {
      rc = launch_step(sk, key, a, refined, s, phase);
      if (rc) return rc;
      if (poll) {
        MIHS_CUDA_TRY(cudaMemcpyAsync(sk->ctl_host, sk->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
        MIHS_CUDA_TRY(cudaStreamSynchronize(s));
        if (sk->ctl_host->done) break;
        if (refined) phase = ctl_gate(sk->ctl_host);
      }
    }
  }
  if (info == nullptr) return MIHS_OK;
  MIHS_CUDA_TRY(cudaMemcpyAsync(sk->ctl_host, sk->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  const SolveCtl& c = *sk->ctl_host;
  info->outer_iters = c.outer;
  info->inner_iters_total = c.inner_total;
  info->rel_resid = c.gnorm0 > 0.f ? (double)c.gnorm / (double)c.gnorm0 : 0.0;
  info->status = c.done ? c.status : MIHS_NOT_CONVERGED;
  if (graph_ran) count_launch((refined ? 8ull : 3ull) * (uint64_t)(c.outer + 1));
  return info->status;
}

int mihs_solve(mihs_sketch_t sk, const float* A, int64_t lda, const float* b, double lambda,
               const mihs_opts* opts, float* x, mihs_info* info, void* stream) {
  set_error("");
  return solve_impl(sk, A, lda, b, lambda, opts, x, false, info, stream);
}

int mihs_solve_refined(mihs_sketch_t sk, const float* A, int64_t lda, const float* b, double lambda,
                       const mihs_opts* opts, double* x, mihs_info* info, void* stream) {
  set_error("");
  return solve_impl(sk, A, lda, b, lambda, opts, x, true, info, stream);
}

int mihs_backward_grads(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const float* x,
                        const float* v, float* dA, int64_t ldda, float* db, double* dlambda, void* stream) {
  set_error("");
  int rc = check_matrix(A, n, d, lda, "mihs_backward_grads");
  if (rc) return rc;
  MIHS_ARG(x != nullptr && v != nullptr, "mihs_backward_grads: null x or v");
  MIHS_ARG(dA == nullptr || (b != nullptr && ldda >= d), "mihs_backward_grads: dA needs b and ldda >= d");
  return launch_backward_grads(A, n, d, lda, b, x, v, dA, ldda, db, dlambda, static_cast<cudaStream_t>(stream));
}

int mihs_backward(mihs_sketch_t sk, const float* A, int64_t lda, const float* b, double lambda, const float* x,
                  const float* gx, const mihs_opts* opts, float* v, float* dA, int64_t ldda, float* db,
                  double* dlambda, mihs_info* info, void* stream) {
  set_error("");
  MIHS_ARG(sk != nullptr, "mihs_backward: null handle");
  MIHS_ARG(gx != nullptr && x != nullptr && v != nullptr, "mihs_backward: null gx, x or v");
  MIHS_ARG(dA == nullptr || (b != nullptr && ldda >= sk->d), "mihs_backward: dA needs b and ldda >= d");
  const int st = solve_impl(sk, A, lda, nullptr, lambda, opts, v, false, info, stream, gx);
  if (st < 0) return st;
  const int rc = launch_backward_grads(A, sk->n, sk->d, lda, b, x, v, dA, ldda, db, dlambda,
                                       static_cast<cudaStream_t>(stream));
  return rc ? rc : st;
}

int mihs_backward_refined(mihs_sketch_t sk, const float* A, int64_t lda, const float* b, double lambda,
                          const double* x, const float* gx, const mihs_opts* opts, double* v, float* dA,
                          int64_t ldda, float* db, double* dlambda, mihs_info* info, void* stream) {
  set_error("");
  MIHS_ARG(sk != nullptr, "mihs_backward_refined: null handle");
  MIHS_ARG(gx != nullptr && x != nullptr && v != nullptr, "mihs_backward_refined: null gx, x or v");
  MIHS_ARG(dA == nullptr || (b != nullptr && ldda >= sk->d), "mihs_backward_refined: dA needs b and ldda >= d");
  const int st = solve_impl(sk, A, lda, nullptr, lambda, opts, v, true, info, stream, gx);
  if (st < 0) return st;
  // The gradients are fp32 outputs: the pass takes x and v rounded to fp32.
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int d = (int)sk->d;
  float* x32 = sk->bw32;
  float* v32 = sk->bw32 + sk->dp;
  f64_to_f32_kernel<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(x, x32, d);
  MIHS_CHECK_LAUNCH();
  f64_to_f32_kernel<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(v, v32, d);
  MIHS_CHECK_LAUNCH();
  count_launch(2);
  const int rc = launch_backward_grads(A, sk->n, sk->d, lda, b, x32, v32, dA, ldda, db, dlambda, s);
  return rc ? rc : st;
}

// Enqueues the λ-path solves of one problem (groups of ≤ 16 λ), copying each
// group's control blocks into the handle's pinned host array when
// want_info.  Does not synchronise unless an sd has to be estimated.
static int path_enqueue(mihs_sketch_t sk, const float* A, int64_t lda, const float* b, int nlambda,
                        const double* lambdas, const double* sds, const mihs_opts* opts, float* X, int64_t ldx,
                        bool want_info, cudaStream_t s) {
  MIHS_ARG(sk != nullptr && opts != nullptr && lambdas != nullptr && X != nullptr && b != nullptr,
           "mihs_solve_path: null argument");
  int rc = check_matrix(A, sk->n, sk->d, lda, "mihs_solve_path");
  if (rc) return rc;
  const int64_t n = sk->n, d = sk->d;
  MIHS_ARG(nlambda >= 1, "mihs_solve_path: nlambda must be >= 1");
  MIHS_ARG(ldx >= d, "mihs_solve_path: ldx=%lld < d", (long long)ldx);
  MIHS_ARG(opts->max_outer >= 0 && opts->max_outer < (1 << 24), "mihs_solve_path: bad max_outer");
  MIHS_ARG(opts->eps_sub >= 0.0, "mihs_solve_path: eps_sub must be >= 0");
  for (int l = 0; l < nlambda; ++l) {
    MIHS_ARG(lambdas[l] > 0.0 && lambdas[l] <= (double)FLT_MAX, "mihs_solve_path: lambda[%d] must be in (0, FLT_MAX]", l);
    if (sds != nullptr)
      MIHS_ARG(sds[l] < (double)sk->m, "mihs_solve_path: sd[%d]=%g must be < m", l, sds[l]);
    rc = check_quantised(sk, lambdas[l], "mihs_solve_path");
    if (rc) return rc;
  }
  if (d > apass_path_max_d()) {
    set_error("mihs_solve_path: d=%lld > %d is not supported", (long long)d, apass_path_max_d());
    return MIHS_ERR_UNSUPPORTED;
  }
  if (sk->path_partials == nullptr) {
    sk->P_path = apass_path_num_partials(n);
    const size_t fl = (size_t)sk->P_path * 16 * sk->dp + 2 * 16 * (size_t)sk->dp + aab_path_ws_floats((int)sk->dp);
    const size_t bytes = fl * sizeof(float) + 16 * sizeof(SolveCtl) + 4 * sizeof(int);
    char* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      set_error("mihs_solve_path: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
    }
    sk->path_partials = reinterpret_cast<float*>(p);
    sk->path_g = sk->path_partials + (size_t)sk->P_path * 16 * sk->dp;
    sk->path_xprev = sk->path_g + 16 * (size_t)sk->dp;
    sk->path_aab_ws = sk->path_xprev + 16 * (size_t)sk->dp;
    sk->path_ctl = reinterpret_cast<SolveCtl*>(p + fl * sizeof(float));
    sk->path_cnt = reinterpret_cast<int*>(sk->path_ctl + 16);
  }
  if (want_info) {
    if (sk->path_ctl_host != nullptr && sk->path_ctl_cap < nlambda) {
      cudaFreeHost(sk->path_ctl_host);
      sk->path_ctl_host = nullptr;
    }
    if (sk->path_ctl_host == nullptr) {
      MIHS_CUDA_TRY(cudaMallocHost(&sk->path_ctl_host, sizeof(SolveCtl) * (size_t)nlambda));
      sk->path_ctl_cap = nlambda;
    }
  }
  for (int l0 = 0; l0 < nlambda; l0 += 16) {
    const int nl = nlambda - l0 < 16 ? nlambda - l0 : 16;
    PathScalars ps = {};
    ps.nl = nl;
    for (int l = 0; l < nl; ++l) {
      const double lam = lambdas[l0 + l];
      double sd = sds != nullptr ? sds[l0 + l] : 0.0;
      if (!(sd > 0.0)) {  // Algorithm 4 on SA (T = 2, ε_tr = 0.5), capped below m
        rc = estimate_sd(sk->SA, sk->m, sk->d, sk->dp, lam, 2, 0.5, sk->seed ^ 0x4855544348ull, &sd, s);
        if (rc) return rc;
        if (!(sd > 0.0)) sd = 1.0;
        if (sd > 0.95 * (double)sk->m) sd = 0.95 * (double)sk->m;
      }
      const double beta = sd / (double)sk->m;  // Corollary 3
      ps.lam[l] = (float)lam;
      ps.beta[l] = (float)beta;
      ps.alpha[l] = (float)((1.0 - beta) * (1.0 - beta));
    }
    float* Xg = X + (size_t)l0 * ldx;
    MIHS_CUDA_TRY(cudaMemsetAsync(sk->path_aab_ws, 0, 256, s));  // the grid form's barrier word
    path_init_kernel<<<1, 32, 0, s>>>(sk->path_ctl, sk->path_cnt, nl, opts->max_outer, (float)opts->tol);
    MIHS_CHECK_LAUNCH();
    count_launch();
    if (opts->warm_start) {
      rc = launch_apass_partial(A, n, d, lda, b, nullptr, sk->partials, nullptr, s);
      if (!rc) rc = launch_apass_finalize(sk->partials, sk->P, d, nullptr, 0.f, sk->g, nullptr, s);
      if (rc) return rc;
      path_set_gnorm0_kernel<<<1, 256, 0, s>>>(sk->path_ctl, nl, sk->g, (int)d);
      MIHS_CHECK_LAUNCH();
      count_launch();
    } else {
      MIHS_CUDA_TRY(cudaMemset2DAsync(Xg, (size_t)ldx * sizeof(float), 0, (size_t)d * sizeof(float), nl, s));
    }
    MIHS_CUDA_TRY(cudaMemcpy2DAsync(sk->path_xprev, (size_t)sk->dp * sizeof(float), Xg, (size_t)ldx * sizeof(float),
                                    (size_t)d * sizeof(float), nl, cudaMemcpyDeviceToDevice, s));
    AabLaunch a = {};
    set_sa(a, sk);
    a.m = (int)sk->m;
    a.d = (int)d;
    a.g = sk->path_g;
    a.eps = (float)opts->eps_sub;
    a.max_passes = cap_passes(sk->m, d, opts->max_inner);
    a.x = Xg;
    a.x_prev = sk->path_xprev;
    a.ctl = sk->path_ctl;
    a.path = 1;
    a.ps = ps;
    a.path_ldg = sk->dp;
    a.path_ldx = ldx;
    a.path_ndone = sk->path_cnt;
    a.path_all_done = sk->path_cnt + 1;
    const mihs_sketch_s::PathKey key = {A, lda, b, Xg, ldx, ps, a.eps, a.max_passes, sk->sa_prec};
    bool graph_ran = false;
    if (!timing_on() && !sk->path_graph_failed && std::getenv("MIHS_NO_GRAPH") == nullptr) {
      if (!(sk->path_exec && sk->path_key == key)) {
        retire_graph(sk, sk->path_exec, sk->path_graph);
        const int brc = build_while_graph(sk, (int)sk->m, (int)d, sk->path_graph, sk->path_exec,
                                          [&](unsigned long long cond, cudaStream_t cs) {
                                            AabLaunch b2 = a;
                                            b2.cond = cond;
                                            return launch_path_step(sk, key, b2, cs);
                                          });
        if (brc == MIHS_OK) {
          sk->path_key = key;
        } else {
          retire_graph(sk, sk->path_exec, sk->path_graph);
          sk->path_graph_failed = true;  // host-driven steps from now on
          cudaGetLastError();
        }
      }
      if (sk->path_exec) {
        MIHS_CUDA_TRY(cudaGraphLaunch(sk->path_exec, s));
        graph_ran = true;
      }
    }
    if (!graph_ran) {
      const bool poll = timing_on();
      for (int it = 0; it <= opts->max_outer; ++it) {
        rc = launch_path_step(sk, key, a, s);
        if (rc) return rc;
        if (poll) {
          int flag = 0;
          MIHS_CUDA_TRY(cudaMemcpyAsync(&flag, sk->path_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
          MIHS_CUDA_TRY(cudaStreamSynchronize(s));
          if (flag) break;
        }
      }
    }
    if (want_info)
      MIHS_CUDA_TRY(cudaMemcpyAsync(sk->path_ctl_host + l0, sk->path_ctl, sizeof(SolveCtl) * (size_t)nl,
                                    cudaMemcpyDeviceToHost, s));
  }
  return MIHS_OK;
}

// Fills infos[0..nlambda) from the handle's host copies (after a sync) and
// returns the worst status.
static int path_infos(mihs_sketch_t sk, int nlambda, mihs_info* infos) {
  int worst = MIHS_OK;
  for (int l = 0; l < nlambda; ++l) {
    const SolveCtl& c = sk->path_ctl_host[l];
    infos[l].outer_iters = c.outer;
    infos[l].inner_iters_total = c.inner_total;
    infos[l].rel_resid = c.gnorm0 > 0.f ? (double)c.gnorm / (double)c.gnorm0 : 0.0;
    infos[l].status = c.done ? c.status : MIHS_NOT_CONVERGED;
    if (infos[l].status < 0) worst = infos[l].status;
    else if (worst == MIHS_OK && infos[l].status != MIHS_OK) worst = infos[l].status;
  }
  return worst;
}

int mihs_gradient_path(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, int nl,
                       const double* lambdas, const float* X, int64_t ldx, float* G, int64_t ldg, void* stream) {
  set_error("");
  int rc = check_matrix(A, n, d, lda, "mihs_gradient_path");
  if (rc) return rc;
  MIHS_ARG(b != nullptr && X != nullptr && G != nullptr && lambdas != nullptr, "mihs_gradient_path: null argument");
  MIHS_ARG(nl >= 1 && nl <= 16, "mihs_gradient_path: nl=%d must be in 1..16", nl);
  MIHS_ARG(ldx >= d && ldg >= d, "mihs_gradient_path: ldx and ldg must be >= d");
  if (d > apass_path_max_d()) {
    set_error("mihs_gradient_path: d=%lld > %d is not supported", (long long)d, apass_path_max_d());
    return MIHS_ERR_UNSUPPORTED;
  }
  PathScalars ps = {};
  ps.nl = nl;
  for (int l = 0; l < nl; ++l) {
    MIHS_ARG(lambdas[l] >= 0.0 && lambdas[l] <= (double)FLT_MAX, "mihs_gradient_path: lambda[%d] must be in [0, FLT_MAX]", l);
    ps.lam[l] = (float)lambdas[l];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = apass_path_num_partials(n);
  StreamScratch scratch;
  rc = scratch.alloc(sizeof(float) * (size_t)P * 16 * apass_dpad(d), s);
  if (rc) return rc;
  float* part = static_cast<float*>(scratch.p);
  rc = launch_apass_path(A, n, d, lda, b, X, ldx, nl, part, nullptr, s);
  if (rc) return rc;
  return launch_apass_path_finalize(part, P, d, X, ldx, ps, G, ldg, nullptr, s);
}

int mihs_solve_path(mihs_sketch_t sk, const float* A, int64_t lda, const float* b, int nlambda,
                    const double* lambdas, const double* sds, const mihs_opts* opts, float* X, int64_t ldx,
                    mihs_info* infos, void* stream) {
  set_error("");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = path_enqueue(sk, A, lda, b, nlambda, lambdas, sds, opts, X, ldx, infos != nullptr, s);
  if (rc || infos == nullptr) return rc;
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  return path_infos(sk, nlambda, infos);
}

// Internal streams of the batched entry points (per device, created on first
// use): batch_stream_count() streams and one more event than streams, the
// last one the fork event.  Problems whose solves use the cooperative grid
// form of AAb_Solver share stream 0; the others are spread over the rest, so
// that the small sketches' cluster kernels (1–8 SMs each) fill the GPU.
static int batch_stream_count() {
  static const int n = [] {
    int v = 8;
    if (const char* e = std::getenv("MIHS_BATCH_STREAMS")) v = std::atoi(e);
    return v < 2 ? 2 : (v > 32 ? 32 : v);
  }();
  return n;
}
static int batch_streams(std::vector<cudaStream_t>& st, std::vector<cudaEvent_t>& ev) {
  const int kBatchStreams = batch_stream_count();
  static std::mutex mu;
  static std::vector<std::vector<cudaStream_t>> pool;  // per device
  static std::vector<std::vector<cudaEvent_t>> evs;
  int dev = 0;
  MIHS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)pool.size() <= dev) {
    pool.resize(dev + 1);
    evs.resize(dev + 1);
  }
  if (pool[dev].empty()) {
    for (int k = 0; k < kBatchStreams; ++k) {
      cudaStream_t t;
      cudaEvent_t e;
      MIHS_CUDA_TRY(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
      MIHS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      pool[dev].push_back(t);
      evs[dev].push_back(e);
    }
    cudaEvent_t e;
    MIHS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    evs[dev].push_back(e);  // the fork event
  }
  st = pool[dev];
  ev = evs[dev];
  return MIHS_OK;
}

int mihs_solve_batched(int nprob, const mihs_problem* probs, int nlambda, const double* lambdas,
                       const double* sds, const mihs_opts* opts, mihs_info* infos, void* stream) {
  set_error("");
  MIHS_ARG(nprob >= 0 && (nprob == 0 || probs != nullptr), "mihs_solve_batched: bad problem array");
  for (int i = 0; i < nprob; ++i)
    for (int j = 0; j < i; ++j)
      MIHS_ARG(probs[i].sk != probs[j].sk, "mihs_solve_batched: problems %d and %d share a handle", j, i);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Independent problems run on internal streams forked from and joined back
  // into the caller's stream.  Problems whose path steps use the cooperative
  // grid form all go to stream 0 (two such grids must never wait for each
  // other's blocks, so they never run concurrently); the others are spread
  // over the other streams (or all of them when no problem uses the grid form).
  const int kStreams = batch_stream_count();
  const int nstreams = kStreams;
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> ev;
  int rc0 = batch_streams(st, ev);
  if (rc0) return rc0;
  MIHS_CUDA_TRY(cudaEventRecord(ev[kStreams], s));
  for (int k = 0; k < nstreams; ++k) MIHS_CUDA_TRY(cudaStreamWaitEvent(st[k], ev[kStreams], 0));
  int rc = MIHS_OK;
  bool any_grid = false;
  for (int i = 0; i < nprob; ++i) any_grid = any_grid || path_uses_grid(probs[i].sk);
  int next = 0;
  for (int i = 0; i < nprob && rc == MIHS_OK; ++i) {
    const mihs_problem& q = probs[i];
    int k;
    if (path_uses_grid(q.sk)) {
      k = 0;
    } else if (any_grid) {
      k = 1 + next % (nstreams - 1);
      ++next;
    } else {
      k = next % nstreams;
      ++next;
    }
    rc = path_enqueue(q.sk, q.A, q.lda, q.b, nlambda, lambdas, sds != nullptr ? sds + (size_t)i * nlambda : nullptr,
                      opts, q.X, q.ldx, infos != nullptr, st[k]);
    if (rc) set_error("mihs_solve_batched: problem %d: %s", i, mihs_last_error());
  }
  for (int k = 0; k < nstreams; ++k) {
    MIHS_CUDA_TRY(cudaEventRecord(ev[k], st[k]));
    MIHS_CUDA_TRY(cudaStreamWaitEvent(s, ev[k], 0));
  }
  if (rc || infos == nullptr) return rc;
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  int worst = MIHS_OK;
  for (int i = 0; i < nprob; ++i) {
    const int w = path_infos(probs[i].sk, nlambda, infos + (size_t)i * nlambda);
    if (w < 0) worst = w;
    else if (worst == MIHS_OK && w != MIHS_OK) worst = w;
  }
  return worst;
}

int mihs_refine_batched(int nprob, const mihs_problem* probs, int nlambda, const double* lambdas,
                        const double* sds, const double* tols, const mihs_opts* opts, mihs_info* infos,
                        void* stream) {
  set_error("");
  MIHS_ARG(nprob >= 0 && (nprob == 0 || probs != nullptr), "mihs_refine_batched: bad problem array");
  MIHS_ARG(nlambda >= 1 && lambdas != nullptr && tols != nullptr && opts != nullptr,
           "mihs_refine_batched: null lambdas, tols or opts, or nlambda < 1");
  for (int i = 0; i < nprob; ++i) {
    MIHS_ARG(probs[i].sk != nullptr && probs[i].X != nullptr && probs[i].b != nullptr,
             "mihs_refine_batched: problem %d: null handle, b or X", i);
    MIHS_ARG(probs[i].ldx >= probs[i].sk->d, "mihs_refine_batched: problem %d: ldx < d", i);
    for (int j = 0; j < i; ++j)
      MIHS_ARG(probs[i].sk != probs[j].sk, "mihs_refine_batched: problems %d and %d share a handle", j, i);
  }
  for (int l = 0; l < nlambda; ++l) {
    if (!(tols[l] > 0.0)) continue;
    MIHS_ARG(lambdas[l] > 0.0 && lambdas[l] <= (double)FLT_MAX,
             "mihs_refine_batched: lambda[%d] must be in (0, FLT_MAX]", l);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Workspace first (cudaMalloc synchronises the device): the fp64 iterate
  // and, with infos, pinned copies of the control blocks.
  for (int i = 0; i < nprob; ++i) {
    mihs_sketch_s* sk = probs[i].sk;
    if (sk->ref_x64 == nullptr) {
      cudaError_t e = cudaMalloc(&sk->ref_x64, sizeof(double) * (size_t)sk->dp);
      if (e != cudaSuccess) {
        sk->ref_x64 = nullptr;
        set_error("mihs_refine_batched: cudaMalloc: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
      }
    }
    if (infos != nullptr && sk->ref_ctl_cap < nlambda) {
      if (sk->ref_ctl_host) cudaFreeHost(sk->ref_ctl_host);
      sk->ref_ctl_host = nullptr;
      sk->ref_ctl_cap = 0;
      MIHS_CUDA_TRY(cudaMallocHost(&sk->ref_ctl_host, sizeof(SolveCtl) * (size_t)nlambda));
      sk->ref_ctl_cap = nlambda;
    }
  }
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> ev;
  int rc = batch_streams(st, ev);
  if (rc) return rc;
  const int kBatchStreams = batch_stream_count();
  // Refined solves whose AAb_Solver takes the cooperative grid form run one
  // after another on stream 0 (two such grids must never wait for each
  // other's blocks); the others are spread over the other streams.
  auto uses_grid = [](const mihs_sketch_s* sk) {
    const int sa_type = sk->sa_prec != MIHS_SA_FP32 && sk->SAq != nullptr ? sk->sa_prec : MIHS_SA_FP32;
    return aab_grid_wanted((int)sk->m, (int)sk->d, sa_type, sk->aab_form);
  };
  MIHS_CUDA_TRY(cudaEventRecord(ev[kBatchStreams], s));
  for (int k = 0; k < kBatchStreams; ++k) MIHS_CUDA_TRY(cudaStreamWaitEvent(st[k], ev[kBatchStreams], 0));
  int next = 0;
  for (int i = 0; i < nprob && rc == MIHS_OK; ++i) {
    const mihs_problem& q = probs[i];
    mihs_sketch_s* sk = q.sk;
    const int k = uses_grid(sk) ? 0 : 1 + (next++) % (kBatchStreams - 1);
    const unsigned blocks = (unsigned)((sk->d + 255) / 256);
    for (int l = 0; l < nlambda && rc == MIHS_OK; ++l) {
      if (!(tols[l] > 0.0)) continue;
      float* xrow = q.X + (size_t)l * q.ldx;
      f32_to_f64_kernel<<<blocks, 256, 0, st[k]>>>(xrow, sk->ref_x64, (int)sk->d);
      MIHS_CHECK_LAUNCH();
      count_launch();
      mihs_opts o = *opts;
      o.tol = tols[l];
      o.sd = sds != nullptr ? sds[(size_t)i * nlambda + l] : 0.0;
      o.warm_start = 1;
      rc = solve_impl(sk, q.A, q.lda, q.b, lambdas[l], &o, sk->ref_x64, true, nullptr, st[k]);
      if (rc) {
        set_error("mihs_refine_batched: problem %d, lambda[%d]: %s", i, l, mihs_last_error());
        break;
      }
      f64_to_f32_kernel<<<blocks, 256, 0, st[k]>>>(sk->ref_x64, xrow, (int)sk->d);
      MIHS_CHECK_LAUNCH();
      count_launch();
      if (infos != nullptr)
        MIHS_CUDA_TRY(cudaMemcpyAsync(sk->ref_ctl_host + l, sk->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost,
                                      st[k]));
    }
  }
  for (int k = 0; k < kBatchStreams; ++k) {
    MIHS_CUDA_TRY(cudaEventRecord(ev[k], st[k]));
    MIHS_CUDA_TRY(cudaStreamWaitEvent(s, ev[k], 0));
  }
  if (rc || infos == nullptr) return rc;
  MIHS_CUDA_TRY(cudaStreamSynchronize(s));
  int worst = MIHS_OK;
  for (int i = 0; i < nprob; ++i) {
    for (int l = 0; l < nlambda; ++l) {
      if (!(tols[l] > 0.0)) continue;
      const SolveCtl& c = probs[i].sk->ref_ctl_host[l];
      mihs_info& inf = infos[(size_t)i * nlambda + l];
      inf.outer_iters = c.outer;
      inf.inner_iters_total = c.inner_total;
      inf.rel_resid = c.gnorm0 > 0.f ? (double)c.gnorm / (double)c.gnorm0 : 0.0;
      inf.status = c.done ? c.status : MIHS_NOT_CONVERGED;
      if (inf.status < 0) worst = inf.status;
      else if (worst == MIHS_OK && inf.status != MIHS_OK) worst = inf.status;
    }
  }
  return worst;
}

int mihs_gradient_refined(const float* A, int64_t n, int64_t d, int64_t lda, const float* b,
                          const double* x, double lambda, double* g, void* stream) {
  set_error("");
  int rc = check_matrix(A, n, d, lda, "mihs_gradient_refined");
  if (rc) return rc;
  MIHS_ARG(b != nullptr && x != nullptr && g != nullptr, "mihs_gradient_refined: null vector");
  MIHS_ARG(lambda >= 0.0 && std::isfinite(lambda), "mihs_gradient_refined: lambda must be finite, >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = apass_dd_num_partials(n, d);
  StreamScratch scratch;
  rc = scratch.alloc(sizeof(float2) * (size_t)P * apass_dpad(d), s);
  if (rc) return rc;
  float2* part = static_cast<float2*>(scratch.p);
  rc = launch_apass_dd(A, n, d, lda, b, x, part, nullptr, s);
  if (rc) return rc;
  return launch_apass_dd_finalize(part, P, d, x, lambda, g, nullptr, nullptr, s);
}

}  // extern "C"
