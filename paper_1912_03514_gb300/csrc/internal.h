// Host-side launchers shared between the translation units of libmihs.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mihs {

// ---- gradient A-pass (apass.cu) -------------------------------------------
// Number of split-K partial d-vectors the A-pass writes for an n×d problem.
int apass_num_partials(int64_t n, int64_t d);
// Row pitch (floats) of the partial buffer.
inline int64_t apass_dpad(int64_t d) { return round_up(d, 4); }
// partials[p][j] = Σ_{rows of block p} A[i][j]·(b[i] − A[i]·x).  x and b
// may be NULL (taken as 0).  Skips all work when ctl != NULL and ctl->done.
// A bounded wait that runs out sets ctl->status = MIHS_ERR_TIMEOUT and
// ctl->done (when ctl != NULL) and the library-wide device error word.
// gate ≥ 0: run only while ctl->phase == gate (refinement solves).
int launch_apass_partial(const float* A, int64_t n, int64_t d, int64_t lda,
                         const float* b, const float* x, float* partials,
                         SolveCtl* ctl, cudaStream_t s, int gate = -1);
// Reads and clears the library-wide device error word (synchronises).
int apass_device_error(int* code);
// g[j] = rhs[j] + Σ_p partials[p][j] − λ·x[j] in a fixed order (rhs may be
// null); with base64, g[j] = fp32(base64[j] + that) (refinement corrections).
int launch_apass_finalize(const float* partials, int P, int64_t d,
                          const float* x, float lambda, float* g,
                          const SolveCtl* ctl, cudaStream_t s, int gate = -1,
                          const float* rhs = nullptr, const double* base64 = nullptr);

// ---- λ-path gradient (apass_path.cu) ---------------------------------------
// Per-λ scalars of a path solve (passed by value to the kernels).
struct PathScalars {
  int nl;              // λ values in use (≤ 16)
  float lam[16], alpha[16], beta[16];
};
int apass_path_num_partials(int64_t n);
int apass_path_max_d();
// partials[p][l][j] (p < P, l < 16, row pitch dpad) = Σ_{rows of block p}
// A[i][j]·(b[i] − A[i]·X[l]) for l < nl; X λ-major with row pitch ldx.  Skips
// all work when *all_done (may be NULL).
int launch_apass_path(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const float* X,
                      int64_t ldx, int nl, float* partials, const int* all_done, cudaStream_t s);
// G[l][j] = Σ_p partials[p][l][j] − λ_l·X[l][j] (fixed order), G λ-major (ldg).
int launch_apass_path_finalize(const float* partials, int P, int64_t d, const float* X, int64_t ldx,
                               const PathScalars& sc, float* G, int64_t ldg, const int* all_done,
                               cudaStream_t s);
int apass_path_device_error(int* code);

// ---- quantised SA (sa_quant.cu) ---------------------------------------------
int64_t sa_quant_ld(int64_t d);                 // row pitch (elements) of quantised SA
int64_t sa_scale_count(int64_t m, int64_t d);   // fp8 tile scales
int launch_quantize_sa(const float* SA, int64_t m, int64_t d, int64_t ldsa, int prec, void* out, int64_t ldq,
                       float* scales, cudaStream_t s);
// ‖decode(q) − SA‖_F² in fp64 (deterministic: kQuantErrBlocks block partials
// in `scratch`, summed in order) into *err_out (device).
constexpr int kQuantErrBlocks = 512;
int launch_quant_error(const float* SA, int64_t m, int64_t d, int64_t ldsa, int prec, const void* q, int64_t ldq,
                       const float* scales, double* scratch, double* err_out, cudaStream_t s);
// The quantisation guard: storing SA as SA_q = SA + E keeps the sketched
// Hessian within a factor 2 of the exact one's (SA_qᵀSA_q + λI ⪰ ½(SAᵀSA + λI))
// when ‖E‖₂² ≤ λ/2.  ‖E‖₂² is estimated from ‖E‖_F² as for a matrix of
// independent equal-variance entries, ‖E‖_F²·(1/√m + 1/√d)².
inline double quant_spectral_estimate(double fro2, int64_t m, int64_t d) {
  const double f = 1.0 / ::sqrt((double)m) + 1.0 / ::sqrt((double)d);
  return fro2 * f * f;
}

// ---- gradients of the solution (backward.cu) ------------------------------
// dlambda = −xᵀv (fp64); db = Av; dA = r vᵀ − (Av) xᵀ with r = b − Ax.  Any of
// dA, db, dlambda may be NULL; b may be NULL only when dA is.
int launch_backward_grads(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const float* x,
                          const float* v, float* dA, int64_t ldda, float* db, double* dlambda, cudaStream_t s);

// ---- compensated gradient (apass_dd.cu) -------------------------------------
// Same pass with x in fp64 and double-float sums; partials are (hi, lo) pairs.
int apass_dd_num_partials(int64_t n, int64_t d);
int launch_apass_dd(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const double* x,
                    float2* partials, SolveCtl* ctl, cudaStream_t s, int gate = -1);
// g64[j] = rhs[j] + Σ_p (hi + lo) − λ·x[j] in fp64 (rhs may be null); g32
// (optional) its fp32 rounding; xref (optional) receives x.  b of
// launch_apass_dd may be null (taken as 0).
int launch_apass_dd_finalize(const float2* partials, int P, int64_t d, const double* x, double lambda,
                             double* g64, float* g32, const SolveCtl* ctl, cudaStream_t s, int gate = -1,
                             const float* rhs = nullptr, double* xref = nullptr);
int apass_dd_device_error(int* code);

// ---- AAb_Solver (aab.cu) --------------------------------------------------
struct AabLaunch {
  const void* SA;      // element type per sa_type; ldsa in elements
  int sa_type;         // MIHS_SA_FP32 (0), MIHS_SA_BF16, MIHS_SA_FP8E4M3 (quantised: ldsa % 16 == 0)
  const float* sa_scale;  // fp8: one scale per 128 × 128 tile, ⌈dp/128⌉ per tile row
  int m, d;
  int64_t ldsa;
  const float* g;
  float lambda, eps;
  int max_passes;      // already capped at min(m, d)
  float* delta;        // written when non-NULL
  int* passes;         // device, optional
  // heavy ball (when x != NULL): x⁺ = x + αΔ + β(x − x⁻), x⁻ ← x
  float alpha, beta;
  float* x;
  float* x_prev;
  double* x64;         // refinement mode: fp64 iterate (heavy ball in fp64)
  double* x_prev64;
  float* x32_shadow;   // refinement mode: fp32 copy of the fp64 iterate (plain phase)
  double alpha64, beta64;
  SolveCtl* ctl;       // solve mode (stop test, counters); may be NULL
  float* hist;         // solve mode: ‖g‖ of every gradient step (kHistCap entries); may be NULL
  unsigned long long cond;  // graph conditional handle to clear when the solve stops (0: none)
  // λ-path mode (path != 0): one cluster per λ_l (l < ps.nl) with g, x, x⁻
  // and ctl offset by l (g and x⁻ pitch path_ldg, x pitch path_ldx), the
  // scalars from ps; *path_ndone counts stopped λ and the last one sets
  // *path_all_done and clears cond.  delta, passes, hist and x64 unused.
  int path;
  PathScalars ps;
  int64_t path_ldg, path_ldx;
  int* path_ndone;
  int* path_all_done;
  // Global scratch of the grid form (aab_grid_ws_bytes(d) bytes, barrier
  // word zeroed); NULL: the grid form is not used.
  void* grid_ws;
  int aab_form;     // MIHS_AAB_AUTO / _CLUSTER / _GRID
  int grid_blocks;  // grid form: blocks wanted (0: one per SM, at most m)
};
// Runs one cluster (aab.cu), or — when SA does not fit one cluster's shared
// memory and a.grid_ws is given — one grid over the SMs (aab_grid.cu).
int launch_aab(const AabLaunch& a, cudaStream_t s);
// Single-λ AAb_Solver as one grid that keeps SA in the shared memory of up to
// every SM.  `ws` holds aab_grid_ws_bytes(d) bytes whose first
// kAabGridBarBytes hold the grid barrier word, which must be zero before a
// solve (it returns to zero after every completed launch).  Returns
// MIHS_ERR_UNSUPPORTED (nothing launched) when SA does not fit.
constexpr size_t kAabGridBarBytes = 256;
size_t aab_grid_ws_bytes(int d);
int launch_aab_grid(const AabLaunch& a, void* ws, cudaStream_t s);
int aab_grid_device_error(int* code);
// True when launch_aab would take the grid form given scratch: `form` is
// MIHS_AAB_GRID, or MIHS_AAB_AUTO and SA of m × d does not fit in the shared
// memory of one cluster (for AUTO, MIHS_AAB_FORM=grid or =cluster in the
// environment overrides).
bool aab_grid_wanted(int m, int d, int sa_type, int form = 0);
// λ-path mode with all λ in one cooperative grid that keeps SA in the
// shared memory of all SMs (aab_path.cu); `ws` holds aab_path_ws_floats(dp)
// floats.  Returns MIHS_ERR_UNSUPPORTED (nothing launched) when SA or d does
// not fit, so that the caller can use launch_aab's one-cluster-per-λ form.
size_t aab_path_ws_floats(int dp);
int aab_path_device_error(int* code);
int launch_aab_path(const AabLaunch& a, float* ws, cudaStream_t s);
// Picks and caches the cluster shape for (m, d) (call outside stream capture).
void aab_prepare(int m, int d, int sa_type = 0);

constexpr int kHistCap = 1024;

// ---- sketches (sketch_*.cu) ------------------------------------------------
int sketch_gaussian(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m,
                    uint64_t seed, float* SA, int64_t ldsa, cudaStream_t s);
// tcgen05 version of the Gaussian sketch (sketch_gaussian_tc.cu).
bool gaussian_tc_available();
// A tiled tensor map over the rows × cols fp32 matrix A (row pitch ld
// elements, 16-byte aligned, ld·4 a multiple of 16), box box_cols × box_rows,
// no swizzle, zero fill out of bounds, L2 promotion of 128 or 256 bytes.
// UNSUPPORTED without the driver entry point or when the driver rejects the
// layout.
int encode_tmap_2d_f32(CUtensorMap* map, const float* A, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                       int box_rows, int l2_promotion);
// prec: 0 tf32 operands, 1 S and A rounded to bf16, 2 S and A·256/max|A|
// rounded to fp8 e4m3 (the scale undone in the reduction).
int sketch_gaussian_tc(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m,
                       uint64_t seed, float* SA, int64_t ldsa, cudaStream_t s, int prec = 0);
int gauss_tc_device_error(int* code);
int sketch_countsketch(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m,
                       uint64_t seed, float* SA, int64_t ldsa, cudaStream_t s);
int sketch_srht(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m,
                uint64_t seed, float* SA, int64_t ldsa, cudaStream_t s);
int srht_device_error(int* code);

// ---- statistical dimension (hutchinson.cu) ----------------------------------
// Algorithm 4; synchronises `s` and writes the estimate to *sd_out (host).
int estimate_sd(const float* SA, int64_t m, int64_t d, int64_t ldsa, double lambda, int T, double eps_tr,
                uint64_t seed, double* sd_out, cudaStream_t s);

// ---- per-kernel event timing (api.cu) -------------------------------------
enum TimerId { kTimerApass = 0, kTimerAab = 1, kTimerSketch = 2, kTimerApassDd = 3, kTimerBackward = 4, kTimerApassPath = 5,
               kTimerApassCorr = 6, kNumTimers = 7 };
bool timing_on();
void timing_begin(int which, cudaStream_t s);
void timing_end(int which, cudaStream_t s);

// Stream-ordered scratch that frees itself on the same stream.
struct StreamScratch {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~StreamScratch() {
    if (p) cudaFreeAsync(p, s);
  }
  int alloc(size_t bytes, cudaStream_t stream) {
    s = stream;
    cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, stream);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? MIHS_ERR_OOM : MIHS_ERR_CUDA;
    }
    return MIHS_OK;
  }
};

}  // namespace mihs
