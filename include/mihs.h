/*
 * mihs.h — C ABI of the GB300 Momentum Iterative Hessian Sketch (M-IHS) ridge
 * solver (Ozaslan, Pilanci, Arikan, "M-IHS: A Momentum-based Iterative
 * Hessian Sketch ...", arXiv 1912.03514).
 *
 * Problem (Section 1, Eq. "intro"):
 *     x* = argmin_x  ½‖Ax − b‖² + (λ/2)‖x‖²,   A ∈ R^{n×d}, n ≥ d, λ > 0.
 *
 * Conventions shared by every entry point
 *   - Matrices are fp32, row-major, with a leading dimension (row pitch, in
 *     elements) `ld* ≥ columns`; `lda` must be a multiple of 4 and `A` 16-byte
 *     aligned (the kernels read rows with 128-bit loads).  Vectors are fp32.
 *   - Every pointer to array data is DEVICE memory owned by the caller unless
 *     the argument says otherwise.  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; only calls that return
 *     host-visible results (an `info` struct, a host scalar) synchronise it.
 *   - Return value: MIHS_OK (0) on success, MIHS_NOT_CONVERGED (+1) when a
 *     solve stopped at its iteration cap (the output is still written), or a
 *     negative MIHS_ERR_* code.  mihs_last_error() gives a message for the
 *     most recent failure on the calling host thread.  No C++ exception
 *     crosses this boundary.
 *   - Limits: 1 ≤ d ≤ 2048, d ≤ n < 2^31, 1 ≤ m ≤ n.
 */
#ifndef MIHS_H
#define MIHS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MIHS_OK = 0,
  MIHS_NOT_CONVERGED = 1,
  MIHS_ERR_INVALID_ARG = -1,
  MIHS_ERR_CUDA = -2,
  MIHS_ERR_OOM = -3,
  MIHS_ERR_TIMEOUT = -4,
  MIHS_ERR_NUMERIC = -5,
  MIHS_ERR_UNSUPPORTED = -6
};

/* Sketch families of Lemma 3 (cases iv, i, iii).  All satisfy E[SᵀS] = I
 * (text after Algorithm 1).  S is never stored: it is a function of (family,
 * seed, m, n) through the counter-based generator Philox4x32-10.
 *   MIHS_GAUSSIAN    S_ij ~ N(0, 1/m) (proof of Lemma 3, case iv).  Entry
 *                    (i, j) is a Box–Muller normal from Philox counter
 *                    (⌊j/4⌋, i, 0, 0), key (seed mod 2³², seed div 2³²).
 *   MIHS_COUNTSKETCH one ±1 per column (Lemma 3, case i): column j goes to
 *                    row h(j) = ⌊w0·m/2³²⌋ with sign + if w1 even, from
 *                    counter (j, 0, 1, 0).
 *   MIHS_SRHT        S = √(n_p/m)·P·(H/√n_p)·D (Lemma 3, case iii) with
 *                    n_p = 2^⌈log₂ n⌉ (A zero-padded), D_j from counter
 *                    (j, 0, 2, 0), P's m rows drawn with replacement from
 *                    counter (i, 0, 3, 0).                                  */
enum { MIHS_GAUSSIAN = 0, MIHS_COUNTSKETCH = 1, MIHS_SRHT = 2 };

/* Storage precision of SA inside AAb_Solver (arithmetic is fp32 in all). */
enum { MIHS_SA_FP32 = 0, MIHS_SA_BF16 = 1, MIHS_SA_FP8E4M3 = 2 };

/* Human-readable name of a return code (static string). */
const char* mihs_strerror(int code);
/* Message describing the last failure on this host thread ("" if none). */
const char* mihs_last_error(void);
/* Number of kernels this library has launched in this process so far. */
uint64_t mihs_launch_count(void);

/* Device-side failure report: every wait inside the library's kernels is
 * bounded (2 s); a wait that runs out makes its kernel stop early and record
 * MIHS_ERR_TIMEOUT here (and in the status of the solve it belongs to).
 * Writes the recorded code (0 if none) to *code and clears it; synchronises
 * the current device. */
int mihs_device_status(int* code);

/* Failure-detection self-test of those bounded waits: one kernel runs the
 * library's own wait on a condition that nothing satisfies, with a limit of
 * limit_ns (10⁶ … 10¹⁰ ns) instead of 2 s, and *status receives what the
 * waiting kernel reported — MIHS_ERR_TIMEOUT when the wait ran out (the
 * expected outcome), MIHS_OK if the condition was somehow met.
 *   which 0: an mbarrier expecting one arrival that never comes (the wait of
 *            the bulk-copy rings of the gradient passes, the AAb staging copy
 *            and the tensor-core sketch pipeline);
 *   which 1: a grid barrier of two blocks, one of which leaves without
 *            arriving (the barrier of the grid forms of AAb_Solver).
 * Nothing faults: the kernel returns, the device stays usable and the
 * device error word of mihs_device_status is left alone.  Synchronises
 * `stream`.  Errors: INVALID_ARG, CUDA, OOM. */
int mihs_selftest_wait(int which, int64_t limit_ns, int* status, void* stream);

/* Host → device copy of `bytes` bytes for the end-to-end forms: when `src`
 * is pinned host memory mapped into the device's address space (memory from
 * cudaHostAlloc / cudaHostRegister under unified addressing) and both
 * pointers are 16-byte aligned, the SMs load it directly over the CPU–GPU
 * link (NVLink-C2C on Grace systems); otherwise, and for the last bytes not
 * filling 16, cudaMemcpyAsync.  dst: DEVICE memory.  Asynchronous on
 * `stream`; src must stay valid and unchanged until the copy has run.
 * Errors: INVALID_ARG (null pointers, bytes < 0, dst not device memory),
 * CUDA. */
int mihs_copy_to_device(void* dst, const void* src, int64_t bytes, void* stream);

/* The same host → device copy by a copy engine (cudaMemcpyAsync): no SM
 * takes part, so the copy can overlap solves running on other streams
 * without slowing them — the form for double-buffered inputs, where the
 * next problem is copied in while the current one solves (measured on
 * 262144×1024: 187 solves/s end to end in one run, against 181 with the SM copy on 8
 * SMs beside the solves and 148 copying then solving).  Alone, the SM copy
 * of mihs_copy_to_device is faster.  Arguments and errors as
 * mihs_copy_to_device. */
int mihs_copy_to_device_dma(void* dst, const void* src, int64_t bytes, void* stream);

/* Per-kernel timing (profiling aid, off by default).  mihs_timing(1) clears
 * the records and starts recording CUDA events on the launching stream around
 * every launch of: the gradient A-pass (timer 0), AAb_Solver (timer 1), a
 * sketch call (timer 2), the compensated A-pass (timer 3), the backward
 * gradient pass (timer 4), the λ-path gradient pass (timer 5) and the fp32
 * correction passes of refinement solves (timer 6).  While it
 * is on, solves run their steps as host-driven launches and read the stop
 * state back after each step, so only launches that did work are recorded.
 * mihs_timing(0) stops recording.  mihs_timing_read synchronises on the
 * recorded events and returns the summed duration (ms) and the number of
 * launches of one timer. */
int mihs_timing(int on);
int mihs_timing_read(int which, double* total_ms, int64_t* count);

/* ------------------------------------------------------------------------
 * Building blocks: one call per step of Algorithm 1.
 * ---------------------------------------------------------------------- */

/* RP_fun of Algorithm 1 (sketch step): SA = S·A.
 *   A      n×d, leading dimension lda.
 *   SA     output, m×d, leading dimension ldsa ≥ d (overwritten).
 *   family MIHS_GAUSSIAN | MIHS_COUNTSKETCH | MIHS_SRHT; seed keys S.
 * May allocate stream-ordered scratch (cudaMallocAsync) that it frees on the
 * same stream.  Errors: INVALID_ARG (sizes, alignment, family), CUDA, OOM. */
int mihs_sketch_apply(const float* A, int64_t n, int64_t d, int64_t lda,
                      int family, int64_t m, uint64_t seed,
                      float* SA, int64_t ldsa, void* stream);

/* The Gaussian sketch of mihs_sketch_apply (Lemma 3, case iv) formed from
 * bf16 operands on the tensor cores: every entry of S and of A is rounded to
 * bf16 (round to nearest even) and the products are accumulated in fp32,
 * then scaled by 1/√m.  S is the same Philox/Box–Muller matrix as the fp32
 * form.  The sketch only preconditions Algorithm 1 (the fixed point is where
 * the exact gradient vanishes, Section 3.1), so the rounding changes the
 * rate, not the solution.  Arguments, scratch and errors as
 * mihs_sketch_apply; UNSUPPORTED when the tensor-core path is unavailable. */
int mihs_sketch_gaussian_bf16(const float* A, int64_t n, int64_t d, int64_t lda,
                              int64_t m, uint64_t seed, float* SA, int64_t ldsa,
                              void* stream);

/* The same Gaussian sketch formed from fp8 e4m3 operands on the tensor
 * cores (tcgen05.mma kind::f8f6f4, fp32 accumulation): every entry of S is
 * rounded to e4m3, A is multiplied by the power of two 2^k that puts max|A|
 * in [128, 256) (exact; one extra pass over A for the maximum; k ≤ 127) and
 * rounded to e4m3 (round to nearest even, saturating), and the sum is
 * multiplied by 2^−k and 1/√m.  e4m3 keeps 3 mantissa
 * bits, so this sketch perturbs the preconditioner by a relative 2⁻⁴ of A's
 * entries; it is what a handle storing SA in fp8 forms, and the guard of
 * mihs_sketch_set_precision decides at which λ that storage is accepted.
 * Arguments, scratch and errors as mihs_sketch_gaussian_bf16. */
int mihs_sketch_gaussian_fp8(const float* A, int64_t n, int64_t d, int64_t lda,
                             int64_t m, uint64_t seed, float* SA, int64_t ldsa,
                             void* stream);

/* Gradient step of Algorithm 1: g = Aᵀ(b − Ax) − λx, reading A once.
 *   b (n), x (d) inputs; g (d) output.  0 ≤ λ ≤ FLT_MAX (fp32 arithmetic).
 * Allocates stream-ordered scratch for the split-K partial sums (one d-vector
 * per thread block) and frees it on the same stream.  The reduction order is
 * fixed, so repeated calls give bit-identical g.
 * Errors: INVALID_ARG, CUDA, OOM. */
int mihs_gradient(const float* A, int64_t n, int64_t d, int64_t lda,
                  const float* b, const float* x, double lambda, float* g,
                  void* stream);

/* The gradient of mihs_gradient (same arguments, same result) without any
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc/cudaMallocAsync at the moment they
 * need a gradient — e.g. code inside an allocator or memory-pool callback
 * that must not re-enter the allocator, code that may allocate only at
 * start-up, or a process whose device-memory budget is fixed up front.
 * Its split-K scratch is a fixed 1.25 MiB array in the library's own device
 * memory, reserved on every GPU that loads the library and held until exit.
 *   - The first call on each device looks the array's device address up
 *     (cudaGetSymbolAddress) with that device current and caches it; make
 *     that first call before any stream capture.  A cudaDeviceReset of the
 *     device invalidates the cached address: do not call this entry point
 *     on a device after resetting it.
 *   - λ must lie in [0, FLT_MAX] (the kernels compute in fp32).
 *   - Limit: (partial rows = min(#SMs, ⌈n/rows per block step⌉)) × d rounded
 *     up to 4 must fit in 160 × 2048 floats; larger cases return
 *     MIHS_ERR_UNSUPPORTED with a message (only GPUs with more than 160 SMs
 *     can reach it, since d ≤ 2048).
 *   - Every call shares the array.  Calls whose kernels overlap on the GPU
 *     (different streams or host threads) race on it; serialise them.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
int mihs_gradient_noalloc(const float* A, int64_t n, int64_t d, int64_t lda,
                          const float* b, const float* x, double lambda,
                          float* g, void* stream);

/* AAb_Solver (Algorithm 5, Section 3.6): approximately solve
 *     (SAᵀSA + λI) Δ = g
 * by upper bidiagonalisation of SA, stopping when the relative residual
 * estimate t < eps_sub or after `max_inner` loop passes (≤ 0: min(m, d)).
 *   SA m×d (ld ldsa), g (d) inputs; delta (d) output.
 *   passes: optional DEVICE int* receiving the number of loop passes.
 * Any ldsa ≥ d is accepted when SA fits in the cluster's shared memory
 * (m·d ≲ 800K); larger SA must have 16-byte aligned rows (ldsa % 4 == 0).
 * Runs as one thread-block cluster with SA in its shared memory; an SA too
 * large for that runs as one cooperative grid of up to one block per SM with
 * SA spread over their shared memory, whose scratch (one d-vector per SM,
 * about 1.2 MB at d = 2048) comes from the stream-ordered pool and is freed
 * on the same stream (the environment variable MIHS_AAB_FORM=cluster keeps
 * one cluster reading SA from L2 instead).  Grid-form calls on different
 * streams should not overlap: two grids that wait for each other's blocks
 * end with MIHS_ERR_TIMEOUT after 2 s.
 * Errors: INVALID_ARG (λ ≤ 0, eps_sub < 0, sizes), CUDA, OOM, TIMEOUT. */
int mihs_aab_solve(const float* SA, int64_t m, int64_t d, int64_t ldsa,
                   const float* g, double lambda, double eps_sub, int max_inner,
                   float* delta, int* passes, void* stream);

/* Quantised copy of an SA (device memory), as mihs_sketch_set_precision
 * stores it: out is m × ldq elements of bf16 or fp8 e4m3 (ldq ≥ d, a multiple
 * of 16; columns ≥ d are zero); for fp8, scales receives ⌈m/128⌉ × ⌈d₄/128⌉
 * floats (row-major, d₄ = d rounded up to 4), scale = max |SA| over the
 * 128 × 128 tile / 448 (1 for a zero tile), q = e4m3(SA/scale) rounded to
 * nearest even and saturated.  Errors: INVALID_ARG, CUDA. */
int mihs_quantize_sa(const float* SA, int64_t m, int64_t d, int64_t ldsa,
                     int sa_prec, void* out, int64_t ldq, float* scales,
                     void* stream);

/* mihs_aab_solve on a quantised SA (the output of mihs_quantize_sa): the
 * products decode each element (times its tile scale for fp8) and run in
 * fp32.  Same arguments and errors as mihs_aab_solve otherwise. */
int mihs_aab_solve_q(const void* SAq, int sa_prec, const float* scales,
                     int64_t m, int64_t d, int64_t ldq, const float* g,
                     double lambda, double eps_sub, int max_inner,
                     float* delta, int* passes, void* stream);

/* AAb_Solver followed by the heavy-ball step of Eq. mihs1:
 *     x⁺ = x + αΔ + β(x − x⁻),  then x⁻ ← x, x ← x⁺   (in place).
 * Same arguments as mihs_aab_solve plus α, β and the DEVICE d-vectors x and
 * x_prev (both read and overwritten).  Δ is not written out. */
int mihs_aab_heavy_ball(const float* SA, int64_t m, int64_t d, int64_t ldsa,
                        const float* g, double lambda, double eps_sub,
                        int max_inner, double alpha, double beta,
                        float* x, float* x_prev, int* passes, void* stream);

/* Statistical dimension estimate (Algorithm 4, inexact Hutchinson):
 *     sd ≈ d − (λ/T)·Σ_ℓ ⟨v^ℓ, z^ℓ⟩,   z^ℓ = AAb_Solver(SA, v^ℓ, λ, eps_tr),
 * with Rademacher probes v^ℓ_j = ±1 from Philox counter (j, ℓ, 4, 0) keyed by
 * `seed`.  The paper uses T = 2 or 3 and eps_tr = 0.5.  Synchronises the
 * stream and writes the estimate to the HOST double *sd_out.  Allocates
 * stream-ordered scratch (2d floats).  Errors: INVALID_ARG, CUDA, OOM. */
int mihs_estimate_sd(const float* SA, int64_t m, int64_t d, int64_t ldsa,
                     double lambda, int T, double eps_tr, uint64_t seed,
                     double* sd_out, void* stream);

/* ------------------------------------------------------------------------
 * The solver (Algorithm 1, M-IHS for n ≥ d).
 * ---------------------------------------------------------------------- */

typedef struct mihs_sketch_s* mihs_sketch_t;

/* Form and keep SA = S·A (Algorithm 1, sketch step) for later solves with
 * the same A.  The handle owns SA and the solver's workspace (allocated here
 * with cudaMalloc; freed by mihs_sketch_destroy).  `A` itself is not kept.
 * Errors: INVALID_ARG, CUDA, OOM. */
int mihs_sketch(const float* A, int64_t n, int64_t d, int64_t lda, int family,
                int64_t m, uint64_t seed, void* stream, mihs_sketch_t* out);

/* Recompute the handle's SA for a new matrix of the same shape (n×d) and/or
 * a new seed, reusing its memory (no allocation of the handle's own buffers;
 * the sketch kernels' stream-ordered scratch as in mihs_sketch_apply).  A
 * Gaussian handle whose SA is stored in bf16 or fp8
 * (mihs_sketch_set_precision) forms S·A from bf16 operands
 * (mihs_sketch_gaussian_bf16) before quantising it.
 * Errors: INVALID_ARG, CUDA, OOM. */
int mihs_resketch(mihs_sketch_t sk, const float* A, int64_t lda, uint64_t seed,
                  void* stream);

/* Read-only view of a handle: device pointer to SA (m×d, leading dimension
 * d rounded up to a multiple of 4) and sizes.
 * Any output pointer may be NULL. */
int mihs_sketch_info(mihs_sketch_t sk, const float** SA, int64_t* m,
                     int64_t* d, int64_t* n, int* family);

/* Copy the handle's SA (m×d) into the caller's DEVICE buffer `dst` with
 * leading dimension ldd ≥ d, on `stream`. */
int mihs_sketch_copy(mihs_sketch_t sk, float* dst, int64_t ldd, void* stream);

/* Mixed-precision inner solve: store SA for AAb_Solver in bf16 or
 * in fp8 e4m3 with one fp32 scale per 128 × 128 tile (scale = tile max / 448)
 * while its arithmetic stays fp32.  The sketch only preconditions Algorithm 1
 * (its fixed point is where the exact gradient vanishes, Section 3.1), so the
 * solution is unchanged and only the rate can be; use mihs_solve_refined for
 * targets below the fp32 floor.  Converts the current SA now and after every
 * mihs_resketch; the first call for a quantised precision allocates the
 * quantised copy (cudaMalloc).  MIHS_SA_FP32 switches back.  Sd estimation
 * (Algorithm 4) keeps using the fp32 SA.
 * A Gaussian handle re-forms S·A from operands of the storage precision
 * (mihs_sketch_gaussian_bf16 / _fp8) on every mihs_resketch.
 * Guard: each conversion also measures the rounding E = SA_q − SA (‖E‖_F²,
 * read back to the host, so this call and mihs_resketch synchronise the
 * stream for a quantised handle).  A solve (mihs_solve, _refined, _path,
 * mihs_backward*) at a λ with ‖E‖_F²·(1/√m + 1/√d)² > λ/2 (an estimate of
 * ‖E‖₂²) returns MIHS_ERR_UNSUPPORTED before launching anything: past that
 * point the sketched Hessian is no longer within a factor 2 of the exact
 * one, and the preconditioned spectrum can leave the region where the heavy
 * ball of Theorem 1 converges (fp8 at κ(AᵀA + λI) ≈ 1e6 does).
 * Errors: INVALID_ARG, OOM, CUDA. */
int mihs_sketch_set_precision(mihs_sketch_t sk, int sa_prec, void* stream);

/* Form of the inner solver (AAb_Solver, Algorithm 5) in a handle's solves
 * (mihs_solve, mihs_solve_refined, mihs_backward*):
 *   MIHS_AAB_AUTO     one thread-block cluster holding SA in its distributed
 *                     shared memory when it fits, else one cooperative grid
 *                     holding SA in the shared memory of up to every SM;
 *   MIHS_AAB_CLUSTER  always one cluster (SA read from L2 when it does not
 *                     fit);
 *   MIHS_AAB_GRID     one cooperative grid of `grid_blocks` blocks (0: one per
 *                     SM, at most m), raised to the fewest that hold SA in
 *                     shared memory; the cluster form when the grid cannot be
 *                     made resident.
 * The cluster form is the faster one for a solve that has the GPU to itself.
 * A small grid (about 24 blocks) is the better choice when several solves
 * share the GPU on concurrent streams: its blocks start on any free SMs,
 * while a 16-block cluster waits until one GPU processing cluster has 16
 * free SMs.  Grids of handles solving on concurrent streams never wait for
 * one another while their block counts sum to at most the number of SMs
 * (the other kernels' blocks end by themselves and free their SMs); beyond
 * that, a grid barrier that stalls ends the solve with MIHS_ERR_TIMEOUT
 * after 2 s rather than hanging.  Results agree to fp32 rounding (the
 * summation order differs).  λ-paths, batched and dual solves and the
 * row-level mihs_aab_* calls keep MIHS_AAB_AUTO.  Not to be called while a
 * solve on the handle is in flight.
 * Errors: INVALID_ARG (unknown form, grid_blocks < 0). */
enum { MIHS_AAB_AUTO = 0, MIHS_AAB_CLUSTER = 1, MIHS_AAB_GRID = 2 };
int mihs_sketch_set_aab(mihs_sketch_t sk, int form, int grid_blocks);

/* Release a handle (synchronises the device first).  NULL is a no-op. */
int mihs_sketch_destroy(mihs_sketch_t sk);

typedef struct {
  double tol;       /* stop when ‖g‖ ≤ tol·‖Aᵀb‖ (relative normal-equation
                       residual; checked after every gradient step); ≤ 0
                       disables the test                                   */
  int max_outer;    /* N of Algorithm 1: at most this many momentum steps   */
  double eps_sub;   /* forcing term ε_sub of AAb_Solver (0.1 in the paper)  */
  int max_inner;    /* cap on AAb_Solver passes per step (≤ 0: min(m, d))   */
  double sd;        /* statistical dimension estimate, sd < m; gives
                       β = sd/m and α = (1 − β)² (Corollary 3).  sd ≤ 0:
                       estimated from SA by Algorithm 4 (T = 2, eps 0.5,
                       capped at 0.95·m); the call then synchronises      */
  int warm_start;   /* 0: x is ignored and the iteration starts at 0;
                       1: x holds x¹ (costs one extra pass over A for ‖Aᵀb‖) */
} mihs_opts;

typedef struct {
  int outer_iters;        /* momentum steps taken                          */
  int inner_iters_total;  /* AAb_Solver passes summed over the steps       */
  double rel_resid;       /* ‖g(x)‖/‖Aᵀb‖ of the returned x                */
  int status;             /* MIHS_OK, MIHS_NOT_CONVERGED or MIHS_ERR_NUMERIC */
} mihs_info;

/* Default options: tol 1e-6, max_outer 100, eps_sub 0.1, max_inner 0,
 * sd must still be set by the caller. */
mihs_opts mihs_default_opts(void);

/* Run Algorithm 1 with the handle's SA on the problem (A, b, λ).
 * The outer loop runs on the device: a CUDA graph with a conditional WHILE
 * node (body: gradient A-pass, partial-sum reduce, AAb_Solver + heavy ball)
 * that the AAb kernel stops when the test fires, so a solve costs one graph
 * launch plus two small launches.  Up to eight graphs per kind of solve are
 * cached in the handle, keyed by A, lda, b, x, λ, α, β, eps_sub and
 * max_inner and replaced least recently used, so that solves alternating
 * between input buffers or cycling through a few λ relaunch cached graphs.
 * A replaced graph is kept until the handle is destroyed (or until 64 have
 * gathered, when they are freed together, which waits for the GPU):
 * destroying an executable graph waits for the work in flight.  Setting
 * the environment variable MIHS_NO_GRAPH makes the host drive the steps.
 *   A     n×d (same n, d as the handle), leading dimension lda.
 *   b     n-vector.  0 < λ ≤ FLT_MAX (AAb_Solver computes in fp32).
 *   x     d-vector: x¹ on entry if opts->warm_start, the solution on exit.
 *   info  optional HOST struct; when non-NULL the call synchronises the
 *         stream and fills it, and the return value reflects convergence
 *         (MIHS_NOT_CONVERGED / MIHS_ERR_NUMERIC).  When NULL the call only
 *         enqueues work and returns MIHS_OK.
 * A handle must not be used by two solves that overlap in time.
 * Errors: INVALID_ARG (λ ≤ 0, sd ∉ (0, m), sizes), CUDA, NUMERIC. */
int mihs_solve(mihs_sketch_t sk, const float* A, int64_t lda, const float* b,
               double lambda, const mihs_opts* opts, float* x, mihs_info* info,
               void* stream);

/* Algorithm 1 with compensated refinement: the same iteration with the
 * iterate x in fp64.  Steps use the plain fp32 gradient until the relative
 * residual is below 1e-7 or has set no new minimum for three steps, then the
 * gradient g = Aᵀ(b − Ax) − λx computed by a
 * compensated pass over A (double-float sums: TwoProduct/TwoSum in fp32
 * pairs, fp64 partial sums), while SA, AAb_Solver and its stop test stay
 * fp32 (the sketch only preconditions; the fixed point of the iteration is
 * where the gradient vanishes).  Between compensated passes ("refreshes" at
 * x_ref), steps may take g(x) = g(x_ref) − (AᵀA + λI)(x − x_ref) with the
 * product from the plain fp32 pass: its rounding is relative to
 * ‖x − x_ref‖, not to ‖x‖; a refresh follows when that gradient stops
 * falling, after 8 such steps, or before the solve may stop (only a
 * compensated gradient ends a solve), and the corrections are switched off
 * for the rest of the solve once a refresh cycle gains less than 4×
 * (ill-conditioned problems; environment MIHS_REFINE_CORR=0 switches them
 * off from the start).  For targets below the fp32 floor (relative error
 * ~1e-6 and beyond).  x is a DEVICE double array (x¹ on entry if
 * warm_start).  The first refined solve on a handle allocates its workspace
 * (double-float partials, fp64 previous iterate, reference point and
 * gradient) with cudaMalloc.  Same arguments, semantics and errors as
 * mihs_solve otherwise. */
int mihs_solve_refined(mihs_sketch_t sk, const float* A, int64_t lda, const float* b,
                       double lambda, const mihs_opts* opts, double* x,
                       mihs_info* info, void* stream);

/* The compensated gradient of mihs_solve_refined on its own:
 * g = Aᵀ(b − Ax) − λx with x and g DEVICE double arrays (d), A and b fp32.
 * Allocates stream-ordered scratch for the double-float partials.
 * Errors: INVALID_ARG, CUDA, OOM. */
int mihs_gradient_refined(const float* A, int64_t n, int64_t d, int64_t lda,
                          const float* b, const double* x, double lambda,
                          double* g, void* stream);

/* ------------------------------------------------------------------------
 * λ-paths and batches.  Algorithm 1 for several regularisation values on
 * one matrix: SA does not depend on λ (AAb_Solver takes λ as an argument,
 * Algorithm 5), so one sketch serves the whole path, and the gradients of
 * all iterates are formed in ONE pass over A per outer step.  Each λ_l keeps
 * its own iterate, momentum parameters β_l = sd_l/m, α_l = (1 − β_l)²
 * (Corollary 3) and stop test; the path stops when every λ has.
 * ---------------------------------------------------------------------- */

/* The path's gradient step on its own: G_l = Aᵀ(b − A·X_l) − λ_l·X_l for
 * l < nl ≤ 16 in one pass over A.  X and G DEVICE, λ-major (row l of pitch
 * ldx / ldg ≥ d); lambdas HOST (λ_l ≥ 0).  d ≤ 1024.  Allocates
 * stream-ordered scratch for the split-K partials.  Errors: INVALID_ARG,
 * UNSUPPORTED, CUDA, OOM. */
int mihs_gradient_path(const float* A, int64_t n, int64_t d, int64_t lda,
                       const float* b, int nl, const double* lambdas,
                       const float* X, int64_t ldx, float* G, int64_t ldg,
                       void* stream);

/* Solve the ridge problem (A, b, λ_l) for l < nlambda with the handle's SA.
 *   lambdas  HOST array of nlambda values > 0.
 *   sds      HOST array of nlambda statistical dimensions (< m), or NULL:
 *            each estimated from SA by Algorithm 4 (T = 2, ε_tr = 0.5,
 *            capped at 0.95·m; the call then synchronises).
 *   opts     tol, max_outer, eps_sub, max_inner, warm_start as in
 *            mihs_solve (opts->sd is ignored).
 *   X        DEVICE nlambda × d, λ-major: X + l·ldx is x(λ_l) (the starting
 *            point when opts->warm_start, the solution on exit); ldx ≥ d.
 *   infos    optional HOST array of nlambda; when non-NULL the call
 *            synchronises and returns the worst status.
 * λ values are processed in groups of 16 (one device-side graph loop per
 * group, cached in the handle).  d ≤ 1024 (MIHS_ERR_UNSUPPORTED beyond).
 * Each step runs AAb_Solver as one thread-block cluster per λ; with the
 * environment variable MIHS_PATH_AAB=grid, as one cooperative grid for all λ
 * that holds SA in the shared memory of up to every SM (when it fits).  Do
 * not run two path solves at the same time on different streams.
 * The first path solve on a handle allocates its workspace (cudaMalloc). */
int mihs_solve_path(mihs_sketch_t sk, const float* A, int64_t lda,
                    const float* b, int nlambda, const double* lambdas,
                    const double* sds, const mihs_opts* opts, float* X,
                    int64_t ldx, mihs_info* infos, void* stream);

/* One problem of a batch: its handle (sketched from its A), A, b and the
 * λ-major output X (nlambda × d, pitch ldx), all device memory. */
typedef struct {
  mihs_sketch_t sk;
  const float* A;
  int64_t lda;
  const float* b;
  float* X;
  int64_t ldx;
} mihs_problem;

/* mihs_solve_path for nprob independent problems sharing one λ list:
 * the problems run concurrently on internal streams (8 by default; the
 * environment variable MIHS_BATCH_STREAMS sets 2 … 32) forked from and
 * joined back into `stream`; problems whose steps use the cooperative grid
 * form of AAb_Solver share one of them.  sds: HOST nprob × nlambda (row i
 * for problem i) or NULL; infos: HOST nprob × nlambda or NULL (then no
 * synchronisation).  Every problem must have its own handle.  Returns the
 * worst status. */
int mihs_solve_batched(int nprob, const mihs_problem* probs, int nlambda,
                       const double* lambdas, const double* sds,
                       const mihs_opts* opts, mihs_info* infos, void* stream);

/* Compensated refinement of chosen λ of a batch of paths, as
 * mihs_solve_refined (Algorithm 1 with the fp64 iterate and the double-float
 * gradient; the sketch only preconditions, Section 3.1, so the handle's SA
 * serves unchanged).  Where κ(AᵀA + λI) is large, the fp32 fixed point of
 * mihs_solve_batched lies far from x*(λ): at κ ≈ 1e6 a relative residual of
 * 1e-6 leaves a relative error near 1e-3, and no fp32 residual certifies
 * 1e-5.  For every problem i and every l with tols[l] > 0 this runs one
 * refined solve of (A_i, b_i, λ_l) warm-started from row l of X_i (fp32, e.g.
 * the result of mihs_solve_batched), stopping at the relative residual
 * tols[l] (or after opts->max_outer steps), and writes the fp32 rounding of
 * the fp64 solution back into that row.  Rows with tols[l] ≤ 0 are left as
 * they are.
 *   probs, nlambda, lambdas, sds  as mihs_solve_batched (sds NULL: each λ's
 *            sd estimated by Algorithm 4, which synchronises).
 *   tols     HOST array of nlambda target residuals (≤ 0: skip that λ).
 *   opts     eps_sub, max_inner, max_outer; tol, sd and warm_start are
 *            taken from tols, sds and the warm start above.
 *   infos    HOST nprob × nlambda or NULL: the entries of refined λ are
 *            overwritten (status, steps and residual of the refined solve),
 *            the others left unchanged; non-NULL makes the call synchronise.
 * Problems run concurrently on the internal streams of mihs_solve_batched
 * (those whose refined solves use the grid form of AAb_Solver one after
 * another on one of them), forked from and joined back into `stream`; the λ
 * of one problem run in order on its handle.  The first refinement on a
 * handle allocates its refinement workspace and one fp64 d-vector
 * (cudaMalloc).  Returns the worst status.  Errors: INVALID_ARG, CUDA, OOM,
 * TIMEOUT, NUMERIC. */
int mihs_refine_batched(int nprob, const mihs_problem* probs, int nlambda,
                        const double* lambdas, const double* sds, const double* tols,
                        const mihs_opts* opts, mihs_info* infos, void* stream);

/* ------------------------------------------------------------------------
 * Differentiation of the solution x(A, b, λ) = (AᵀA + λI)⁻¹Aᵀb.  The paper
 * does not differentiate the solve; these follow from differentiating the
 * normal equations (AᵀA + λI)x = Aᵀb of the ridge problem of Section 1:
 * with the adjoint v = (AᵀA + λI)⁻¹ḡ of an upstream gradient ḡ = ∂L/∂x and
 * the residual r = b − Ax,
 *   ∂L/∂A = r vᵀ − (Av) xᵀ,   ∂L/∂b = Av,   ∂L/∂λ = −xᵀv.
 * ---------------------------------------------------------------------- */

/* The gradients above for a given v, in one pass over A (reads A, writes dA).
 *   A, b   as in mihs_solve (n×d, leading dimension lda; b n).
 *   x, v   d-vectors (the solution and the adjoint).
 *   dA     optional n×d output, leading dimension ldda ≥ d.
 *   db     optional n-vector output.
 *   dlambda optional DEVICE double: −xᵀv accumulated in fp64.
 * b may be NULL only when dA is (then r is not needed).  All device memory,
 * enqueued on `stream`, no synchronisation, no allocation.
 * Errors: INVALID_ARG, CUDA. */
int mihs_backward_grads(const float* A, int64_t n, int64_t d, int64_t lda,
                        const float* b, const float* x, const float* v,
                        float* dA, int64_t ldda, float* db, double* dlambda,
                        void* stream);

/* Backward of mihs_solve: the adjoint system (AᵀA + λI)v = ḡ is solved by
 * Algorithm 1 with the handle's SA (the Hessian is symmetric, so the sketch
 * of the forward solve preconditions it as well; the stop test is
 * ‖ḡ − (AᵀA + λI)v‖ ≤ tol·‖ḡ‖), then mihs_backward_grads runs.
 *   gx     d-vector ḡ.
 *   v      d-vector output (the adjoint; its input value is the starting
 *          point when opts->warm_start, else ignored).
 *   other arguments as in mihs_solve and mihs_backward_grads.
 * The adjoint solve has its own cached graph in the handle, so forward and
 * backward solves that alternate do not rebuild each other's graphs.
 * Returns like mihs_solve: with info non-NULL the status of the adjoint
 * solve (the gradients are written in every case). */
int mihs_backward(mihs_sketch_t sk, const float* A, int64_t lda, const float* b,
                  double lambda, const float* x, const float* gx,
                  const mihs_opts* opts, float* v, float* dA, int64_t ldda,
                  float* db, double* dlambda, mihs_info* info, void* stream);

/* mihs_backward with the adjoint solved by compensated refinement (as in
 * mihs_solve_refined): x (the solution, e.g. from mihs_solve_refined) and v
 * (the adjoint: output, and the starting point when opts->warm_start) are
 * DEVICE double arrays.  For adjoint right-hand sides whose fp32 residual
 * floor (≈ κ(H)·u₃₂·‖ḡ‖ at worst) is above the wanted tolerance.  The
 * gradients stay fp32 and are formed from x and v rounded to fp32.  The
 * first refined solve on a handle allocates its workspace (cudaMalloc).
 * Errors and return value as mihs_backward. */
int mihs_backward_refined(mihs_sketch_t sk, const float* A, int64_t lda,
                          const float* b, double lambda, const double* x,
                          const float* gx, const mihs_opts* opts, double* v,
                          float* dA, int64_t ldda, float* db, double* dlambda,
                          mihs_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Dual M-IHS (Algorithm 2) for n ≤ d: M-IHS on the dual problem
 * ν* = argmin ½‖Aᵀν‖² + (λ/2)‖ν‖² − ⟨b, ν⟩ (Eq. intro_dual) with the sketch
 * taken along the d coordinates, SAᵀ (m × n), and x* = Aᵀν* (Eq.
 * dual_relation).  Each step: g = b − AAᵀν − λν (two passes over A),
 * Δν = AAb_Solver(SAᵀ, g, λ, ε_sub), ν⁺ = ν + αΔν + β(ν − ν⁻) with
 * β = sd/m, α = (1 − β)² (Theorem 1 / Corollary 3 hold for the dual form).
 * A is n × d row-major (lda ≥ d, a multiple of 4, 16-byte aligned rows),
 * 1 ≤ n ≤ 2048, n ≤ d.
 * ---------------------------------------------------------------------- */
typedef struct mihs_dual_s* mihs_dual_t;

/* Sketch Aᵀ: a d × n transposed copy of A is formed in stream-ordered
 * scratch, then sketched along its d rows by `family` with m ≤ d rows.  The
 * handle owns SAᵀ and the workspace of mihs_solve_dual.
 * Errors: INVALID_ARG, CUDA, OOM. */
int mihs_dual_sketch(const float* A, int64_t n, int64_t d, int64_t lda,
                     int family, int64_t m, uint64_t seed, void* stream,
                     mihs_dual_t* out);
/* Recompute SAᵀ for a new A of the handle's shape. */
int mihs_dual_resketch(mihs_dual_t dk, const float* A, int64_t lda,
                       uint64_t seed, void* stream);
/* Copy SAᵀ (m × n) into dst (device, leading dimension ldd ≥ n). */
int mihs_dual_copy(mihs_dual_t dk, float* dst, int64_t ldd, void* stream);
int mihs_dual_destroy(mihs_dual_t dk);

/* The dual gradient step on its own: g = b − A(Aᵀν) − λν (n-vectors).
 * Allocates stream-ordered scratch for Aᵀν and its row-split partials. */
int mihs_gradient_dual(const float* A, int64_t n, int64_t d, int64_t lda,
                       const float* b, const float* nu, double lambda,
                       float* g, void* stream);
/* x = Aᵀν (d-vector, 16-byte aligned).  Allocates stream-ordered scratch
 * for the row-split partials (summed in a fixed order). */
int mihs_dual_recover(const float* A, int64_t n, int64_t d, int64_t lda,
                      const float* nu, float* x, void* stream);

/* Algorithm 2 with the handle's SAᵀ.  nu: DEVICE n-vector, ν¹ on entry if
 * opts->warm_start (else zeroed), the dual solution on exit; x: optional
 * DEVICE d-vector receiving Aᵀν.  The stop test is ‖g‖ ≤ tol·‖b‖.  opts,
 * info and the return value as in mihs_solve (sd ≤ 0: Algorithm 4 on SAᵀ). */
int mihs_solve_dual(mihs_dual_t dk, const float* A, int64_t lda,
                    const float* b, double lambda, const mihs_opts* opts,
                    float* x, float* nu, mihs_info* info, void* stream);

/* Trace of the last solve on this handle: the relative residual
 * ‖g(xⁱ)‖/‖Aᵀb‖ of every gradient step (i = 0, 1, …, at most 1024 entries)
 * into the HOST array host_out[0..cap), the number written in *count.
 * Synchronises the device. */
int mihs_solve_history(mihs_sketch_t sk, float* host_out, int cap, int* count);

#ifdef __cplusplus
}
#endif

#endif /* MIHS_H */
