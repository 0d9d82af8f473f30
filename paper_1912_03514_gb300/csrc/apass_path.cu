// Gradient A-pass for a λ-path: G[l] = Aᵀ(b − A·X[l]) for up to 16 iterates
// X[l] (one per λ_l) in ONE pass over A (Algorithm 1's gradient step, run for
// every λ of the path at once; A, b and the sketch are shared by the path,
// only λ, the iterate and β/α differ).  Streaming A once for 16 iterates
// turns the pass from HBM-bound (1 FMA per 4 bytes, two for the pass) into
// FP32-bound (32 FMAs per element): a register-tiled SIMT contraction whose
// operands come from shared memory.
//
// Block: one producer warp streams blocks of kRows = 16 rows of A into a
// two-stage shared-memory ring (one bulk copy per row, row pitch dpad + 4
// floats so that the phase-1 reads are free of bank conflicts); eight
// consumer warps then, per stage:
//   phase 1  R[16 rows][16 λ] = A_stage · Xᵀ — the 256 threads split the
//            columns into 32 interleaved K-groups (warp w, lane bits 3–4) of
//            float4 columns 4k + 128i, each thread holding 2 rows × 16 λ
//            accumulators; X (λ-major, 16 × dpad) sits in shared memory and is
//            read as broadcast float4s.  Partials are summed over the four
//            lane groups with shuffles and over the eight warps through
//            shared memory, then r = b − R.
//   phase 2  each thread owns 4 columns × 16 λ accumulators of Aᵀr over its
//            share of the rows (for d < 1024 several threads share a column
//            group and split the rows; they are summed at the end).
// Per-block column sums go to partials[block][l][j]; a finalize kernel adds
// them in a fixed order and subtracts λ_l·X[l].
#include "internal.h"

namespace mihs {

namespace {

constexpr int kL = 16;          // iterates per pass
constexpr int kRows = 16;       // rows per stage
constexpr int kStagesPath = 2;
constexpr int kConsumers = 8;   // consumer warps
constexpr int kPathThreads = (kConsumers + 1) * 32;
constexpr int kPathMaxD = 1024;

__device__ int g_apass_path_error = 0;

struct PathSmem {
  // offsets in floats from the dynamic shared-memory base
  size_t ring, xs, rpart, rfull, bars;
};

__host__ __device__ inline int path_pitch(int dpad) { return dpad + 4; }

// Threads per column group in phase 2 (they split the stage's rows).
__host__ __device__ inline int path_rsub(int dpad) {
  const int ngroups = dpad >> 2;
  return ngroups >= 256 ? 1 : 256 / ngroups;
}

__host__ __device__ inline PathSmem path_layout(int dpad) {
  PathSmem L;
  L.ring = 0;
  // the ring is reused at the end to sum the phase-2 row subsets
  size_t ring = (size_t)kStagesPath * kRows * path_pitch(dpad);
  const size_t red = (size_t)path_rsub(dpad) * kL * dpad;
  if (red > ring) ring = red;
  L.xs = L.ring + ring;
  L.rpart = L.xs + (size_t)kL * dpad;
  L.rfull = L.rpart + (size_t)kConsumers * kRows * kL;
  L.bars = L.rfull + (size_t)kRows * kL;
  return L;
}

__host__ inline size_t path_smem_bytes(int dpad) {
  return path_layout(dpad).bars * sizeof(float) + 2 * kStagesPath * sizeof(uint64_t);
}

template <int CH>
__global__ void __launch_bounds__(kPathThreads, 1)
apass_path_kernel(const float* __restrict__ A, int n, int d, long long lda, const float* __restrict__ b,
                  const float* __restrict__ X, long long ldx, int nl, float* __restrict__ partials, int dpad,
                  int rows_per_cta, const int* __restrict__ all_done) {
  if (all_done != nullptr && *all_done) return;  // every λ of the path has stopped
  extern __shared__ __align__(128) float sm[];
  const PathSmem L = path_layout(dpad);
  const int pitch = path_pitch(dpad);
  float* ring = sm + L.ring;
  float* xs = sm + L.xs;
  float* rpart = sm + L.rpart;
  float* rfull = sm + L.rfull;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* empty = full + kStagesPath;
  __shared__ int issued;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min((long long)n, r0 + rows_per_cta);
  const int nst = r1 > r0 ? (int)((r1 - r0 + kRows - 1) / kRows) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesPath; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumers);
    }
    issued = 0;
    fence_mbar_init();
  }
  // X, λ-major and zero beyond nl and d.
  for (int i = threadIdx.x; i < kL * dpad; i += kPathThreads) {
    const int l = i / dpad, j = i - l * dpad;
    xs[i] = (l < nl && j < d) ? X[(long long)l * ldx + j] : 0.f;
  }
  __syncthreads();

  if (warp == kConsumers) {  // producer: one bulk copy per row of the stage
    for (int it = 0; it < nst; ++it) {
      const int s = it % kStagesPath;
      const uint32_t ph = (uint32_t)(it / kStagesPath) & 1u;
      bool ok = true;
      if (it >= kStagesPath) {
        if (lane == 0) ok = mbar_wait(&empty[s], ph ^ 1u, kWaitLimitNs);
        ok = __shfl_sync(0xffffffffu, ok, 0);
      }
      if (!ok) {
        if (lane == 0) atomicExch(&g_apass_path_error, MIHS_ERR_TIMEOUT);
        break;
      }
      const long long row0 = r0 + (long long)it * kRows;
      const int rows = (int)min((long long)kRows, r1 - row0);
      const uint32_t row_bytes = (uint32_t)dpad * 4u;
      if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)rows * row_bytes);
      __syncwarp();
      if (lane < rows)
        bulk_copy_g2s(ring + ((size_t)s * kRows + lane) * pitch, A + (row0 + lane) * lda, row_bytes, &full[s]);
      if (lane == 0) *(volatile int*)&issued = it + 1;
    }
    return;
  }

  // ---- consumers
  const int tid = threadIdx.x;            // 0..255
  const int kg = warp * 4 + (lane >> 3);  // K-group 0..31
  const int rl = lane & 7;                // rows rl and rl + 8 of the stage
  // phase-2 mapping: column group cg (4 columns), row subset rs
  const int ngroups = dpad >> 2;          // ≤ 256
  const int rsub = path_rsub(dpad);
  const int cg = tid % ngroups, rs = tid / ngroups;
  const bool p2 = rs < rsub && cg < ngroups;
  float acc2[4][kL];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int l = 0; l < kL; ++l) acc2[q][l] = 0.f;

  int consumed = 0;
  for (int it = 0; it < nst; ++it) {
    const int s = it % kStagesPath;
    const uint32_t ph = (uint32_t)(it / kStagesPath) & 1u;
    const long long row0 = r0 + (long long)it * kRows;
    const int rows = (int)min((long long)kRows, r1 - row0);
    if (!mbar_wait(&full[s], ph, kWaitLimitNs)) {
      atomicExch(&g_apass_path_error, MIHS_ERR_TIMEOUT);
      break;
    }
    const float* st = ring + (size_t)s * kRows * pitch;
    // phase 1: 2 rows × 16 λ over this thread's K-group
    float acc1[2][kL];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int l = 0; l < kL; ++l) acc1[q][l] = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int c = 4 * kg + 128 * i;
      if (c < dpad) {
        // rows beyond `rows` hold stale data: their products are discarded below
        float4 a0 = *reinterpret_cast<const float4*>(st + (size_t)rl * pitch + c);
        float4 a1 = *reinterpret_cast<const float4*>(st + (size_t)(rl + 8) * pitch + c);
        if (c + 4 > d) {  // the copied padding of a ragged row may hold anything
          if (c + 1 >= d) a0.y = a1.y = 0.f;
          if (c + 2 >= d) a0.z = a1.z = 0.f;
          a0.w = a1.w = 0.f;
        }
#pragma unroll
        for (int l = 0; l < kL; ++l) {
          const float4 xv = *reinterpret_cast<const float4*>(xs + (size_t)l * dpad + c);
          acc1[0][l] = fmaf(a0.x, xv.x, fmaf(a0.y, xv.y, fmaf(a0.z, xv.z, fmaf(a0.w, xv.w, acc1[0][l]))));
          acc1[1][l] = fmaf(a1.x, xv.x, fmaf(a1.y, xv.y, fmaf(a1.z, xv.z, fmaf(a1.w, xv.w, acc1[1][l]))));
        }
      }
    }
    // sum over the four lane groups of the warp (lane bits 3 and 4)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int l = 0; l < kL; ++l) {
        float v = acc1[q][l];
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        acc1[q][l] = v;
      }
    if ((lane >> 3) == 0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float4* dst = reinterpret_cast<float4*>(rpart + ((size_t)warp * kRows + rl + 8 * q) * kL);
#pragma unroll
        for (int l4 = 0; l4 < kL / 4; ++l4)
          dst[l4] = make_float4(acc1[q][4 * l4], acc1[q][4 * l4 + 1], acc1[q][4 * l4 + 2], acc1[q][4 * l4 + 3]);
      }
    }
    named_sync(1, kConsumers * 32);
    {  // r = b − Σ_warps R, one (row, λ) per thread, in a fixed order
      const int row = tid >> 4, l = tid & (kL - 1);
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < kConsumers; ++w) t += rpart[((size_t)w * kRows + row) * kL + l];
      const float bi = (row < rows && b != nullptr) ? __ldg(b + row0 + row) : 0.f;
      rfull[row * kL + l] = row < rows ? bi - t : 0.f;  // padded rows contribute nothing
    }
    named_sync(1, kConsumers * 32);
    // phase 2: acc2[q][l] += A[row][4cg + q] · r[row][l] over this thread's rows
    if (p2) {
      for (int row = rs; row < rows; row += rsub) {
        const float4 a = *reinterpret_cast<const float4*>(st + (size_t)row * pitch + 4 * cg);
        const float4* rr = reinterpret_cast<const float4*>(rfull + row * kL);
#pragma unroll
        for (int l4 = 0; l4 < kL / 4; ++l4) {
          const float4 r4 = rr[l4];
          const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc2[0][4 * l4 + k] = fmaf(a.x, rv[k], acc2[0][4 * l4 + k]);
            acc2[1][4 * l4 + k] = fmaf(a.y, rv[k], acc2[1][4 * l4 + k]);
            acc2[2][4 * l4 + k] = fmaf(a.z, rv[k], acc2[2][4 * l4 + k]);
            acc2[3][4 * l4 + k] = fmaf(a.w, rv[k], acc2[3][4 * l4 + k]);
          }
        }
      }
    }
    __syncwarp();  // the warp's reads of the stage are done
    if (lane == 0) mbar_arrive(&empty[s]);
    consumed = it + 1;
  }
  if (consumed < nst && tid == 0) {
    // Aborted: let the copies already issued land before the block exits.
    const int iss = *(volatile int*)&issued;
    for (int it = consumed; it < iss; ++it)
      if (!mbar_wait(&full[it % kStagesPath], (uint32_t)(it / kStagesPath) & 1u, kWaitLimitNs)) break;
  }
  named_sync(1, kConsumers * 32);
  // Sum the row subsets (fixed order) through the ring memory, then write.
  float* red = ring;  // rsub × kL × dpad floats (the ring region is sized for it)
  float* out = partials + (size_t)blockIdx.x * kL * dpad;
  if (rsub == 1) {
    if (p2)
#pragma unroll
      for (int l = 0; l < kL; ++l)
        *reinterpret_cast<float4*>(out + (size_t)l * dpad + 4 * cg) =
            make_float4(acc2[0][l], acc2[1][l], acc2[2][l], acc2[3][l]);
  } else {
    if (p2)
#pragma unroll
      for (int l = 0; l < kL; ++l)
        *reinterpret_cast<float4*>(red + ((size_t)rs * kL + l) * dpad + 4 * cg) =
            make_float4(acc2[0][l], acc2[1][l], acc2[2][l], acc2[3][l]);
    named_sync(1, kConsumers * 32);
    for (int i = tid; i < kL * dpad; i += kConsumers * 32) {
      float t = 0.f;
      for (int q = 0; q < rsub; ++q) t += red[(size_t)q * kL * dpad + i];
      out[i] = t;
    }
  }
}

// G[l][j] = Σ_p partials[p][l][j] − λ_l·X[l][j] (fixed order), l < nl.
__global__ void apass_path_finalize_kernel(const float* __restrict__ partials, int P, int d, int dpad,
                                           const float* __restrict__ X, long long ldx, PathScalars sc,
                                           float* __restrict__ G, long long ldg, const int* __restrict__ all_done) {
  if (all_done != nullptr && *all_done) return;
  const int l = blockIdx.y;
  if (l >= sc.nl) return;
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < d)
    for (int p = grp; p < P; p += 8) s += partials[((size_t)p * kL + l) * dpad + j];
  red[grp][lane] = s;
  __syncthreads();
  if (grp == 0 && j < d) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    G[(long long)l * ldg + j] = t - (X != nullptr ? sc.lam[l] * X[(long long)l * ldx + j] : 0.f);
  }
}

}  // namespace

int apass_path_num_partials(int64_t n) {
  const int64_t by_rows = (n + kRows - 1) / kRows;
  int64_t P = num_sms();
  if (P > by_rows) P = by_rows;
  return (int)(P < 1 ? 1 : P);
}

int apass_path_max_d() { return kPathMaxD; }

int launch_apass_path(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, const float* X,
                      int64_t ldx, int nl, float* partials, const int* all_done, cudaStream_t s) {
  const int64_t dpad = apass_dpad(d);
  if (d > kPathMaxD || nl < 1 || nl > kL) {
    set_error("path A-pass: d=%lld (max %d) or nl=%d (1..%d) unsupported", (long long)d, kPathMaxD, nl, kL);
    return MIHS_ERR_UNSUPPORTED;
  }
  const int P = apass_path_num_partials(n);
  const int rows_per_cta = (int)round_up((n + P - 1) / P, kRows);
  const size_t smem = path_smem_bytes((int)dpad);
  const int ch = (int)((dpad + 127) / 128);
  const void* fn;
  if (ch <= 1) fn = (const void*)&apass_path_kernel<1>;
  else if (ch <= 2) fn = (const void*)&apass_path_kernel<2>;
  else if (ch <= 4) fn = (const void*)&apass_path_kernel<4>;
  else fn = (const void*)&apass_path_kernel<8>;
  MIHS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int n32 = (int)n, d32 = (int)d, dp32 = (int)dpad;
  long long lda64 = lda, ldx64 = ldx;
  void* args[] = {(void*)&A, &n32, &d32, &lda64, (void*)&b, (void*)&X, &ldx64, &nl,
                  (void*)&partials, &dp32, (void*)&rows_per_cta, (void*)&all_done};
  timing_begin(kTimerApassPath, s);
  MIHS_CUDA_TRY(cudaLaunchKernel(fn, dim3(P), dim3(kPathThreads), args, smem, s));
  timing_end(kTimerApassPath, s);
  count_launch();
  return MIHS_OK;
}

int launch_apass_path_finalize(const float* partials, int P, int64_t d, const float* X, int64_t ldx,
                               const PathScalars& sc, float* G, int64_t ldg, const int* all_done,
                               cudaStream_t s) {
  apass_path_finalize_kernel<<<dim3((unsigned)((d + 31) / 32), (unsigned)sc.nl), 256, 0, s>>>(
      partials, P, (int)d, (int)apass_dpad(d), X, ldx, sc, G, ldg, all_done);
  MIHS_CHECK_LAUNCH();
  count_launch();
  return MIHS_OK;
}

int apass_path_device_error(int* code) {
  int v = 0, z = 0;
  MIHS_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_apass_path_error, sizeof(int)));
  MIHS_CUDA_TRY(cudaMemcpyToSymbol(g_apass_path_error, &z, sizeof(int)));
  *code = v;
  return MIHS_OK;
}

}  // namespace mihs
