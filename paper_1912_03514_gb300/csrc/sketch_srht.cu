// Subsampled randomized Hadamard transform (Lemma 3, case iii):
//     SA = √(n_p/m) · P · (H_{n_p}/√n_p) · D · A = (1/√m) · P · H_{n_p} · D · A,
// n_p = 2^⌈log₂ n⌉ with A zero-padded, D = diag(±1), P = m rows of H_{n_p}
// sampled uniformly with replacement.
//
// Only the m sampled rows of H·D·A are needed.  With n_p = B·(n_p/B) the
// Sylvester matrix factors as H_{n_p} = H_{n_p/B} ⊗ H_B, so for a sampled row
// r = (r_hi, r_lo):
//     (H·D·A)[r] = Σ_blk (−1)^popc(r_hi ∧ blk) · (H_B · D·A[blk·B : (blk+1)·B])[r_lo].
// Each thread block therefore streams B-row blocks of a 32-column slice of A,
// applies the length-B fast Walsh–Hadamard transform in registers and shared
// memory (two radix-32 register stages around one shared-memory transpose),
// and adds the signed sampled rows into an m×32 accumulator kept in shared
// memory.  A is read once (O(nd log B) additions on the SIMT pipes); the
// cross-block combine costs O(m·d·n_p/B).
//
// Pipelined form (srht_tma_kernel, n > 256 with 16-byte aligned rows): B =
// 512, a producer warp loads each 512-row × 32-column unit with two TMA
// tile loads into a two-deep shared-memory ring (rows past n read as zeros),
// and 16 consumer warps transform one unit in place while the next one is in
// flight.  Blocks of H·D·A that lie wholly in the zero padding (rows ≥ n) are
// skipped: they add nothing.
#include <cmath>
#include <cstdlib>

#include "internal.h"

namespace mihs {

namespace {

constexpr int kW = 32;          // columns per slice (one warp lane per column)
constexpr int kThreads = 512;   // 16 warps
constexpr int kWarps = kThreads / 32;
constexpr int kMaxLB = 10;      // block length B = 2^LB ≤ 1024

// signs[w] bit t = 1 when D_{32w+t} = −1 (counter (j,0,2,0), w0 odd);
// rows[i] = ⌊w0 / 2^(32−L)⌋ from counter (i,0,3,0).
__global__ void srht_prep_kernel(int n, int m, int L, uint32_t k0, uint32_t k1,
                                 uint32_t* __restrict__ signs, int* __restrict__ rows) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nwords = (n + 31) / 32;
  if (idx < nwords) {
    uint32_t word = 0;
    for (int t = 0; t < 32; ++t) {
      const int j = 32 * idx + t;
      if (j < n) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)j, 0u, kTagSrhtSigns, 0u), k0, k1);
        word |= (w.x & 1u) << t;
      }
    }
    signs[idx] = word;
  }
  if (idx < m) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)idx, 0u, kTagSrhtRows, 0u), k0, k1);
    rows[idx] = L > 0 ? (int)(w.x >> (32 - L)) : 0;
  }
}

template <int N>
__device__ __forceinline__ void fwht_reg(float (&x)[N]) {
#pragma unroll
  for (int h = 1; h < N; h <<= 1) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if ((i & h) == 0) {
        const float a = x[i], b = x[i + h];
        x[i] = a + b;
        x[i + h] = a - b;
      }
    }
  }
}

struct SrhtArgs {
  const float* A;
  int n, d;
  long long lda;
  int m;
  int LB;               // log2 B
  int nblk;             // n_p / B
  long long units;      // column slices × nblk
  const uint32_t* signs;
  const int* rows;
  float* partial;       // [gridDim.x][smax][m][kW]
  int smax;
  int acc_in_smem;
};

template <int L1, int L2>
__global__ void __launch_bounds__(kThreads, 1) srht_block_kernel(const SrhtArgs a) {
  constexpr int N1 = 1 << L1, N2 = 1 << L2, B = N1 * N2;
  extern __shared__ float4 smem4[];
  float* Y = reinterpret_cast<float*>(smem4);  // B × kW
  int* rlo = reinterpret_cast<int*>(Y + B * kW);
  int* rhi = rlo + a.m;
  float* acc_s = reinterpret_cast<float*>(rhi + a.m);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const long long u0 = (long long)blockIdx.x * a.units / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * a.units / gridDim.x;
  if (u0 >= u1) return;
  for (int i = tid; i < a.m; i += kThreads) {
    const int r = a.rows[i];
    rlo[i] = r & (B - 1);
    rhi[i] = r >> a.LB;
  }
  const size_t slot_elems = (size_t)a.m * kW;
  float* part_base = a.partial + (size_t)blockIdx.x * a.smax * slot_elems;
  int slot = 0;
  float* acc = a.acc_in_smem ? acc_s : part_base;
  for (size_t e = tid; e < slot_elems; e += kThreads) acc[e] = 0.f;
  long long cur_slice = u0 / a.nblk;
  __syncthreads();

  for (long long u = u0; u < u1; ++u) {
    const long long slice = u / a.nblk;
    const int blk = (int)(u - slice * a.nblk);
    if (slice != cur_slice) {  // flush the finished slice into its slot
      float* dst = part_base + (size_t)slot * slot_elems;
      if (a.acc_in_smem) {
        for (size_t e = tid; e < slot_elems; e += kThreads) {
          dst[e] = acc[e];
          acc[e] = 0.f;
        }
      }
      ++slot;
      if (!a.acc_in_smem) {
        acc = part_base + (size_t)slot * slot_elems;
        for (size_t e = tid; e < slot_elems; e += kThreads) acc[e] = 0.f;
      }
      cur_slice = slice;
      __syncthreads();
    }
    const int c = (int)slice * kW + lane;
    const long long rbase = (long long)blk * B;

    // Stage 1: transform over the high L1 bits of the in-block row index.
    for (int t = warp; t < N2; t += kWarps) {
      float x[N1];
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const long long row = rbase + t + (k << L2);
        float v = 0.f;
        if (row < a.n && c < a.d) {
          v = __ldcs(a.A + row * a.lda + c);
          if ((__ldg(a.signs + (row >> 5)) >> (row & 31)) & 1u) v = -v;
        }
        x[k] = v;
      }
      fwht_reg<N1>(x);
#pragma unroll
      for (int k = 0; k < N1; ++k) Y[(t + (k << L2)) * kW + lane] = x[k];
    }
    __syncthreads();
    // Stage 2: transform over the low L2 bits.
    for (int t = warp; t < N1; t += kWarps) {
      float y[N2];
#pragma unroll
      for (int k = 0; k < N2; ++k) y[k] = Y[((t << L2) + k) * kW + lane];
      fwht_reg<N2>(y);
#pragma unroll
      for (int k = 0; k < N2; ++k) Y[((t << L2) + k) * kW + lane] = y[k];
    }
    __syncthreads();
    // Signed sampled rows into the accumulator.
    for (int i = warp; i < a.m; i += kWarps) {
      const float yv = Y[rlo[i] * kW + lane];
      acc[(size_t)i * kW + lane] += (__popc(rhi[i] & blk) & 1) ? -yv : yv;
    }
    __syncthreads();
  }
  if (a.acc_in_smem) {
    float* dst = part_base + (size_t)slot * slot_elems;
    for (size_t e = tid; e < slot_elems; e += kThreads) dst[e] = acc[e];
  }
}

__device__ int g_srht_error = 0;

constexpr int kTB = 512;                        // rows per unit of the pipelined form
constexpr int kTL1 = 5, kTL2 = 4;               // B = 2^5 · 2^4
constexpr int kTBoxRows = 256;                  // rows per TMA tile load
constexpr int kTNBuf = 2;                       // ring depth
constexpr uint32_t kTUnitBytes = kTB * kW * 4;  // 64 KB
constexpr int kTCons = 16;                      // consumer warps (one per stage-1 row class)
constexpr int kTThreads = (kTCons + 1) * 32;    // + the producer warp

__host__ __device__ constexpr size_t srht_tma_smem(int m, bool acc_in_smem) {
  return 128 /*align*/ + (size_t)kTNBuf * kTUnitBytes + 64 /*barriers, flags*/ + 8 * (size_t)m +
         (acc_in_smem ? (size_t)m * kW * 4 : 0);
}

// kTCons consumer warps and one producer; the m × 32 accumulator lives in
// shared memory (acc_in_smem) or in the block's global partial slot.  (A
// register accumulator, 8 consumer warps owning m/8 rows each, measured
// slower: the sampled-row gathers then form one long dependent chain per
// warp.)
__global__ void __launch_bounds__(kTThreads, 1) srht_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                 const SrhtArgs a) {
  constexpr int NC = kTCons, NT = NC * 32;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);  // TMA destinations: 128-byte aligned
  float* ring = reinterpret_cast<float*>(base);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)kTNBuf * kTUnitBytes);
  uint64_t* empty = full + kTNBuf;
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(empty + kTNBuf);
  // sampled row r: {offset of r_lo = r mod B in a unit (floats), r_hi = ⌊r/B⌋}
  int2* rows_s = reinterpret_cast<int2*>(base + (size_t)kTNBuf * kTUnitBytes + 64);
  float* acc_s = reinterpret_cast<float*>(rows_s + a.m);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const long long u0 = (long long)blockIdx.x * a.units / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * a.units / gridDim.x;
  if (u0 >= u1) return;
  if (tid == 0) {
    for (int q = 0; q < kTNBuf; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    *abort_flag = 0u;
    fence_mbar_init();
  }
  for (int i = tid; i < a.m; i += blockDim.x) {
    const int r = a.rows[i];
    rows_s[i] = make_int2((r & (kTB - 1)) * kW, r >> a.LB);
  }
  __syncthreads();

  if (warp == NC) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      for (long long u = u0; u < u1; ++u) {
        const int j = (int)(u - u0), q = j % kTNBuf;
        if (j >= kTNBuf && !mbar_wait(&empty[q], ((uint32_t)(j / kTNBuf) & 1u) ^ 1u, kWaitLimitNs)) {
          atomicExch(&g_srht_error, MIHS_ERR_TIMEOUT);
          break;
        }
        const long long slice = u / a.nblk;
        const int blk = (int)(u - slice * a.nblk);
        float* dst = ring + (size_t)q * (kTB * kW);
        mbar_arrive_expect_tx(&full[q], kTUnitBytes);
        for (int h = 0; h < kTB / kTBoxRows; ++h)
          tma_load_2d(dst + h * kTBoxRows * kW, &tmap, (int)slice * kW, blk * kTB + h * kTBoxRows, &full[q]);
      }
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  constexpr int N1 = 1 << kTL1, N2 = 1 << kTL2;
  const size_t slot_elems = (size_t)a.m * kW;
  float* part_base = a.partial + (size_t)blockIdx.x * a.smax * slot_elems;
  int slot = 0;
  float* acc = a.acc_in_smem ? acc_s : part_base;
  for (size_t e = tid; e < slot_elems; e += NT) acc[e] = 0.f;
  long long cur_slice = u0 / a.nblk;
  const int nwords = (a.n + 31) >> 5;
  named_sync(1, NT);

  for (long long u = u0; u < u1; ++u) {
    const int j = (int)(u - u0), q = j % kTNBuf;
    const long long slice = u / a.nblk;
    const int blk = (int)(u - slice * a.nblk);
    if (slice != cur_slice) {  // flush the finished slice into its slot
      float* dst = part_base + (size_t)slot * slot_elems;
      if (a.acc_in_smem) {
        for (size_t e = tid; e < slot_elems; e += NT) {
          dst[e] = acc[e];
          acc[e] = 0.f;
        }
      }
      ++slot;
      if (!a.acc_in_smem) {
        acc = part_base + (size_t)slot * slot_elems;
        for (size_t e = tid; e < slot_elems; e += NT) acc[e] = 0.f;
      }
      cur_slice = slice;
      named_sync(1, NT);
    }
    // One thread waits (bounded) for the unit; every consumer takes its decision.
    if (tid == 0 && !mbar_wait(&full[q], (uint32_t)(j / kTNBuf) & 1u, kWaitLimitNs)) {
      atomicExch(&g_srht_error, MIHS_ERR_TIMEOUT);
      *abort_flag = 1u;
    }
    named_sync(1, NT);
    if (*abort_flag) return;
    float* Y = ring + (size_t)q * (kTB * kW);
    // D: word w of the unit's 16 sign words covers rows 32w … 32w + 31, so
    // row t + 16k (k = 2w + h) is bit t + 16h of word w: gathered into two
    // masks, bit w of neg_h = the sign of row t + 16(2w + h).
    const int wi = blk * (kTB / 32) + (lane & 15);
    const uint32_t sw = (lane < 16 && wi < nwords) ? __ldg(a.signs + wi) : 0u;

    // Stage 1 (with D): rows t + 16k, k = 0 … 31 (the high 5 bits of the row).
    for (int t = warp; t < N2; t += NC) {
      const uint32_t neg0 = __ballot_sync(0xffffffffu, (sw >> t) & 1u);
      const uint32_t neg1 = __ballot_sync(0xffffffffu, (sw >> (t + 16)) & 1u);
      float x[N1];
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const uint32_t nm = (k & 1) ? neg1 : neg0;
        const uint32_t flip = (nm << (31 - (k >> 1))) & 0x80000000u;
        x[k] = __uint_as_float(__float_as_uint(Y[(t + (k << kTL2)) * kW + lane]) ^ flip);
      }
      fwht_reg<N1>(x);
#pragma unroll
      for (int k = 0; k < N1; ++k) Y[(t + (k << kTL2)) * kW + lane] = x[k];
    }
    named_sync(1, NT);
    // Stage 2: rows 16t + k, k = 0 … 15 (the low 4 bits).
    for (int t = warp; t < N1; t += NC) {
      float y[N2];
#pragma unroll
      for (int k = 0; k < N2; ++k) y[k] = Y[((t << kTL2) + k) * kW + lane];
      fwht_reg<N2>(y);
#pragma unroll
      for (int k = 0; k < N2; ++k) Y[((t << kTL2) + k) * kW + lane] = y[k];
    }
    named_sync(1, NT);
    // Signed sampled rows into the accumulator: row r = (r_hi, r_lo) takes
    // entry r_lo of this block's transform with the sign (−1)^popc(r_hi ∧ blk).
    const float* Yl = Y + lane;
    float* accl = acc + lane;
#pragma unroll 4
    for (int i = warp; i < a.m; i += NC) {
      const int2 r = rows_s[i];
      const uint32_t flip = (uint32_t)__popc(r.y & blk) << 31;
      accl[(size_t)i * kW] += __uint_as_float(__float_as_uint(Yl[r.x]) ^ flip);
    }
    fence_async_shared();            // this thread's writes to the unit → before the next TMA write
    named_sync(1, NT);
    if (tid == 0) mbar_arrive(&empty[q]);
  }
  if (a.acc_in_smem) {
    float* dst = part_base + (size_t)slot * slot_elems;
    for (size_t e = tid; e < slot_elems; e += NT) dst[e] = acc[e];
  }
}

// SA[i][slice·32 + c] = (1/√m) Σ_b partial[b][slice − first_slice(b)][i][c],
// summed over the blocks b whose unit range meets the slice, in order of b.
__global__ void __launch_bounds__(256)
srht_reduce_kernel(const float* __restrict__ partial, int NB, int smax, long long units,
                   int nblk, int m, int d, float scale, float* __restrict__ SA, long long ldsa) {
  const int slice = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int c = slice * kW + lane;
  if (i >= m || c >= d) return;
  const long long s0 = (long long)slice * nblk, s1 = s0 + nblk;
  float s = 0.f;
  // Blocks b own units [⌊b·units/NB⌋, ⌊(b+1)·units/NB⌋): start one block below
  // the owner of unit s0 and stop past the slice, in order of b.
  int b = (int)((s0 * NB) / units);
  if (b > 0) --b;
  for (; b < NB; ++b) {
    const long long u0 = (long long)b * units / NB, u1 = (long long)(b + 1) * units / NB;
    if (u0 >= s1) break;
    if (u1 <= s0 || u0 >= u1) continue;
    const int slot = (int)(slice - u0 / nblk);
    s += partial[(((size_t)b * smax + slot) * m + i) * kW + lane];
  }
  SA[(long long)i * ldsa + c] = s * scale;
}

using KernelFn = void (*)(const SrhtArgs);

KernelFn pick_kernel(int LB) {
  switch (LB) {
    case 0: return srht_block_kernel<0, 0>;
    case 1: return srht_block_kernel<0, 1>;
    case 2: return srht_block_kernel<0, 2>;
    case 3: return srht_block_kernel<0, 3>;
    case 4: return srht_block_kernel<0, 4>;
    case 5: return srht_block_kernel<0, 5>;
    case 6: return srht_block_kernel<1, 5>;
    case 7: return srht_block_kernel<2, 5>;
    case 8: return srht_block_kernel<3, 5>;
    case 9: return srht_block_kernel<4, 5>;
    default: return srht_block_kernel<5, 5>;
  }
}

}  // namespace

int srht_device_error(int* code) {
  int v = 0, zero = 0;
  MIHS_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_srht_error, sizeof(int)));
  if (v != 0) MIHS_CUDA_TRY(cudaMemcpyToSymbol(g_srht_error, &zero, sizeof(int)));
  *code = v;
  return MIHS_OK;
}

int sketch_srht(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed,
                float* SA, int64_t ldsa, cudaStream_t s) {
  int L = 0;
  while ((1LL << L) < n) ++L;
  int dev_max = 0, dev = 0;
  MIHS_CUDA_TRY(cudaGetDevice(&dev));
  MIHS_CUDA_TRY(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // The pipelined form needs n > 256, TMA-compatible rows and room for its
  // ring (the accumulator goes to global memory when it does not fit too).
  static const bool force_plain = [] {
    const char* e = std::getenv("MIHS_SRHT_PLAIN");
    return e != nullptr && std::atoi(e) == 1;
  }();
  CUtensorMap tmap;
  const bool tma = !force_plain && L >= 9 && lda % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0 &&
                   srht_tma_smem((int)m, false) <= (size_t)dev_max &&
                   encode_tmap_2d_f32(&tmap, A, n, d, lda, kW, kTBoxRows, 128) == MIHS_OK;
  const int LB = tma ? 9 : (L < kMaxLB ? L : kMaxLB);
  const int B = 1 << LB;
  // n_p/B blocks of rows; the pipelined form skips those wholly past n.
  const int nblk = tma ? (int)((n + B - 1) / B) : (int)((1LL << L) / B);
  const int ncs = (int)((d + kW - 1) / kW);
  const long long units = (long long)ncs * nblk;
  int NB = num_sms();
  if (NB > units) NB = (int)units;
  // slots per block: slices met by its unit range
  int smax = 1;
  for (int b = 0; b < NB; ++b) {
    const long long u0 = (long long)b * units / NB, u1 = (long long)(b + 1) * units / NB;
    if (u1 > u0) {
      const int k = (int)((u1 - 1) / nblk - u0 / nblk + 1);
      if (k > smax) smax = k;
    }
  }
  bool acc_in_smem;
  size_t smem;
  if (tma) {
    acc_in_smem = srht_tma_smem((int)m, true) <= (size_t)dev_max;
    smem = srht_tma_smem((int)m, acc_in_smem);
  } else {
    const size_t base_smem = (size_t)B * kW * sizeof(float) + 2 * sizeof(int) * (size_t)m;
    const size_t acc_bytes = (size_t)m * kW * sizeof(float);
    acc_in_smem = base_smem + acc_bytes <= (size_t)dev_max;
    smem = base_smem + (acc_in_smem ? acc_bytes : 0);
  }
  if (smem > (size_t)dev_max) {
    set_error("srht: m=%lld needs %zu bytes of shared memory", (long long)m, smem);
    return MIHS_ERR_UNSUPPORTED;
  }

  StreamScratch scratch;
  const size_t nwords = (size_t)(n + 31) / 32;
  const size_t part_elems = (size_t)NB * smax * m * kW;
  int rc = scratch.alloc(sizeof(uint32_t) * nwords + sizeof(int) * (size_t)m +
                             sizeof(float) * part_elems + 64,
                         s);
  if (rc) return rc;
  float* partial = static_cast<float*>(scratch.p);
  uint32_t* signs = reinterpret_cast<uint32_t*>(partial + part_elems);
  int* rows = reinterpret_cast<int*>(signs + nwords);

  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int nprep = (int)((nwords > (size_t)m ? nwords : (size_t)m) + 255) / 256;
  srht_prep_kernel<<<nprep, 256, 0, s>>>((int)n, (int)m, L, k0, k1, signs, rows);
  MIHS_CHECK_LAUNCH();

  SrhtArgs a;
  a.A = A;
  a.n = (int)n;
  a.d = (int)d;
  a.lda = lda;
  a.m = (int)m;
  a.LB = LB;
  a.nblk = nblk;
  a.units = units;
  a.signs = signs;
  a.rows = rows;
  a.partial = partial;
  a.smax = smax;
  a.acc_in_smem = acc_in_smem ? 1 : 0;
  if (tma) {
    MIHS_CUDA_TRY(cudaFuncSetAttribute((const void*)srht_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    srht_tma_kernel<<<NB, kTThreads, smem, s>>>(tmap, a);
  } else {
    KernelFn fn = pick_kernel(LB);
    MIHS_CUDA_TRY(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fn<<<NB, kThreads, smem, s>>>(a);
  }
  MIHS_CHECK_LAUNCH();
  dim3 rg((unsigned)ncs, (unsigned)((m + 7) / 8));
  srht_reduce_kernel<<<rg, 256, 0, s>>>(partial, NB, smax, units, nblk, (int)m, (int)d,
                                        (float)(1.0 / std::sqrt((double)m)), SA, ldsa);
  MIHS_CHECK_LAUNCH();
  count_launch(3);
  return MIHS_OK;
}

}  // namespace mihs
