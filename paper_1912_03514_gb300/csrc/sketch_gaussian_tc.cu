// Gaussian sketch on the 5th-generation tensor cores (tcgen05, TMEM, TMA):
//     SA = S·A,  S_ij ~ N(0, 1/m)  (Lemma 3, case iv).
//
// GEMM orientation: D[M = 128 sketch rows][N = 256 columns of A] accumulates
// over K = rows of A.  The tf32 MMA reads both operands K-major, while A is
// stored with its columns contiguous, so per K-block of 32 rows:
//   * a TMA lane loads the 32×256 tile of A (fp32) into a staging ring;
//   * four transposer warps rewrite it K-major (one 128-byte row per column
//     of A, 16-byte chunks XOR-swizzled by row mod 8 — the canonical 128-byte
//     swizzle layout), rounding to tf32;
//   * sixteen generator warps write the 128×32 tile of S (Philox4x32-10 counter
//     (⌊k/4⌋, i, 0, 0), Box–Muller, rounded to tf32) in the same layout — S
//     never leaves shared memory;
//   * one thread issues four tcgen05.mma.kind::tf32 (K = 8 each) into a
//     128×256 fp32 accumulator in tensor memory and commits the operand stage
//     back to the producers.
// The blocks that share a tile of S (the same sketch rows and rows of A, one
// per 256-column tile of A) form one thread-block cluster: block r of the
// cluster generates only its slice of the tile's rows (a contiguous byte
// range of the swizzled layout) and pushes it into the other blocks' stage by
// bulk shared::cta → shared::cluster copies that complete on their `full`
// barrier, and every MMA commit arrives on the `empty` barrier of every block
// of the cluster (a stage is refilled once all of them have consumed it).
// So each element of S is generated once, not once per column tile of A.
// Rings: 3 operand stages (48 KB) and 2 staging stages (32 KB).  The K range is
// split across blocks (split-K); each block's accumulator goes to a partial
// buffer that a small kernel sums in a fixed order and scales by 1/√m.
// Every mbarrier wait is bounded; a wait that runs out records
// MIHS_ERR_TIMEOUT, the block still frees its tensor memory and returns.
// Operand precisions (the sketch only preconditions, Section 3.1): tf32
// (32 K per 128-byte row), bf16 (64 K) or fp8 e4m3 (128 K; A scaled by the
// power of two that puts max|A| in [128, 256) before rounding, the scale
// undone exactly in the reduction).
#include <cuda.h>

#include <cmath>
#include <cstdlib>
#include <mutex>

#include "internal.h"

namespace mihs {

namespace {

constexpr int TM = 128;          // sketch rows per tile (MMA M)
constexpr int TN = 256;          // columns of A per tile (MMA N)
constexpr int TK = 32;           // rows of A per TMA load (a tf32 stage: 4 MMAs of K = 8)
constexpr int kGenWarps = 16;    // S generators (warps 2–17); warps 2–5 then run the epilogue
constexpr int kTrWarps = 4;      // A transposers (warps 18–21)
constexpr int kThreads = (2 + kGenWarps + kTrWarps) * 32;  // warp 0: MMA, warp 1: TMA
constexpr uint32_t kSBytes = TM * TK * 4;       // one 128-row S tile: 16 KB
constexpr uint32_t kABytes = TK * TN * 4;       // one 32-row fp32 A tile: 32 KB

// Shape of one kernel variant.  PREC: 0 tf32 (32 K per 128-byte swizzled
// row), 1 bf16 (64 K), 2 fp8 e4m3 (128 K): all use the same layout and
// descriptors, and each MMA consumes 32 bytes of K.
// MT: sketch-row tiles per block (two TMEM accumulators of 256 columns when
// MT = 2, so that each staged and transposed A tile feeds twice the MMA
// work — the kernel is bound by shared-memory traffic, not by the MMA).
// Operand ring and staging ring (TMA → transposers) depths fill ≤ 227 KB.
template <int PREC, int MT>
struct TcCfg {
  static constexpr int KT = 32 << PREC;          // K rows per operand stage
  static constexpr int NSLOT = KT / TK;          // 32-row TMA loads per stage
  static constexpr uint32_t SBytes = MT * kSBytes;
  static constexpr uint32_t StageBytes = SBytes + kABytes;
  static constexpr int NSTAGE = MT == 1 ? (PREC > 0 ? 2 : 3) : 2;
  static constexpr int NSTG = MT == 1 ? (PREC > 0 ? 4 : 2) : 3;
  static constexpr uint32_t TmemCols = 256u * MT;
  static constexpr size_t Smem = (size_t)NSTAGE * StageBytes + (size_t)NSTG * kABytes + 1024 /*align*/ +
                                 256 /*barriers*/;
};

__device__ int g_gauss_tc_error = 0;

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // tcgen05 shared-memory matrix descriptor: start >> 4, leading/stride byte
  // offsets >> 4, descriptor version 1 (bit 46), 128-byte swizzle (mode 2).
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptors: D f32 (bits 4–5 = 1), A and B both K-major,
// N/8 at bit 17, M/16 at bit 24; operand format at bits 7–9 / 10–12:
// kind::tf32 takes tf32 (2), kind::f16 takes bf16 (1).
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | (0u << 15) | (0u << 16) |
                                ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (0u << 16) |
                                ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
// kind::f8f6f4 with both operands e4m3 (format 0).
constexpr uint32_t kIdescFp8 = (1u << 4) | (0u << 7) | (0u << 10) | (0u << 15) | (0u << 16) |
                               ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescBf16), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_fp8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescFp8), "r"(accumulate)
      : "memory");
}

// Four fp32 values → four e4m3 bytes (round to nearest even, saturating to
// ±448), the first in the lowest byte (the lowest K index).
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  uint16_t lo, hi;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Two fp32 values → one bf16x2 word (round to nearest even); `lo` lands in
// the low half (the lower K index).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Commit that arrives on the barrier at the same offset in every block of
// `mask` (the blocks of this cluster).
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// shared::cluster address of the same location in block `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// Bulk copy of `bytes` (multiple of 16) from this block's shared memory to a
// block of the cluster; completes `bytes` on the barrier `rbar` there.
__device__ __forceinline__ void bulk_copy_s2c(uint32_t rdst, uint32_t src, uint32_t bytes, uint32_t rbar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   rdst),
               "r"(src), "r"(bytes), "r"(rbar)
               : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }



// Box–Muller with CUDA's fast intrinsics (its results are rounded to tf32,
// 2⁻¹¹ relative, so the intrinsics' ~2⁻²¹ error is invisible): the same
// u1 = (⌊a/2⁸⌋+1)·2⁻²⁴, u2 = ⌊b/2⁸⌋·2⁻²⁴ as box_muller(); the angle is taken
// as 2π(u2 − ½) ∈ [−π, π), where the intrinsics are accurate, and the
// half-turn is undone by negating both outputs.
__device__ __forceinline__ float2 box_muller_fast(uint32_t a, uint32_t b) {
  const float u1 = (float)((a >> 8) + 1u) * 0x1p-24f;
  const float u2 = (float)(b >> 8) * 0x1p-24f;
  const float t = -2.0f * __logf(u1);
  const float r = t > 0.f ? t * rsqrtf(t) : 0.f;
  float sn, cs;
  __sincosf(6.283185307179586f * (u2 - 0.5f), &sn, &cs);
  return make_float2(-r * cs, -r * sn);
}

__device__ __forceinline__ uint32_t to_tf32(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

// 32 lanes × 32 consecutive columns of the accumulator → 32 registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct GaussTcArgs {
  int n, d, m;
  int rows_per_split;   // multiple of TK
  uint32_t k0, k1;      // Philox key
  float* part;          // [gridDim.z][m][dp]
  int dp;
  int cn;               // blocks per cluster (= column tiles of A, gridDim.x)
  const float* ascale;  // fp8: [0] = the power-of-two scale applied before rounding A, [1] = its inverse
};

// PREC 0: tf32 operands (kind::tf32, 32 K per stage); 1: S and A rounded to
// bf16 (kind::f16, 64 K per stage, two TMA loads of 32 rows); 2: S and the
// scaled A rounded to e4m3 (kind::f8f6f4, 128 K per stage, four loads).
// MT sketch-row tiles of 128 per block, one TMEM accumulator each.
template <int PREC, int MT>
__global__ void __launch_bounds__(kThreads, 1)
gauss_tc_kernel(const __grid_constant__ CUtensorMap tmap_a, const GaussTcArgs a) {
  using C = TcCfg<PREC, MT>;
  constexpr int KT = C::KT;
  constexpr int NSLOT = C::NSLOT;  // TMA loads (staging slots) per operand stage
  constexpr int NSTAGE = C::NSTAGE;
  constexpr int NSTG = C::NSTG;
  constexpr uint32_t kStageBytes = C::StageBytes;
  constexpr int MROWS = MT * TM;   // sketch rows of the block
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment for the 128-byte swizzle atoms.
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* stg = base + (size_t)NSTAGE * kStageBytes;           // staging ring
  uint64_t* full = reinterpret_cast<uint64_t*>(stg + (size_t)NSTG * kABytes);
  uint64_t* empty = full + NSTAGE;
  uint64_t* stg_full = empty + NSTAGE;
  uint64_t* stg_empty = stg_full + NSTG;
  uint64_t* accum = stg_empty + NSTG;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accum + 1);
  volatile uint32_t* gen_abort = tmem_holder + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * MROWS;          // first sketch row
  const int c0 = blockIdx.x * TN;             // first column of A
  const int kb0 = blockIdx.z * a.rows_per_split;
  const int kb1 = min(a.n, kb0 + a.rows_per_split);
  const int nkb = kb1 > kb0 ? (kb1 - kb0 + KT - 1) / KT : 0;

  const int cn = a.cn;
  const uint32_t crank = cn > 1 ? cluster_rank() : 0u;
  // This block's slice of the stage's S rows (contiguous bytes: row g of the
  // MT stacked swizzled tiles occupies bytes [128g, 128g + 128)).
  const int g_lo = (int)((MROWS * crank) / (uint32_t)cn), g_hi = (int)((MROWS * (crank + 1)) / (uint32_t)cn);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1 + kTrWarps);  // generator leader (+ peers' bytes), transposer warps
      mbar_init(&empty[s], cn);           // MMA commits of every block of the cluster
    }
    for (int s = 0; s < NSTG; ++s) {
      mbar_init(&stg_full[s], 1);                 // TMA expect_tx arrival
      mbar_init(&stg_empty[s], kTrWarps);
    }
    mbar_init(accum, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(C::TmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  if (cn > 1) cluster_sync_all();  // every block's barriers initialised before any remote access

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NSTAGE;
        const uint32_t ph = (uint32_t)(kb / NSTAGE) & 1u;
        if (!mbar_wait(&full[s], ph, kWaitLimitNs)) {
          atomicExch(&g_gauss_tc_error, MIHS_ERR_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t sS = smem_u32(base + (size_t)s * kStageBytes);
        const uint32_t sA = sS + C::SBytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          // Both operands K-major: 8-row atoms of 1024 B; each MMA covers 32
          // bytes of K (8 tf32 or 16 bf16 values).  Tile t of S (rows
          // 128t … 128t + 127) accumulates into TMEM columns 256t ….
          const uint64_t bd = smem_desc_sw128(sA + kk * 32, 16, 1024);
#pragma unroll
          for (int t = 0; t < MT; ++t) {
            const uint64_t ad = smem_desc_sw128(sS + t * kSBytes + kk * 32, 16, 1024);
            if constexpr (PREC == 2)
              mma_fp8(tmem + 256u * t, ad, bd, (kb > 0 || kk > 0) ? 1u : 0u);
            else if constexpr (PREC == 1)
              mma_bf16(tmem + 256u * t, ad, bd, (kb > 0 || kk > 0) ? 1u : 0u);
            else
              mma_tf32(tmem + 256u * t, ad, bd, (kb > 0 || kk > 0) ? 1u : 0u);
          }
        }
        if (cn > 1)
          mma_commit_mc(&empty[s], (uint16_t)((1u << cn) - 1u));
        else
          mma_commit(&empty[s]);
      }
      mma_commit(accum);  // fires when every MMA issued above has completed
      // Drain: the last rounds' commits of every block of the cluster have
      // arrived here before this block may exit (its barriers stay valid).
      for (int kb = nkb > NSTAGE ? nkb - NSTAGE : 0; kb < nkb; ++kb)
        if (!mbar_wait(&empty[kb % NSTAGE], (uint32_t)(kb / NSTAGE) & 1u, kWaitLimitNs)) {
          atomicExch(&g_gauss_tc_error, MIHS_ERR_TIMEOUT);
          break;
        }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ TMA loads of A
    if (lane == 0) {
      // load j covers rows kb0 + 32j … (NSLOT loads per operand stage)
      for (int j = 0; j < nkb * NSLOT; ++j) {
        const int s = j % NSTG;
        const uint32_t ph = (uint32_t)(j / NSTG) & 1u;
        if (j >= NSTG && !mbar_wait(&stg_empty[s], ph ^ 1u, kWaitLimitNs)) {
          atomicExch(&g_gauss_tc_error, MIHS_ERR_TIMEOUT);
          break;
        }
        mbar_arrive_expect_tx(&stg_full[s], kABytes);
        tma_load_2d(stg + (size_t)s * kABytes, &tmap_a, c0, kb0 + j * TK, &stg_full[s]);
      }
    }
    __syncwarp();
  } else if (warp >= 2 + kGenWarps) {
    // ------------------------------------------------ A transposers: staging → K-major
    const int tt = threadIdx.x - (2 + kGenWarps) * 32;  // 0..127: columns tt, tt + 128
    const float as = PREC == 2 ? a.ascale[0] : 1.f;
    bool stop = false;
    for (int kb = 0; kb < nkb && !stop; ++kb) {
      const int s = kb % NSTAGE;
      if (kb >= NSTAGE && !mbar_wait(&empty[s], ((uint32_t)(kb / NSTAGE) & 1u) ^ 1u, kWaitLimitNs)) {
        atomicExch(&g_gauss_tc_error, MIHS_ERR_TIMEOUT);
        break;
      }
      unsigned char* dstA = base + (size_t)s * kStageBytes + C::SBytes;
#pragma unroll
      for (int sl = 0; sl < NSLOT; ++sl) {
        const int j = kb * NSLOT + sl;
        const int q = j % NSTG;
        if (!mbar_wait(&stg_full[q], (uint32_t)(j / NSTG) & 1u, kWaitLimitNs)) {
          atomicExch(&g_gauss_tc_error, MIHS_ERR_TIMEOUT);
          stop = true;
          break;
        }
        const float* src = reinterpret_cast<const float*>(stg + (size_t)q * kABytes);  // [32 rows][256 cols]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = tt + 128 * h;
          unsigned char* row = dstA + (c >> 3) * 1024 + (c & 7) * 128;
          if constexpr (PREC == 2) {
            // 16-byte chunk ch = 2·sl + hh holds K = 16ch … 16ch + 15 as e4m3
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const float* r = src + (size_t)(16 * hh) * TN + c;
              uint4 v;
              v.x = pack_e4m3x4(r[0 * TN] * as, r[1 * TN] * as, r[2 * TN] * as, r[3 * TN] * as);
              v.y = pack_e4m3x4(r[4 * TN] * as, r[5 * TN] * as, r[6 * TN] * as, r[7 * TN] * as);
              v.z = pack_e4m3x4(r[8 * TN] * as, r[9 * TN] * as, r[10 * TN] * as, r[11 * TN] * as);
              v.w = pack_e4m3x4(r[12 * TN] * as, r[13 * TN] * as, r[14 * TN] * as, r[15 * TN] * as);
              const int ch = 2 * sl + hh;
              *reinterpret_cast<uint4*>(row + ((ch ^ (c & 7)) << 4)) = v;
            }
          } else if constexpr (PREC == 1) {
            // 16-byte chunk ch = 4·sl + cc holds K = 8ch … 8ch + 7 as bf16
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              const float* r = src + (size_t)(8 * cc) * TN + c;
              uint4 v;
              v.x = pack_bf16x2(r[0 * TN], r[1 * TN]);
              v.y = pack_bf16x2(r[2 * TN], r[3 * TN]);
              v.z = pack_bf16x2(r[4 * TN], r[5 * TN]);
              v.w = pack_bf16x2(r[6 * TN], r[7 * TN]);
              const int ch = 4 * sl + cc;
              *reinterpret_cast<uint4*>(row + ((ch ^ (c & 7)) << 4)) = v;
            }
          } else {
#pragma unroll
            for (int ch = 0; ch < TK / 4; ++ch) {
              uint4 v;
              v.x = to_tf32(src[(4 * ch + 0) * TN + c]);
              v.y = to_tf32(src[(4 * ch + 1) * TN + c]);
              v.z = to_tf32(src[(4 * ch + 2) * TN + c]);
              v.w = to_tf32(src[(4 * ch + 3) * TN + c]);
              *reinterpret_cast<uint4*>(row + ((ch ^ (c & 7)) << 4)) = v;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&stg_empty[q]);  // this warp's reads of the slot are done
      }
      if (stop) break;
      fence_async_shared();  // generic-proxy writes → visible to the tensor core
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
    }
  } else {
    // ------------------------------------------------------------ S generators
    // Item e of this block's slice: tile row g_lo + e/8, 16-byte chunk e mod 8
    // (one Philox call, four consecutive K).  The slice is then pushed to the
    // other blocks of the cluster by the leader (generator thread 0).
    const int g = threadIdx.x - 64;
    const int nitems = (g_hi - g_lo) * 8;
    const uint32_t slice_off = (uint32_t)g_lo * 128u, slice_bytes = (uint32_t)(g_hi - g_lo) * 128u;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % NSTAGE;
      const uint32_t ph = (uint32_t)(kb / NSTAGE) & 1u;
      if (kb >= NSTAGE) {
        // One thread waits (bounded) and every generator takes its decision, so
        // that all of them reach the same named barriers.
        if (g == 0) *gen_abort = mbar_wait(&empty[s], ph ^ 1u, kWaitLimitNs) ? 0u : 1u;
        named_sync(1, kGenWarps * 32);
        if (*gen_abort) {
          if (g == 0) atomicExch(&g_gauss_tc_error, MIHS_ERR_TIMEOUT);
          break;
        }
      }
      unsigned char* sS = base + (size_t)s * kStageBytes;
      const int kbase = kb0 + kb * KT;
      for (int e = g; e < nitems; e += kGenWarps * 32) {
        const int gt = g_lo + (e >> 3), c = e & 7;
        const int gi = i0 + gt;
        uint4 out = make_uint4(0u, 0u, 0u, 0u);
        if constexpr (PREC == 2) {
          // chunk c: K = kbase + 16c … + 15, four Philox counters
          const int j0 = kbase + 16 * c;
          if (gi < a.m && j0 < kb1) {
            float z[16];
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
              const uint4 w = philox4x32_10(make_uint4((uint32_t)((j0 >> 2) + hh), (uint32_t)gi, kTagGaussian, 0u),
                                            a.k0, a.k1);
              const float2 za = box_muller_fast(w.x, w.y);
              const float2 zb = box_muller_fast(w.z, w.w);
              z[4 * hh + 0] = za.x;
              z[4 * hh + 1] = za.y;
              z[4 * hh + 2] = zb.x;
              z[4 * hh + 3] = zb.y;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (j0 + q >= kb1) z[q] = 0.f;
            out = make_uint4(pack_e4m3x4(z[0], z[1], z[2], z[3]), pack_e4m3x4(z[4], z[5], z[6], z[7]),
                             pack_e4m3x4(z[8], z[9], z[10], z[11]), pack_e4m3x4(z[12], z[13], z[14], z[15]));
          }
        } else if constexpr (PREC == 1) {
          // chunk c: K = kbase + 8c … + 7, two Philox counters
          const int j0 = kbase + 8 * c;
          if (gi < a.m && j0 < kb1) {
            float z[8];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const uint4 w = philox4x32_10(make_uint4((uint32_t)((j0 >> 2) + hh), (uint32_t)gi, kTagGaussian, 0u),
                                            a.k0, a.k1);
              const float2 za = box_muller_fast(w.x, w.y);
              const float2 zb = box_muller_fast(w.z, w.w);
              z[4 * hh + 0] = za.x;
              z[4 * hh + 1] = za.y;
              z[4 * hh + 2] = zb.x;
              z[4 * hh + 3] = zb.y;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
              if (j0 + q >= kb1) z[q] = 0.f;
            out = make_uint4(pack_bf16x2(z[0], z[1]), pack_bf16x2(z[2], z[3]), pack_bf16x2(z[4], z[5]),
                             pack_bf16x2(z[6], z[7]));
          }
        } else {
          const int j0 = kbase + 4 * c;
          if (gi < a.m && j0 < kb1) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(j0 >> 2), (uint32_t)gi, kTagGaussian, 0u), a.k0, a.k1);
            const float2 za = box_muller_fast(w.x, w.y);
            const float2 zb = box_muller_fast(w.z, w.w);
            out = make_uint4(to_tf32(za.x), j0 + 1 < kb1 ? to_tf32(za.y) : 0u,
                             j0 + 2 < kb1 ? to_tf32(zb.x) : 0u, j0 + 3 < kb1 ? to_tf32(zb.y) : 0u);
          }
        }
        *reinterpret_cast<uint4*>(sS + (size_t)gt * 128 + ((c ^ (gt & 7)) << 4)) = out;
      }
      fence_async_shared();            // the slice → visible to the async proxy (MMA, bulk copies)
      named_sync(1, kGenWarps * 32);   // every generator has written its part
      if (g == 0) {
        // This block's stage is complete once the peers' slices have landed.
        mbar_arrive_expect_tx(&full[s], (uint32_t)(MROWS * 128) - slice_bytes);
        const uint32_t src = smem_u32(sS) + slice_off;
        for (int p = 1; p < cn; ++p) {
          const uint32_t peer = (crank + (uint32_t)p) % (uint32_t)cn;
          bulk_copy_s2c(mapa(src, peer), src, slice_bytes, mapa(smem_u32(&full[s]), peer));
        }
      }
    }
    if (warp >= 6) goto done;  // warps 2–5 (one per TMEM lane quarter) run the epilogue
    {
    // -------------------------------------------------------------- epilogue
    const bool ok = mbar_wait(accum, 0u, kWaitLimitNs);
    if (!ok) atomicExch(&g_gauss_tc_error, MIHS_ERR_TIMEOUT);
    tc_fence_after();
    const int qw = warp & 3;                 // TMEM lanes 32·qw … 32·qw + 31
    const int row_local = 32 * qw + lane;
#pragma unroll 1
    for (int t = 0; t < MT; ++t) {          // tile t: TMEM columns 256t …
    const int grow = i0 + TM * t + row_local;
    float* dst = a.part + ((size_t)blockIdx.z * a.m + (size_t)(grow < a.m ? grow : 0)) * a.dp;
    for (int cc = 0; cc < TN; cc += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)(256 * t + cc), v);
      if (grow < a.m) {
        const int col = c0 + cc;
        const bool have = ok && nkb > 0;
        if (col + 32 <= a.d) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<float4*>(dst + col + 4 * q) =
                have ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
          for (int q = 0; q < 32; ++q)
            if (col + q < a.d) dst[col + q] = have ? v[q] : 0.f;
        }
      }
    }
    }
    }
  }
done:
  tc_fence_before();
  __syncthreads();
  if (cn > 1) cluster_sync_all();  // no block exits while a peer may still copy into it
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TmemCols) : "memory");
  }
}

// SA[i][c] = scale · (ascale ? ascale[1] : 1) · Σ_z part[z][i][c] (fixed order).
__global__ void gauss_tc_reduce_kernel(const float* __restrict__ part, int KS, int m, int d, int dp,
                                       float scale, const float* __restrict__ ascale, float* __restrict__ SA,
                                       long long ldsa) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * d) return;
  const int i = (int)(idx / d), c = (int)(idx - (long long)i * d);
  float s = 0.f;
  for (int z = 0; z < KS; ++z) s += part[((size_t)z * m + i) * dp + c];
  if (ascale != nullptr) s *= ascale[1];
  SA[(long long)i * ldsa + c] = s * scale;
}

// max |A| over the matrix (fp32 bit patterns of non-negative values order as
// unsigned integers, so an atomic max on them is exact and order-free).
// max|A| over the n×d matrix (fp32 bits, atomicMax: the order of non-negative
// floats is that of their bit patterns).  One warp per row at a time, 16-byte
// loads when the rows allow them (vec: lda % 4 == 0, A 16-byte aligned).
__global__ void __launch_bounds__(256) absmax_kernel(const float* __restrict__ A, long long n, int d, long long lda,
                                                     int vec, unsigned int* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long wpb = blockDim.x >> 5;
  float mx = 0.f;
  const int d4 = vec ? (d & ~3) : 0;
  for (long long i = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (long long)gridDim.x * wpb) {
    const float* row = A + i * lda;
    for (int j = 4 * lane; j < d4; j += 128) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(row + j));
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int j = d4 + lane; j < d; j += 32) mx = fmaxf(mx, fabsf(__ldcs(row + j)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) atomicMax(out, __float_as_uint(mx));
}

// ascale[0] = 2^(8−e) with max|A| = f·2^e, f ∈ [½, 1), so that max|A|·ascale[0]
// lies in [128, 256) (e4m3 reaches 448) and the scaling is exact; ascale[1]
// its inverse.  The exponent is capped at 127 (a max|A| below 2⁻¹¹⁹ then
// maps below 128); A = 0 takes the scale 1.
__global__ void ascale_kernel(const unsigned int* __restrict__ mx, float* __restrict__ ascale) {
  const float m = __uint_as_float(*mx);
  int e = 0;
  if (m > 0.f) (void)frexpf(m, &e);
  const int k = m > 0.f ? min(8 - e, 127) : 0;
  ascale[0] = ldexpf(1.0f, k);
  ascale[1] = ldexpf(1.0f, -k);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

}  // namespace

bool gaussian_tc_available() { return encode_fn() != nullptr; }

int encode_tmap_2d_f32(CUtensorMap* map, const float* A, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                       int box_rows, int l2_promotion) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return MIHS_ERR_UNSUPPORTED;
  const cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         l2_promotion == 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? MIHS_OK : MIHS_ERR_UNSUPPORTED;
}

int sketch_gaussian_tc(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed, float* SA,
                       int64_t ldsa, cudaStream_t s, int prec) {
  using KernFn = void (*)(const CUtensorMap, const GaussTcArgs);
  // Two 128-row sketch tiles per block whenever there are two to share the
  // staged A tiles (MIHS_GAUSSIAN_MT=1 keeps one).
  static const bool force_mt1 = [] {
    const char* e = std::getenv("MIHS_GAUSSIAN_MT");
    return e != nullptr && std::atoi(e) == 1;
  }();
  const int tm = (int)((m + TM - 1) / TM);
  const int MT = (tm >= 2 && !force_mt1) ? 2 : 1;
  const KernFn kern = prec == 2   ? (MT == 2 ? gauss_tc_kernel<2, 2> : gauss_tc_kernel<2, 1>)
                     : prec == 1 ? (MT == 2 ? gauss_tc_kernel<1, 2> : gauss_tc_kernel<1, 1>)
                                 : (MT == 2 ? gauss_tc_kernel<0, 2> : gauss_tc_kernel<0, 1>);
  const size_t kSmemBytes = prec == 2   ? (MT == 2 ? TcCfg<2, 2>::Smem : TcCfg<2, 1>::Smem)
                            : prec == 1 ? (MT == 2 ? TcCfg<1, 2>::Smem : TcCfg<1, 1>::Smem)
                                        : (MT == 2 ? TcCfg<0, 2>::Smem : TcCfg<0, 1>::Smem);
  const int KT = 32 << prec;
  const int tmb = (tm + MT - 1) / MT;  // blocks along the sketch rows
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) {
    set_error("gaussian sketch: cuTensorMapEncodeTiled unavailable");
    return MIHS_ERR_UNSUPPORTED;
  }
  CUtensorMap tmap;
  const cuuint64_t gdim[2] = {(cuuint64_t)d, (cuuint64_t)n};
  const cuuint64_t gstride[1] = {(cuuint64_t)lda * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)TN, (cuuint32_t)TK};
  const cuuint32_t estr[2] = {1u, 1u};
  CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim, gstride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("gaussian sketch: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MIHS_ERR_UNSUPPORTED;
  }
  const int tn = (int)((d + TN - 1) / TN);
  const int64_t kblocks = (n + KT - 1) / KT;
  MIHS_CUDA_TRY(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  // One cluster per (sketch-row tile, K split) holds the tn column tiles.
  // Clusters that run at once on this GPU (a cluster needs tn SMs of one GPC):
  int active = 0;
  {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)tn;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)tn, 1, 1);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&active, (const void*)kern, &cfg) != cudaSuccess || active < 1) {
      cudaGetLastError();
      active = num_sms() / tn;
    }
  }
  // K splits: minimise waves × (a block's fixed cost + its K blocks), the
  // fixed cost (barrier set-up, TMEM, pipeline fill, the 128 KB partial
  // write) counted as 64 K blocks.
  int64_t KS = 1;
  {
    double best = 1e300;
    for (int64_t ks = 1; ks <= kblocks && ks <= 256; ++ks) {
      const int64_t cl = (int64_t)tmb * ks;
      const int64_t waves = (cl + active - 1) / active;
      const double cost = (double)waves * (64.0 + (double)((kblocks + ks - 1) / ks));
      if (cost < best * 0.999) {
        best = cost;
        KS = ks;
      }
    }
  }
  const int rows_per_split = (int)(((n + KS - 1) / KS + KT - 1) / KT * KT);
  KS = (n + rows_per_split - 1) / rows_per_split;
  const int dp = (int)round_up(d, 4);
  StreamScratch scratch;
  int rc = scratch.alloc(sizeof(float) * (size_t)KS * m * dp + 64, s);
  if (rc) return rc;
  float* ascale = nullptr;
  if (prec == 2) {  // the scale of A for e4m3: one pass over A for max |A|
    unsigned int* mx = reinterpret_cast<unsigned int*>(static_cast<float*>(scratch.p) + (size_t)KS * m * dp);
    ascale = reinterpret_cast<float*>(mx) + 4;
    MIHS_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned int), s));
    const int vec = (lda % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0) ? 1 : 0;
    absmax_kernel<<<(unsigned)(4 * num_sms()), 256, 0, s>>>(A, n, (int)d, lda, vec, mx);
    MIHS_CHECK_LAUNCH();
    ascale_kernel<<<1, 1, 0, s>>>(mx, ascale);
    MIHS_CHECK_LAUNCH();
    count_launch(2);
  }
  GaussTcArgs args;
  args.n = (int)n;
  args.d = (int)d;
  args.m = (int)m;
  args.rows_per_split = rows_per_split;
  args.k0 = (uint32_t)seed;
  args.k1 = (uint32_t)(seed >> 32);
  args.part = static_cast<float*>(scratch.p);
  args.dp = dp;
  args.cn = tn;
  args.ascale = ascale;
  {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)tn;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)tn, (unsigned)tmb, (unsigned)KS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MIHS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, tmap, args));
  }
  const long long tot = (long long)m * d;
  gauss_tc_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      args.part, (int)KS, (int)m, (int)d, dp, (float)(1.0 / std::sqrt((double)m)), ascale, SA, ldsa);
  MIHS_CHECK_LAUNCH();
  count_launch(2);
  return MIHS_OK;
}

int gauss_tc_device_error(int* code) {
  int v = 0, zero = 0;
  MIHS_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_gauss_tc_error, sizeof(int)));
  if (v != 0) MIHS_CUDA_TRY(cudaMemcpyToSymbol(g_gauss_tc_error, &zero, sizeof(int)));
  *code = v;
  return MIHS_OK;
}

}  // namespace mihs
