// Sparse embedding with one ±1 per column (Lemma 3, case i; "CountSketch"):
//     SA[h(j), :] += s(j) · A[j, :],   j = 0 … n−1.
//
// Instead of scattering rows of A into SA with atomics, the rows are bucketed
// by h once (a counting sort of n 32-bit keys: ~4 B/row of extra traffic) and
// one thread block then owns each output row h and streams its rows of A in
// ascending j.  A is read exactly once, in whole coalesced rows, every output
// row is written exactly once (no memset, no atomics on SA), and the sum order
// is fixed, so SA is bit-reproducible.
#include "internal.h"

namespace mihs {

namespace {

constexpr int kGatherThreads = 256;
constexpr int kSortCap = 8192;  // bucket entries sorted in shared memory
// Rows loaded before they are added (16-byte loads in flight per thread):
// 4 left the gather bound by load latency (55 % of DRAM bandwidth).
constexpr int kRowsInFlight = 8;

// h(j) = ⌊w0·m/2³²⌋, s(j) = + if w1 even; Philox counter (j, 0, 1, 0).
__global__ void cs_hash_kernel(int n, uint32_t m, uint32_t k0, uint32_t k1,
                               int* __restrict__ code, int* __restrict__ counts) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)j, 0u, kTagCountSketch, 0u), k0, k1);
  const int h = (int)(((uint64_t)w.x * m) >> 32);
  const int neg = (int)(w.y & 1u);
  code[j] = h | (neg ? (int)0x80000000 : 0);  // the sign travels in bit 31
  atomicAdd(counts + h, 1);
}

// Exclusive scan of counts[0..m) → offsets[0..m], cursor = offsets (one block).
__global__ void __launch_bounds__(1024) cs_scan_kernel(const int* __restrict__ counts, int m,
                                                       int* __restrict__ offsets,
                                                       int* __restrict__ cursor) {
  __shared__ int buf[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < m; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < m ? counts[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // Hillis–Steele inclusive scan
      const int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < m) {
      const int ex = carry + buf[threadIdx.x] - v;
      offsets[i] = ex;
      cursor[i] = ex;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[m] = carry;
}

// list[offsets[h] + k] = j | (sign << 31)  (order within a bucket is fixed later)
__global__ void cs_scatter_kernel(int n, const int* __restrict__ code, int* __restrict__ cursor,
                                  int* __restrict__ list) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int c = code[j];
  const int h = c & 0x7fffffff;
  const int pos = atomicAdd(cursor + h, 1);
  list[pos] = j | (c & (int)0x80000000);
}

__device__ __forceinline__ int entry_row(int e) { return e & 0x7fffffff; }
__device__ __forceinline__ float entry_sign(int e) { return e < 0 ? -1.f : 1.f; }

// One block per output row h: sort the bucket by j, then SA[h] = Σ s(j) A[j].
__global__ void __launch_bounds__(kGatherThreads)
cs_gather_kernel(const float* __restrict__ A, int d, long long lda,
                 const int* __restrict__ offsets, const int* __restrict__ list, int m,
                 float* __restrict__ SA, long long ldsa) {
  __shared__ int keys[kSortCap];
  for (int h = blockIdx.x; h < m; h += gridDim.x) {
    const int beg = offsets[h], cnt = offsets[h + 1] - beg;
    const bool sorted = cnt <= kSortCap;
    if (sorted) {
      int np2 = 1;
      while (np2 < cnt) np2 <<= 1;
      for (int e = threadIdx.x; e < np2; e += kGatherThreads)
        keys[e] = e < cnt ? list[beg + e] : 0x7fffffff;
      __syncthreads();
      // bitonic sort by row index (bit 31 carries the sign, so sort on j)
      for (int k = 2; k <= np2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
          for (int e = threadIdx.x; e < np2; e += kGatherThreads) {
            const int p = e ^ jj;
            if (p > e) {
              const int a = keys[e], b = keys[p];
              const bool up = (e & k) == 0;
              const bool gt = (a & 0x7fffffff) > (b & 0x7fffffff);
              if (gt == up) {
                keys[e] = b;
                keys[p] = a;
              }
            }
          }
          __syncthreads();
        }
      }
    }
    // Each thread owns float4 column groups q = tid + 256·c.
    for (int q0 = 0; 4 * q0 < d; q0 += kGatherThreads) {
      const int q = q0 + threadIdx.x;
      const int col = 4 * q;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (col < d) {
        const bool full = col + 4 <= d;
        int e = 0;
        for (; e + kRowsInFlight <= cnt; e += kRowsInFlight) {
          int en[kRowsInFlight];
          float4 a[kRowsInFlight];
#pragma unroll
          for (int u = 0; u < kRowsInFlight; ++u) en[u] = sorted ? keys[e + u] : list[beg + e + u];
#pragma unroll
          for (int u = 0; u < kRowsInFlight; ++u) {
            const float* row = A + (long long)entry_row(en[u]) * lda + col;
            if (full) {
              a[u] = __ldcs(reinterpret_cast<const float4*>(row));
            } else {
              a[u] = make_float4(row[0], col + 1 < d ? row[1] : 0.f, col + 2 < d ? row[2] : 0.f, 0.f);
            }
          }
#pragma unroll
          for (int u = 0; u < kRowsInFlight; ++u) {
            const float sg = entry_sign(en[u]);
            acc.x = fmaf(sg, a[u].x, acc.x);
            acc.y = fmaf(sg, a[u].y, acc.y);
            acc.z = fmaf(sg, a[u].z, acc.z);
            acc.w = fmaf(sg, a[u].w, acc.w);
          }
        }
        for (; e < cnt; ++e) {
          const int en = sorted ? keys[e] : list[beg + e];
          const float* row = A + (long long)entry_row(en) * lda + col;
          const float sg = entry_sign(en);
          float4 a;
          if (full) {
            a = __ldcs(reinterpret_cast<const float4*>(row));
          } else {
            a = make_float4(row[0], col + 1 < d ? row[1] : 0.f, col + 2 < d ? row[2] : 0.f, 0.f);
          }
          acc.x = fmaf(sg, a.x, acc.x);
          acc.y = fmaf(sg, a.y, acc.y);
          acc.z = fmaf(sg, a.z, acc.z);
          acc.w = fmaf(sg, a.w, acc.w);
        }
        float* out = SA + (long long)h * ldsa + col;
        if (full && (ldsa % 4) == 0) {
          *reinterpret_cast<float4*>(out) = acc;
        } else {
          out[0] = acc.x;
          if (col + 1 < d) out[1] = acc.y;
          if (col + 2 < d) out[2] = acc.z;
          if (col + 3 < d) out[3] = acc.w;
        }
      }
    }
    __syncthreads();  // keys reused by the next bucket
  }
}

}  // namespace

int sketch_countsketch(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m,
                       uint64_t seed, float* SA, int64_t ldsa, cudaStream_t s) {
  StreamScratch scratch;
  // code[n], list[n], counts[m], offsets[m+1], cursor[m]
  const size_t bytes = sizeof(int) * ((size_t)2 * n + 3 * (size_t)m + 1);
  int rc = scratch.alloc(bytes, s);
  if (rc) return rc;
  int* code = static_cast<int*>(scratch.p);
  int* list = code + n;
  int* counts = list + n;
  int* offsets = counts + m;
  int* cursor = offsets + m + 1;
  MIHS_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)m, s));
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int nb = (int)((n + 255) / 256);
  cs_hash_kernel<<<nb, 256, 0, s>>>((int)n, (uint32_t)m, k0, k1, code, counts);
  MIHS_CHECK_LAUNCH();
  cs_scan_kernel<<<1, 1024, 0, s>>>(counts, (int)m, offsets, cursor);
  MIHS_CHECK_LAUNCH();
  cs_scatter_kernel<<<nb, 256, 0, s>>>((int)n, code, cursor, list);
  MIHS_CHECK_LAUNCH();
  const int grid = (int)(m < 65535 ? m : 65535);
  cs_gather_kernel<<<grid, kGatherThreads, 0, s>>>(A, (int)d, (long long)lda, offsets, list,
                                                    (int)m, SA, (long long)ldsa);
  MIHS_CHECK_LAUNCH();
  count_launch(4);
  return MIHS_OK;
}

}  // namespace mihs
