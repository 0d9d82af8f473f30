/* Compensated gradient for the oracle (TEST INFRASTRUCTURE ONLY; shares no
 * code with the CUDA path).
 *
 *   g = Aᵀ(b − Ax) − λx      (the gradient step of Algorithm 1)
 *
 * for fp32 A (n × d, row pitch lda) and b, fp64 x and λ, with every product
 * and every sum carried as an unevaluated pair hi + lo of doubles
 * ("double-double"): products split exactly by a fused multiply-add
 * (TwoProduct) and sums by Knuth's TwoSum, as in Ogita, Rump and Oishi,
 * "Accurate sum and dot product" (SIAM J. Sci. Comput. 26, 2005).  The
 * residual r = b − Ax of each row is formed in double-double and kept in
 * double-double; Aᵀr is accumulated in double-double.  Rows are split into
 * `nthreads` contiguous chunks, each summed in row order, and the chunk sums
 * are added in chunk order, so the result does not depend on scheduling.
 * Relative accuracy ≈ 2⁻¹⁰⁴ per operation: used to refine the oracle's
 * Cholesky solution to fp64 rounding on problems with κ(AᵀA + λI) ≈ 1e6. */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>

typedef struct {
  double hi, lo;
} dd;

static dd two_sum(double a, double b) {
  dd r;
  r.hi = a + b;
  double bv = r.hi - a;
  r.lo = (a - (r.hi - bv)) + (b - bv);
  return r;
}

static dd quick_two_sum(double a, double b) { /* |a| ≥ |b| */
  dd r;
  r.hi = a + b;
  r.lo = b - (r.hi - a);
  return r;
}

static dd two_prod(double a, double b) {
  dd r;
  r.hi = a * b;
  r.lo = fma(a, b, -r.hi);
  return r;
}

static dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

/* (a.hi + a.lo)·(double) b */
static dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo = fma(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

typedef struct {
  const float* A;
  const float* b;
  const double* x;
  long r0, r1, d, lda;
  dd* g; /* d entries, this chunk's Σ A_iᵀ r_i */
} chunk_t;

static void* run_chunk(void* p) {
  chunk_t* c = (chunk_t*)p;
  for (long j = 0; j < c->d; ++j) c->g[j].hi = c->g[j].lo = 0.0;
  for (long i = c->r0; i < c->r1; ++i) {
    const float* row = c->A + i * c->lda;
    dd r = {(double)c->b[i], 0.0};
    for (long j = 0; j < c->d; ++j) {
      dd p = two_prod((double)row[j], c->x[j]);
      p.hi = -p.hi;
      p.lo = -p.lo;
      r = dd_add(r, p);
    }
    for (long j = 0; j < c->d; ++j) c->g[j] = dd_add(c->g[j], dd_mul_d(r, (double)row[j]));
  }
  return NULL;
}

/* g_hi[j] + g_lo[j] = (Aᵀ(b − Ax) − λx)_j.  Returns 0, or −1 if memory or a
 * thread could not be had. */
int oracle_gradient_dd(const float* A, long n, long d, long lda, const float* b, const double* x, double lam,
                       int nthreads, double* g_hi, double* g_lo) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n) nthreads = (int)(n > 0 ? n : 1);
  chunk_t* cs = (chunk_t*)calloc((size_t)nthreads, sizeof(chunk_t));
  dd* gs = (dd*)calloc((size_t)nthreads * (size_t)d, sizeof(dd));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!cs || !gs || !th) {
    free(cs);
    free(gs);
    free(th);
    return -1;
  }
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    cs[t].A = A;
    cs[t].b = b;
    cs[t].x = x;
    cs[t].r0 = n * t / nthreads;
    cs[t].r1 = n * (t + 1) / nthreads;
    cs[t].d = d;
    cs[t].lda = lda;
    cs[t].g = gs + (size_t)t * (size_t)d;
  }
  int started = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, run_chunk, &cs[t]) != 0) {
      rc = -1;
      break;
    }
    started = t;
  }
  run_chunk(&cs[0]);
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  if (rc == 0) {
    for (long j = 0; j < d; ++j) {
      dd s = {0.0, 0.0};
      for (int t = 0; t < nthreads; ++t) s = dd_add(s, gs[(size_t)t * (size_t)d + j]);
      dd lx = two_prod(lam, x[j]);
      lx.hi = -lx.hi;
      lx.lo = -lx.lo;
      s = dd_add(s, lx);
      g_hi[j] = s.hi;
      g_lo[j] = s.lo;
    }
  }
  free(cs);
  free(gs);
  free(th);
  return rc;
}
