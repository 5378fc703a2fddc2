/*
 * gk_oracle.c -- plain FP64 CPU oracle for "Accurate and fast matrix
 * factorization for low-rank learning" (arXiv 2104.10785).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA library.
 *
 * Each routine restates one passage of the paper, or the textbook definition
 * the paper relies on, in double precision.  Loops are written out; the only
 * liberties are (a) OpenMP work-sharing over independent outputs, which never
 * changes any sum's order, and (b) dot products summed in fixed 4096-element
 * chunks so that results do not depend on the thread count.
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  - Algorithm 1's indices follow the Bidiag-1 recurrences of Eqs. 2.1-2.2.
 *  - The break test of Algorithm 1 compares the norm *before* normalization
 *    (beta_{j+1}) with the threshold, and uses <= so that a zero matrix stops.
 *  - The threshold is eps * sigma_est (relative reading; sigma_est is a running
 *    lower bound on sigma_1 built from row/column norms of B) unless the caller
 *    asks for the absolute reading.
 *  - A vanishing alpha_{j+1} also ends Algorithm 1 (division by it would only
 *    amplify rounding noise); the paper tests beta only.
 *  - Algorithm 3 counts singular values of B above eps * sigma_1(B); the
 *    literal eigenvalue count of B^T B above eps is available as an option.
 *  - The restarted partial SVD (thick restart with Ritz vectors) is not
 *    printed in the paper, which cites augmented restarting; it is written
 *    here in the upper-bidiagonal form started from v1 = A^T q1 / ||A^T q1||
 *    (Algorithm 1).
 *
 * The fused sweep (fused != 0) is not in the paper: it is the one-pass
 * ordering the CUDA path uses, restated here step by step.  The left step's
 * vector w (A p_j minus its recurrence term, before reorthogonalization) is
 * multiplied by A^T right away, and the right step uses A^T w / beta_{j+1} in
 * place of A^T q_{j+1}.  The two differ by A^T Q_j h / beta_{j+1} (h the
 * Gram-Schmidt coefficients), and A^T Q_j lies in span(P_j) by Eq. 2.2
 * (A^T q_i = alpha_i p_i + beta_i p_{i-1}), so the Gram-Schmidt pass against
 * P_j removes the difference: in exact arithmetic the recurrence is unchanged.
 */
#include "gk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CHUNK 4096

/* ------------------------------------------------------------------------ */
/* value promotion                                                           */
/* ------------------------------------------------------------------------ */

static double bf16_bits_to_double(uint16_t b)
{
  /* bf16 is the top half of an IEEE binary32 word */
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

static double f16_bits_to_double(uint16_t h)
{
  /* IEEE binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits */
  int s = (h >> 15) & 1;
  int e = (h >> 10) & 31;
  int f = h & 1023;
  double v;
  if (e == 0)
    v = ldexp((double)f, -24);              /* subnormal: f * 2^-14 / 2^10 */
  else if (e == 31)
    v = f ? NAN : INFINITY;
  else
    v = ldexp((double)(1024 + f), e - 25);  /* (1 + f/2^10) * 2^(e-15) */
  return s ? -v : v;
}

static inline double stored_value(const gko_op *A, int64_t idx)
{
  double v;
  switch (A->dtype) {
  case GKO_F64: v = ((const double *)A->vals)[idx]; break;
  case GKO_F32: v = (double)((const float *)A->vals)[idx]; break;
  case GKO_BF16: v = bf16_bits_to_double(((const uint16_t *)A->vals)[idx]); break;
  default: v = f16_bits_to_double(((const uint16_t *)A->vals)[idx]); break;
  }
  return v * A->scale;
}

double gko_elem_value(const gko_op *A, int64_t idx) { return stored_value(A, idx); }

void gko_set_threads(int nthreads)
{
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

/* ------------------------------------------------------------------------ */
/* products with A and A^T                                                   */
/* ------------------------------------------------------------------------ */

/* y = A x : y_i = sum_j a_ij x_j */
void gko_apply(const gko_op *A, const double *x, double *y)
{
  const int64_t m = A->m;
  if (A->kind == GKO_DENSE) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < A->n; ++j) s += stored_value(A, i * A->ld + j) * x[j];
      y[i] = s;
    }
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
        s += stored_value(A, p) * x[A->colind[p]];
      y[i] = s;
    }
  }
}

/* y = A^T x : y_j = sum_i a_ij x_i, each y_j summed in increasing i */
void gko_apply_t(const gko_op *A, const double *x, double *y)
{
  const int64_t n = A->n;
  if (A->kind == GKO_DENSE) {
    const int64_t nblk = (n + 63) / 64;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
      const int64_t j0 = b * 64, j1 = (j0 + 64 < n) ? j0 + 64 : n;
      double acc[64];
      for (int64_t j = j0; j < j1; ++j) acc[j - j0] = 0.0;
      for (int64_t i = 0; i < A->m; ++i)
        for (int64_t j = j0; j < j1; ++j) acc[j - j0] += stored_value(A, i * A->ld + j) * x[i];
      for (int64_t j = j0; j < j1; ++j) y[j] = acc[j - j0];
    }
  } else {
    for (int64_t j = 0; j < n; ++j) y[j] = 0.0;
    for (int64_t i = 0; i < A->m; ++i)
      for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
        y[A->colind[p]] += stored_value(A, p) * x[i];
  }
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */

static double dot(const double *a, const double *b, int64_t len)
{
  const int64_t nc = (len + CHUNK - 1) / CHUNK;
  if (nc <= 1) {
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += a[i] * b[i];
    return s;
  }
  double *part = (double *)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t i0 = c * CHUNK, i1 = (i0 + CHUNK < len) ? i0 + CHUNK : len;
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) s += a[i] * b[i];
    part[c] = s;
  }
  double s = 0.0;
  for (int64_t c = 0; c < nc; ++c) s += part[c];
  free(part);
  return s;
}

static double norm2(const double *a, int64_t len) { return sqrt(dot(a, a, len)); }

static void scale_into(double *dst, const double *src, double f, int64_t len)
{
  for (int64_t i = 0; i < len; ++i) dst[i] = src[i] * f;
}

/* One classical Gram-Schmidt pass: h = Q^T w, then w <- w - Q h, with Q the
 * first j columns of a column-major basis (leading dimension ld). */
static void cgs_pass(double *w, const double *Qb, int64_t len, int64_t ld, int j, double *h)
{
  if (j <= 0) return;
#pragma omp parallel for schedule(static) if (len * (int64_t)j > 65536)
  for (int c = 0; c < j; ++c) {
    const double *q = Qb + (int64_t)c * ld;
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += q[i] * w[i];
    h[c] = s;
  }
  const int64_t nblk = (len + 255) / 256;
#pragma omp parallel for schedule(static) if (len * (int64_t)j > 65536)
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t i0 = b * 256, i1 = (i0 + 256 < len) ? i0 + 256 : len;
    for (int c = 0; c < j; ++c) {
      const double *q = Qb + (int64_t)c * ld;
      const double hc = h[c];
      for (int64_t i = i0; i < i1; ++i) w[i] -= hc * q[i];
    }
  }
}

static double norm2sq(const double *w, int64_t len)
{
  double s = 0.0;
  for (int64_t i = 0; i < len; ++i) s += w[i] * w[i];
  return s;
}

/* passes = 1 or 2: that many classical Gram-Schmidt passes.  passes = 0: one
 * pass, then a second only if the first left less than 1/sqrt(2) of the norm
 * (||w1||^2 < ||w0||^2 / 2; Daniel, Gragg, Kaufman and Stewart, Math. Comp.
 * 1976, the test ARPACK applies after its Gram-Schmidt step). */
static void cgs(int passes, double *w, const double *Qb, int64_t len, int64_t ld, int j)
{
  if (j <= 0) return;
  double *h = (double *)malloc(sizeof(double) * (size_t)j);
  if (passes == 0) {
    const double n0 = norm2sq(w, len);
    cgs_pass(w, Qb, len, ld, j, h);
    if (norm2sq(w, len) < 0.5 * n0) cgs_pass(w, Qb, len, ld, j, h);
  } else {
    for (int p = 0; p < passes; ++p) cgs_pass(w, Qb, len, ld, j, h);
  }
  free(h);
}

/* The Gram-Schmidt step on its own (len x j column-major basis), for the tests. */
void gko_cgs(int passes, double *w, const double *Q, int64_t len, int64_t ld, int j)
{
  cgs(passes, w, Q, len, ld, j);
}

/* ------------------------------------------------------------------------ */
/* counter-based generators (seeded inputs and replacement directions)       */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
 * 4x32 multiply-xor bijection keyed by a 64-bit key bumped by the Weyl
 * constants between rounds. */
void gko_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The start vector of Algorithm 1, q_i ~ N(2,1): Philox block b = i/2 with
 * counter (b, 0, 0, 0) and key (seed_lo, seed_hi) gives two 53-bit uniforms
 * in (0,1); Box-Muller maps them to a normal pair (z0 for even i, z1 for odd). */
void gko_start_vector(uint64_t seed, int64_t m, double *q)
{
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t i = 0; i < m; ++i) {
    const uint64_t b = (uint64_t)i >> 1;
    const uint32_t ctr[4] = {(uint32_t)b, (uint32_t)(b >> 32), 0u, 0u};
    uint32_t x[4];
    gko_philox4x32_10(ctr, key, x);
    const double ua = ((double)(((uint64_t)(x[0] >> 5) << 26) | (x[1] >> 6)) + 0.5) * 0x1.0p-53;
    const double ub = ((double)(((uint64_t)(x[2] >> 5) << 26) | (x[3] >> 6)) + 0.5) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(ua));
    const double z = (i & 1) ? r * sin(two_pi * ub) : r * cos(two_pi * ub);
    q[i] = 2.0 + z;
  }
}

/* SplitMix64 finalizer (Steele, Lea, Flood, OOPSLA'14). */
uint64_t gko_splitmix64(uint64_t x)
{
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Replacement direction number d after an exact breakdown: entries uniform in
 * [-1, 1) from SplitMix64 of (mixed seed + index). */
static void fresh_direction(uint64_t seed, int64_t d, double *x, int64_t len)
{
  const uint64_t base = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(d + 1));
  for (int64_t i = 0; i < len; ++i) {
    const uint64_t r = gko_splitmix64(base + (uint64_t)i);
    x[i] = (double)(r >> 11) * 0x1.0p-52 - 1.0;
  }
}

/* ------------------------------------------------------------------------ */
/* one-sided Jacobi SVD and cyclic Jacobi eigensolver                        */
/* ------------------------------------------------------------------------ */

int gko_jacobi_svd(int64_t rows, int64_t cols, const double *M, double *sigma, double *Uc, double *Vc)
{
  if (rows < cols || cols <= 0) return -1000;
  double *W = (double *)malloc(sizeof(double) * (size_t)(rows * cols));
  double *Vt = (double *)calloc((size_t)(cols * cols), sizeof(double));
  memcpy(W, M, sizeof(double) * (size_t)(rows * cols));
  for (int64_t i = 0; i < cols; ++i) Vt[i * cols + i] = 1.0;
  const double tol = 2.0 * sqrt((double)rows) * 0x1.0p-52;
  int sweep, done = 0;
  for (sweep = 1; sweep <= 80 && !done; ++sweep) {
    int rotated = 0;
    for (int64_t p = 0; p + 1 < cols; ++p) {
      for (int64_t q = p + 1; q < cols; ++q) {
        double *wp = W + p * rows, *wq = W + q * rows;
        double a = 0.0, b = 0.0, c = 0.0;
        for (int64_t i = 0; i < rows; ++i) {
          a += wp[i] * wp[i];
          b += wq[i] * wq[i];
          c += wp[i] * wq[i];
        }
        if (c == 0.0 || fabs(c) <= tol * sqrt(a) * sqrt(b)) continue;
        rotated = 1;
        /* rotation that makes columns p and q orthogonal (Rutishauser) */
        const double zeta = (b - a) / (2.0 * c);
        double t;
        if (fabs(zeta) > 1e150)
          t = 0.5 / zeta;
        else
          t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int64_t i = 0; i < rows; ++i) {
          const double x = wp[i], y = wq[i];
          wp[i] = cs * x - sn * y;
          wq[i] = sn * x + cs * y;
        }
        double *vp = Vt + p * cols, *vq = Vt + q * cols;
        for (int64_t i = 0; i < cols; ++i) {
          const double x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
      }
    }
    if (!rotated) done = 1;
  }
  /* singular values are the column norms; order them descending (stable) */
  double *nrm = (double *)malloc(sizeof(double) * (size_t)cols);
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)cols);
  for (int64_t j = 0; j < cols; ++j) {
    nrm[j] = norm2(W + j * rows, rows);
    ord[j] = j;
  }
  for (int64_t a = 1; a < cols; ++a) { /* insertion sort, stable */
    int64_t v = ord[a], b = a - 1;
    while (b >= 0 && nrm[ord[b]] < nrm[v]) {
      ord[b + 1] = ord[b];
      --b;
    }
    ord[b + 1] = v;
  }
  for (int64_t j = 0; j < cols; ++j) {
    const int64_t s = ord[j];
    sigma[j] = nrm[s];
    for (int64_t i = 0; i < rows; ++i) Uc[j * rows + i] = nrm[s] > 0.0 ? W[s * rows + i] / nrm[s] : 0.0;
    for (int64_t i = 0; i < cols; ++i) Vc[j * cols + i] = Vt[s * cols + i];
  }
  free(nrm);
  free(ord);
  free(W);
  free(Vt);
  return done ? sweep - 1 : -(sweep - 1);
}

int gko_jacobi_eig(int64_t n, const double *S0, double *theta, double *G)
{
  double *S = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *Gt = (double *)calloc((size_t)(n * n), sizeof(double));
  memcpy(S, S0, sizeof(double) * (size_t)(n * n));
  for (int64_t i = 0; i < n; ++i) Gt[i * n + i] = 1.0;
#define SS(i, j) S[(j) * n + (i)]
  int sweep, done = 0;
  for (sweep = 1; sweep <= 80 && !done; ++sweep) {
    int rotated = 0;
    for (int64_t p = 0; p + 1 < n; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        const double apq = SS(p, q);
        if (apq == 0.0 || fabs(apq) <= 0x1.0p-53 * sqrt(fabs(SS(p, p)) * fabs(SS(q, q)))) continue;
        rotated = 1;
        /* symmetric Schur rotation J(p,q) with (J^T S J)_pq = 0 */
        const double tau = (SS(q, q) - SS(p, p)) / (2.0 * apq);
        double t;
        if (fabs(tau) > 1e150)
          t = 0.5 / tau;
        else
          t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int64_t k = 0; k < n; ++k) { /* S <- S J */
          const double x = SS(k, p), y = SS(k, q);
          SS(k, p) = c * x - s * y;
          SS(k, q) = s * x + c * y;
        }
        for (int64_t k = 0; k < n; ++k) { /* S <- J^T S */
          const double x = SS(p, k), y = SS(q, k);
          SS(p, k) = c * x - s * y;
          SS(q, k) = s * x + c * y;
        }
        for (int64_t k = 0; k < n; ++k) { /* G <- G J */
          const double x = Gt[p * n + k], y = Gt[q * n + k];
          Gt[p * n + k] = c * x - s * y;
          Gt[q * n + k] = s * x + c * y;
        }
      }
    }
    if (!rotated) done = 1;
  }
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < n; ++j) ord[j] = j;
  for (int64_t a = 1; a < n; ++a) {
    int64_t v = ord[a], b = a - 1;
    while (b >= 0 && SS(ord[b], ord[b]) < SS(v, v)) {
      ord[b + 1] = ord[b];
      --b;
    }
    ord[b + 1] = v;
  }
  for (int64_t j = 0; j < n; ++j) {
    theta[j] = SS(ord[j], ord[j]);
    for (int64_t i = 0; i < n; ++i) G[j * n + i] = Gt[ord[j] * n + i];
  }
#undef SS
  free(ord);
  free(S);
  free(Gt);
  return done ? sweep - 1 : -(sweep - 1);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (lower-bidiagonal Bidiag-1 with reorthogonalization)          */
/* ------------------------------------------------------------------------ */

int gko_gk_lower(const gko_op *A, int k, double eps, int eps_relative, int passes, const double *q1,
                 double *alpha, double *beta, double *Q, double *P, gko_gk_info *info, int fused)
{
  const int64_t m = A->m, n = A->n;
  const int64_t mn = m < n ? m : n;
  if (k < 1 || k > mn || passes < 0 || passes > 3) return -1;
  memset(alpha, 0, sizeof(double) * (size_t)(k + 1));
  memset(beta, 0, sizeof(double) * (size_t)(k + 2));
  memset(Q, 0, sizeof(double) * (size_t)(m * (k + 1)));
  memset(P, 0, sizeof(double) * (size_t)(n * (k + 1)));
  info->kprime = 0;
  info->stop_reason = 0;

  /* beta_1 = ||q_1||, q_1 = q_1 / beta_1 (Eq. 2.1, beta_1 q_1 = q_1) */
  const double b1 = norm2(q1, m);
  if (!(b1 > 0.0)) return -2;
  beta[0] = b1;
  scale_into(Q, q1, 1.0 / b1, m);

  /* p_1 = A^T q_1, alpha_1 = ||p_1||, p_1 = p_1 / alpha_1 (Eq. 2.1) */
  double *w = (double *)malloc(sizeof(double) * (size_t)m);
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double *zr = fused ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
  gko_apply_t(A, Q, z);
  const double a1 = norm2(z, n);
  alpha[0] = a1;
  double sest = a1;
  if (a1 <= (eps_relative ? eps * sest : eps)) {
    info->stop_reason = 2;
    info->sigma_est = sest;
    free(w);
    free(z);
    free(zr);
    return 0;
  }
  scale_into(P, z, 1.0 / a1, n);

  int j;
  for (j = 1; j <= k; ++j) {
    /* column j-1 (0-based) holds q_j and p_j; alpha[j-1] is alpha_j */
    const double *pj = P + (int64_t)(j - 1) * n;
    const double *qj = Q + (int64_t)(j - 1) * m;
    const double aj = alpha[j - 1];

    /* beta_{j+1} q_{j+1} = A p_j - alpha_j q_j, reorthogonalized against Q_j (Eq. 2.2) */
    gko_apply(A, pj, w);
    for (int64_t i = 0; i < m; ++i) w[i] -= aj * qj[i];
    if (fused) gko_apply_t(A, w, zr); /* fused sweep: A^T w before reorthogonalization */
    cgs(passes, w, Q, m, m, j);
    const double b = norm2(w, m);
    beta[j] = b;
    sest = fmax(sest, hypot(aj, b));
    if (b <= (eps_relative ? eps * sest : eps)) { /* break test on beta_{j+1} */
      info->kprime = j;
      info->stop_reason = 1;
      break;
    }
    scale_into(Q + (int64_t)j * m, w, 1.0 / b, m);

    /* alpha_{j+1} p_{j+1} = A^T q_{j+1} - beta_{j+1} p_j, reorthogonalized against P_j;
     * the fused sweep takes A^T w / beta_{j+1} for A^T q_{j+1} (equal up to span(P_j)) */
    if (fused) {
      for (int64_t i = 0; i < n; ++i) z[i] = zr[i] / b - b * pj[i];
    } else {
      gko_apply_t(A, Q + (int64_t)j * m, z);
      for (int64_t i = 0; i < n; ++i) z[i] -= b * pj[i];
    }
    cgs(passes, z, P, n, n, j);
    const double a = norm2(z, n);
    alpha[j] = a;
    sest = fmax(sest, hypot(b, a));
    if (a <= (eps_relative ? eps * sest : eps)) {
      info->kprime = j;
      info->stop_reason = 2;
      break;
    }
    scale_into(P + (int64_t)j * n, z, 1.0 / a, n);
  }
  if (j > k) {
    info->kprime = k;
    info->stop_reason = 0;
  }
  info->sigma_est = sest;
  free(w);
  free(z);
  free(zr);
  return 0;
}

/* dense (k'+1) x k' lower-bidiagonal B, column-major */
static double *build_lower_B(int kp, const double *alpha, const double *beta)
{
  double *B = (double *)calloc((size_t)((kp + 1) * kp), sizeof(double));
  for (int j = 0; j < kp; ++j) {
    B[(int64_t)j * (kp + 1) + j] = alpha[j];         /* alpha_{j+1} on the diagonal */
    B[(int64_t)j * (kp + 1) + j + 1] = beta[j + 1];  /* beta_{j+2} below it */
  }
  return B;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3: rank determination                                           */
/* ------------------------------------------------------------------------ */

int gko_numrank(const gko_op *A, int kmax, double eps, int eps_relative, int literal, int passes,
                const double *q1, int *rank, gko_gk_info *info, double *sigma_out, int fused)
{
  const int64_t m = A->m, n = A->n;
  const int64_t mn = m < n ? m : n;
  if (kmax <= 0 || kmax > mn) kmax = (int)mn; /* k = min(m, n) */
  double *alpha = (double *)malloc(sizeof(double) * (size_t)(kmax + 1));
  double *beta = (double *)malloc(sizeof(double) * (size_t)(kmax + 2));
  double *Q = (double *)malloc(sizeof(double) * (size_t)(m * (kmax + 1)));
  double *P = (double *)malloc(sizeof(double) * (size_t)(n * (kmax + 1)));
  /* run Algorithm 1 */
  int rc = gko_gk_lower(A, kmax, eps, eps_relative, passes, q1, alpha, beta, Q, P, info, fused);
  if (rc != 0) goto out;
  const int kp = info->kprime;
  *rank = 0;
  if (kp > 0) {
    double *B = build_lower_B(kp, alpha, beta);
    double *sig = (double *)malloc(sizeof(double) * (size_t)kp);
    if (!literal) {
      /* singular values of B (= square roots of the eigenvalues of B^T B) */
      double *Uc = (double *)malloc(sizeof(double) * (size_t)((kp + 1) * kp));
      double *Vc = (double *)malloc(sizeof(double) * (size_t)(kp * kp));
      gko_jacobi_svd(kp + 1, kp, B, sig, Uc, Vc);
      const double thr = eps_relative ? eps * sig[0] : eps;
      for (int i = 0; i < kp; ++i) *rank += sig[i] > thr ? 1 : 0;
      free(Uc);
      free(Vc);
    } else {
      /* eigenvalues of B^T B, counted against eps */
      double *S = (double *)calloc((size_t)(kp * kp), sizeof(double));
      double *G = (double *)malloc(sizeof(double) * (size_t)(kp * kp));
      for (int c = 0; c < kp; ++c)
        for (int r = 0; r < kp; ++r) {
          double s = 0.0;
          for (int i = 0; i < kp + 1; ++i) s += B[(int64_t)r * (kp + 1) + i] * B[(int64_t)c * (kp + 1) + i];
          S[(int64_t)c * kp + r] = s;
        }
      gko_jacobi_eig(kp, S, sig, G);
      for (int i = 0; i < kp; ++i) *rank += sig[i] > eps ? 1 : 0;
      for (int i = 0; i < kp; ++i) sig[i] = sig[i] > 0.0 ? sqrt(sig[i]) : 0.0;
      free(S);
      free(G);
    }
    if (sigma_out)
      for (int i = 0; i < kp; ++i) sigma_out[i] = sig[i];
    free(sig);
    free(B);
  }
out:
  free(alpha);
  free(beta);
  free(Q);
  free(P);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* sign convention for reported singular vectors                             */
/* ------------------------------------------------------------------------ */

static void sign_normalize(int64_t m, int64_t n, int k, double *U, double *V)
{
  for (int i = 0; i < k; ++i) {
    double *v = V + (int64_t)i * n, *u = U + (int64_t)i * m;
    int64_t best = 0;
    for (int64_t r = 1; r < n; ++r)
      if (fabs(v[r]) > fabs(v[best])) best = r;
    if (v[best] < 0.0) {
      for (int64_t r = 0; r < n; ++r) v[r] = -v[r];
      for (int64_t r = 0; r < m; ++r) u[r] = -u[r];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: F-SVD                                                        */
/* ------------------------------------------------------------------------ */

int gko_fsvd(const gko_op *A, int k, int r, int route, int passes, const double *q1, double *U, double *S,
             double *V, gko_gk_info *info, int fused)
{
  const int64_t m = A->m, n = A->n;
  double *alpha = (double *)malloc(sizeof(double) * (size_t)(k + 1));
  double *beta = (double *)malloc(sizeof(double) * (size_t)(k + 2));
  double *Q = (double *)malloc(sizeof(double) * (size_t)(m * (k + 1)));
  double *P = (double *)malloc(sizeof(double) * (size_t)(n * (k + 1)));
  memset(U, 0, sizeof(double) * (size_t)(m * r));
  memset(V, 0, sizeof(double) * (size_t)(n * r));
  memset(S, 0, sizeof(double) * (size_t)r);
  /* Algorithm 1 with k iterations and no break (eps = 0, absolute) */
  int rc = gko_gk_lower(A, k, 0.0, 0, passes, q1, alpha, beta, Q, P, info, fused);
  if (rc != 0) goto out;
  const int kp = info->kprime;
  if (kp == 0) goto out;
  double *B = build_lower_B(kp, alpha, beta);
  const int rr = r < kp ? r : kp;
  if (route == 0) {
    /* eigen-decomposition of B^T B */
    double *Sm = (double *)calloc((size_t)(kp * kp), sizeof(double));
    double *G = (double *)malloc(sizeof(double) * (size_t)(kp * kp));
    double *th = (double *)malloc(sizeof(double) * (size_t)kp);
    for (int c = 0; c < kp; ++c)
      for (int rw = 0; rw < kp; ++rw) {
        double s = 0.0;
        for (int i = 0; i < kp + 1; ++i) s += B[(int64_t)rw * (kp + 1) + i] * B[(int64_t)c * (kp + 1) + i];
        Sm[(int64_t)c * kp + rw] = s;
      }
    gko_jacobi_eig(kp, Sm, th, G);
    /* V_2 = P V_1, keep the r largest, Sigma_r = sqrt(Sigma_1) */
    for (int i = 0; i < rr; ++i) {
      S[i] = th[i] > 0.0 ? sqrt(th[i]) : 0.0;
      for (int64_t row = 0; row < n; ++row) {
        double s = 0.0;
        for (int c = 0; c < kp; ++c) s += P[(int64_t)c * n + row] * G[(int64_t)i * kp + c];
        V[(int64_t)i * n + row] = s;
      }
      /* u_i = A v_i / sigma_i (Eq. svdV, read as the left vector) */
      gko_apply(A, V + (int64_t)i * n, U + (int64_t)i * m);
      if (S[i] > 0.0)
        for (int64_t row = 0; row < m; ++row) U[(int64_t)i * m + row] /= S[i];
    }
    free(Sm);
    free(G);
    free(th);
  } else {
    /* SVD of B itself: B = X Sigma Y^T, V = P Y, U = Q X */
    double *sg = (double *)malloc(sizeof(double) * (size_t)kp);
    double *X = (double *)malloc(sizeof(double) * (size_t)((kp + 1) * kp));
    double *Y = (double *)malloc(sizeof(double) * (size_t)(kp * kp));
    gko_jacobi_svd(kp + 1, kp, B, sg, X, Y);
    for (int i = 0; i < rr; ++i) {
      S[i] = sg[i];
      for (int64_t row = 0; row < n; ++row) {
        double s = 0.0;
        for (int c = 0; c < kp; ++c) s += P[(int64_t)c * n + row] * Y[(int64_t)i * kp + c];
        V[(int64_t)i * n + row] = s;
      }
      for (int64_t row = 0; row < m; ++row) {
        double s = 0.0;
        for (int c = 0; c < kp + 1; ++c) s += Q[(int64_t)c * m + row] * X[(int64_t)i * (kp + 1) + c];
        U[(int64_t)i * m + row] = s;
      }
    }
    free(sg);
    free(X);
    free(Y);
  }
  sign_normalize(m, n, rr, U, V);
  free(B);
out:
  free(alpha);
  free(beta);
  free(Q);
  free(P);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* restarted partial SVD (upper-bidiagonal form, thick restart)              */
/* ------------------------------------------------------------------------ */

/* Orthonormal extension after an exact breakdown: a replacement direction,
 * orthogonalized twice against the first j basis columns.  Returns 0 if the
 * basis already spans the space (then x is left zero). */
static int extend_basis(double *x, const double *Bs, int64_t len, int64_t ld, int j, uint64_t seed, int64_t *nfresh)
{
  fresh_direction(seed, (*nfresh)++, x, len);
  const double n0 = norm2(x, len);
  cgs(2, x, Bs, len, ld, j);
  const double n1 = norm2(x, len);
  if (!(n1 > 1e-8 * n0)) {
    memset(x, 0, sizeof(double) * (size_t)len);
    return 0;
  }
  for (int64_t i = 0; i < len; ++i) x[i] /= n1;
  return 1;
}

/* relative size below which a new alpha or beta counts as an exact breakdown */
#define BREAKDOWN 0x1.0p-46

static int bidiag_upper_cycle(const gko_op *A, int l, int K, int passes, uint64_t seed, int64_t *nfresh,
                              const double *rho, double *Ub, double *Vb, double *Bm, double *betaK,
                              double *sest, int64_t *matvecs, int fused)
{
  const int64_t m = A->m, n = A->n;
  double *w = (double *)malloc(sizeof(double) * (size_t)m);
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double *zr = fused ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
  double bprev = 0.0;
  for (int j = l; j < K; ++j) {
    /* left step: A v_j minus its components along the kept/previous u's */
    gko_apply(A, Vb + (int64_t)j * n, w);
    ++*matvecs;
    if (j == l && l > 0) {
      for (int i = 0; i < l; ++i)
        for (int64_t r = 0; r < m; ++r) w[r] -= rho[i] * Ub[(int64_t)i * m + r];
    } else if (j > 0) {
      for (int64_t r = 0; r < m; ++r) w[r] -= bprev * Ub[(int64_t)(j - 1) * m + r];
    }
    /* fused sweep: A^T w before reorthogonalization, except at the first step after a
     * restart (w there subtracts the whole kept block) */
    const int fuse = fused && !(j == l && l > 0);
    if (fuse) gko_apply_t(A, w, zr);
    cgs(passes, w, Ub, m, m, j);
    double a = norm2(w, m);
    *sest = fmax(*sest, a);
    if (a <= BREAKDOWN * *sest) {
      a = 0.0;
      extend_basis(Ub + (int64_t)j * m, Ub, m, m, j, seed, nfresh);
    } else {
      scale_into(Ub + (int64_t)j * m, w, 1.0 / a, m);
    }
    Bm[(int64_t)j * K + j] = a;

    /* right step: A^T u_j - alpha_j v_j, orthogonalized against V_{j+1}; the fused sweep
     * takes A^T w / alpha_j for A^T u_j (equal up to span(V_j), since A^T U_{j-1} lies in
     * span(V_j)), unless u_j was replaced after a breakdown */
    if (fuse && a > 0.0) {
      for (int64_t r = 0; r < n; ++r) z[r] = zr[r] / a - a * Vb[(int64_t)j * n + r];
    } else {
      gko_apply_t(A, Ub + (int64_t)j * m, z);
      for (int64_t r = 0; r < n; ++r) z[r] -= a * Vb[(int64_t)j * n + r];
    }
    ++*matvecs;
    cgs(passes, z, Vb, n, n, j + 1);
    double b = norm2(z, n);
    *sest = fmax(*sest, b);
    if (b <= BREAKDOWN * *sest) {
      b = 0.0;
      extend_basis(Vb + (int64_t)(j + 1) * n, Vb, n, n, j + 1, seed, nfresh);
    } else {
      scale_into(Vb + (int64_t)(j + 1) * n, z, 1.0 / b, n);
    }
    if (j + 1 < K) Bm[(int64_t)(j + 1) * K + j] = b; /* superdiagonal B[j, j+1] */
    bprev = b;
  }
  *betaK = bprev;
  free(w);
  free(z);
  free(zr);
  return 0;
}

int gko_gk_upper(const gko_op *A, int K, int passes, const double *q1, uint64_t seed, double *alpha,
                 double *beta, double *Ub, double *Vb, int fused)
{
  const int64_t m = A->m, n = A->n;
  const int64_t mn = m < n ? m : n;
  if (K < 1 || K > mn) return -1;
  memset(Ub, 0, sizeof(double) * (size_t)(m * K));
  memset(Vb, 0, sizeof(double) * (size_t)(n * (K + 1)));
  double *qn = (double *)malloc(sizeof(double) * (size_t)m);
  const double b1 = norm2(q1, m);
  scale_into(qn, q1, 1.0 / b1, m);
  gko_apply_t(A, qn, Vb);
  int64_t nfresh = 0, mv = 0;
  const double nv = norm2(Vb, n);
  if (nv > 0.0)
    for (int64_t r = 0; r < n; ++r) Vb[r] /= nv;
  else
    extend_basis(Vb, Vb, n, n, 0, seed, &nfresh);
  double *Bm = (double *)calloc((size_t)K * K, sizeof(double));
  double sest = 0.0, betaK = 0.0;
  bidiag_upper_cycle(A, 0, K, passes, seed, &nfresh, NULL, Ub, Vb, Bm, &betaK, &sest, &mv, fused);
  for (int j = 0; j < K; ++j) {
    alpha[j] = Bm[(int64_t)j * K + j];
    beta[j] = (j + 1 < K) ? Bm[(int64_t)(j + 1) * K + j] : betaK;
  }
  free(Bm);
  free(qn);
  return 0;
}

int gko_psvd(const gko_op *A, int k, int K, int keep, double tol, int max_restarts, int passes,
             const double *q1, uint64_t seed, double *U, double *S, double *V, gko_psvd_info *info, int fused)
{
  const int64_t m = A->m, n = A->n;
  const int64_t mn = m < n ? m : n;
  memset(info, 0, sizeof(*info));
  if (k < 1 || k > mn || K < k || K > mn || passes < 0 || passes > 3) return -1;
  if (K == k && K < mn) return -1; /* a restart needs room beyond the k wanted vectors */
  if (keep <= 0) keep = k + (K - k) / 2;
  if (keep < k) keep = k;
  if (keep >= K) keep = K - 1;
  if (keep < 0) keep = 0;

  double *Ub = (double *)calloc((size_t)(m * K), sizeof(double));
  double *Vb = (double *)calloc((size_t)(n * (K + 1)), sizeof(double));
  double *Un = (double *)calloc((size_t)(m * K), sizeof(double));
  double *Vn = (double *)calloc((size_t)(n * (K + 1)), sizeof(double));
  double *Bm = (double *)calloc((size_t)K * K, sizeof(double));
  double *sg = (double *)malloc(sizeof(double) * (size_t)K);
  double *X = (double *)malloc(sizeof(double) * (size_t)K * K);
  double *Y = (double *)malloc(sizeof(double) * (size_t)K * K);
  double *rho = (double *)calloc((size_t)K, sizeof(double));
  double *res = (double *)malloc(sizeof(double) * (size_t)K);
  int64_t nfresh = 0;
  double sest = 0.0;

  /* v_1 = A^T q_1 / ||A^T q_1|| (Algorithm 1) */
  {
    double *qn = (double *)malloc(sizeof(double) * (size_t)m);
    const double b1 = norm2(q1, m);
    scale_into(qn, q1, 1.0 / b1, m);
    gko_apply_t(A, qn, Vb);
    info->matvecs++;
    const double nv = norm2(Vb, n);
    if (nv > 0.0)
      for (int64_t r = 0; r < n; ++r) Vb[r] /= nv;
    else
      extend_basis(Vb, Vb, n, n, 0, seed, &nfresh);
    free(qn);
  }

  int l = 0, rc = 1;
  for (int cycle = 0;; ++cycle) {
    memset(Bm, 0, sizeof(double) * (size_t)K * K);
    for (int i = 0; i < l; ++i) {
      Bm[(int64_t)i * K + i] = sg[i];  /* kept Ritz values on the diagonal */
      Bm[(int64_t)l * K + i] = rho[i]; /* coupling column l */
    }
    double betaK = 0.0;
    bidiag_upper_cycle(A, l, K, passes, seed, &nfresh, rho, Ub, Vb, Bm, &betaK, &sest, &info->matvecs, fused);
    info->cycles = cycle + 1;

    /* SVD of the small K x K matrix: B = X Sigma Y^T */
    gko_jacobi_svd(K, K, Bm, sg, X, Y);
    sest = fmax(sest, sg[0]);
    /* Ritz residuals: ||A^T u~_i - sigma_i v~_i|| = |beta_K X_{K,i}| */
    double rmax = 0.0;
    for (int i = 0; i < K; ++i) res[i] = fabs(betaK * X[(int64_t)i * K + (K - 1)]);
    for (int i = 0; i < k; ++i) rmax = fmax(rmax, res[i]);
    const int conv = rmax <= tol * sg[0];
    info->resid_est_max = sg[0] > 0.0 ? rmax / sg[0] : 0.0;
    info->kdim_used = K;

    if (conv || cycle >= max_restarts) {
      for (int i = 0; i < k; ++i) {
        S[i] = sg[i];
        for (int64_t r = 0; r < m; ++r) {
          double s = 0.0;
          for (int c = 0; c < K; ++c) s += Ub[(int64_t)c * m + r] * X[(int64_t)i * K + c];
          U[(int64_t)i * m + r] = s;
        }
        for (int64_t r = 0; r < n; ++r) {
          double s = 0.0;
          for (int c = 0; c < K; ++c) s += Vb[(int64_t)c * n + r] * Y[(int64_t)i * K + c];
          V[(int64_t)i * n + r] = s;
        }
      }
      sign_normalize(m, n, k, U, V);
      info->converged = conv;
      rc = conv ? 0 : 1;
      break;
    }

    /* thick restart: keep the `keep` leading Ritz vectors and v_{K+1} */
    for (int i = 0; i < keep; ++i) {
      for (int64_t r = 0; r < m; ++r) {
        double s = 0.0;
        for (int c = 0; c < K; ++c) s += Ub[(int64_t)c * m + r] * X[(int64_t)i * K + c];
        Un[(int64_t)i * m + r] = s;
      }
      for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int c = 0; c < K; ++c) s += Vb[(int64_t)c * n + r] * Y[(int64_t)i * K + c];
        Vn[(int64_t)i * n + r] = s;
      }
      rho[i] = betaK * X[(int64_t)i * K + (K - 1)];
    }
    memcpy(Vn + (int64_t)keep * n, Vb + (int64_t)K * n, sizeof(double) * (size_t)n);
    double *t;
    t = Ub; Ub = Un; Un = t;
    t = Vb; Vb = Vn; Vn = t;
    l = keep;
    info->restarts++;
  }

  free(Ub); free(Vb); free(Un); free(Vn); free(Bm);
  free(sg); free(X); free(Y); free(rho); free(res);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* error metrics (Section 5: err_rel, err_res) and per-triplet residuals    */
/* ------------------------------------------------------------------------ */

void gko_residuals(const gko_op *A, int k, const double *U, const double *S, const double *V, double *res_av,
                   double *res_atu)
{
  const int64_t m = A->m, n = A->n;
  double *w = (double *)malloc(sizeof(double) * (size_t)m);
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < k; ++i) {
    gko_apply(A, V + (int64_t)i * n, w);
    for (int64_t r = 0; r < m; ++r) w[r] -= S[i] * U[(int64_t)i * m + r];
    res_av[i] = norm2(w, m);
    gko_apply_t(A, U + (int64_t)i * m, z);
    for (int64_t r = 0; r < n; ++r) z[r] -= S[i] * V[(int64_t)i * n + r];
    res_atu[i] = norm2(z, n);
  }
  free(w);
  free(z);
}

double gko_err_rel(const gko_op *A, int k, const double *U, const double *S, const double *V)
{
  const int64_t m = A->m, n = A->n;
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double num = 0.0, den = 0.0;
  for (int i = 0; i < k; ++i) {
    gko_apply_t(A, U + (int64_t)i * m, z);
    for (int64_t r = 0; r < n; ++r) {
      const double d = z[r] - V[(int64_t)i * n + r] * S[i];
      num += d * d;
    }
    den += S[i] * S[i];
  }
  free(z);
  return den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
}

double gko_err_res(const gko_op *A, int k, const double *U, const double *S, const double *V)
{
  if (A->kind != GKO_DENSE) return -1.0;
  const int64_t m = A->m, n = A->n;
  double tot = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : tot)
  for (int64_t r = 0; r < m; ++r) {
    for (int64_t c = 0; c < n; ++c) {
      double s = stored_value(A, r * A->ld + c);
      for (int i = 0; i < k; ++i) s -= U[(int64_t)i * m + r] * S[i] * V[(int64_t)i * n + c];
      tot += s * s;
    }
  }
  return sqrt(tot);
}
