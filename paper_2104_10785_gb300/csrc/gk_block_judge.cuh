// gk_block_judge.cuh -- the arithmetic of one block judge of block Golub-Kahan: the 2-norm of a
// block's triangular factor T = triu(raw) (s x s, column-major) and the break tests on it.
//
// ||T||_2 = mu sqrt(lambda_max(G)) with mu = max |t_ac| and G = (T / mu)^T (T / mu): the scaling
// keeps G inside the exponent range for any finite T (an unscaled G overflows past ~1e154 and
// underflows below ~1e-162, where a nonzero block would read as zero and pass the break test).
// lambda_max by cyclic Jacobi: a rotation for each pair (p, q) while |g_pq| > 1e-16 sqrt(|g_pp
// g_qq|), at most kBlockSweeps sweeps; the largest diagonal entry is a lower bound on lambda_max
// at any point and equals it on convergence.  Each rotation updates columns p, q of G and then
// rows p, q, one entry per lane (distinct entries in each phase), so the warp's lanes run the
// updates in parallel between two warp barriers and the host tests run the same functions lane
// after lane.  The break tests (Algorithm 1's, with block norms):
//   side 0 (S_{j+1}, left block): sest = max(sest, ||T||), break when eps > 0 and ||T|| <= eps sest;
//   side 1 (R_{j+1}, right block): break when eps > 0 and ||T|| <= eps max(sest, ||T||), else
//     sest = max(sest, ||T||);
//   side 2 (R_1, the first right block): no test, sest = max(sest, ||T||);
// a non-finite norm breaks with status 2.
#pragma once

#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace gk {

constexpr int kBlockSweeps = 60;

// entry e = a + c s of T = triu(raw)
__host__ __device__ inline double bj_triu(const double *raw, int s, int e) {
  return (e % s) <= (e / s) ? raw[e] : 0.0;
}

// max(m, v) that propagates NaN (fmax would drop it, and a NaN block would then read as finite)
__host__ __device__ inline double bj_absmax(double m, double v) { return (v != v || m != m) ? v + m : fmax(m, v); }

// 1 / mu for a positive finite mu, else 0 (a zero block: G = 0; a non-finite one: the norm is
// non-finite through mu)
__host__ __device__ inline double bj_rscale(double mu) { return (mu > 0.0 && isfinite(mu)) ? 1.0 / mu : 0.0; }

// entry e = p + q s of G = (T / mu)^T (T / mu), rmu = bj_rscale(mu)
__host__ __device__ inline double bj_gram(const double *T, int s, double rmu, int e) {
  const int p = e % s, q = e / s;
  double v = 0.0;
  for (int a = 0; a < s; ++a) v = fma(T[a + p * s] * rmu, T[a + q * s] * rmu, v);
  return v;
}

// the rotation [c sn; -sn c] that zeroes g_pq in J^T G J (the symmetric 2 x 2 Schur
// decomposition); false when g_pq is already negligible
__host__ __device__ inline bool bj_rotation(const double *G, int s, int p, int q, double *c, double *sn) {
  const double apq = G[p + q * s], app = G[p + p * s], aqq = G[q + q * s];
  if (apq == 0.0 || fabs(apq) <= 1e-16 * sqrt(fabs(app) * fabs(aqq))) return false;
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = fabs(tau) > 1e150 ? 0.5 / tau : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  *c = 1.0 / sqrt(1.0 + t * t);
  *sn = t * *c;
  return true;
}

// G <- G J on columns p, q: the lane's row
__host__ __device__ inline void bj_col(double *G, int s, int p, int q, double c, double sn, int lane) {
  const double gp = G[lane + p * s], gq = G[lane + q * s];
  G[lane + p * s] = c * gp - sn * gq;
  G[lane + q * s] = sn * gp + c * gq;
}

// G <- J^T G on rows p, q: the lane's column
__host__ __device__ inline void bj_row(double *G, int s, int p, int q, double c, double sn, int lane) {
  const double gp = G[p + lane * s], gq = G[q + lane * s];
  G[p + lane * s] = c * gp - sn * gq;
  G[q + lane * s] = sn * gp + c * gq;
}

// ||T||_2 from the converged G and mu, then the side's break test: updates *sest, returns the
// break status (0 go on, 1 break, 2 non-finite)
__host__ __device__ inline int bj_decide(const double *G, int s, double mu, int side, double eps, double *sest,
                                         double *nrm_out) {
  double lmax = 0.0;
  for (int p = 0; p < s; ++p) lmax = bj_absmax(lmax, G[p + p * s]);
  const double nrm = isfinite(mu) ? mu * sqrt(lmax) : mu + mu;  // inf or NaN for a non-finite block
  *nrm_out = nrm;
  if (!isfinite(nrm)) return 2;
  if (side == 0) {
    *sest = fmax(*sest, nrm);
    return (eps > 0.0 && nrm <= eps * *sest) ? 1 : 0;
  }
  if (side == 1) {
    if (eps > 0.0 && nrm <= eps * fmax(*sest, nrm)) return 1;
    *sest = fmax(*sest, nrm);
    return 0;
  }
  *sest = fmax(*sest, nrm);
  return 0;
}

// where entry (a, c), a <= c, of T goes in B (column-major, ld ldb): T at (row0 + a, col0 + c)
// for a left block (side 0), T^T at (row0 + c, col0 + a) for a right block
__host__ __device__ inline long long bj_place(int side, int row0, int col0, int a, int c, long long ldb) {
  return side == 0 ? (long long)(row0 + a) + (long long)(col0 + c) * ldb
                   : (long long)(row0 + c) + (long long)(col0 + a) * ldb;
}

}  // namespace gk
