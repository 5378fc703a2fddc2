// gk_bdsvd.cuh -- SVD of an upper-bidiagonal matrix by implicitly shifted QR sweeps: the
// Golub-Kahan SVD step with a Wilkinson shift (Golub & Van Loan, "Matrix Computations",
// Algorithm 8.6.2), with the zero-diagonal chases of the same section.
//
// B (n x n): d[k] = B[k][k], e[k] = B[k][k+1].  B = X diag(sigma) Y^T is reached as a product of
// plane rotations: each step of the iteration records its rotations -- left ones, acting on two
// rows of B, and right ones, acting on two columns -- and the singular-vector matrices take them
// column pair by column pair (X from the left rotations, Y from the right ones; both start as
// the identity).  The work splits in two:
//   * bd_step, scalar: deflation (|e_k| <= tol (|d_k| + |d_k+1|) is set to zero), the active
//     block, then either one Golub-Kahan step on it (shift: the eigenvalue of the trailing 2 x 2
//     of B^T B closer to its last entry) or, for a diagonal entry <= tol ||B||, the chase that
//     zeroes its row's (or, at the block's end, its column's) off-diagonal entry;
//   * bd_apply_row / bd_apply_chase, per row of X or Y: the step's rotations in order, on that
//     row's entries (bd_apply_chase for the adjacent pairs of a Golub-Kahan step, with the
//     running entry in a register).
// The GPU kernel runs bd_step on one thread and the row functions on one thread per row; the
// CPU tests run the same functions on the host.
#pragma once

#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace gk {

// a plane rotation of entries (i, j) of a row: x_i' = c x_i + s x_j, x_j' = -s x_i + c x_j
struct BdRot {
  int i, j;
  double c, s;
};

struct BdState {
  int n;
  double tol;     // relative threshold of the deflation test
  double small;   // absolute threshold below which a diagonal entry counts as zero
  int steps;      // steps taken
  int max_steps;  // the iteration gives up after this many (then bd_step reports -1)
};

// c, s with [a b] [c -s; s c] = [r 0] (r = hypot(a, b) >= 0); c = 1, s = 0 for a = b = 0
__host__ __device__ inline void bd_givens(double a, double b, double *c, double *s, double *r) {
  if (b == 0.0) {
    *c = a >= 0.0 ? 1.0 : -1.0;
    *s = 0.0;
    *r = fabs(a);
    return;
  }
  const double h = hypot(a, b), inv = 1.0 / h;  // one division per rotation
  *c = a * inv;
  *s = b * inv;
  *r = h;
}

__host__ __device__ inline void bd_init(BdState *st, const double *d, const double *e, int n) {
  double nb = 0.0;
  for (int k = 0; k < n; ++k) nb = fmax(nb, fabs(d[k]));
  for (int k = 0; k + 1 < n; ++k) nb = fmax(nb, fabs(e[k]));
  st->n = n;
  st->tol = 4.0 * 1.1102230246251565e-16;  // a few units of roundoff
  st->small = st->tol * nb;
  st->steps = 0;
  st->max_steps = 30 * n * n + 100;
}

// One step.  Returns 0 when B is diagonal (done), -1 when the step budget is spent, else the
// step's rotations are in rotL[0..*nL) (left: rows) and rotR[0..*nR) (right: columns) and the
// return value says their shape: 1 for a Golub-Kahan step (both lists are (k, k+1) for
// k = lo, lo+1, ..., hi-1, so bd_apply_chase may apply them), 2 for a zero-diagonal chase
// (any pairs: bd_apply_row).  rotL and rotR need room for n - 1 rotations each.
__host__ __device__ inline int bd_step(double *d, double *e, BdState *st, BdRot *rotL, int *nL, BdRot *rotR, int *nR) {
  const int n = st->n;
  *nL = 0;
  *nR = 0;
  for (int k = 0; k + 1 < n; ++k)
    if (fabs(e[k]) <= st->tol * (fabs(d[k]) + fabs(d[k + 1]))) e[k] = 0.0;
  // the active block [lo, hi]: the lowest run of nonzero off-diagonal entries
  int hi = n - 1;
  while (hi > 0 && e[hi - 1] == 0.0) --hi;
  if (hi == 0) return 0;
  if (st->steps >= st->max_steps) return -1;
  ++st->steps;
  int lo = hi - 1;
  while (lo > 0 && e[lo - 1] != 0.0) --lo;
  // a (numerically) zero diagonal entry inside the block: chase its off-diagonal entry out
  for (int k = lo; k <= hi; ++k) {
    if (fabs(d[k]) > st->small) continue;
    d[k] = 0.0;
    if (k < hi) {
      // row k holds f = e[k] at column k+1: left rotations of rows (j, k), j = k+1..hi, move it
      // right until it leaves the block (B[k][j] zeroed against B[j][j])
      double f = e[k];
      e[k] = 0.0;
      for (int j = k + 1; j <= hi; ++j) {
        double c, s, r;
        bd_givens(d[j], f, &c, &s, &r);
        d[j] = r;
        rotL[(*nL)++] = BdRot{j, k, c, s};
        if (j < hi) {
          f = -s * e[j];
          e[j] = c * e[j];
        }
      }
    } else {
      // the last diagonal entry is zero: right rotations of columns (j, hi), j = hi-1..lo, move
      // B[j][hi] up (B[j][hi] zeroed against B[j][j])
      double f = e[hi - 1];
      e[hi - 1] = 0.0;
      for (int j = hi - 1; j >= lo; --j) {
        double c, s, r;
        bd_givens(d[j], f, &c, &s, &r);
        d[j] = r;
        rotR[(*nR)++] = BdRot{j, hi, c, s};
        if (j > lo) {
          f = -s * e[j - 1];
          e[j - 1] = c * e[j - 1];
        }
      }
    }
    return 2;
  }
  // Wilkinson shift from the trailing 2 x 2 of B^T B on the block
  const double dm = d[hi - 1], dn = d[hi], em = e[hi - 1];
  const double el = hi - 1 > lo ? e[hi - 2] : 0.0;
  const double t11 = dm * dm + el * el, t12 = dm * em, t22 = dn * dn + em * em;
  const double del = 0.5 * (t11 - t22);
  const double den = del + (del >= 0.0 ? 1.0 : -1.0) * hypot(del, t12);
  const double mu = den != 0.0 ? t22 - t12 * t12 / den : t22;
  // the bulge chase: right rotation (k, k+1) from [y z], then left rotation (k, k+1) to clear
  // the subdiagonal entry it made
  double y = d[lo] * d[lo] - mu, z = d[lo] * e[lo];
  for (int k = lo; k < hi; ++k) {
    double c, s, r;
    bd_givens(y, z, &c, &s, &r);
    rotR[(*nR)++] = BdRot{k, k + 1, c, s};
    // columns k, k+1 of rows k-1, k, k+1
    if (k > lo) e[k - 1] = r;  // row k-1: [e_{k-1}, bulge] -> [r, 0]
    double bkk = c * d[k] + s * e[k];
    double bk1 = -s * d[k] + c * e[k];
    double bulge = s * d[k + 1];  // B[k+1][k]
    double bk11 = c * d[k + 1];   // B[k+1][k+1]
    // left rotation of rows k, k+1 zeroing B[k+1][k]
    bd_givens(bkk, bulge, &c, &s, &r);
    rotL[(*nL)++] = BdRot{k, k + 1, c, s};
    d[k] = r;
    e[k] = c * bk1 + s * bk11;
    d[k + 1] = -s * bk1 + c * bk11;
    if (k + 1 < hi) {
      y = e[k];
      z = s * e[k + 1];  // the new bulge B[k][k+2]
      e[k + 1] = c * e[k + 1];
    }
  }
  return 1;
}

// the rotations rot[0..nrot) in order on one row, entries at x[k * stride]
__host__ __device__ inline void bd_apply_row(double *x, long long stride, const BdRot *rot, int nrot) {
  for (int t = 0; t < nrot; ++t) {
    const BdRot R = rot[t];
    double *pi = x + (long long)R.i * stride, *pj = x + (long long)R.j * stride;
    const double a = *pi, b = *pj;
    *pi = R.c * a + R.s * b;
    *pj = -R.s * a + R.c * b;
  }
}

// the rotations of a Golub-Kahan step (pairs (k, k+1), k increasing from rot[0].i) on one row:
// each entry is read once and written once, the running entry carried in a register
__host__ __device__ inline void bd_apply_chase(double *x, long long stride, const BdRot *rot, int nrot) {
  if (nrot <= 0) return;
  const int k0 = rot[0].i;
  double carry = x[(long long)k0 * stride];
  for (int t = 0; t < nrot; ++t) {
    const double b = x[(long long)(k0 + t + 1) * stride];
    const double c = rot[t].c, s = rot[t].s;
    x[(long long)(k0 + t) * stride] = c * carry + s * b;
    carry = -s * carry + c * b;
  }
  x[(long long)(k0 + nrot) * stride] = carry;
}

}  // namespace gk
