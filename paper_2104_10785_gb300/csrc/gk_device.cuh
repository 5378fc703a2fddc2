// gk_device.cuh -- device routines shared by the stand-alone kernels and the
// batched solver: the cluster-parallel one-sided Jacobi SVD and the Sturm-count
// rank of a lower-bidiagonal matrix.
#pragma once

#include <cooperative_groups.h>
#include <float.h>
#include <math.h>

#include "gk_internal.cuh"

namespace gk {
namespace dev {
namespace {  // internal linkage: each translation unit keeps its own copy

namespace cg = cooperative_groups;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// tournament (circle method) pairing: round r, slot s of Kp players
__device__ __forceinline__ int player(int r, int s, int Kp) { return s == 0 ? 0 : ((s - 1 + r) % (Kp - 1)) + 1; }

// One-sided (Hestenes) Jacobi SVD of the K x K matrix B on the calling thread-block
// cluster.  Each round of the tournament ordering rotates Kp/2 disjoint column
// pairs, one pair per warp across the cluster; the cluster barrier
// (release/acquire at cluster scope) separates the rounds.  The columns of B
// and of the accumulated right rotations Yw live in global memory, read with
// ld.global.cg so that no stale L1 line survives a round.  A sweep that rotates
// no pair ends the iteration; the CTAs agree on that through their
// shared-memory flags s_rot (read by the others through distributed shared
// memory).  Outputs: sigma (descending, stable by index), X = B's columns
// normalized, Y = the rotations, in that order.  Returns the sweeps used
// (negative if the sweep limit was reached).  Every thread of the cluster must
// call it.
// NL > 0 (K <= 32 NL): each lane loads its NL elements of the four columns of its pair
// (B's p and q, Yw's p and q) at once into registers, so a round costs one L2 round trip
// instead of one per element group and pass; the arithmetic and its order are the same
// as with NL = 0, which walks the columns in memory (any K).
template <int NL = 0>
__device__ int cluster_jacobi(cg::cluster_group &cl, double *__restrict__ B, double *__restrict__ Yw, int K,
                              double *__restrict__ sigma, double *__restrict__ X, double *__restrict__ Y,
                              double *__restrict__ nrm, int *__restrict__ pos, int *s_rot, int *s_any) {
  const unsigned crank = cl.block_rank(), csize = cl.num_blocks();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int gw = (int)crank * nw + warp, gnw = (int)csize * nw;
  const int64_t gtid = (int64_t)crank * blockDim.x + threadIdx.x, gthreads = (int64_t)csize * blockDim.x;
  for (int64_t idx = gtid; idx < (int64_t)K * K; idx += gthreads) Yw[idx] = ((idx % K) == (idx / K)) ? 1.0 : 0.0;
  const int Kp = K + (K & 1);
  const double tol = fmax(2.0 * sqrt((double)K) * 0x1.0p-52, (double)K * 0x1.0p-53);
  int sweep, done = 0;
  cl.sync();
  for (sweep = 1; sweep <= 80; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    for (int r = 0; r < Kp - 1; ++r) {
      for (int pi = gw; pi < Kp / 2; pi += gnw) {
        int p = player(r, pi, Kp), q = player(r, Kp - 1 - pi, Kp);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q >= K) continue;
        double *bp = B + (int64_t)p * K, *bq = B + (int64_t)q * K;
        double *yp = Yw + (int64_t)p * K, *yq = Yw + (int64_t)q * K;
        if constexpr (NL > 0) {
          double xb[NL], yb[NL], xy[NL], yy[NL];
#pragma unroll
          for (int e = 0; e < NL; ++e) {
            const int i = lane + 32 * e;
            xb[e] = yb[e] = xy[e] = yy[e] = 0.0;
            if (i < K) {
              xb[e] = __ldcg(bp + i);
              yb[e] = __ldcg(bq + i);
              xy[e] = __ldcg(yp + i);
              yy[e] = __ldcg(yq + i);
            }
          }
          double a = 0.0, b = 0.0, c = 0.0;
#pragma unroll
          for (int e = 0; e < NL; ++e) {
            if (lane + 32 * e < K) {
              a = fma(xb[e], xb[e], a);
              b = fma(yb[e], yb[e], b);
              c = fma(xb[e], yb[e], c);
            }
          }
          a = warp_sum_d(a);
          b = warp_sum_d(b);
          c = warp_sum_d(c);
          if (c == 0.0 || fabs(c) <= tol * sqrt(a) * sqrt(b)) continue;
          if (lane == 0) *s_rot = 1;
          const double zeta = (b - a) / (2.0 * c);
          const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                              : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
#pragma unroll
          for (int e = 0; e < NL; ++e) {
            const int i = lane + 32 * e;
            if (i < K) {
              bp[i] = cs * xb[e] - sn * yb[e];
              bq[i] = sn * xb[e] + cs * yb[e];
              yp[i] = cs * xy[e] - sn * yy[e];
              yq[i] = sn * xy[e] + cs * yy[e];
            }
          }
        } else {
          double a = 0.0, b = 0.0, c = 0.0;
          for (int i = lane; i < K; i += 32) {
            const double x = __ldcg(bp + i), y = __ldcg(bq + i);
            a = fma(x, x, a);
            b = fma(y, y, b);
            c = fma(x, y, c);
          }
          a = warp_sum_d(a);
          b = warp_sum_d(b);
          c = warp_sum_d(c);
          if (c == 0.0 || fabs(c) <= tol * sqrt(a) * sqrt(b)) continue;
          if (lane == 0) *s_rot = 1;
          // rotation that makes columns p and q orthogonal (Rutishauser's formula)
          const double zeta = (b - a) / (2.0 * c);
          const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                              : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          for (int i = lane; i < K; i += 32) {
            const double x = __ldcg(bp + i), y = __ldcg(bq + i);
            bp[i] = cs * x - sn * y;
            bq[i] = sn * x + cs * y;
          }
          for (int i = lane; i < K; i += 32) {
            const double x = __ldcg(yp + i), y = __ldcg(yq + i);
            yp[i] = cs * x - sn * y;
            yq[i] = sn * x + cs * y;
          }
        }
      }
      cl.sync();
    }
    if (threadIdx.x == 0) {
      int any = 0;
      for (unsigned qr = 0; qr < csize; ++qr) any |= *cl.map_shared_rank(s_rot, qr);
      *s_any = any;
    }
    cl.sync();  // every CTA has read every flag before any CTA clears its own
    if (!*s_any) {
      done = 1;
      break;
    }
  }
  // singular values = column norms, ordered descending (stable by index)
  for (int c = gw; c < K; c += gnw) {
    const double *bc = B + (int64_t)c * K;
    double sq = 0.0;
    for (int i = lane; i < K; i += 32) {
      const double v = __ldcg(bc + i);
      sq = fma(v, v, sq);
    }
    sq = warp_sum_d(sq);
    if (lane == 0) nrm[c] = sqrt(sq);
  }
  cl.sync();
  for (int64_t c = gtid; c < K; c += gthreads) {
    const double nc = __ldcg(nrm + c);
    int rk = 0;
    for (int o = 0; o < K; ++o) {
      const double no = __ldcg(nrm + o);
      rk += (no > nc) || (no == nc && o < c);
    }
    pos[c] = rk;
  }
  cl.sync();
  for (int c = gw; c < K; c += gnw) {
    const int pc = __ldcg(pos + c);
    const double nc = __ldcg(nrm + c);
    for (int i = lane; i < K; i += 32) {
      X[(int64_t)pc * K + i] = nc > 0.0 ? __ldcg(B + (int64_t)c * K + i) / nc : 0.0;
      Y[(int64_t)pc * K + i] = __ldcg(Yw + (int64_t)c * K + i);
    }
    if (lane == 0) sigma[pc] = nc;
  }
  cl.sync();
  return done ? sweep : -(sweep - 1);
}

// Rank count of Algorithm 3 for the lower-bidiagonal B_{kp+1,kp} (diagonal
// alpha[0..kp-1], subdiagonal beta[1..kp]): its Golub-Kahan tridiagonal (zero
// diagonal, off-diagonals alpha_1, beta_2, alpha_2, ..., beta_{kp+1}) has the
// eigenvalues +-sigma_i(B) and 0, so Sturm counts (negative pivots of T - xI)
// count singular values.  sigma_1 by multisection with one evaluation point per
// thread, rank = #{sigma > eps*sigma_1} (or > eps) by one more count; sigma
// (optional) gets every singular value by bisection.  Called by every thread of
// one block (blockDim.x <= 1024).
// off-diagonal i (0-based) of the Golub-Kahan tridiagonal of the lower-bidiagonal B:
// alpha_1, beta_2, alpha_2, beta_3, ..., alpha_kp, beta_{kp+1}
__device__ __forceinline__ double gk_offdiag(const double *alpha, const double *beta, int i) {
  return (i & 1) ? beta[(i + 1) >> 1] : alpha[i >> 1];
}

// number of eigenvalues of T (size N = 2kp+1, zero diagonal) below x: negative pivots of T - xI
__device__ __forceinline__ int count_below(const double *alpha, const double *beta, int kp, double x, double pivmin) {
  const int N = 2 * kp + 1;
  double d = -x;
  if (fabs(d) < pivmin) d = -pivmin;
  int cnt = d < 0.0;
  for (int i = 1; i < N; ++i) {
    const double e = gk_offdiag(alpha, beta, i - 1);
    d = -x - (e * e) / d;
    if (fabs(d) < pivmin) d = -pivmin;
    cnt += d < 0.0;
  }
  return cnt;
}

// red: shared scratch of blockDim.x doubles
__device__ void block_bidiag_rank(const double *__restrict__ alpha, const double *__restrict__ beta, int kp, double eps,
                                  int eps_rel, int *__restrict__ rank, double *__restrict__ sigma1,
                                  double *__restrict__ sigma, double *__restrict__ red) {
  __shared__ int tbest;
  __shared__ double lo_s, hi_s;
  const int T = blockDim.x;
  if (kp <= 0) {
    if (threadIdx.x == 0) {
      *rank = 0;
      *sigma1 = 0.0;
    }
    return;
  }
  const int N = 2 * kp + 1;
  // Gershgorin bound on the spectrum and the pivot floor
  double g = 0.0, emax = 0.0;
  for (int i = threadIdx.x; i < N; i += T) {
    const double l = i > 0 ? fabs(gk_offdiag(alpha, beta, i - 1)) : 0.0;
    const double r = i < N - 1 ? fabs(gk_offdiag(alpha, beta, i)) : 0.0;
    g = fmax(g, l + r);
    emax = fmax(emax, r);
  }
  red[threadIdx.x] = g;
  __syncthreads();
  for (int o = T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const double gmax = red[0];
  __syncthreads();
  red[threadIdx.x] = emax;
  __syncthreads();
  for (int o = T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const double pivmin = DBL_MIN * fmax(1.0, red[0] * red[0]);
  if (threadIdx.x == 0) {
    lo_s = 0.0;
    hi_s = gmax * (1.0 + 0x1.0p-40) + DBL_MIN;
  }
  __syncthreads();
  // sigma_1 by multisection: T evaluation points per round
  for (int round = 0; round < 10; ++round) {
    const double lo = lo_s, hi = hi_s;
    if (!(hi - lo > 0x1.0p-54 * hi)) break;
    const double x = lo + (hi - lo) * (double)(threadIdx.x + 1) / (double)(T + 1);
    const int above = N - count_below(alpha, beta, kp, x, pivmin);  // eigenvalues >= x
    if (threadIdx.x == 0) tbest = -1;
    __syncthreads();
    if (above >= 1) atomicMax(&tbest, (int)threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int t = tbest;
      const double nlo = t >= 0 ? lo + (hi - lo) * (double)(t + 1) / (double)(T + 1) : lo;
      const double nhi = (t + 1 < T) ? lo + (hi - lo) * (double)(t + 2) / (double)(T + 1) : hi;
      lo_s = nlo;
      hi_s = nhi;
    }
    __syncthreads();
  }
  const double s1 = 0.5 * (lo_s + hi_s);
  if (threadIdx.x == 0) {
    *sigma1 = s1;
    const double thr = eps_rel ? eps * s1 : eps;
    // #{sigma > thr} = #{eigenvalues >= next double above thr}
    const double xt = thr > 0.0 ? __longlong_as_double(__double_as_longlong(thr) + 1) : DBL_MIN;
    *rank = (s1 > 0.0) ? N - count_below(alpha, beta, kp, xt, pivmin) : 0;
  }
  if (sigma) {
    // every singular value of B by bisection on its index
    for (int i = threadIdx.x; i < kp; i += T) {
      double lo = 0.0, hi = hi_s;
      for (int it = 0; it < 100 && hi - lo > 0x1.0p-53 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (N - count_below(alpha, beta, kp, mid > 0.0 ? mid : DBL_MIN, pivmin) >= i + 1)
          lo = mid;
        else
          hi = mid;
      }
      sigma[i] = 0.5 * (lo + hi);
    }
  }
}


}  // namespace
}  // namespace dev
}  // namespace gk
