// gk_block.cu -- the small kernels of block Golub-Kahan with s start vectors (gk_block_numrank).
//
// The block recurrence replaces each vector of Algorithm 1 by an m x s (or n x s) block and
// each normalization by a QR factorization with diag(R) >= 0:
//   Q_1 R_0 = Q0,  P_1 R_1 = A^T Q_1,
//   Q_{j+1} S_{j+1} = A P_j - Q_j R_j^T,   P_{j+1} R_{j+1} = A^T Q_{j+1} - P_j S_{j+1}^T,
// each new block reorthogonalized against the earlier ones, so that A [P_1..P_k] =
// [Q_1..Q_{k+1}] B with B block lower bidiagonal (diagonal blocks R_j^T, subdiagonal blocks
// S_{j+1}), the block form of Eq. 2.2.  The host driver (gk_api.cu) forms a block's columns
// one at a time by classical Gram-Schmidt (two passes) against every basis column so far:
// that is the QR of the block after its reorthogonalization, and the triangular factor is
// Q_{j+1}^T (A P_j) (resp. P_{j+1}^T (A^T Q_{j+1})) because each new column is orthogonal to
// the earlier blocks.  These kernels form those s x s inner products, keep their upper
// triangle, place it (or its transpose) into B, and judge the block's 2-norm:
//   * k_block_dots / k_block_dots_sum: raw = X^T Y for two len x s column blocks, f64, the
//     row chunks summed in a fixed order;
//   * k_block_judge: T = triu(raw), ||T||_2 by cyclic Jacobi on the scaled T^T T on one warp,
//     the running estimate of sigma_1 and the block break tests (the arithmetic in
//     gk_block_judge.cuh, which the CPU tests also build for the host);
//   * k_block_count: Algorithm 3's count of the singular values of B above eps sigma_1(B);
//   * k_bgs_dots, k_bgs_sub (with k_block_dots_sum and the double-f32 Ritz product): the block
//     Gram-Schmidt's projection out = X - Q (Q^T X) of a whole block, the basis read twice per
//     block instead of four times per column (GK_FLAG_BLOCK_GS).
#include <math.h>

#include "gk_block_judge.cuh"
#include "gk_internal.cuh"
#include "gk_ritz_df.cuh"

namespace gk {

namespace {

constexpr int kDotThreads = 256;
constexpr int kDotRows = 8192;  // rows per partial sum of k_block_dots

__device__ __forceinline__ double warp_sum_b(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// part[pair * G + g] = sum over rows [g kDotRows, (g + 1) kDotRows) of X[i, a] Y[i, b],
// pair = a + b s (grid: G x s^2)
__global__ void __launch_bounds__(kDotThreads) k_block_dots(const double *__restrict__ X, int64_t ldx,
                                                            const double *__restrict__ Y, int64_t ldy, int64_t len,
                                                            int s, int G, double *__restrict__ part) {
  __shared__ double red[kDotThreads / 32];
  const int g = blockIdx.x, pair = blockIdx.y;
  const int a = pair % s, b = pair / s;
  const int64_t i0 = (int64_t)g * kDotRows;
  const int64_t i1 = i0 + kDotRows < len ? i0 + kDotRows : len;
  const double *x = X + (int64_t)a * ldx;
  const double *y = Y + (int64_t)b * ldy;
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kDotThreads) acc = fma(x[i], y[i], acc);
  acc = warp_sum_b(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kDotThreads / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum_b(v);
    if (threadIdx.x == 0) part[(int64_t)pair * G + g] = v;
  }
}

// raw[pair] = sum_g part[pair * G + g], g ascending
__global__ void k_block_dots_sum(const double *__restrict__ part, int G, int pairs, double *__restrict__ raw) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pairs) return;
  double v = 0.0;
  for (int g = 0; g < G; ++g) v += part[(int64_t)p * G + g];
  raw[p] = v;
}

// One warp: the block judge of gk_block_judge.cuh -- T = triu(raw), mu = max |t_ac| (a warp
// reduction), G = (T / mu)^T (T / mu), cyclic Jacobi with the rotations' column and row updates
// spread over the lanes, then lane 0 takes ||T||_2 and the side's break test (sest, nrm, brk and
// the sweeps in *bc).  T (side 0) or T^T (sides 1, 2) is placed into Bf at (row0, col0) unless the
// block broke (a left block that breaks is placed: it is B's last row block).
__global__ void __launch_bounds__(32) k_block_judge(const double *__restrict__ raw, int s, double *__restrict__ Bf,
                                                    int64_t ldb, int row0, int col0, int side, double eps,
                                                    BlockCtl *bc) {
  __shared__ double T[kBlockMaxS * kBlockMaxS];
  __shared__ double G[kBlockMaxS * kBlockMaxS];
  __shared__ int s_brk;
  const int lane = threadIdx.x;
  const int ss = s * s;
  double mu = 0.0;
  for (int e = lane; e < ss; e += 32) {
    T[e] = bj_triu(raw, s, e);
    mu = bj_absmax(mu, fabs(T[e]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mu = bj_absmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
  const double rmu = bj_rscale(mu);
  __syncwarp();
  for (int e = lane; e < ss; e += 32) G[e] = bj_gram(T, s, rmu, e);
  __syncwarp();
  int sweeps = 0;
  if (rmu > 0.0) {
    for (; sweeps < kBlockSweeps; ++sweeps) {
      bool rotated = false;
      for (int p = 0; p < s - 1; ++p) {
        for (int q = p + 1; q < s; ++q) {
          __syncwarp();
          double c, sn;
          if (!bj_rotation(G, s, p, q, &c, &sn)) continue;  // the same on every lane
          rotated = true;
          __syncwarp();
          if (lane < s) bj_col(G, s, p, q, c, sn, lane);
          __syncwarp();
          if (lane < s) bj_row(G, s, p, q, c, sn, lane);
        }
      }
      if (!rotated) break;
    }
  }
  __syncwarp();
  if (lane == 0) {
    double sest = bc->sest, nrm = 0.0;
    const int brk = bj_decide(G, s, mu, side, eps, &sest, &nrm);
    bc->sest = sest;
    bc->nrm = nrm;
    bc->brk = brk;
    bc->sweeps = sweeps;
    s_brk = brk;
  }
  __syncwarp();
  const bool place = s_brk == 0 || (side == 0 && s_brk == 1);
  if (!place) return;
  for (int e = lane; e < ss; e += 32) {
    const int a = e % s, c = e / s;
    if (a <= c) Bf[bj_place(side, row0, col0, a, c, ldb)] = T[e];
  }
}

// est[i] = || R x_i' || for i < r: R = triu(raw) (s x s), x_i' = X[row0 .. row0 + s), column i
// (column-major, ld ldx) -- the right residual of the block form of Algorithm 2's i-th triplet
__global__ void k_block_resid(const double *__restrict__ raw, int s, const double *__restrict__ X, int ldx, int row0,
                              int r, double *__restrict__ est) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r) return;
  const double *x = X + (int64_t)i * ldx + row0;
  double t = 0.0;
  for (int a = 0; a < s; ++a) {
    double v = 0.0;
    for (int c = a; c < s; ++c) v = fma(raw[a + c * s], x[c], v);
    t = fma(v, v, t);
  }
  est[i] = sqrt(t);
}

// *rank = #{i < n : sigma[i] > eps * sigma[0]}
__global__ void k_block_count(const double *__restrict__ sigma, int n, double eps, int *rank) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int r = 0;
  if (n > 0) {
    const double thr = eps * sigma[0];
    for (int i = 0; i < n; ++i) r += sigma[i] > thr ? 1 : 0;
  }
  *rank = r;
}

// ---- block Gram-Schmidt (GK_FLAG_BLOCK_GS): out = X - Q (Q^T X) for an s-column block X ----
// part[(v * j + c) * G + g] = sum over rows [g kBgsRows, (g + 1) kBgsRows) of q_ic x_iv, from the
// double-f32 copies of Q (Qs) and of X (Xs): each thread's terms in double-f32 (gk_ritz_df.cuh's
// df_fma, renormalized every four), then the threads' f64 sums in a fixed tree (grid: G x j)
constexpr int kBgsThreads = 256;
constexpr int kBgsRows = 4096;

template <int S>
__global__ void __launch_bounds__(kBgsThreads) k_bgs_dots(const float2 *__restrict__ Qs, int64_t ldq, int64_t len,
                                                          int j, const float2 *__restrict__ Xs, int64_t ldxs, int s,
                                                          int G, double *__restrict__ part) {
  __shared__ double red[kBgsThreads / 32][S];
  const int g = blockIdx.x, c = blockIdx.y;
  const int64_t i0 = (int64_t)g * kBgsRows;
  const int64_t i1 = i0 + kBgsRows < len ? i0 + kBgsRows : len;
  const DfPair *q = reinterpret_cast<const DfPair *>(Qs) + (int64_t)c * ldq;
  const DfPair *x = reinterpret_cast<const DfPair *>(Xs);
  float hi[S], lo[S];
#pragma unroll
  for (int v = 0; v < S; ++v) hi[v] = lo[v] = 0.f;
  int t = 0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kBgsThreads) {
    const DfPair qi = q[i];
#pragma unroll
    for (int v = 0; v < S; ++v)
      if (v < s) df_fma(hi[v], lo[v], qi, x[(int64_t)v * ldxs + i]);
    if ((++t & 3) == 0) {
#pragma unroll
      for (int v = 0; v < S; ++v) df_renorm(hi[v], lo[v]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < S; ++v) {
    double a = (double)hi[v] + (double)lo[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[warp][v] = a;
  }
  __syncthreads();
  if (threadIdx.x < s) {
    double a = 0.0;
    for (int w = 0; w < kBgsThreads / 32; ++w) a += red[w][threadIdx.x];
    part[((int64_t)threadIdx.x * j + c) * G + g] = a;
  }
}

// out[v * len + i] = X[v * ldx + i] - C[v * len + i]
__global__ void k_bgs_sub(const double *__restrict__ X, int64_t ldx, const double *__restrict__ C, int64_t len, int s,
                          double *__restrict__ out) {
  const int64_t total = len * (int64_t)s;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / len, i = t % len;
    out[t] = X[v * ldx + i] - C[t];
  }
}

}  // namespace

int bgs_dot_chunks(int64_t len) { return (int)((len + kBgsRows - 1) / kBgsRows); }

cudaError_t bgs_project(const float2 *Qs, int64_t ldq, int64_t len, int j, const double *X, int64_t ldx,
                        const float2 *Xs, int64_t ldxs, int s, double *part, double *H, float2 *Hs, double *C,
                        double *out, cudaStream_t st) {
  if (s < 1 || s > kBlockMaxS || j < 1 || len < 1) return cudaErrorInvalidValue;
  const int G = bgs_dot_chunks(len);
  const dim3 grid((unsigned)G, (unsigned)j);
  if (s <= 8)
    GK_LAUNCH(k_bgs_dots<8><<<grid, kBgsThreads, 0, st>>>(Qs, ldq, len, j, Xs, ldxs, s, G, part));
  else if (s <= 16)
    GK_LAUNCH(k_bgs_dots<16><<<grid, kBgsThreads, 0, st>>>(Qs, ldq, len, j, Xs, ldxs, s, G, part));
  else
    GK_LAUNCH(k_bgs_dots<32><<<grid, kBgsThreads, 0, st>>>(Qs, ldq, len, j, Xs, ldxs, s, G, part));
  const int pairs = j * s;  // H (j x s, column-major): the partials of each entry summed in chunk order
  GK_LAUNCH(k_block_dots_sum<<<(pairs + 127) / 128, 128, 0, st>>>(part, G, pairs, H));
  cudaError_t e = ritz_gemm_df(Qs, ldq, len, j, H, j, s, C, len, Hs, st);  // C = Q H
  if (e != cudaSuccess) return e;
  int64_t b = (len * s + 255) / 256;
  if (b > 4096) b = 4096;
  GK_LAUNCH(k_bgs_sub<<<(int)b, 256, 0, st>>>(X, ldx, C, len, s, out));
  return cudaGetLastError();
}

int block_dot_chunks(int64_t len) { return (int)((len + kDotRows - 1) / kDotRows); }

cudaError_t block_dots(const double *X, int64_t ldx, const double *Y, int64_t ldy, int64_t len, int s, double *part,
                       double *raw, cudaStream_t st) {
  if (s < 1 || s > kBlockMaxS || len < 1) return cudaErrorInvalidValue;
  const int G = block_dot_chunks(len);
  const int pairs = s * s;
  GK_LAUNCH(k_block_dots<<<dim3((unsigned)G, (unsigned)pairs), kDotThreads, 0, st>>>(X, ldx, Y, ldy, len, s, G, part));
  GK_LAUNCH(k_block_dots_sum<<<(pairs + 127) / 128, 128, 0, st>>>(part, G, pairs, raw));
  return cudaGetLastError();
}

cudaError_t block_judge(const double *raw, int s, double *Bf, int64_t ldb, int row0, int col0, int side, double eps,
                        BlockCtl *bc, cudaStream_t st) {
  if (s < 1 || s > kBlockMaxS) return cudaErrorInvalidValue;
  GK_LAUNCH(k_block_judge<<<1, 32, 0, st>>>(raw, s, Bf, ldb, row0, col0, side, eps, bc));
  return cudaGetLastError();
}

cudaError_t block_resid(const double *raw, int s, const double *X, int ldx, int row0, int r, double *est,
                        cudaStream_t st) {
  if (r <= 0) return cudaSuccess;
  GK_LAUNCH(k_block_resid<<<(r + 127) / 128, 128, 0, st>>>(raw, s, X, ldx, row0, r, est));
  return cudaGetLastError();
}

cudaError_t block_count(const double *sigma, int n, double eps, int *rank, cudaStream_t st) {
  GK_LAUNCH(k_block_count<<<1, 32, 0, st>>>(sigma, n, eps, rank));
  return cudaGetLastError();
}

}  // namespace gk
