// gk_small.cu -- the small dense steps of the method:
//  * the SVD of the projected matrix B (Eq. 2.13; Algorithm 2),
//    by one-sided Jacobi in f64 with a parallel (round-robin) pair ordering;
//  * the Ritz residual estimates |beta_K X_{K,i}| and the restart coupling;
//  * Ritz vectors U_K X and V_K Y (Algorithm 2: V_2 = P V_1);
//  * the rank count of Algorithm 3 from Sturm sequences of the Golub-Kahan
//    tridiagonal of B_{k'+1,k'} (its eigenvalues are +-sigma_i(B) and 0).
#include <float.h>
#include <math.h>

#include <mutex>

#include <cooperative_groups.h>

#include "gk_bdsvd.cuh"
#include "gk_ritz_df.cuh"
#include "gk_device.cuh"
#include "gk_internal.cuh"

namespace cg = cooperative_groups;

namespace gk {

namespace {

__device__ __forceinline__ bool halted(const Ctl *ctl) {
  return ctl != nullptr && *reinterpret_cast<const volatile int *>(&ctl->halt) != 0;
}


__global__ void k_assemble_B(double *__restrict__ Bm, int K, int l, const double *__restrict__ sigma,
                             const double *__restrict__ rho, const double *__restrict__ alpha,
                             const double *__restrict__ beta, const Ctl *ctl) {
  if (halted(ctl)) return;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)K * K;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % K), c = (int)(idx / K);
    double v = 0.0;
    if (r < l) {
      if (c == r) v = sigma[r];
      else if (c == l) v = rho[r];
    } else {
      if (c == r) v = alpha[r];
      else if (c == r + 1) v = beta[r];
    }
    Bm[idx] = v;
  }
}

// The lower-bidiagonal B_{kp+1,kp} of Algorithm 1 (alpha_1..alpha_kp on the diagonal,
// beta_2..beta_{kp+1} below it: alpha[c] at (c, c), beta[c + 1] at (c + 1, c)) padded with a
// zero last column to the square K = kp + 1 (column-major) that the Jacobi kernel takes.
__global__ void k_assemble_lower(double *__restrict__ Bm, int kp, const double *__restrict__ alpha,
                                 const double *__restrict__ beta) {
  const int K = kp + 1;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)K * K;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % K), c = (int)(idx / K);
    double v = 0.0;
    if (c < kp) {
      if (r == c) v = alpha[c];
      else if (r == c + 1) v = beta[c + 1];
    }
    Bm[idx] = v;
  }
}

// Bm = B^T B (kp x kp, column-major) for the lower-bidiagonal B_{kp+1,kp} (alpha[0..kp-1] on its
// diagonal, beta[1..kp] below it): tridiagonal, diag alpha_c^2 + beta_{c+1}^2, off-diagonal
// beta_{c+1} alpha_{c+1}
__global__ void k_assemble_btb(double *__restrict__ Bm, int kp, const double *__restrict__ alpha,
                               const double *__restrict__ beta) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)kp * kp;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % kp), c = (int)(idx / kp);
    double v = 0.0;
    if (r == c) v = alpha[c] * alpha[c] + beta[c + 1] * beta[c + 1];
    else if (r == c + 1) v = beta[c + 1] * alpha[c + 1];
    else if (c == r + 1) v = beta[r + 1] * alpha[r + 1];
    Bm[idx] = v;
  }
}

// theta[i] = sqrt(max(theta[i], 0)) for i < n
__global__ void k_sqrt_vals(double *__restrict__ theta, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    theta[i] = theta[i] > 0.0 ? sqrt(theta[i]) : 0.0;
}

// column i of U (len x ncol, column-major) /= sigma[i] (left as is when sigma[i] is not positive)
__global__ void k_scale_cols(double *__restrict__ U, int64_t len, int ncol, const double *__restrict__ sigma) {
  const int c = blockIdx.y;
  const double v = sigma[c];
  if (!(v > 0.0)) return;
  const double f = 1.0 / v;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    U[(int64_t)c * len + i] *= f;
}

// y[i] /= *d for i < len (left as is when *d is not positive)
__global__ void k_scale_inv(double *__restrict__ y, int64_t len, const double *__restrict__ d) {
  const double v = *d;
  if (!(v > 0.0)) return;
  const double f = 1.0 / v;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    y[i] *= f;
}

// NL: elements of a column per lane held in registers during a rotation (0: none, any K)
template <int NL>
__global__ void __launch_bounds__(256) k_jacobi_cluster(double *__restrict__ B, double *__restrict__ Yw, int K,
                                                        double *__restrict__ sigma, double *__restrict__ X,
                                                        double *__restrict__ Y, double *__restrict__ nrm,
                                                        int *__restrict__ pos, int *sweeps_out, const Ctl *ctl) {
  cg::cluster_group cl = cg::this_cluster();
  if (halted(ctl)) return;  // every CTA of the cluster sees the same flag
  __shared__ int s_rot, s_any;
  const int sw = dev::cluster_jacobi<NL>(cl, B, Yw, K, sigma, X, Y, nrm, pos, &s_rot, &s_any);
  if (cl.block_rank() == 0 && threadIdx.x == 0 && sweeps_out) *sweeps_out = sw;
}

__global__ void k_ritz_check(const double *__restrict__ sigma, const double *__restrict__ X, int K, int k,
                             const double *__restrict__ betaK, double tol, double *__restrict__ rho,
                             double *__restrict__ out, Ctl *ctl) {
  if (halted(ctl)) return;
  __shared__ double red[256];
  const double bK = *betaK;
  double mx = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double r = bK * X[(int64_t)i * K + (K - 1)];
    rho[i] = r;
    if (i < k) mx = fmax(mx, fabs(r));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double s1 = sigma[0];
    out[0] = red[0];
    out[1] = s1;
    out[2] = (red[0] <= tol * s1) ? 1.0 : 0.0;
    ctl->sest = fmax(ctl->sest, s1);
  }
}

// C[:, c] = Q[:, 0:K] X[:, c], 16 output columns per block, X staged in tiles of 64 rows
__global__ void __launch_bounds__(256) k_ritz_gemm(const double *__restrict__ Q, int64_t ldq, int64_t len, int K,
                                                   const double *__restrict__ X, int ldx, int ncol,
                                                   double *__restrict__ C, int64_t ldc) {
  __shared__ double xs[64][16];
  const int col0 = blockIdx.y * 16;
  const int nc = (ncol - col0) < 16 ? (ncol - col0) : 16;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) acc[t] = 0.0;
  for (int kt = 0; kt < K; kt += 64) {
    const int kk = (K - kt) < 64 ? (K - kt) : 64;
    for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
      const int r = e / 16, t = e % 16;
      xs[r][t] = (r < kk && t < nc) ? X[(int64_t)(col0 + t) * ldx + kt + r] : 0.0;
    }
    __syncthreads();
    if (i < len) {
      for (int r = 0; r < kk; ++r) {
        const double q = Q[(int64_t)(kt + r) * ldq + i];
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[t] = fma(q, xs[r][t], acc[t]);
      }
    }
    __syncthreads();
  }
  if (i < len) {
#pragma unroll
    for (int t = 0; t < 16; ++t)
      if (t < nc) C[(int64_t)(col0 + t) * ldc + i] = acc[t];
  }
}

__global__ void __launch_bounds__(256) k_sign_normalize(double *__restrict__ U, int64_t ldu, int64_t m,
                                                        double *__restrict__ V, int64_t ldv, int64_t n) {
  __shared__ double bv[256];
  __shared__ int64_t bi[256];
  __shared__ int flip;
  double *v = V + (int64_t)blockIdx.x * ldv;
  double *u = U + (int64_t)blockIdx.x * ldu;
  double best = -1.0;
  int64_t bidx = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double a = fabs(v[r]);
    if (a > best) {
      best = a;
      bidx = r;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double b2 = bv[threadIdx.x + o];
      const int64_t i2 = bi[threadIdx.x + o];
      if (b2 > bv[threadIdx.x] || (b2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = b2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) flip = v[bi[0]] < 0.0;
  __syncthreads();
  if (!flip) return;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) v[r] = -v[r];
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) u[r] = -u[r];
}

__global__ void __launch_bounds__(256) k_bidiag_rank(const double *__restrict__ alpha,
                                                     const double *__restrict__ beta, int kp, double eps, int eps_rel,
                                                     int *__restrict__ rank, double *__restrict__ sigma1,
                                                     double *__restrict__ sigma) {
  __shared__ double red[256];
  dev::block_bidiag_rank(alpha, beta, kp, eps, eps_rel, rank, sigma1, sigma, red);
}

// SVD of the upper-bidiagonal B (d = alpha[0..K), e = beta[0..K-1)) by Golub-Kahan SVD steps
// (gk_bdsvd.cuh) on one CTA: thread 0 takes the steps, then every thread applies the step's
// rotations to its rows of the work copies Xw (left) and Yw (right), column-major K x K; at the
// end the values are made nonnegative (a sign flip of Y's column), ordered descending (stable
// by index) by counting ranks, and X, Y gathered in that order.  sweeps_out: steps taken
// (negative if the step budget was spent).
constexpr int kBdThreads = 256;

__global__ void __launch_bounds__(kBdThreads) k_bdsvd(const double *__restrict__ alpha, const double *__restrict__ beta,
                                                     int K, double *__restrict__ sigma, double *__restrict__ X,
                                                     double *__restrict__ Y, double *__restrict__ Xw,
                                                     double *__restrict__ Yw, int *__restrict__ sweeps_out,
                                                     const Ctl *ctl) {
  if (halted(ctl)) return;
  extern __shared__ __align__(16) unsigned char bd_smem[];
  double *d = reinterpret_cast<double *>(bd_smem);
  double *e = d + K;
  BdRot *rl = reinterpret_cast<BdRot *>(e + K);
  BdRot *rr = rl + K;
  int *rank = reinterpret_cast<int *>(rr + K);
  __shared__ int s_rc, s_nl, s_nr;
  __shared__ BdState st;
  const int tid = threadIdx.x;
  for (int64_t idx = tid; idx < (int64_t)K * K; idx += blockDim.x) {
    const double v = (idx % K) == (idx / K) ? 1.0 : 0.0;
    Xw[idx] = v;
    Yw[idx] = v;
  }
  for (int k = tid; k < K; k += blockDim.x) {
    d[k] = alpha[k];
    e[k] = k + 1 < K ? beta[k] : 0.0;
  }
  __syncthreads();
  if (tid == 0) bd_init(&st, d, e, K);
  int rc;
  for (;;) {
    if (tid == 0) {
      int nl = 0, nr = 0;
      s_rc = bd_step(d, e, &st, rl, &nl, rr, &nr);
      s_nl = nl;
      s_nr = nr;
    }
    __syncthreads();
    rc = s_rc;
    if (rc <= 0) break;
    const int nl = s_nl, nr = s_nr;
    for (int i = tid; i < K; i += blockDim.x) {
      if (rc == 1) {
        bd_apply_chase(Xw + i, K, rl, nl);
        bd_apply_chase(Yw + i, K, rr, nr);
      } else {
        bd_apply_row(Xw + i, K, rl, nl);
        bd_apply_row(Yw + i, K, rr, nr);
      }
    }
    __syncthreads();  // the rotations are applied before thread 0 records the next step's
  }
  for (int k = tid; k < K; k += blockDim.x) {
    const double a = fabs(d[k]);
    int r = 0;
    for (int j = 0; j < K; ++j) {
      const double b = fabs(d[j]);
      r += (b > a || (b == a && j < k)) ? 1 : 0;
    }
    rank[k] = r;
  }
  __syncthreads();
  for (int k = tid; k < K; k += blockDim.x) sigma[rank[k]] = fabs(d[k]);
  for (int64_t idx = tid; idx < (int64_t)K * K; idx += blockDim.x) {
    const int k = (int)(idx / K), i = (int)(idx % K);
    const int64_t t = (int64_t)rank[k] * K + i;
    X[t] = Xw[idx];
    Y[t] = d[k] < 0.0 ? -Yw[idx] : Yw[idx];
  }
  if (tid == 0 && sweeps_out) *sweeps_out = rc < 0 ? -st.steps : st.steps;
}

// C[:, c] = Q[:, 0:K] X[:, c] from the double-f32 copy Qs of Q (gk_ritz_df.cuh): one thread per row
// and group of kRitzCols columns; Xs = X split into f32 pairs (K x ncol, ld K)
__global__ void __launch_bounds__(256) k_ritz_df(const float2 *__restrict__ Qs, int64_t ldq, int64_t len, int K,
                                                 const float2 *__restrict__ Xs, int ncol, double *__restrict__ C,
                                                 int64_t ldc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const int c0 = blockIdx.y * kRitzCols;
  const int nc = ncol - c0 < kRitzCols ? ncol - c0 : kRitzCols;
  ritz_df_row(reinterpret_cast<const DfPair *>(Qs), ldq, i, K, reinterpret_cast<const DfPair *>(Xs), K, c0, nc, C,
              ldc);
}

// Xs[c * K + k] = the f32 pair of X[c * ldx + k]
__global__ void k_split_x(const double *__restrict__ X, int ldx, int K, int ncol, float2 *__restrict__ Xs) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)K * ncol;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / K), k = (int)(idx % K);
    const DfPair v = df_split(X[(int64_t)c * ldx + k]);
    Xs[idx] = make_float2(v.hi, v.lo);
  }
}

}  // namespace

cudaError_t assemble_B(double *Bm, int K, int l, const double *sigma, const double *rho, const double *alpha,
                       const double *beta, const Ctl *ctl, cudaStream_t s) {
  int64_t blocks = ((int64_t)K * K + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  GK_LAUNCH(k_assemble_B<<<(int)blocks, 256, 0, s>>>(Bm, K, l, sigma, rho, alpha, beta, ctl));
  return cudaGetLastError();
}

cudaError_t assemble_lower(double *Bm, int kp, const double *alpha, const double *beta, cudaStream_t s) {
  int64_t blocks = ((int64_t)(kp + 1) * (kp + 1) + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  GK_LAUNCH(k_assemble_lower<<<(int)blocks, 256, 0, s>>>(Bm, kp, alpha, beta));
  return cudaGetLastError();
}

cudaError_t assemble_btb(double *Bm, int kp, const double *alpha, const double *beta, cudaStream_t s) {
  int64_t blocks = ((int64_t)kp * kp + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  GK_LAUNCH(k_assemble_btb<<<(int)blocks, 256, 0, s>>>(Bm, kp, alpha, beta));
  return cudaGetLastError();
}

cudaError_t sqrt_vals(double *theta, int n, cudaStream_t s) {
  GK_LAUNCH(k_sqrt_vals<<<1, 256, 0, s>>>(theta, n));
  return cudaGetLastError();
}

cudaError_t scale_cols(double *U, int64_t len, int ncol, const double *sigma, cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  int64_t bx = (len + 255) / 256;
  if (bx > 256) bx = 256;
  if (bx < 1) bx = 1;
  GK_LAUNCH(k_scale_cols<<<dim3((unsigned)bx, (unsigned)ncol), 256, 0, s>>>(U, len, ncol, sigma));
  return cudaGetLastError();
}

cudaError_t scale_inv(double *y, int64_t len, const double *d, cudaStream_t s) {
  int64_t blocks = (len + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  GK_LAUNCH(k_scale_inv<<<(int)blocks, 256, 0, s>>>(y, len, d));
  return cudaGetLastError();
}

cudaError_t small_svd(double *Bm, double *Yw, int K, double *sigma, double *X, double *Y, double *nrm, int *pos,
                      int *sweeps, const Ctl *ctl, cudaStream_t s) {
  // registers per lane for a column pair: the smallest of 1, 2, 4, 8, 16 covering K (K <= 512)
  using Kern = void (*)(double *, double *, int, double *, double *, double *, double *, int *, int *, const Ctl *);
  Kern kern = K <= 32 ? k_jacobi_cluster<1>
            : K <= 64 ? k_jacobi_cluster<2>
            : K <= 128 ? k_jacobi_cluster<4>
            : K <= 256 ? k_jacobi_cluster<8>
            : K <= 512 ? k_jacobi_cluster<16>
                       : k_jacobi_cluster<0>;
  // cluster size: enough warps for the Kp/2 pairs of a round (8 per CTA), a power of two up to 16
  const int pairs = (K + (K & 1)) / 2;
  int want = 1;
  while (want < 16 && want * 8 < pairs) want *= 2;
  {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  for (int cs = want; cs >= 1; cs /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int maxc = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&maxc, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (maxc < cs) continue;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, Bm, Yw, K, sigma, X, Y, nrm, pos, sweeps, ctl);
    if (e == cudaSuccess) {
      note_launch();
      return cudaSuccess;
    }
    cudaGetLastError();
  }
  return cudaErrorLaunchFailure;
}

cudaError_t ritz_check(const double *sigma, const double *X, int K, int k, const double *betaK, double tol,
                       double *rho, double *out, Ctl *ctl, cudaStream_t s) {
  GK_LAUNCH(k_ritz_check<<<1, 256, 0, s>>>(sigma, X, K, k, betaK, tol, rho, out, ctl));
  return cudaGetLastError();
}

cudaError_t ritz_gemm(const double *Q, int64_t ldq, int64_t len, int K, const double *X, int ldx, int ncol,
                      double *C, int64_t ldc, cudaStream_t s, const Dev &d) {
  (void)d;
  if (ncol <= 0 || len <= 0) return cudaSuccess;
  dim3 grid((unsigned)((len + 255) / 256), (unsigned)((ncol + 15) / 16));
  GK_LAUNCH(k_ritz_gemm<<<grid, 256, 0, s>>>(Q, ldq, len, K, X, ldx, ncol, C, ldc));
  return cudaGetLastError();
}

cudaError_t ritz_gemm_df(const float2 *Qs, int64_t ldq, int64_t len, int K, const double *X, int ldx, int ncol,
                         double *C, int64_t ldc, float2 *Xs, cudaStream_t s) {
  if (ncol <= 0 || len <= 0) return cudaSuccess;
  int64_t b = ((int64_t)K * ncol + 255) / 256;
  if (b > 1024) b = 1024;
  GK_LAUNCH(k_split_x<<<(int)b, 256, 0, s>>>(X, ldx, K, ncol, Xs));
  dim3 grid((unsigned)((len + 255) / 256), (unsigned)((ncol + kRitzCols - 1) / kRitzCols));
  GK_LAUNCH(k_ritz_df<<<grid, 256, 0, s>>>(Qs, ldq, len, K, Xs, ncol, C, ldc));
  return cudaGetLastError();
}

cudaError_t bd_svd(const double *alpha, const double *beta, int K, double *sigma, double *X, double *Y, double *Xw,
                   double *Yw, int *sweeps, const Ctl *ctl, cudaStream_t s) {
  if (K < 1 || K > kBdMaxK) return cudaErrorInvalidValue;
  const size_t per = 2 * sizeof(double) + 2 * sizeof(BdRot) + sizeof(int);
  static std::mutex mu;
  static int attr_dev = -1;  // the device whose shared-memory limit for the kernel was raised
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (attr_dev != dev) {
      e = cudaFuncSetAttribute(k_bdsvd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per * kBdMaxK));
      if (e != cudaSuccess) return e;
      attr_dev = dev;
    }
  }
  GK_LAUNCH(k_bdsvd<<<1, kBdThreads, per * (size_t)K, s>>>(alpha, beta, K, sigma, X, Y, Xw, Yw, sweeps, ctl));
  return cudaGetLastError();
}

cudaError_t sign_normalize(double *U, int64_t ldu, int64_t m, double *V, int64_t ldv, int64_t n, int k,
                           cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  GK_LAUNCH(k_sign_normalize<<<k, 256, 0, s>>>(U, ldu, m, V, ldv, n));
  return cudaGetLastError();
}

cudaError_t bidiag_rank(const double *alpha, const double *beta, int kp, double eps, int eps_rel, int *rank,
                        double *sigma1, double *sigma, cudaStream_t s) {
  GK_LAUNCH(k_bidiag_rank<<<1, 256, 0, s>>>(alpha, beta, kp, eps, eps_rel, rank, sigma1, sigma));
  return cudaGetLastError();
}

}  // namespace gk
