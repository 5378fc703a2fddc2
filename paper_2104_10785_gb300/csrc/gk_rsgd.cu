// gk_rsgd.cu -- Algorithm 4 (fast Riemannian mini-batch gradient descent, Section 4) for
// P independent problems of one shape: the mini-batch gradient, the projection onto the
// tangent space of the rank-r manifold (the Riemannian gradient equation) and the SVD
// retraction as kernels over all problems; the two rank-r SVDs of a step (Algorithm 2: fixed
// Golub-Kahan steps, no restart) as one gk_psvd_batched launch each.
//
// Layouts (f64): W, Gr, M = W - eta Z: P x d1 x d2 row-major; U: P x (d1 x r) column-major,
// V: P x (d2 x r) column-major (the batched solver's outputs); GV = Gr V: P x d1 x r
// row-major; UG = U^T Gr: P x r x d2 row-major; D = U (U^T GV): P x d1 x r row-major.
// With those, Z = Gr V V^T + U U^T Gr - U U^T Gr V V^T = (GV - D) V^T + U UG, so a step costs
// two passes over each d1 x d2 matrix besides the inner solves.  Every sum has a fixed order.
#include <chrono>
#include <cstring>
#include <vector>

#include "gk_internal.cuh"

namespace gk {

namespace {

constexpr int kRMax = 16;   // largest rank r
constexpr int kGTile = 32;  // gradient: 32 x 32 output tile per block
constexpr int kGChunk = 16; // samples staged per round

// Gr[p] = (1/b) sum_s y_i(s) x_i(s) v_i(s)^T - lam W[p], i(s) = idx[p * b + s], s ascending
__global__ void __launch_bounds__(256) k_rsgd_grad(const double *__restrict__ X, const double *__restrict__ Vd,
                                                   const double *__restrict__ y, const int32_t *__restrict__ idx,
                                                   const double *__restrict__ W, int N, int d1, int d2, int b,
                                                   double lam, double *__restrict__ G) {
  __shared__ double xs[kGChunk][kGTile];
  __shared__ double vs[kGChunk][kGTile];
  const int p = blockIdx.z;
  const int a0 = blockIdx.y * kGTile, c0 = blockIdx.x * kGTile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads, 4 rows each
  const int32_t *ip = idx + (int64_t)p * b;
  const double *Xp = X + (int64_t)p * N * d1;
  const double *Vp = Vd + (int64_t)p * N * d2;
  const double *yp = y + (int64_t)p * N;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s0 = 0; s0 < b; s0 += kGChunk) {
    for (int t = threadIdx.x; t < kGChunk * kGTile; t += blockDim.x) {
      const int s = t / kGTile, e = t % kGTile;
      double xv = 0.0, vv = 0.0;
      if (s0 + s < b) {
        const int64_t i = ip[s0 + s];
        if (a0 + e < d1) xv = yp[i] * Xp[i * d1 + a0 + e];
        if (c0 + e < d2) vv = Vp[i * d2 + c0 + e];
      }
      xs[s][e] = xv;
      vs[s][e] = vv;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kGChunk; ++s) {
      const double vv = vs[s][tx];
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = fma(xs[s][ty + 8 * k], vv, acc[k]);
    }
    __syncthreads();
  }
  const int c = c0 + tx;
  if (c >= d2) return;
  const double inv_b = 1.0 / (double)b;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a = a0 + ty + 8 * k;
    if (a < d1) {
      const int64_t o = ((int64_t)p * d1 + a) * d2 + c;
      G[o] = acc[k] * inv_b - lam * W[o];
    }
  }
}

// GV[p][a][s] = sum_c Gr[p][a][c] V[p][c][s]: one warp per row a (lanes over c, a fixed tree)
__global__ void __launch_bounds__(256) k_rsgd_gv(const double *__restrict__ G, const double *__restrict__ V, int d1,
                                                 int d2, int r, double *__restrict__ GV) {
  const int p = blockIdx.y;
  const int a = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= d1) return;
  const double *g = G + ((int64_t)p * d1 + a) * d2;
  const double *Vp = V + (int64_t)p * d2 * r;
  double acc[kRMax];
#pragma unroll
  for (int s = 0; s < kRMax; ++s) acc[s] = 0.0;
  for (int c = lane; c < d2; c += 32) {
    const double gv = g[c];
#pragma unroll
    for (int s = 0; s < kRMax; ++s)
      if (s < r) acc[s] = fma(gv, Vp[(int64_t)s * d2 + c], acc[s]);
  }
#pragma unroll
  for (int s = 0; s < kRMax; ++s) {
    if (s < r) {
      double v = acc[s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) GV[((int64_t)p * d1 + a) * r + s] = v;
    }
  }
}

// UG[p][s][c] = sum_a U[p][a][s] Gr[p][a][c]: one thread per column c, rows in order
__global__ void __launch_bounds__(256) k_rsgd_ug(const double *__restrict__ G, const double *__restrict__ U, int d1,
                                                 int d2, int r, double *__restrict__ UG) {
  const int p = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d2) return;
  const double *Gp = G + (int64_t)p * d1 * d2;
  const double *Up = U + (int64_t)p * d1 * r;
  double acc[kRMax];
#pragma unroll
  for (int s = 0; s < kRMax; ++s) acc[s] = 0.0;
  for (int a = 0; a < d1; ++a) {
    const double gv = Gp[(int64_t)a * d2 + c];
#pragma unroll
    for (int s = 0; s < kRMax; ++s)
      if (s < r) acc[s] = fma(Up[(int64_t)s * d1 + a], gv, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < kRMax; ++s)
    if (s < r) UG[((int64_t)p * r + s) * d2 + c] = acc[s];
}

// C = U^T GV (r x r, one block per problem), then D = U C (d1 x r)
__global__ void __launch_bounds__(256) k_rsgd_cd(const double *__restrict__ U, const double *__restrict__ GV, int d1,
                                                 int r, double *__restrict__ D) {
  __shared__ double Cs[kRMax * kRMax];
  __shared__ double red[8];
  const int p = blockIdx.x;
  const double *Up = U + (int64_t)p * d1 * r;
  const double *GVp = GV + (int64_t)p * d1 * r;
  for (int e = 0; e < r * r; ++e) {  // C[s][t] = sum_a U[a][s] GV[a][t], a fixed tree per entry
    const int s = e / r, t = e % r;
    double v = 0.0;
    for (int a = threadIdx.x; a < d1; a += blockDim.x) v = fma(Up[(int64_t)s * d1 + a], GVp[(int64_t)a * r + t], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < 8; ++w) tot += red[w];
      Cs[s * r + t] = tot;
    }
    __syncthreads();
  }
  for (int a = threadIdx.x; a < d1; a += blockDim.x)
    for (int t = 0; t < r; ++t) {
      double v = 0.0;
      for (int s = 0; s < r; ++s) v = fma(Up[(int64_t)s * d1 + a], Cs[s * r + t], v);
      D[((int64_t)p * d1 + a) * r + t] = v;
    }
}

// M[p][a][c] = W[p][a][c] - eta (sum_s (GV - D)[a][s] V[c][s] + sum_s U[a][s] UG[s][c])
__global__ void __launch_bounds__(256) k_rsgd_m(const double *__restrict__ W, const double *__restrict__ GV,
                                                const double *__restrict__ D, const double *__restrict__ U,
                                                const double *__restrict__ UG, const double *__restrict__ V, int d1,
                                                int d2, int r, double eta, double *__restrict__ M) {
  const int p = blockIdx.z;
  const int a = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d1 || c >= d2) return;
  const double *gv = GV + ((int64_t)p * d1 + a) * r;
  const double *dd = D + ((int64_t)p * d1 + a) * r;
  const double *Up = U + (int64_t)p * d1 * r;
  const double *Vp = V + (int64_t)p * d2 * r;
  const double *UGp = UG + (int64_t)p * r * d2;
  double z = 0.0;
  for (int s = 0; s < r; ++s) z = fma(gv[s] - dd[s], Vp[(int64_t)s * d2 + c], z);
  for (int s = 0; s < r; ++s) z = fma(Up[(int64_t)s * d1 + a], UGp[(int64_t)s * d2 + c], z);
  const int64_t o = ((int64_t)p * d1 + a) * d2 + c;
  M[o] = W[o] - eta * z;
}

// W[p][a][c] = sum_s U[a][s] S[s] V[c][s]  (the retraction)
__global__ void __launch_bounds__(256) k_rsgd_retract(const double *__restrict__ U, const double *__restrict__ S,
                                                      const double *__restrict__ V, int d1, int d2, int r,
                                                      double *__restrict__ W) {
  const int p = blockIdx.z;
  const int a = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d1 || c >= d2) return;
  const double *Up = U + (int64_t)p * d1 * r;
  const double *Vp = V + (int64_t)p * d2 * r;
  const double *Sp = S + (int64_t)p * r;
  double w = 0.0;
  for (int s = 0; s < r; ++s) w = fma(Up[(int64_t)s * d1 + a] * Sp[s], Vp[(int64_t)s * d2 + c], w);
  W[((int64_t)p * d1 + a) * d2 + c] = w;
}

}  // namespace

namespace {

bool device_memory(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// the inner rank-r SVDs of the P matrices mats[p] (d1 x d2 row-major): Algorithm 2 as one
// restart-free cycle of the batched solver
int inner_svds(const double *mats, const gk_rsgd_args &a, const gk_opts &oi, double *U, double *S, double *V,
               std::vector<gk_batch_item> &items, gk_info *acc) {
  for (int p = 0; p < a.P; ++p) {
    gk_batch_item &it = items[p];
    memset(&it, 0, sizeof(it));
    it.A.kind = GK_DENSE;
    it.A.dtype = GK_F64;
    it.A.m = a.d1;
    it.A.n = a.d2;
    it.A.ld = a.d2;
    it.A.scale = 1.0;
    it.A.vals = mats + (int64_t)p * a.d1 * a.d2;
    it.k = a.r;
    it.krylov_dim = a.k_inner;
    it.tol = 1e-8;
    it.U = U + (int64_t)p * a.d1 * a.r;
    it.S = S + (int64_t)p * a.r;
    it.V = V + (int64_t)p * a.d2 * a.r;
    it.start = a.q1 + (int64_t)p * a.d1;
  }
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  const int rc = gk_psvd_batched(items.data(), a.P, &oi, &inf);
  acc->matvecs += inf.matvecs;
  acc->steps += inf.steps;
  acc->breakdowns += inf.breakdowns;
  // GK_NOT_CONVERGED / GK_RANK_DEFICIENT: a fixed number of steps, as Algorithm 2 takes
  return rc < 0 ? rc : GK_OK;
}

}  // namespace
}  // namespace gk

extern "C" int gk_rsgd_batched(const gk_rsgd_args *a, const gk_opts *opts, gk_info *info) {
  using namespace gk;
  const auto t0 = std::chrono::steady_clock::now();
  if (!a) return GK_INVALID_ARG;
  const int64_t P = a->P, N = a->N, d1 = a->d1, d2 = a->d2;
  const int mn = (int)(d1 < d2 ? d1 : d2);
  if (P < 1 || P > 65535 || a->b < 1 || N < a->b || d1 < 2 || d1 > 65535 || d2 < 2 || d2 > 4096 || a->r < 1 ||
      a->r > kRMax || a->k_inner < a->r + 2 || a->k_inner > mn || a->k_inner > 510 || a->steps < 0)
    return GK_INVALID_ARG;
  if (!(a->eta == a->eta) || !(a->lam == a->lam)) return GK_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return GK_NO_DEVICE;
  }
  if (!device_memory(a->X) || !device_memory(a->Vd) || !device_memory(a->y) || !device_memory(a->q1) ||
      !device_memory(a->W) || (a->steps > 0 && !device_memory(a->batches)))
    return GK_INVALID_ARG;
  gk_opts o;
  if (opts) {
    o = *opts;
  } else {
    gk_default_opts(&o);
  }
  cudaStream_t s = (cudaStream_t)o.stream;
  // inner solves: one cycle of k_inner steps each, the caller's Gram-Schmidt rule
  gk_opts oi = o;
  oi.max_restarts = 0;
  oi.krylov_dim = 0;
  oi.keep = 0;
  oi.start = nullptr;
  oi.predictor = nullptr;
  oi.workspace = nullptr;
  oi.workspace_bytes = 0;
  oi.flags = o.flags & GK_FLAG_AUTOTUNE;

  const int r = a->r;
  const int64_t nW = P * d1 * d2, nU = P * d1 * r, nV = P * d2 * r, nS = P * r;
  const size_t doubles = 2 * nW + 4 * nU + 3 * nV + 2 * nS;  // G, M; U1, U2, GV, D; V1, V2, UG; S1, S2
  double *base = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void **>(&base), sizeof(double) * doubles, s) != cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  double *G = base, *M = G + nW, *U1 = M + nW, *U2 = U1 + nU, *GV = U2 + nU, *D = GV + nU;
  double *V1 = D + nU, *V2 = V1 + nV, *UG = V2 + nV, *S1 = UG + nV, *S2 = S1 + nS;
  std::vector<gk_batch_item> items((size_t)P);
  gk_info acc;
  memset(&acc, 0, sizeof(acc));
  int rc = GK_OK;
  int done = 0;
  const dim3 blk(256);
  for (int t = 0; t < a->steps && rc == GK_OK; ++t) {
    // Gr = mean over the batch of y x v^T, minus lam W
    GK_LAUNCH(k_rsgd_grad<<<dim3((unsigned)ceil_div(d2, kGTile), (unsigned)ceil_div(d1, kGTile), (unsigned)P), blk, 0,
                            s>>>(a->X, a->Vd, a->y, a->batches + (int64_t)t * P * a->b, a->W, (int)N, (int)d1,
                                 (int)d2, a->b, a->lam, G));
    if (cudaGetLastError() != cudaSuccess) {
      rc = GK_CUDA_ERROR;
      break;
    }
    rc = inner_svds(G, *a, oi, U1, S1, V1, items, &acc);  // U_r, V_r of Gr (Algorithm 2)
    if (rc) break;
    // M = W - eta Z, Z the projection of Gr onto the tangent space at (U_r, V_r)
    GK_LAUNCH(k_rsgd_gv<<<dim3((unsigned)ceil_div(d1, 8), (unsigned)P), blk, 0, s>>>(G, V1, (int)d1, (int)d2, r, GV));
    GK_LAUNCH(k_rsgd_ug<<<dim3((unsigned)ceil_div(d2, 256), (unsigned)P), blk, 0, s>>>(G, U1, (int)d1, (int)d2, r, UG));
    GK_LAUNCH(k_rsgd_cd<<<(unsigned)P, blk, 0, s>>>(U1, GV, (int)d1, r, D));
    GK_LAUNCH(k_rsgd_m<<<dim3((unsigned)ceil_div(d2, 256), (unsigned)d1, (unsigned)P), blk, 0, s>>>(
        a->W, GV, D, U1, UG, V1, (int)d1, (int)d2, r, a->eta, M));
    if (cudaGetLastError() != cudaSuccess) {
      rc = GK_CUDA_ERROR;
      break;
    }
    rc = inner_svds(M, *a, oi, U2, S2, V2, items, &acc);  // the retraction's rank-r SVD
    if (rc) break;
    GK_LAUNCH(k_rsgd_retract<<<dim3((unsigned)ceil_div(d2, 256), (unsigned)d1, (unsigned)P), blk, 0, s>>>(
        U2, S2, V2, (int)d1, (int)d2, r, a->W));
    if (cudaGetLastError() != cudaSuccess) {
      rc = GK_CUDA_ERROR;
      break;
    }
    ++done;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == GK_OK) rc = GK_CUDA_ERROR;
  cudaFreeAsync(base, s);
  cudaStreamSynchronize(s);
  if (info) {
    acc.cycles = done;
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *info = acc;
  }
  return rc;
}
