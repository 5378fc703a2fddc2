// gk_accurate.cu -- FP64-grade products of a reduced-precision operator with a block of
// vectors, for the true residuals of Section 5 (err_rel and the per-triplet residuals
// ||A v_i - s_i u_i||, ||A^T u_i - s_i v_i||) and the refinement check of gk_psvd.
//
// The sweep's products (gk_matvec.cu) multiply in f32 and combine short f32 runs in f64:
// every entry is exact to ~2^-24 sum |a x|, which leaves a floor of about 1e-9 sigma_1 on the
// residuals of the benchmark operator -- a tenth of the 1e-8 tolerance.  A residual that is
// itself ~1e-8 of A v must be formed from products exact to well below that, so these
// kernels carry every product and every sum in double-f32 arithmetic on the FP32 pipes
// (GB300's FP64 rate is 1/64 of its FP32 rate):
//   x = x_hi + x_lo        (the f64 vector split into two f32, exact to 2^-48)
//   p = a x_hi, e = fma(a, x_hi, -p)         (TwoProd: p + e == a x_hi exactly)
//   (hi, t) = TwoSum(hi, p)                   (hi + t == old hi + p exactly)
//   lo += t + e + a x_lo                      (the small terms, in f32)
// so each output is the exact sum to about 2^-47 sum |a x|.  Pairs of vectors share packed
// f32x2 instructions (sm_100 FFMA2/FADD2/FMUL2).
//
// Tile: a CTA computes 128 outputs (rows of A x, or columns of A^T u) times 32 vectors,
// walking the contraction dimension in chunks of 32: the operator chunk is converted to f32
// in shared memory (transposed for A x), the vectors' hi/lo parts are staged beside it, and
// each thread updates 4 outputs x 4 vectors.  The operator is read once per 32 vectors
// (it stays HBM-light: the kernel is bound by the FP32 issue rate).
#include "gk_internal.cuh"

namespace gk {

namespace {

constexpr int kAThreads = 256;
constexpr int kAOut = 128;    // outputs per CTA tile
constexpr int kAVec = 32;     // vectors per CTA tile
constexpr int kAChunk = 32;   // contraction indices per shared-memory chunk
constexpr int kATR = 4;       // outputs per thread
constexpr int kATP = 2;       // vector pairs per thread (4 vectors)
static_assert((kAOut / kATR) * (kAVec / (2 * kATP)) == kAThreads, "thread grid covers the tile");

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// (hi, lo) += a * (xh + xl), pairwise over two vectors
__device__ __forceinline__ void df_madd(float2 &hi, float2 &lo, float2 a2, float2 na2, float2 xh, float2 xl) {
  const float2 m1 = f2(-1.f, -1.f);
  const float2 q = __fmul2_rn(na2, xh);      // -p, p = fl(a xh)
  const float2 e = __ffma2_rn(a2, xh, q);    // a xh - p (exact)
  const float2 s = __ffma2_rn(q, m1, hi);    // hi + p
  const float2 bb = __ffma2_rn(hi, m1, s);   // s - hi
  const float2 t1 = __ffma2_rn(bb, m1, s);   // s - bb
  const float2 d1 = __ffma2_rn(t1, m1, hi);  // hi - (s - bb)
  const float2 d2 = __fadd2_rn(q, bb);       // -(p - bb)
  float2 l = __ffma2_rn(a2, xl, lo);         // lo + a xl
  l = __fadd2_rn(l, e);
  l = __fadd2_rn(l, d1);
  lo = __ffma2_rn(d2, m1, l);                // + (p - bb): TwoSum error = d1 + (p - bb)
  hi = s;
}

// out[j * ldo + o] = scale * sum_c op(A)[o][c] * X[j][c]   (X given as hi/lo f32, [j * ldx + c])
// TRANS = false: op(A) = A (o: row, c: column); TRANS = true: op(A) = A^T (o: column, c: row).
// FAST = true: the same tiling in f32 -- x rounded to f32 (its high word), each 32-term chunk of
// products summed in f32, the chunk sums combined in double-f32 (TwoSum): every output within
// about 2^-24 (32 + 2) sum |a x| of the exact product, the precision model of gk_matvec's kernels,
// at about one FMA per product instead of eleven packed operations per two.
template <typename T, bool TRANS, bool FAST = false>
__global__ void __launch_bounds__(kAThreads) k_acc_gemm(const T *__restrict__ A, int64_t m, int64_t n, int64_t ld,
                                                        double scale, const float *__restrict__ xh,
                                                        const float *__restrict__ xl, int64_t ldx, int k,
                                                        double *__restrict__ out, int64_t ldo) {
  __shared__ float As[kAChunk][kAOut + 4];
  __shared__ float Xh[kAChunk][kAVec + 4];
  __shared__ float Xl[kAChunk][kAVec + 4];
  const int64_t nout = TRANS ? n : m;   // outputs
  const int64_t ncon = TRANS ? m : n;   // contraction length
  const int64_t o0 = (int64_t)blockIdx.x * kAOut;
  const int j0 = blockIdx.y * kAVec;
  const int tid = threadIdx.x;
  const int to = (tid % (kAOut / kATR)) * kATR;       // this thread's first output in the tile
  const int tv = (tid / (kAOut / kATR)) * (2 * kATP);  // this thread's first vector in the tile
  float2 hi[kATR][kATP], lo[kATR][kATP];
#pragma unroll
  for (int r = 0; r < kATR; ++r)
#pragma unroll
    for (int p = 0; p < kATP; ++p) {
      hi[r][p] = f2(0.f, 0.f);
      lo[r][p] = f2(0.f, 0.f);
    }
  for (int64_t c0 = 0; c0 < ncon; c0 += kAChunk) {
    // the operator chunk (f32, zero outside), As[c][o]
    for (int i = tid; i < kAChunk * kAOut; i += kAThreads) {
      int cc, oo;
      if (TRANS) {  // consecutive threads: consecutive columns of one row of A
        cc = i / kAOut;
        oo = i % kAOut;
      } else {      // consecutive threads: consecutive columns of one row of A (= c)
        oo = i / kAChunk;
        cc = i % kAChunk;
      }
      const int64_t o = o0 + oo, c = c0 + cc;
      float v = 0.f;
      if (o < nout && c < ncon) v = Vec<T>::one(TRANS ? A + c * ld + o : A + o * ld + c);
      As[cc][oo] = v;
    }
    for (int i = tid; i < kAChunk * kAVec; i += kAThreads) {
      const int vv = i / kAChunk, cc = i % kAChunk;
      const int64_t c = c0 + cc;
      const int j = j0 + vv;
      float a = 0.f, b = 0.f;
      if (j < k && c < ncon) {
        a = xh[(int64_t)j * ldx + c];
        b = xl[(int64_t)j * ldx + c];
      }
      Xh[cc][vv] = a;
      Xl[cc][vv] = b;
    }
    __syncthreads();
    if constexpr (FAST) {
      float2 cs[kATR][kATP];  // this chunk's f32 sums
#pragma unroll
      for (int r = 0; r < kATR; ++r)
#pragma unroll
        for (int p = 0; p < kATP; ++p) cs[r][p] = f2(0.f, 0.f);
#pragma unroll 4
      for (int cc = 0; cc < kAChunk; ++cc) {
        const float4 a4 = *reinterpret_cast<const float4 *>(&As[cc][to]);
        const float av[kATR] = {a4.x, a4.y, a4.z, a4.w};
        const float4 h4 = *reinterpret_cast<const float4 *>(&Xh[cc][tv]);
        const float2 xhp[kATP] = {f2(h4.x, h4.y), f2(h4.z, h4.w)};
#pragma unroll
        for (int r = 0; r < kATR; ++r) {
          const float2 a2 = f2(av[r], av[r]);
#pragma unroll
          for (int p = 0; p < kATP; ++p) cs[r][p] = __ffma2_rn(a2, xhp[p], cs[r][p]);
        }
      }
      // (hi, lo) += chunk sum, TwoSum
      const float2 m1 = f2(-1.f, -1.f);
#pragma unroll
      for (int r = 0; r < kATR; ++r)
#pragma unroll
        for (int p = 0; p < kATP; ++p) {
          const float2 sm = __fadd2_rn(hi[r][p], cs[r][p]);
          const float2 bb = __ffma2_rn(hi[r][p], m1, sm);                  // s - hi
          const float2 d1 = __ffma2_rn(__ffma2_rn(bb, m1, sm), m1, hi[r][p]);  // hi - (s - bb)
          const float2 d2 = __ffma2_rn(bb, m1, cs[r][p]);                  // c - bb
          lo[r][p] = __fadd2_rn(lo[r][p], __fadd2_rn(d1, d2));
          hi[r][p] = sm;
        }
    } else {
#pragma unroll 4
      for (int cc = 0; cc < kAChunk; ++cc) {
        const float4 a4 = *reinterpret_cast<const float4 *>(&As[cc][to]);
        const float av[kATR] = {a4.x, a4.y, a4.z, a4.w};
        const float4 h4 = *reinterpret_cast<const float4 *>(&Xh[cc][tv]);
        const float4 l4 = *reinterpret_cast<const float4 *>(&Xl[cc][tv]);
        const float2 xhp[kATP] = {f2(h4.x, h4.y), f2(h4.z, h4.w)};
        const float2 xlp[kATP] = {f2(l4.x, l4.y), f2(l4.z, l4.w)};
#pragma unroll
        for (int r = 0; r < kATR; ++r) {
          const float2 a2 = f2(av[r], av[r]), na2 = f2(-av[r], -av[r]);
#pragma unroll
          for (int p = 0; p < kATP; ++p) df_madd(hi[r][p], lo[r][p], a2, na2, xhp[p], xlp[p]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kATR; ++r) {
    const int64_t o = o0 + to + r;
    if (o >= nout) continue;
#pragma unroll
    for (int p = 0; p < kATP; ++p) {
      const int j = j0 + tv + 2 * p;
      if (j < k) out[(int64_t)j * ldo + o] = ((double)hi[r][p].x + (double)lo[r][p].x) * scale;
      if (j + 1 < k) out[(int64_t)(j + 1) * ldo + o] = ((double)hi[r][p].y + (double)lo[r][p].y) * scale;
    }
  }
}

// The block calls' products for narrow blocks (k <= VEC, VEC = 8 or 16 vectors): k_acc_gemm's
// 32-vector tile would spend 3/4 (or 1/2) of its arithmetic on zero padding, which at 8 vectors
// puts a pass over a bf16 operator well above the FP32 pipes' rate at HBM speed.  Same thread work
// (4 outputs x 4 vectors), the 256 threads spread over VEC / 4 vector rows and 1024 / VEC output
// groups: 512 outputs per CTA at VEC = 8 (contraction chunks of 16), 256 at VEC = 16 (chunks of
// 32); shared memory ~35-38 KB.  FAST: each chunk's products summed in f32, the chunk sums
// combined in double-f32 (TwoSum), as k_acc_gemm's FAST instantiation; otherwise every product and
// sum in double-f32 (df_madd), as k_acc_gemm.
template <int VEC>
struct NarrowTile {
  static constexpr int kRows = VEC / 4;                   // thread rows (4 vectors each)
  static constexpr int kCols = kAThreads / kRows;         // thread columns (4 outputs each)
  static constexpr int kOut = kCols * kATR;               // outputs per CTA
  static constexpr int kChunk = VEC == 8 ? 16 : 32;       // contraction indices per chunk
};

// The contraction may be split over blockIdx.z (slices of cspan indices, a multiple of the chunk):
// with part, each slice writes its unscaled sums to part[(z * k + j) * ldo + o] for k_acc_reduce.
template <typename T, bool TRANS, bool FAST, int VEC>
__global__ void __launch_bounds__(kAThreads) k_acc_gemm_narrow(const T *__restrict__ A, int64_t m, int64_t n,
                                                               int64_t ld, double scale, const float *__restrict__ xh,
                                                               const float *__restrict__ xl, int64_t ldx, int k,
                                                               double *__restrict__ out, int64_t ldo, int64_t cspan,
                                                               double *__restrict__ part) {
  using Tl = NarrowTile<VEC>;
  static_assert(VEC == 8 || VEC == 16, "narrow tiles of 8 or 16 vectors");
  static_assert(Tl::kRows * 2 * kATP == VEC && Tl::kRows * Tl::kCols == kAThreads, "thread grid covers the tile");
  __shared__ __align__(16) float As[Tl::kChunk][Tl::kOut + 4];
  __shared__ __align__(16) float Xh[Tl::kChunk][VEC + 4];
  __shared__ __align__(16) float Xl[FAST ? 1 : Tl::kChunk][VEC + 4];
  const int64_t nout = TRANS ? n : m;
  const int64_t ncon = TRANS ? m : n;
  const int64_t o0 = (int64_t)blockIdx.x * Tl::kOut;
  const int j0 = blockIdx.y * VEC;
  const int tid = threadIdx.x;
  const int to = (tid % Tl::kCols) * kATR;        // this thread's first output in the tile
  const int tv = (tid / Tl::kCols) * (2 * kATP);  // this thread's first vector in the tile
  float2 hi[kATR][kATP], lo[kATR][kATP];
#pragma unroll
  for (int r = 0; r < kATR; ++r)
#pragma unroll
    for (int p = 0; p < kATP; ++p) {
      hi[r][p] = f2(0.f, 0.f);
      lo[r][p] = f2(0.f, 0.f);
    }
  const int64_t cbeg = (int64_t)blockIdx.z * cspan;
  const int64_t cend = cbeg + cspan < ncon ? cbeg + cspan : ncon;  // this slice of the contraction
  for (int64_t c0 = cbeg; c0 < cend; c0 += Tl::kChunk) {
    for (int i = tid; i < Tl::kChunk * Tl::kOut; i += kAThreads) {
      int cc, oo;
      if (TRANS) {  // consecutive threads: consecutive columns of one row of A
        cc = i / Tl::kOut;
        oo = i % Tl::kOut;
      } else {      // consecutive threads: consecutive columns of one row of A (= c)
        oo = i / Tl::kChunk;
        cc = i % Tl::kChunk;
      }
      const int64_t o = o0 + oo, c = c0 + cc;
      float v = 0.f;
      if (o < nout && c < cend) v = Vec<T>::one(TRANS ? A + c * ld + o : A + o * ld + c);
      As[cc][oo] = v;
    }
    for (int i = tid; i < Tl::kChunk * VEC; i += kAThreads) {
      const int vv = i / Tl::kChunk, cc = i % Tl::kChunk;
      const int64_t c = c0 + cc;
      const int j = j0 + vv;
      const bool in = j < k && c < cend;
      Xh[cc][vv] = in ? xh[(int64_t)j * ldx + c] : 0.f;
      if constexpr (!FAST) Xl[cc][vv] = in ? xl[(int64_t)j * ldx + c] : 0.f;
    }
    __syncthreads();
    if constexpr (FAST) {
      float2 cs[kATR][kATP];  // this chunk's f32 sums
#pragma unroll
      for (int r = 0; r < kATR; ++r)
#pragma unroll
        for (int p = 0; p < kATP; ++p) cs[r][p] = f2(0.f, 0.f);
#pragma unroll 4
      for (int cc = 0; cc < Tl::kChunk; ++cc) {
        const float4 a4 = *reinterpret_cast<const float4 *>(&As[cc][to]);
        const float av[kATR] = {a4.x, a4.y, a4.z, a4.w};
        const float4 h4 = *reinterpret_cast<const float4 *>(&Xh[cc][tv]);
        const float2 xhp[kATP] = {f2(h4.x, h4.y), f2(h4.z, h4.w)};
#pragma unroll
        for (int r = 0; r < kATR; ++r) {
          const float2 a2 = f2(av[r], av[r]);
#pragma unroll
          for (int p = 0; p < kATP; ++p) cs[r][p] = __ffma2_rn(a2, xhp[p], cs[r][p]);
        }
      }
      const float2 m1 = f2(-1.f, -1.f);
#pragma unroll
      for (int r = 0; r < kATR; ++r)
#pragma unroll
        for (int p = 0; p < kATP; ++p) {  // (hi, lo) += chunk sum, TwoSum
          const float2 sm = __fadd2_rn(hi[r][p], cs[r][p]);
          const float2 bb = __ffma2_rn(hi[r][p], m1, sm);
          const float2 d1 = __ffma2_rn(__ffma2_rn(bb, m1, sm), m1, hi[r][p]);
          const float2 d2 = __ffma2_rn(bb, m1, cs[r][p]);
          lo[r][p] = __fadd2_rn(lo[r][p], __fadd2_rn(d1, d2));
          hi[r][p] = sm;
        }
    } else {
#pragma unroll 4
      for (int cc = 0; cc < Tl::kChunk; ++cc) {
        const float4 a4 = *reinterpret_cast<const float4 *>(&As[cc][to]);
        const float av[kATR] = {a4.x, a4.y, a4.z, a4.w};
        const float4 h4 = *reinterpret_cast<const float4 *>(&Xh[cc][tv]);
        const float4 l4 = *reinterpret_cast<const float4 *>(&Xl[cc][tv]);
        const float2 xhp[kATP] = {f2(h4.x, h4.y), f2(h4.z, h4.w)};
        const float2 xlp[kATP] = {f2(l4.x, l4.y), f2(l4.z, l4.w)};
#pragma unroll
        for (int r = 0; r < kATR; ++r) {
          const float2 a2 = f2(av[r], av[r]), na2 = f2(-av[r], -av[r]);
#pragma unroll
          for (int p = 0; p < kATP; ++p) df_madd(hi[r][p], lo[r][p], a2, na2, xhp[p], xlp[p]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kATR; ++r) {
    const int64_t o = o0 + to + r;
    if (o >= nout) continue;
#pragma unroll
    for (int p = 0; p < kATP; ++p) {
      const int j = j0 + tv + 2 * p;
      const double v0 = (double)hi[r][p].x + (double)lo[r][p].x, v1 = (double)hi[r][p].y + (double)lo[r][p].y;
      if (part) {
        double *pz = part + (int64_t)blockIdx.z * k * ldo;
        if (j < k) pz[(int64_t)j * ldo + o] = v0;
        if (j + 1 < k) pz[(int64_t)(j + 1) * ldo + o] = v1;
      } else {
        if (j < k) out[(int64_t)j * ldo + o] = v0 * scale;
        if (j + 1 < k) out[(int64_t)(j + 1) * ldo + o] = v1 * scale;
      }
    }
  }
}

// out[j * ldo + o] = scale * sum_{z < Z} part[(z * k + j) * ldo + o], z ascending (o < nout, j < k)
__global__ void k_acc_reduce(const double *__restrict__ part, int Z, int k, int64_t nout, int64_t ldo, double scale,
                             double *__restrict__ out) {
  const int64_t total = nout * (int64_t)k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / nout, o = t % nout;
    double a = 0.0;
    for (int z = 0; z < Z; ++z) a += part[((int64_t)z * k + j) * ldo + o];
    out[j * ldo + o] = a * scale;
  }
}

// contraction slices of a narrow-tile launch: enough CTAs for about 1024 in flight, each slice at
// least 8 chunks, at most 64 slices
template <int VEC>
int narrow_splits(int64_t nout, int64_t ncon, int k) {
  using Tl = NarrowTile<VEC>;
  const int64_t ctas = ((nout + Tl::kOut - 1) / Tl::kOut) * ((k + VEC - 1) / VEC);
  int64_t z = (1024 + ctas - 1) / ctas;
  const int64_t zmax = (ncon + 8 * Tl::kChunk - 1) / (8 * Tl::kChunk);
  if (z > zmax) z = zmax;
  if (z > 64) z = 64;
  return z < 1 ? 1 : (int)z;
}

// x = hi + lo (two f32), the f64 vectors of a block (count entries)
__global__ void k_split(const double *__restrict__ x, int64_t count, float *__restrict__ hi, float *__restrict__ lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

// res[j] = || Y[:, j] - s_j W[:, j] ||  (len rows, column-major with ld = len), one block per vector
__global__ void __launch_bounds__(256) k_resid_norm(const double *__restrict__ Y, const double *__restrict__ W,
                                                    const double *__restrict__ s, int64_t len, double *__restrict__ res) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  const double sj = s[j];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
    const double d = Y[(int64_t)j * len + i] - sj * W[(int64_t)j * len + i];
    acc = fma(d, d, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    res[j] = sqrt(t);
  }
}

template <typename T, bool FAST, int VEC>
cudaError_t launch_narrow(const Op &A, bool trans, const float *xh, const float *xl, int64_t ldx, int k, double *out,
                          int64_t ldo, cudaStream_t s, double *npart) {
  using Tl = NarrowTile<VEC>;
  const int64_t nout = trans ? A.n : A.m, ncon = trans ? A.m : A.n;
  const int Z = npart ? narrow_splits<VEC>(nout, ncon, k) : 1;
  int64_t cspan = (ncon + Z - 1) / Z;
  cspan = (cspan + Tl::kChunk - 1) / Tl::kChunk * Tl::kChunk;
  double *part = Z > 1 ? npart : nullptr;
  dim3 grid((unsigned)((nout + Tl::kOut - 1) / Tl::kOut), (unsigned)((k + VEC - 1) / VEC), (unsigned)Z);
  if (trans)
    GK_LAUNCH(k_acc_gemm_narrow<T, true, FAST, VEC><<<grid, kAThreads, 0, s>>>(
        (const T *)A.vals, A.m, A.n, A.ld, A.scale, xh, xl, ldx, k, out, ldo, cspan, part));
  else
    GK_LAUNCH(k_acc_gemm_narrow<T, false, FAST, VEC><<<grid, kAThreads, 0, s>>>(
        (const T *)A.vals, A.m, A.n, A.ld, A.scale, xh, xl, ldx, k, out, ldo, cspan, part));
  if (part) {
    int64_t b = (nout * k + 255) / 256;
    if (b > 4096) b = 4096;
    GK_LAUNCH(k_acc_reduce<<<(int)b, 256, 0, s>>>(part, Z, k, nout, ldo, A.scale, out));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_acc(const Op &A, bool trans, const float *xh, const float *xl, int64_t ldx, int k, double *out,
                       int64_t ldo, cudaStream_t s, bool fast, bool narrow, double *npart) {
  const int64_t nout = trans ? A.n : A.m;
  dim3 grid((unsigned)((nout + kAOut - 1) / kAOut), (unsigned)((k + kAVec - 1) / kAVec));
  if (narrow && k <= 8)
    return fast ? launch_narrow<T, true, 8>(A, trans, xh, xl, ldx, k, out, ldo, s, npart)
                : launch_narrow<T, false, 8>(A, trans, xh, xl, ldx, k, out, ldo, s, npart);
  if (narrow && k <= 16)
    return fast ? launch_narrow<T, true, 16>(A, trans, xh, xl, ldx, k, out, ldo, s, npart)
                : launch_narrow<T, false, 16>(A, trans, xh, xl, ldx, k, out, ldo, s, npart);
  if (fast) {
    if (trans)
      GK_LAUNCH(k_acc_gemm<T, true, true><<<grid, kAThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, A.scale, xh,
                                                                       xl, ldx, k, out, ldo));
    else
      GK_LAUNCH(k_acc_gemm<T, false, true><<<grid, kAThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, A.scale, xh,
                                                                        xl, ldx, k, out, ldo));
    return cudaGetLastError();
  }
  if (trans)
    GK_LAUNCH(k_acc_gemm<T, true><<<grid, kAThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, A.scale, xh, xl, ldx,
                                                               k, out, ldo));
  else
    GK_LAUNCH(k_acc_gemm<T, false><<<grid, kAThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, A.scale, xh, xl,
                                                                ldx, k, out, ldo));
  return cudaGetLastError();
}

}  // namespace

bool accurate_ok(const Op &A) { return A.kind == GK_DENSE && A.dtype != GK_F64; }

size_t accurate_floats(const Op &A, int k) {
  const int64_t len = A.m > A.n ? A.m : A.n;
  return 2 * (size_t)len * (size_t)k;
}

size_t accurate_narrow_doubles(const Op &A, int k) {
  if (k < 1 || k > 16) return 0;
  size_t need = 0;
  for (int t = 0; t < 2; ++t) {
    const int64_t nout = t ? A.n : A.m, ncon = t ? A.m : A.n;
    const int z = k <= 8 ? narrow_splits<8>(nout, ncon, k) : narrow_splits<16>(nout, ncon, k);
    const size_t d = z > 1 ? (size_t)z * (size_t)k * (size_t)nout : 0;
    if (d > need) need = d;
  }
  return need;
}

cudaError_t accurate_products(const Op &A, bool trans, const double *X, int k, double *out, float *split,
                              cudaStream_t s, bool fast, bool narrow, double *npart) {
  const int64_t len = trans ? A.m : A.n;  // length of the input vectors
  const int64_t cnt = len * (int64_t)k;
  float *xh = split, *xl = split + cnt;
  int64_t b = (cnt + 255) / 256;
  if (b > 4096) b = 4096;
  GK_LAUNCH(k_split<<<(int)b, 256, 0, s>>>(X, cnt, xh, xl));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t ldo = trans ? A.n : A.m;
  switch (A.dtype) {
    case GK_F32: return launch_acc<float>(A, trans, xh, xl, len, k, out, ldo, s, fast, narrow, npart);
    case GK_BF16: return launch_acc<__nv_bfloat16>(A, trans, xh, xl, len, k, out, ldo, s, fast, narrow, npart);
    case GK_F16: return launch_acc<__half>(A, trans, xh, xl, len, k, out, ldo, s, fast, narrow, npart);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t resid_norms(const double *Y, const double *W, const double *S, int64_t len, int k, double *res,
                        cudaStream_t s) {
  GK_LAUNCH(k_resid_norm<<<k, 256, 0, s>>>(Y, W, S, len, res));
  return cudaGetLastError();
}

}  // namespace gk
