// gk_learn.cu -- the learned predictor of the rank and the Krylov dimension.
//
// Sketch (per problem, one block per 128-row chunk): Y = A Omega with Omega (n x 32) drawn
// N(0,1) from Philox4x32-10 + Box-Muller (entry (j, c) is draw number 32 j + c of the
// stream seeded with the sketch seed), accumulated in f32 tiles (for bf16 operators on the
// tensor pipe, with Omega rounded to bf16); each chunk's part of the 32 x 32 Gram matrix
// G = Y^T Y and of ||A||_F^2 in f64, the chunks summed in order (one thread per entry); the
// singular values of Y are the square roots of G's eigenvalues (cyclic Jacobi, f64).
// Features (35): log(sigma_i(Y) / (sqrt(32) ||A||_F)) for i = 1..32,
// log ||A||_F, log m, log n.
//
// MLP 35 -> 256 -> 256 -> 2 with exact (erf) GELU, f32.  Parameter vector:
// W1 (256 x 35), b1, W2 (256 x 256), b2, W3 (2 x 256), b3, then the input
// mean/std (35 + 35) and target mean/std (2 + 2) used to standardize.
// Training: forward, mean-squared-error loss on standardized targets,
// backward, Adam; inference may use bf16-rounded weights with f32 sums.
#include <math.h>

#include <algorithm>
#include <vector>

#include "gk_internal.cuh"

namespace gk {
namespace {

constexpr int kS = GK_SKETCH_COLS;  // 32
constexpr int kF = GK_FEATURES;     // 35
constexpr int kH = 256;

// parameter offsets
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH, ob3 = oW3 + 2 * kH;
constexpr int oXmu = ob3 + 2, oXsd = oXmu + kF, oYmu = oXsd + kF, oYsd = oYmu + 2;
static_assert(oYsd + 2 == GK_MLP_PARAMS, "parameter layout");
static_assert(ob3 + 2 == GK_MLP_TRAINABLE, "trainable prefix");

__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// draw i of the N(0,1) stream (the start-vector construction without the +2 shift)
__device__ float normal_draw(uint64_t seed, int64_t i) {
  const uint64_t b = (uint64_t)i >> 1;
  const uint4 x = philox(make_uint4((unsigned)b, (unsigned)(b >> 32), 0u, 0u),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const double ua = ((double)(((uint64_t)(x.x >> 5) << 26) | (x.y >> 6)) + 0.5) * 0x1.0p-53;
  const double ub = ((double)(((uint64_t)(x.z >> 5) << 26) | (x.w >> 6)) + 0.5) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(ua));
  const double two_pi = 6.283185307179586476925286766559;
  return (float)((i & 1) ? r * sin(two_pi * ub) : r * cos(two_pi * ub));
}

__global__ void k_omega(float *__restrict__ om, int64_t rows, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * kS; i += (int64_t)gridDim.x * blockDim.x)
    om[i] = normal_draw(seed, i);
}

struct SkProb {
  const void *A;
  int dtype;
  int64_t m, n, ld;
  double scale;
};

template <typename T>
__device__ __forceinline__ float ld_elem(const T *p) {
  return Vec<T>::one(p);
}
template <>
__device__ __forceinline__ float ld_elem<double>(const double *p) {
  return (float)*p;
}

// ---- sketch, stage 1: Gram partials of 128-row chunks ---------------------
// Work item = (problem, 128-row chunk).  The block computes the chunk's rows of
// Y = A Omega (128 x 32, f32 FMA chains over the columns in increasing order),
// then the chunk's Gram contribution Y_c^T Y_c (upper triangle, 528 entries,
// f64 sums of exact f32 x f32 products) and its f32-accumulated ||A_c||_F^2.
constexpr int kChunk = 128, kTileC = 64, kTri = kS * (kS + 1) / 2;  // 528
constexpr int kSkThreads = 256;

struct SkItem {
  int p;
  int r0;
};

// this thread's 32 elements of the tile at rows r0.., columns c0.. (element q at
// tile position tid + 256 q: row (tid + 256 q) / 64, column (tid + 256 q) % 64),
// zero outside A; all 32 loads are issued before any is used
constexpr int kPerThr = kChunk * kTileC / kSkThreads;  // 32
template <typename T>
__device__ __forceinline__ void sk_load(const T *A, int64_t ld, int64_t m, int64_t n, int64_t r0, int64_t c0,
                                        float *v) {
  // element q sits at row rb + 4 q, column cc (256 threads = 4 rows of 64)
  const int cc = threadIdx.x % kTileC, rb = threadIdx.x / kTileC;
  const bool cok = c0 + cc < n;
  const int64_t avail = m - (r0 + rb);
  const T *p = A + (r0 + rb) * ld + c0 + cc;
  const int64_t step = (kSkThreads / kTileC) * ld;
#pragma unroll
  for (int q = 0; q < kPerThr; ++q) v[q] = (cok && (int64_t)(kSkThreads / kTileC) * q < avail) ? ld_elem<T>(p + q * step) : 0.f;
}

template <typename T>
__global__ void __launch_bounds__(kSkThreads) k_sketch_gram(const SkProb *__restrict__ probs,
                                                           const SkItem *__restrict__ items, int nitems,
                                                           const float *__restrict__ om, double *__restrict__ gpart,
                                                           double *__restrict__ fpart) {
  __shared__ float sA[kChunk * (kTileC + 1)];  // A tile, later Y (pitch 33)
  __shared__ __align__(16) float sO[kTileC * kS];
  __shared__ double sred[kSkThreads / 32];
  const int tid = threadIdx.x;
  const int tr = tid / 8, tc = (tid % 8) * 4;  // rows 4 tr .. 4 tr + 3, columns tc .. tc + 3 of Y
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const SkItem I = items[it];
    const SkProb P = probs[I.p];
    const T *A = (const T *)P.A;
    const int64_t m = P.m, n = P.n, ld = P.ld, r0 = I.r0;
    const float scale = (float)P.scale;
    float y[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) y[i][j] = 0.f;
    double fro = 0.0;
    float v[kPerThr];
    constexpr int kOPer = kTileC * kS / kSkThreads;  // 8 Omega entries per thread and tile
    float ov[kOPer];
    auto load_om = [&](int64_t c0) {
#pragma unroll
      for (int k = 0; k < kOPer; ++k) {
        const int e = tid + kSkThreads * k;
        const int64_t rr = c0 + e / kS;
        ov[k] = rr < n ? om[rr * kS + e % kS] : 0.f;
      }
    };
    sk_load<T>(A, ld, m, n, r0, 0, v);
    load_om(0);
    for (int64_t c0 = 0; c0 < n; c0 += kTileC) {
      float fs = 0.f;
      __syncthreads();  // the previous tile (or item) is consumed
#pragma unroll
      for (int q = 0; q < kPerThr; ++q) {
        const float a = v[q] * scale;
        sA[(tid / kTileC + (kSkThreads / kTileC) * q) * (kTileC + 1) + tid % kTileC] = a;
        fs = fmaf(a, a, fs);
      }
#pragma unroll
      for (int k = 0; k < kOPer; ++k) sO[tid + kSkThreads * k] = ov[k];
      fro += (double)fs;
      __syncthreads();
      if (c0 + kTileC < n) {  // next tile in flight during the products
        sk_load<T>(A, ld, m, n, r0, c0 + kTileC, v);
        load_om(c0 + kTileC);
      }
#pragma unroll 8
      for (int kk = 0; kk < kTileC; ++kk) {
        const float4 o = *reinterpret_cast<const float4 *>(sO + kk * kS + tc);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float a = sA[(tr * 4 + i) * (kTileC + 1) + kk];
          y[i][0] = fmaf(a, o.x, y[i][0]);
          y[i][1] = fmaf(a, o.y, y[i][1]);
          y[i][2] = fmaf(a, o.z, y[i][2]);
          y[i][3] = fmaf(a, o.w, y[i][3]);
        }
      }
    }
    __syncthreads();
    float *sY = sA;  // 128 x 33
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sY[(tr * 4 + i) * (kS + 1) + tc + j] = y[i][j];
    // ||A_c||_F^2: warp sums then a fixed-order block sum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if ((tid & 31) == 0) sred[tid >> 5] = fro;
    __syncthreads();
    const int rows = (int)((m - r0) < kChunk ? (m - r0) : kChunk);
    for (int e = tid; e < kTri; e += kSkThreads) {
      // e -> (a, b), a <= b, row-major over the upper triangle
      int a = 0, rem = e;
      while (rem >= kS - a) {
        rem -= kS - a;
        ++a;
      }
      const int b = a + rem;
      double g = 0.0;
      for (int r = 0; r < rows; ++r) g = fma((double)sY[r * (kS + 1) + a], (double)sY[r * (kS + 1) + b], g);
      gpart[(int64_t)it * kTri + e] = g;
    }
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kSkThreads / 32; ++w) t += sred[w];
      fpart[it] = t;
    }
  }
}

// ---- bf16 operators: Y = A Omega on the tensor pipe ------------------------------------
// Omega is rounded to bf16 (round to nearest even) and stored transposed, omT[c][k] (32 x nk, nk
// a multiple of 64, zero past n).  A block takes a 128-row chunk: each of 8 warps owns 16 rows
// and accumulates its 16 x 32 slice of Y in f32 with mma.sync m16n8k16 (bf16 fragments from
// shared memory by ldmatrix), streaming 64-column tiles of A and omT through registers; then
// the chunk's Gram partial and ||A_c||_F^2 exactly as k_sketch_gram does.
constexpr int kMmK = 64, kMmPitch = kMmK + 8;  // bf16 elements per tile row; padded pitch (144 B)

__global__ void k_omega_t_bf16(const float *__restrict__ om, int64_t n, int64_t nk, __nv_bfloat16 *__restrict__ omT) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nk * kS; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / nk, k = t % nk;
    omT[t] = __float2bfloat16_rn(k < n ? om[k * kS + c] : 0.f);
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t &r0, uint32_t &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__global__ void __launch_bounds__(kSkThreads) k_sketch_mma(const SkProb *__restrict__ probs,
                                                          const SkItem *__restrict__ items, int nitems,
                                                          const __nv_bfloat16 *__restrict__ omT, int64_t nk,
                                                          double *__restrict__ gpart, double *__restrict__ fpart) {
  __shared__ __align__(16) __nv_bfloat16 sA[kChunk * kMmPitch];
  __shared__ __align__(16) __nv_bfloat16 sO[kS * kMmPitch];
  __shared__ float sY[kChunk * (kS + 1)];
  __shared__ double sred[kSkThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t4 = lane & 3;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const SkItem I = items[it];
    const SkProb P = probs[I.p];
    const __nv_bfloat16 *A = (const __nv_bfloat16 *)P.A;
    const int64_t m = P.m, n = P.n, ld = P.ld, r0 = I.r0;
    float acc[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    double fro = 0.0;
    uint4 av[4], ov;
    // this thread's 4 16-byte vectors of the A tile (vector v = tid + 256 q: row v / 8, columns
    // 8 (v % 8)..), zero outside A; one vector of omT (row tid / 8, columns 8 (tid % 8)..)
    auto load = [&](int64_t k0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int v = tid + kSkThreads * q, row = v >> 3, c8 = (v & 7) * 8;
        const int64_t gr = r0 + row, gc = k0 + c8;
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        if (gr < m && gc < n) {
          const __nv_bfloat16 *src = A + gr * ld + gc;
          if (gc + 8 <= n) {
            x = *reinterpret_cast<const uint4 *>(src);
          } else {
            unsigned short e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = 0; i < 8 && gc + i < n; ++i) e[i] = __bfloat16_as_ushort(src[i]);
            x = make_uint4(e[0] | ((unsigned)e[1] << 16), e[2] | ((unsigned)e[3] << 16), e[4] | ((unsigned)e[5] << 16),
                           e[6] | ((unsigned)e[7] << 16));
          }
        }
        av[q] = x;
      }
      ov = *reinterpret_cast<const uint4 *>(omT + (int64_t)(tid >> 3) * nk + k0 + (tid & 7) * 8);
    };
    load(0);
    for (int64_t k0 = 0; k0 < n; k0 += kMmK) {
      __syncthreads();  // the previous tile (or item) is consumed
      float fs = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int v = tid + kSkThreads * q, row = v >> 3, c8 = (v & 7) * 8;
        *reinterpret_cast<uint4 *>(sA + row * kMmPitch + c8) = av[q];
        const unsigned w4[4] = {av[q].x, av[q].y, av[q].z, av[q].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float lo = __uint_as_float(w4[i] << 16), hi = __uint_as_float(w4[i] & 0xffff0000u);
          fs = fmaf(lo, lo, fs);
          fs = fmaf(hi, hi, fs);
        }
      }
      *reinterpret_cast<uint4 *>(sO + (tid >> 3) * kMmPitch + (tid & 7) * 8) = ov;
      fro += (double)fs;
      __syncthreads();
      if (k0 + kMmK < n) load(k0 + kMmK);  // next tile in flight during the products
#pragma unroll
      for (int kk = 0; kk < kMmK / 16; ++kk) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(smem_addr(sA + (warp * 16 + (lane & 15)) * kMmPitch + kk * 16 + (lane >> 4) * 8), a0, a1, a2, a3);
#pragma unroll
        for (int nt = 0; nt < kS / 8; ++nt) {
          uint32_t b0, b1;
          ldsm_x2(smem_addr(sO + (nt * 8 + (lane & 7)) * kMmPitch + kk * 16 + ((lane >> 3) & 1) * 8), b0, b1);
          mma_bf16_16816(acc[nt], a0, a1, a2, a3, b0, b1);
        }
      }
    }
    __syncthreads();
    const float scale = (float)P.scale;
#pragma unroll
    for (int nt = 0; nt < kS / 8; ++nt) {
      const int r = warp * 16 + g, c = nt * 8 + 2 * t4;
      sY[r * (kS + 1) + c] = acc[nt][0] * scale;
      sY[r * (kS + 1) + c + 1] = acc[nt][1] * scale;
      sY[(r + 8) * (kS + 1) + c] = acc[nt][2] * scale;
      sY[(r + 8) * (kS + 1) + c + 1] = acc[nt][3] * scale;
    }
    fro *= P.scale * P.scale;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if (lane == 0) sred[warp] = fro;
    __syncthreads();
    const int rows = (int)((m - r0) < kChunk ? (m - r0) : kChunk);
    for (int e = tid; e < kTri; e += kSkThreads) {
      int a = 0, rem = e;
      while (rem >= kS - a) {
        rem -= kS - a;
        ++a;
      }
      const int b = a + rem;
      double gg = 0.0;
      for (int r = 0; r < rows; ++r) gg = fma((double)sY[r * (kS + 1) + a], (double)sY[r * (kS + 1) + b], gg);
      gpart[(int64_t)it * kTri + e] = gg;
    }
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kSkThreads / 32; ++w) t += sred[w];
      fpart[it] = t;
    }
  }
}

// the chunk partials of problem p summed in chunk order: gsum[p * (kTri + 1) + e] for the 528
// Gram entries and e = kTri for ||A||_F^2 (one thread per entry, each in ascending chunk order)
__global__ void __launch_bounds__(128) k_sketch_sum(const int *__restrict__ first, int count,
                                                    const double *__restrict__ gpart,
                                                    const double *__restrict__ fpart, double *__restrict__ gsum) {
  const int p = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count || e > kTri) return;
  const int c0 = first[p], c1 = first[p + 1];
  double g = 0.0;
  if (e < kTri) {
#pragma unroll 8
    for (int c = c0; c < c1; ++c) g += gpart[(int64_t)c * kTri + e];
  } else {
#pragma unroll 8
    for (int c = c0; c < c1; ++c) g += fpart[c];
  }
  gsum[(int64_t)p * (kTri + 1) + e] = g;
}

// tournament (circle method) pairing of 32 indices: round r, slot s
__device__ __forceinline__ int pair_player(int r, int s) { return s == 0 ? 0 : ((s - 1 + r) % (kS - 1)) + 1; }

// ---- sketch, stage 2: per problem, sum the chunk partials in chunk order,
// eigenvalues of G by parallel cyclic Jacobi (one warp), the 35 features --------
__global__ void __launch_bounds__(32) k_sketch_eig(const SkProb *__restrict__ probs, int count,
                                                  const double *__restrict__ gsum, float *__restrict__ feats) {
  __shared__ double sG[kS * kS];
  __shared__ double2 sRot[kS / 2];
  __shared__ int2 sPair[kS / 2];
  const int lane = threadIdx.x;
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const SkProb P = probs[p];
    const double *gp = gsum + (int64_t)p * (kTri + 1);
    __syncwarp();
    for (int e = lane; e < kTri; e += 32) {
      int a = 0, rem = e;
      while (rem >= kS - a) {
        rem -= kS - a;
        ++a;
      }
      const int b = a + rem;
      const double g = gp[e];
      sG[a * kS + b] = g;
      sG[b * kS + a] = g;
    }
    const double fro2 = gp[kTri];
    __syncwarp();
    // parallel cyclic Jacobi (tournament ordering): each round, lanes 0..15 take one of 16
    // disjoint index pairs and compute its rotation; the warp then applies all 16 to the
    // columns (lane = row) and to the rows (lane = column)
    for (int sweep = 0; sweep < 30; ++sweep) {
      int rotated = 0;
      for (int r = 0; r < kS - 1; ++r) {
        if (lane < kS / 2) {
          int pp = pair_player(r, lane), q = pair_player(r, kS - 1 - lane);
          if (pp > q) {
            const int t = pp;
            pp = q;
            q = t;
          }
          const double apq = sG[pp * kS + q];
          const double app = sG[pp * kS + pp], aqq = sG[q * kS + q];
          double c = 1.0, sn = 0.0;
          if (!(apq == 0.0 || fabs(apq) <= 0x1.0p-52 * sqrt(fabs(app) * fabs(aqq)))) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t =
                fabs(tau) > 1e150 ? 0.5 / tau : (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
            rotated = 1;
          }
          sRot[lane] = make_double2(c, sn);
          sPair[lane] = make_int2(pp, q);
        }
        __syncwarp();
#pragma unroll 4
        for (int k = 0; k < kS / 2; ++k) {  // columns: lane is the row
          const double2 cs = sRot[k];
          const int2 pq = sPair[k];
          const double x = sG[lane * kS + pq.x], y2 = sG[lane * kS + pq.y];
          sG[lane * kS + pq.x] = cs.x * x - cs.y * y2;
          sG[lane * kS + pq.y] = cs.y * x + cs.x * y2;
        }
        __syncwarp();
#pragma unroll 4
        for (int k = 0; k < kS / 2; ++k) {  // rows: lane is the column
          const double2 cs = sRot[k];
          const int2 pq = sPair[k];
          const double x = sG[pq.x * kS + lane], y2 = sG[pq.y * kS + lane];
          sG[pq.x * kS + lane] = cs.x * x - cs.y * y2;
          sG[pq.y * kS + lane] = cs.y * x + cs.x * y2;
        }
        __syncwarp();
      }
      if (!__any_sync(0xffffffffu, rotated)) break;
    }
    // sort the eigenvalues descending and form the features
    const double lam = sG[lane * kS + lane];
    int rk = 0;
    for (int o = 0; o < kS; ++o) {
      const double lo = sG[o * kS + o];
      rk += (lo > lam) || (lo == lam && o < lane);
    }
    const double nf = sqrt(fro2);
    const double ref = sqrt((double)kS) * nf;
    const double sv = sqrt(fmax(lam, 0.0));
    float *f = feats + (int64_t)p * kF;
    f[rk] = (float)log(fmax(sv, 1e-30 * fmax(ref, 1e-300)) / fmax(ref, 1e-300));
    if (lane == 0) {
      f[kS] = (float)log(fmax(nf, 1e-300));
      f[kS + 1] = (float)log((double)P.m);
      f[kS + 2] = (float)log((double)P.n);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// MLP kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// C (M x N) = A (M x K, row-major, lda) * op(B) + bias, op(B) = B^T when B is N x K (row-major, ldb);
// weights may be bf16 (Wb) or f32 (B).  16 x 16 tiles of K.
template <bool BF16W>
__global__ void k_dense(const float *__restrict__ A, int lda, const float *__restrict__ B,
                        const __nv_bfloat16 *__restrict__ Wb, int ldb, const float *__restrict__ bias, float *__restrict__ C,
                        int ldc, int M, int N, int K, int act, float *__restrict__ Zsave) {
  __shared__ float sa[16][17], sb[16][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    sa[ty][tx] = (row < M && k0 + tx < K) ? A[(int64_t)row * lda + k0 + tx] : 0.f;
    const int brow = blockIdx.x * 16 + ty;  // output column index for the B tile load
    float bv = 0.f;
    if (brow < N && k0 + tx < K) bv = BF16W ? __bfloat162float(Wb[(int64_t)brow * ldb + k0 + tx]) : B[(int64_t)brow * ldb + k0 + tx];
    sb[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fmaf(sa[ty][kk], sb[tx][kk], acc);
    __syncthreads();
  }
  if (row < M && col < N) {
    const float z = acc + (bias ? bias[col] : 0.f);
    if (Zsave) Zsave[(int64_t)row * ldc + col] = z;
    C[(int64_t)row * ldc + col] = act ? gelu(z) : z;
  }
}

// C (M x N) = A^T (A: K x M row-major) * B (K x N row-major): weight gradients
__global__ void k_dense_tn(const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
                           float *__restrict__ C, int ldc, int M, int N, int K) {
  __shared__ float sa[16][17], sb[16][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    sa[ty][tx] = (k0 + ty < K && blockIdx.y * 16 + tx < M) ? A[(int64_t)(k0 + ty) * lda + blockIdx.y * 16 + tx] : 0.f;
    sb[ty][tx] = (k0 + ty < K && col < N) ? B[(int64_t)(k0 + ty) * ldb + col] : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fmaf(sa[kk][ty], sb[kk][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) C[(int64_t)row * ldc + col] = acc;
}

// C (M x N) = A (M x K row-major) * B (K x N row-major): backpropagation through a layer
__global__ void k_dense_nn(const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
                           float *__restrict__ C, int ldc, int M, int N, int K, const float *__restrict__ Zmul) {
  __shared__ float sa[16][17], sb[16][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    sa[ty][tx] = (row < M && k0 + tx < K) ? A[(int64_t)row * lda + k0 + tx] : 0.f;
    sb[ty][tx] = (k0 + ty < K && col < N) ? B[(int64_t)(k0 + ty) * ldb + col] : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fmaf(sa[ty][kk], sb[kk][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) C[(int64_t)row * ldc + col] = Zmul ? acc * gelu_grad(Zmul[(int64_t)row * ldc + col]) : acc;
}

// column sums of a (B x N) matrix into out[N] (bias gradients), fixed order
__global__ void k_colsum(const float *__restrict__ X, int B, int N, float *__restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += X[(int64_t)b * N + c];
  out[c] = s;
}

// standardized inputs X~ = (X - mu) / sd
__global__ void k_standardize(const float *__restrict__ X, int B, const float *__restrict__ params,
                              float *__restrict__ Xs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * kF) return;
  const int f = i % kF;
  Xs[i] = (X[i] - params[oXmu + f]) / params[oXsd + f];
}

// dO = (O - (Y - ymu)/ysd) / B and the loss sum 0.5 sum (O - Y~)^2 / B (one block)
__global__ void k_mse(const float *__restrict__ O, const float *__restrict__ Y, int B, const float *__restrict__ params,
                      float *__restrict__ dO, float *__restrict__ loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < 2 * B; i += blockDim.x) {
    const int o = i % 2;
    const float d = O[i] - (Y[i] - params[oYmu + o]) / params[oYsd + o];
    dO[i] = d / (float)B;
    s += 0.5f * d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / (float)B;
}

// de-standardized predictions: out = O * ysd + ymu
__global__ void k_destandardize(float *__restrict__ O, int B, const float *__restrict__ params) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * B) return;
  O[i] = O[i] * params[oYsd + i % 2] + params[oYmu + i % 2];
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                       int n, float lr, float b1, float b2, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void k_gather(const float *__restrict__ x, const float *__restrict__ y, const int *__restrict__ idx, int B,
                         float *__restrict__ xb, float *__restrict__ yb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * kF) xb[i] = x[(int64_t)idx[i / kF] * kF + i % kF];
  if (i < B * 2) yb[i] = y[(int64_t)idx[i / 2] * 2 + i % 2];
}

__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

int cdiv(int a, int b) { return (a + b - 1) / b; }

// activations of one forward pass (B rows)
struct Acts {
  float *Xs, *Z1, *A1, *Z2, *A2, *O;
};

size_t acts_floats(int B) { return (size_t)B * (kF + 4 * kH + 2); }

Acts carve_acts(float *p, int B) {
  Acts a;
  a.Xs = p;
  a.Z1 = a.Xs + (size_t)B * kF;
  a.A1 = a.Z1 + (size_t)B * kH;
  a.Z2 = a.A1 + (size_t)B * kH;
  a.A2 = a.Z2 + (size_t)B * kH;
  a.O = a.A2 + (size_t)B * kH;
  return a;
}

cudaError_t forward(const float *params, const __nv_bfloat16 *wb, const float *X, int B, Acts a, cudaStream_t s) {
  GK_LAUNCH(k_standardize<<<cdiv(B * kF, 256), 256, 0, s>>>(X, B, params, a.Xs));
  const dim3 blk(256);
  if (wb) {
    GK_LAUNCH(k_dense<true><<<dim3(cdiv(kH, 16), cdiv(B, 16)), blk, 0, s>>>(a.Xs, kF, nullptr, wb + oW1, kF,
                                                                            params + ob1, a.A1, kH, B, kH, kF, 1, a.Z1));
    GK_LAUNCH(k_dense<true><<<dim3(cdiv(kH, 16), cdiv(B, 16)), blk, 0, s>>>(a.A1, kH, nullptr, wb + oW2, kH,
                                                                            params + ob2, a.A2, kH, B, kH, kH, 1, a.Z2));
    GK_LAUNCH(k_dense<true><<<dim3(1, cdiv(B, 16)), blk, 0, s>>>(a.A2, kH, nullptr, wb + oW3, kH, params + ob3, a.O, 2,
                                                                 B, 2, kH, 0, nullptr));
  } else {
    GK_LAUNCH(k_dense<false><<<dim3(cdiv(kH, 16), cdiv(B, 16)), blk, 0, s>>>(a.Xs, kF, params + oW1, nullptr, kF,
                                                                             params + ob1, a.A1, kH, B, kH, kF, 1, a.Z1));
    GK_LAUNCH(k_dense<false><<<dim3(cdiv(kH, 16), cdiv(B, 16)), blk, 0, s>>>(a.A1, kH, params + oW2, nullptr, kH,
                                                                             params + ob2, a.A2, kH, B, kH, kH, 1, a.Z2));
    GK_LAUNCH(k_dense<false><<<dim3(1, cdiv(B, 16)), blk, 0, s>>>(a.A2, kH, params + oW3, nullptr, kH, params + ob3,
                                                                  a.O, 2, B, 2, kH, 0, nullptr));
  }
  return cudaGetLastError();
}

// gradient of the loss w.r.t. the trainable parameters (written to grad[0..GK_MLP_TRAINABLE))
cudaError_t backward(const float *params, const float *Y, int B, Acts a, float *grad, float *dbuf, float *loss,
                     cudaStream_t s) {
  float *dO = dbuf, *dZ2 = dO + 2 * (size_t)B, *dZ1 = dZ2 + (size_t)B * kH;
  const dim3 blk(256);
  GK_LAUNCH(k_mse<<<1, 256, 0, s>>>(a.O, Y, B, params, dO, loss));
  // layer 3: dW3 = dO^T A2 (2 x 256), db3 = colsum dO
  GK_LAUNCH(k_dense_tn<<<dim3(cdiv(kH, 16), 1), blk, 0, s>>>(dO, 2, a.A2, kH, grad + oW3, kH, 2, kH, B));
  GK_LAUNCH(k_colsum<<<1, 256, 0, s>>>(dO, B, 2, grad + ob3));
  // dZ2 = (dO W3) .* gelu'(Z2)
  GK_LAUNCH(k_dense_nn<<<dim3(cdiv(kH, 16), cdiv(B, 16)), blk, 0, s>>>(dO, 2, params + oW3, kH, dZ2, kH, B, kH, 2,
                                                                       a.Z2));
  GK_LAUNCH(k_dense_tn<<<dim3(cdiv(kH, 16), cdiv(kH, 16)), blk, 0, s>>>(dZ2, kH, a.A1, kH, grad + oW2, kH, kH, kH, B));
  GK_LAUNCH(k_colsum<<<1, 256, 0, s>>>(dZ2, B, kH, grad + ob2));
  // dZ1 = (dZ2 W2) .* gelu'(Z1)
  GK_LAUNCH(k_dense_nn<<<dim3(cdiv(kH, 16), cdiv(B, 16)), blk, 0, s>>>(dZ2, kH, params + oW2, kH, dZ1, kH, B, kH, kH,
                                                                       a.Z1));
  GK_LAUNCH(k_dense_tn<<<dim3(cdiv(kF, 16), cdiv(kH, 16)), blk, 0, s>>>(dZ1, kH, a.Xs, kF, grad + oW1, kF, kH, kF, B));
  GK_LAUNCH(k_colsum<<<1, 256, 0, s>>>(dZ1, B, kH, grad + ob1));
  return cudaGetLastError();
}


int check(cudaError_t e) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GK_CUDA_ERROR;
  }
  return GK_OK;
}

bool have_device() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return false;
  }
  return true;
}

}  // namespace
}  // namespace gk

using namespace gk;

extern "C" int gk_sketch_batched(const gk_matrix *A, int count, uint64_t seed, float *features, const gk_opts *opts) {
  if (!have_device()) return GK_NO_DEVICE;
  if (!A || count <= 0 || !features) return GK_INVALID_ARG;
  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  std::vector<SkProb> pr(count);
  std::vector<int> first(count + 1, 0);
  std::vector<SkItem> items;
  int64_t nmax = 1;
  const int dtype0 = A[0].dtype;
  for (int i = 0; i < count; ++i) {
    const gk_matrix &M = A[i];
    if (M.kind != GK_DENSE || M.m <= 0 || M.n <= 0 || M.ld < M.n || !M.vals || M.dtype != dtype0 ||
        M.dtype < GK_F64 || M.dtype > GK_F16 || M.m > (int64_t)INT32_MAX)
      return GK_INVALID_ARG;
    pr[i] = SkProb{M.vals, M.dtype, M.m, M.n, M.ld, M.scale};
    nmax = nmax > M.n ? nmax : M.n;
    first[i] = (int)items.size();
    for (int64_t r = 0; r < M.m; r += kChunk) items.push_back(SkItem{i, (int)r});
  }
  first[count] = (int)items.size();
  const int nitems = (int)items.size();
  bool mma_ok = dtype0 == GK_BF16;
  for (int i = 0; i < count && mma_ok; ++i)
    mma_ok = (uintptr_t)A[i].vals % 16 == 0 && (A[i].ld * 2) % 16 == 0;
  const int64_t nk = (nmax + kMmK - 1) / kMmK * kMmK;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_om = up(sizeof(float) * (size_t)nmax * kS), b_pr = up(sizeof(SkProb) * count),
               b_it = up(sizeof(SkItem) * nitems), b_first = up(sizeof(int) * (count + 1)),
               b_g = up(sizeof(double) * (size_t)nitems * kTri), b_f = up(sizeof(double) * nitems),
               b_ot = mma_ok ? up(sizeof(__nv_bfloat16) * (size_t)nk * kS) : 0,
               b_gs = up(sizeof(double) * (size_t)count * (kTri + 1)), b_err = up(sizeof(int));
  // the tensor-core form (opt-in): one bf16 operator whose rows the TMA can address
  const bool tc = mma_ok && count == 1 && opts && (opts->flags & GK_FLAG_SKETCH_TC) &&
                  sketch_tc_ok(A[0].vals, A[0].m, A[0].n, A[0].ld);
  if (opts && (opts->flags & GK_FLAG_SKETCH_TC) && !tc) return GK_INVALID_ARG;
  char *base = nullptr;
  if (cudaMallocAsync((void **)&base, b_om + b_pr + b_it + b_first + b_g + b_f + b_ot + b_gs + b_err, s) !=
      cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  float *om = (float *)base;
  SkProb *dpr = (SkProb *)(base + b_om);
  SkItem *dit = (SkItem *)(base + b_om + b_pr);
  int *dfirst = (int *)(base + b_om + b_pr + b_it);
  double *gpart = (double *)(base + b_om + b_pr + b_it + b_first);
  double *fpart = (double *)(base + b_om + b_pr + b_it + b_first + b_g);
  __nv_bfloat16 *omT = (__nv_bfloat16 *)(base + b_om + b_pr + b_it + b_first + b_g + b_f);
  double *gsum = (double *)(base + b_om + b_pr + b_it + b_first + b_g + b_f + b_ot);
  int *derr = (int *)(base + b_om + b_pr + b_it + b_first + b_g + b_f + b_ot + b_gs);
  int rc = GK_OK, herr = 0;
  do {
    if ((rc = check(cudaMemcpyAsync(dpr, pr.data(), sizeof(SkProb) * count, cudaMemcpyHostToDevice, s)))) break;
    if ((rc = check(cudaMemcpyAsync(dit, items.data(), sizeof(SkItem) * nitems, cudaMemcpyHostToDevice, s)))) break;
    if ((rc = check(cudaMemcpyAsync(dfirst, first.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s))))
      break;
    GK_LAUNCH(k_omega<<<(int)std::min<int64_t>(4096, (nmax * kS + 255) / 256), 256, 0, s>>>(om, nmax, seed));
    if (mma_ok) {  // bf16 rows on 16-byte boundaries: the tensor pipe, Omega rounded to bf16
      GK_LAUNCH(k_omega_t_bf16<<<(int)std::min<int64_t>(4096, (nk * kS + 255) / 256), 256, 0, s>>>(om, nmax, nk, omT));
      if (tc) {
        if ((rc = check(cudaMemsetAsync(derr, 0, sizeof(int), s)))) break;
        if ((rc = check(sketch_tc(A[0].vals, A[0].m, A[0].n, A[0].ld, A[0].scale, omT, nk, gpart, fpart, derr, s))))
          break;
      } else {
        GK_LAUNCH(k_sketch_mma<<<nitems, kSkThreads, 0, s>>>(dpr, dit, nitems, omT, nk, gpart, fpart));
      }
    } else switch (dtype0) {
      case GK_F64: GK_LAUNCH(k_sketch_gram<double><<<nitems, kSkThreads, 0, s>>>(dpr, dit, nitems, om, gpart, fpart)); break;
      case GK_F32: GK_LAUNCH(k_sketch_gram<float><<<nitems, kSkThreads, 0, s>>>(dpr, dit, nitems, om, gpart, fpart)); break;
      case GK_BF16:
        GK_LAUNCH(k_sketch_gram<__nv_bfloat16><<<nitems, kSkThreads, 0, s>>>(dpr, dit, nitems, om, gpart, fpart));
        break;
      default: GK_LAUNCH(k_sketch_gram<__half><<<nitems, kSkThreads, 0, s>>>(dpr, dit, nitems, om, gpart, fpart)); break;
    }
    GK_LAUNCH(k_sketch_sum<<<dim3((kTri + 1 + 127) / 128, count), 128, 0, s>>>(dfirst, count, gpart, fpart, gsum));
    GK_LAUNCH(k_sketch_eig<<<count, 32, 0, s>>>(dpr, count, gsum, features));
    if ((rc = check(cudaGetLastError()))) break;
    if (tc && (rc = check(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s)))) break;
    rc = check(cudaStreamSynchronize(s));
    if (rc == GK_OK && herr != 0) rc = GK_TIMEOUT;
  } while (0);
  cudaFreeAsync(base, s);
  cudaStreamSynchronize(s);
  return rc;
}

extern "C" int gk_mlp_forward(const float *params, const float *x, int B, float *out, int bf16_weights,
                              const gk_opts *opts) {
  if (!have_device()) return GK_NO_DEVICE;
  if (!params || !x || !out || B <= 0) return GK_INVALID_ARG;
  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  const size_t na = acts_floats(B);
  char *base = nullptr;
  const size_t bytes = sizeof(float) * na + sizeof(__nv_bfloat16) * GK_MLP_TRAINABLE + 512;
  if (cudaMallocAsync((void **)&base, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  Acts a = carve_acts((float *)base, B);
  __nv_bfloat16 *wb = bf16_weights ? (__nv_bfloat16 *)(base + (sizeof(float) * na + 255) / 256 * 256) : nullptr;
  int rc = GK_OK;
  do {
    if (wb) GK_LAUNCH(k_to_bf16<<<cdiv(GK_MLP_TRAINABLE, 256), 256, 0, s>>>(params, wb, GK_MLP_TRAINABLE));
    if ((rc = check(forward(params, wb, x, B, a, s)))) break;
    GK_LAUNCH(k_destandardize<<<cdiv(2 * B, 256), 256, 0, s>>>(a.O, B, params));
    if ((rc = check(cudaMemcpyAsync(out, a.O, sizeof(float) * 2 * B, cudaMemcpyDefault, s)))) break;
    rc = check(cudaStreamSynchronize(s));
  } while (0);
  cudaFreeAsync(base, s);
  cudaStreamSynchronize(s);
  return rc;
}

extern "C" int gk_mlp_grad(const float *params, const float *x, const float *y, int B, float *grad, float *loss,
                           const gk_opts *opts) {
  if (!have_device()) return GK_NO_DEVICE;
  if (!params || !x || !y || !grad || B <= 0) return GK_INVALID_ARG;
  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  const size_t na = acts_floats(B), nd = (size_t)B * (2 + 2 * kH);
  char *base = nullptr;
  if (cudaMallocAsync((void **)&base, sizeof(float) * (na + nd + 1) + 512, s) != cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  Acts a = carve_acts((float *)base, B);
  float *dbuf = (float *)base + na;
  float *dloss = dbuf + nd;
  int rc = GK_OK;
  do {
    if ((rc = check(forward(params, nullptr, x, B, a, s)))) break;
    if ((rc = check(backward(params, y, B, a, grad, dbuf, dloss, s)))) break;
    if (loss && (rc = check(cudaMemcpyAsync(loss, dloss, sizeof(float), cudaMemcpyDefault, s)))) break;
    rc = check(cudaStreamSynchronize(s));
  } while (0);
  cudaFreeAsync(base, s);
  cudaStreamSynchronize(s);
  return rc;
}

extern "C" int gk_mlp_train(float *params, float *adam_m, float *adam_v, int t0, const float *x, const float *y,
                            int n, int batch, int epochs, float lr, uint64_t seed, float *losses, const gk_opts *opts) {
  if (!have_device()) return GK_NO_DEVICE;
  if (!params || !adam_m || !adam_v || !x || !y || n <= 0 || batch <= 0 || epochs <= 0 || !(lr > 0.f))
    return GK_INVALID_ARG;
  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  const int B = batch < n ? batch : n;
  const size_t na = acts_floats(B), nd = (size_t)B * (2 + 2 * kH);
  char *base = nullptr;
  const size_t bytes =
      sizeof(float) * (na + nd + GK_MLP_TRAINABLE + (size_t)B * (kF + 2) + (size_t)epochs) + sizeof(int) * (size_t)n + 2048;
  if (cudaMallocAsync((void **)&base, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  Acts a = carve_acts((float *)base, B);
  float *dbuf = (float *)base + na;
  float *grad = dbuf + nd;
  float *xb = grad + GK_MLP_TRAINABLE;
  float *yb = xb + (size_t)B * kF;
  float *eloss = yb + (size_t)B * 2;
  int *dperm = (int *)(eloss + epochs + 64);
  // minibatches: a seeded permutation per epoch, drawn on the host (SplitMix64 keys)
  std::vector<int> perm(n);
  int rc = GK_OK;
  int t = t0;
  const float b1 = 0.9f, b2 = 0.999f;
  uint64_t st = seed;
  for (int ep = 0; ep < epochs && rc == GK_OK; ++ep) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) {  // Fisher-Yates with SplitMix64
      st += 0x9E3779B97F4A7C15ull;
      uint64_t z = st;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const int j = (int)(z % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    float *lsum = eloss + ep;
    if ((rc = check(cudaMemsetAsync(lsum, 0, sizeof(float), s)))) break;
    if ((rc = check(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)))) break;
    // the host copy of perm is rewritten next epoch: wait for this one to land
    if ((rc = check(cudaStreamSynchronize(s)))) break;
    for (int b0 = 0; b0 + B <= n && rc == GK_OK; b0 += B) {
      GK_LAUNCH(k_gather<<<cdiv(B * kF, 256), 256, 0, s>>>(x, y, dperm + b0, B, xb, yb));
      if ((rc = check(forward(params, nullptr, xb, B, a, s)))) break;
      if ((rc = check(backward(params, yb, B, a, grad, dbuf, nullptr, s)))) break;
      ++t;
      const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
      GK_LAUNCH(k_adam<<<cdiv(GK_MLP_TRAINABLE, 256), 256, 0, s>>>(params, adam_m, adam_v, grad, GK_MLP_TRAINABLE, lr, b1,
                                                                   b2, c1, c2));
    }
    // epoch loss on the last minibatch after the update
    if (rc == GK_OK) {
      if ((rc = check(forward(params, nullptr, xb, B, a, s)))) break;
      GK_LAUNCH(k_mse<<<1, 256, 0, s>>>(a.O, yb, B, params, dbuf, lsum));
    }
  }
  if (rc == GK_OK && losses) rc = check(cudaMemcpyAsync(losses, eloss, sizeof(float) * epochs, cudaMemcpyDefault, s));
  if (rc == GK_OK) rc = check(cudaStreamSynchronize(s));
  cudaFreeAsync(base, s);
  cudaStreamSynchronize(s);
  return rc;
}
