// gk_ritz_df.cuh -- Ritz vectors C = Q X (Eq. 2.13: U_K X_k, V_K Y_k; the thick restart's kept
// columns) from the double-f32 copy of the basis, on the FP32 pipes.
//
// Q (len x K, column-major, ld) is read as its copy Qs (every entry the pair hi + lo of f32
// values, exact to ~2^-48 of the f64 entry), X (K x ncol) as the same kind of pairs.  Each output
// is accumulated in double-f32: the product of the high words exactly (TwoProd, one FMA for its
// rounding error), added to the running high word by TwoSum, and the small terms (the rounding
// errors and both cross products) summed in f32 beside it, the pair renormalized every four
// terms; the f64 result is hi + lo, exact to about 2^-46 of sum_k |q_ik x_kj|.  GB300's FP64 rate is 1/64 of its FP32 rate, which is why
// this form exists.  One thread per output row and kRitzCols columns: a row of Q is read once
// per column group, X from the cache.  The per-thread function runs on the host in the CPU tests.
#pragma once

#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define GK_RITZ_ALIGN8 alignas(8)
#else
#define GK_RITZ_ALIGN8 __align__(8)
#endif
#ifdef __CUDA_ARCH__
#define GK_RITZ_UNROLL _Pragma("unroll")
#else
#define GK_RITZ_UNROLL
#endif

namespace gk {

constexpr int kRitzCols = 16;  // output columns per thread

struct GK_RITZ_ALIGN8 DfPair {
  float hi, lo;
};

__host__ __device__ inline DfPair df_split(double v) {
  const float h = (float)v;
  return DfPair{h, (float)(v - (double)h)};
}

// f32 operations that the compiler must not fuse into FMAs (the error-free transformations below
// rely on each rounding): the device's round-to-nearest intrinsics; on the host the tests compile
// with -ffp-contract=off
__host__ __device__ inline float rn_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ inline float rn_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ inline float rn_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

// (hi, lo) += q * x in double-f32
__host__ __device__ inline void df_fma(float &hi, float &lo, DfPair q, DfPair x) {
  const float p = rn_mul(q.hi, x.hi);
  const float e = fmaf(q.hi, x.hi, -p);  // q.hi x.hi = p + e exactly
  const float s = rn_add(hi, p);         // TwoSum(hi, p) = s + t exactly
  const float bb = rn_sub(s, hi);
  const float t = rn_add(rn_sub(hi, rn_sub(s, bb)), rn_sub(p, bb));
  hi = s;
  lo = rn_add(lo, rn_add(rn_add(t, e), fmaf(q.hi, x.lo, rn_mul(q.lo, x.hi))));
}

// (hi, lo) <- (hi + lo, the rounding error of that sum) when |hi| >= |lo| (QuickTwoSum): keeps
// the f32 sum of the small terms small, so its own rounding stays near 2^-48 of the result
__host__ __device__ inline void df_renorm(float &hi, float &lo) {
  const float s = rn_add(hi, lo);
  lo = rn_sub(lo, rn_sub(s, hi));
  hi = s;
}

// C[(c0 + c) * ldc + i] = sum_k Q[k * ldq + i] X[(c0 + c) * ldx + k] for c < nc (<= kRitzCols):
// one thread's outputs, row i, columns c0 .. c0 + nc - 1 (renormalized every 4 terms)
__host__ __device__ inline void ritz_df_row(const DfPair *Qs, long long ldq, long long i, int K, const DfPair *Xs,
                                            long long ldx, int c0, int nc, double *C, long long ldc) {
  float hi[kRitzCols], lo[kRitzCols];
  GK_RITZ_UNROLL
  for (int c = 0; c < kRitzCols; ++c) hi[c] = lo[c] = 0.f;
  for (int k = 0; k < K; ++k) {
    const DfPair q = Qs[(long long)k * ldq + i];
    GK_RITZ_UNROLL
    for (int c = 0; c < kRitzCols; ++c)
      if (c < nc) df_fma(hi[c], lo[c], q, Xs[(long long)(c0 + c) * ldx + k]);
    if ((k & 3) == 3) {
      GK_RITZ_UNROLL
      for (int c = 0; c < kRitzCols; ++c) df_renorm(hi[c], lo[c]);
    }
  }
  GK_RITZ_UNROLL
  for (int c = 0; c < kRitzCols; ++c)
    if (c < nc) C[(long long)(c0 + c) * ldc + i] = (double)hi[c] + (double)lo[c];
}

}  // namespace gk
