// gk_batched_kernel.cuh -- many independent problems in one persistent launch.
//
// The grid is a set of thread-block clusters; each cluster is a worker that
// takes problems from a device queue (ordered longest-first by the host's cost
// model) and solves each one completely on the device: the restarted partial
// SVD (upper-bidiagonal Golub-Kahan with two-pass Gram-Schmidt, Jacobi SVD of
// B, thick restarts) or Algorithm 3 (lower-bidiagonal Algorithm 1 with the
// break test, then the Sturm-count rank of B).  The CTAs of a cluster split the
// rows of A and of the basis vectors; coefficient vectors and the partial sums
// of A^T u are combined through distributed shared memory in a fixed CTA order,
// so every CTA obtains bitwise the same norms and takes the same decisions.
// Rounds are separated by hardware cluster barriers: the kernel has no
// software spin-wait.
#pragma once

#include <cooperative_groups.h>

#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "gk_device.cuh"
#include "gk_internal.cuh"

namespace gk {
namespace {

namespace cg = cooperative_groups;

constexpr int kBThreads = 256;
constexpr int kNMax = 4096;  // columns per problem (shared-memory copies of v and of A^T u partial sums)
constexpr int kKMax = 512;   // basis columns per problem
constexpr int kRunRows = 32; // f32 run length in rows before an f64 combine (A^T u)
// row ring: the CTA's rows of A stream through shared memory by 1-D bulk copies (TMA),
// kRingStages stages of kRingStage bytes, one mbarrier per stage
constexpr int kRingStages = 3;
constexpr int kRingStage = 16384;
constexpr long long kRingWait = 4000000000ll;  // ~2 s at 2 GHz before a wait gives up
constexpr size_t kSmemFixed = sizeof(float) * kNMax + sizeof(double) * (kNMax + 2 * (kKMax + 8)) + sizeof(int) * kKMax;
constexpr size_t kRingOffset = (kSmemFixed + 127) / 128 * 128;
constexpr size_t kSmemBytes = kRingOffset + (size_t)kRingStages * kRingStage;


struct BProb {
  const void *A;
  int dtype, mode;  // mode 0: restarted partial SVD, 1: Algorithm 3
  int64_t m, n, ld;
  double scale;
  int k, K, keep, max_restarts, passes, eps_rel;
  double tol;  // psvd tolerance or Algorithm 3 eps
  double cut;  // psvd: relative rank cut (0 = none)
  int prof;    // accumulate phase clocks
  double *U, *S, *V;
  const double *start;
  uint64_t seed;
  int64_t out;  // index of this problem's result row
};

struct BRes {
  int status, cycles, restarts, steps, rank, breakdowns, sweeps, pad;
  long long matvecs;
  double resid_est, sigma_est, sigma_next;
  // with profiling: SM clock cycles of the leading CTA in each phase (A v, A^T u with its
  // cluster reduction, Gram-Schmidt and normalization, small SVD and test, setup/restart/output)
  long long cyc[5];
};

// phase clock of the leading thread (clock64 of one SM; every phase ends at a cluster
// barrier); the per-phase sums live in shared memory
struct PhaseClock {
  long long *acc;  // null: off
  long long t;
  __device__ static long long now() {
#ifdef __CUDA_ARCH__
    return clock64();
#else
    return 0;
#endif
  }
  __device__ explicit PhaseClock(long long *a) : acc(a), t(a ? now() : 0) {}
  __device__ __forceinline__ void mark(int ph) {
    if (acc) {
      const long long n = now();
      acc[ph] += n - t;
      t = n;
    }
  }
};

struct BDims {
  int64_t ldu, ldv;  // basis leading dimensions
  int cols;          // basis columns per buffer
  int K;             // small-matrix dimension
};

struct BWork {
  double *Ub, *Ub2, *Vb, *Vb2, *w, *z, *alpha, *beta, *Bm, *Yw, *X, *Y, *sigma, *rho, *nrm;
  int *pos;
};

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline size_t work_bytes(const BDims &d) {
  const size_t bu = al256(sizeof(double) * d.ldu * d.cols), bv = al256(sizeof(double) * d.ldv * d.cols);
  const size_t kk = al256(sizeof(double) * (size_t)d.K * d.K), kv = al256(sizeof(double) * (d.K + 2));
  return 2 * bu + 2 * bv + al256(8 * d.ldu) + al256(8 * d.ldv) + 2 * kv + 4 * kk + 3 * kv + al256(4 * (d.K + 2));
}

__device__ BWork carve(char *p, const BDims &d) {
  BWork w;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += al256(bytes);
    return q;
  };
  w.Ub = (double *)take(sizeof(double) * d.ldu * d.cols);
  w.Ub2 = (double *)take(sizeof(double) * d.ldu * d.cols);
  w.Vb = (double *)take(sizeof(double) * d.ldv * d.cols);
  w.Vb2 = (double *)take(sizeof(double) * d.ldv * d.cols);
  w.w = (double *)take(8 * d.ldu);
  w.z = (double *)take(8 * d.ldv);
  w.alpha = (double *)take(sizeof(double) * (d.K + 2));
  w.beta = (double *)take(sizeof(double) * (d.K + 2));
  w.Bm = (double *)take(sizeof(double) * (size_t)d.K * d.K);
  w.Yw = (double *)take(sizeof(double) * (size_t)d.K * d.K);
  w.X = (double *)take(sizeof(double) * (size_t)d.K * d.K);
  w.Y = (double *)take(sizeof(double) * (size_t)d.K * d.K);
  w.sigma = (double *)take(sizeof(double) * (d.K + 2));
  w.rho = (double *)take(sizeof(double) * (d.K + 2));
  w.nrm = (double *)take(sizeof(double) * (d.K + 2));
  w.pos = (int *)take(4 * (d.K + 2));
  return w;
}

// per-CTA shared memory of the solver
struct Shm {
  float *xs;     // kNMax: f32 copy of the vector A multiplies
  double *zp;    // kNMax: this CTA's partial sums of A^T u (read by the others)
  double *red;   // kKMax + 8: this CTA's partial coefficients (read by the others)
  double *hv;    // kKMax + 8: the cluster totals
  int *redi;     // kKMax: argmax indices
  int *s_rot, *s_any, *s_idx;
  long long *cyc;  // 5 phase-clock sums (profiling)
  unsigned char *ring;  // kRingStages x kRingStage bytes
  uint64_t *bar;        // kRingStages mbarriers (one arrival + the copies' bytes per phase)
  int *dead;            // set when a ring wait timed out: the ring stays unused afterwards
  int *err;             // kernel-wide timeout flag (global memory) read by the host
  unsigned seq;         // ring stages consumed so far (the same value in every thread)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// bounded wait for the phase of the given parity; false if it did not complete in time
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit = kRingWait) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// L2 prefetch of `bytes` (a multiple of 16) at a 16-byte aligned global address
__device__ __forceinline__ void l2_prefetch(const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// geometry of the ring for one operator: rows of n elements at a pitch of whole 16-byte
// groups; the bulk copies move the whole groups (bulk bytes), the consumers read the
// last partial group, if any, from global memory
struct RingGeom {
  int pitch, bulk, rows;  // bytes per staged row, bytes copied per row, rows per stage
  bool contig;            // rows adjacent in memory: one copy per stage
};

template <typename T>
__device__ __forceinline__ bool ring_geom(const BProb &P, const Shm &S, RingGeom *g) {
  if constexpr (std::is_same<T, double>::value) {
    return false;
  } else {
    const int64_t rowb = P.n * (int64_t)sizeof(T);
    if (*S.dead || ((uintptr_t)P.A & 15) || ((P.ld * (int64_t)sizeof(T)) & 15) || rowb > kRingStage) return false;
    g->bulk = (int)(rowb & ~(int64_t)15);
    g->pitch = (int)((rowb + 15) & ~(int64_t)15);
    g->rows = kRingStage / g->pitch;
    g->contig = (P.ld * (int64_t)sizeof(T) == rowb) && (rowb & 15) == 0;
    return true;
  }
}

// thread 0: stage `st` of the rows [r0, r1) into ring slot `slot`
template <typename T>
__device__ __forceinline__ void ring_issue(const BProb &P, Shm &S, const RingGeom &g, int64_t r0, int64_t r1,
                                           int64_t st, int slot) {
  const int64_t row0 = r0 + st * g.rows;
  const int cnt = (int)((r1 - row0) < g.rows ? (r1 - row0) : g.rows);
  uint64_t *b = S.bar + slot;
  unsigned char *dst = S.ring + (size_t)slot * kRingStage;
  const char *src = (const char *)P.A + row0 * P.ld * (int64_t)sizeof(T);
  mbar_expect(b, (unsigned)(cnt * g.bulk));
  if (g.bulk == 0) return;
  if (g.contig) {
    bulk_copy(dst, src, (unsigned)(cnt * g.bulk), b);
  } else {
    for (int i = 0; i < cnt; ++i)
      bulk_copy(dst + (size_t)i * g.pitch, src + (int64_t)i * P.ld * (int64_t)sizeof(T), (unsigned)g.bulk, b);
  }
}

// stream the rows [r0, r1) through the ring; consume(stage, first row, rows) runs on every
// thread once per stage.  Returns false (nothing done) if the ring cannot serve this operator;
// on a timed-out wait sets the error flags, marks the ring dead and returns true with the
// remaining stages unconsumed (the caller poisons its result).
template <typename T, typename F>
__device__ bool ring_rows(const BProb &P, Shm &S, const RingGeom &g, int64_t r0, int64_t r1, F &&consume,
                          bool *timed_out) {
  *timed_out = false;
  const int64_t nst = (r1 - r0 + g.rows - 1) / g.rows;
  if (nst <= 0) return true;
  if (threadIdx.x == 0)
    for (int64_t st = 0; st < nst && st < kRingStages; ++st) ring_issue<T>(P, S, g, r0, r1, st, (int)((S.seq + st) % kRingStages));
  for (int64_t st = 0; st < nst; ++st) {
    const unsigned q = S.seq + (unsigned)st;
    const int slot = (int)(q % kRingStages);
    const bool ok = mbar_wait_bounded(S.bar + slot, (q / kRingStages) & 1u);
    // every thread has finished the previous stage: its slot may be refilled
    const int bad = __syncthreads_or(!ok);
    if (threadIdx.x == 0 && st >= 1 && st - 1 + kRingStages < nst && !bad) {
      ring_issue<T>(P, S, g, r0, r1, st - 1 + kRingStages, (int)((q - 1) % kRingStages));
    }
    if (bad) {
      if (threadIdx.x == 0) {
        atomicExch(S.err, 1);
        *S.dead = 1;
        // copies still in flight: give each outstanding stage one more bounded wait
        for (int64_t t = st; t < nst && t < st - 1 + kRingStages; ++t) {
          const unsigned qt = S.seq + (unsigned)t;
          mbar_wait_bounded(S.bar + (qt % kRingStages), (qt / kRingStages) & 1u);
        }
      }
      __syncthreads();
      *timed_out = true;
      return true;
    }
    const int64_t row0 = r0 + st * g.rows;
    const int cnt = (int)((r1 - row0) < g.rows ? (r1 - row0) : g.rows);
    consume(S.ring + (size_t)slot * kRingStage, row0, cnt);
  }
  __syncthreads();  // the last stage is consumed before the ring is reused
  S.seq += (unsigned)nst;
  return true;
}

__device__ __forceinline__ void slice(int64_t len, unsigned r, unsigned cs, int64_t *a, int64_t *b) {
  *a = len * (int64_t)r / (int64_t)cs;
  *b = len * (int64_t)(r + 1) / (int64_t)cs;
}

// sum of the CTAs' red[0..L) in rank order into hv[0..L) of every CTA
__device__ void cl_allreduce(cg::cluster_group &cl, Shm &S, int L) {
  cl.sync();
  const unsigned cs = cl.num_blocks();
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    double t = 0.0;
    for (unsigned c = 0; c < cs; ++c) t += cl.map_shared_rank(S.red, c)[i];
    S.hv[i] = t;
  }
  cl.sync();
}

template <typename T>
__device__ __forceinline__ float load_val(const T *p) {
  return Vec<T>::one(p);
}

// w[r] = scale * (A x)_r - sum_c coefs[c] Qb[(c0 + c) ld + r], rows [r0, r1); x staged in S.xs (f32)
template <typename T>
__device__ void rows_matvec(const BProb &P, Shm &S, int64_t r0, int64_t r1, double *w, const double *Qb, int64_t ldq,
                            int c0, int cn, const double *coefs) {
  const T *A = (const T *)P.A;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t n = P.n;
  using VT = Vec<T>;
  constexpr int E = VT::E;
  const bool vec = (((uintptr_t)A % 16) == 0 && ((P.ld * (int64_t)sizeof(T)) % 16) == 0);
  // two rows per warp at a time: 2 x 4 loads of 16 bytes in flight per lane; lane 0 asks L2
  // for the warp's row pair two passes ahead
  const unsigned pf_bytes = (unsigned)((n * (int64_t)sizeof(T)) & ~(int64_t)15);
  for (int64_t rb = r0 + 2 * warp; rb < r1; rb += 2 * nw) {
    if (vec && lane == 0 && pf_bytes > 0) {
      const int64_t pr = rb + 4 * nw;
      if (pr < r1) l2_prefetch(A + pr * P.ld, pf_bytes);
      if (pr + 1 < r1) l2_prefetch(A + (pr + 1) * P.ld, pf_bytes);
    }
    double acc[2] = {0.0, 0.0};
    const int nr = (r1 - rb) >= 2 ? 2 : 1;  // the second row repeats the first when the slice is odd
    int64_t tail0 = 0;
    if (vec) {
      const int64_t nv = n / E;
      const typename VT::V *av0 = reinterpret_cast<const typename VT::V *>(A + rb * P.ld);
      const typename VT::V *av1 = reinterpret_cast<const typename VT::V *>(A + (rb + (nr - 1)) * P.ld);
      // four 16-byte groups per row and lane in flight; the last pass is predicated
      for (int64_t i = lane; i < nv; i += 32 * 4) {
        typename VT::V b0[4] = {}, b1[4] = {};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (i + 32 * q < nv) {
            b0[q] = __ldcs(av0 + i + 32 * q);
            b1[q] = __ldcs(av1 + i + 32 * q);
          }
        }
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (i + 32 * q < nv) {
            float f0[E], f1[E];
            VT::unpack(b0[q], f0);
            VT::unpack(b1[q], f1);
            const float4 *xv = reinterpret_cast<const float4 *>(S.xs + (i + 32 * q) * E);
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
              const float4 x4 = xv[h];
              s0 = fmaf(f0[4 * h], x4.x, s0);
              s0 = fmaf(f0[4 * h + 1], x4.y, s0);
              s0 = fmaf(f0[4 * h + 2], x4.z, s0);
              s0 = fmaf(f0[4 * h + 3], x4.w, s0);
              s1 = fmaf(f1[4 * h], x4.x, s1);
              s1 = fmaf(f1[4 * h + 1], x4.y, s1);
              s1 = fmaf(f1[4 * h + 2], x4.z, s1);
              s1 = fmaf(f1[4 * h + 3], x4.w, s1);
            }
          }
        }
        acc[0] += (double)s0;
        acc[1] += (double)s1;
      }
      tail0 = nv * E;
    }
    for (int h = 0; h < nr; ++h) {
      const T *a = A + (rb + h) * P.ld;
      float s = 0.f;
      int cnt = 0;
      for (int64_t c = tail0 + lane; c < n; c += 32) {
        s = fmaf(load_val<T>(a + c), S.xs[c], s);
        if (++cnt == 32) {
          acc[h] += (double)s;
          s = 0.f;
          cnt = 0;
        }
      }
      acc[h] += (double)s;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) acc[h] = dev::warp_sum_d(acc[h]);
    if (lane == 0)
      for (int h = 0; h < nr; ++h) w[rb + h] = acc[h] * P.scale;
  }
  // the basis combination after all rows (coalesced, off the rows' load chain)
  if (cn > 0) {
    __syncthreads();
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      double v = w[r];
      for (int c = 0; c < cn; ++c) v -= coefs[c] * Qb[(int64_t)(c0 + c) * ldq + r];
      w[r] = v;
    }
  }
}

// f64 operator: products in f64 with x read from the f64 basis column
__device__ void rows_matvec_f64(const BProb &P, int64_t r0, int64_t r1, const double *x, double *w, const double *Qb,
                                int64_t ldq, int c0, int cn, const double *coefs) {
  const double *A = (const double *)P.A;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t r = r0 + warp; r < r1; r += nw) {
    const double *a = A + r * P.ld;
    double acc = 0.0;
    for (int64_t c = lane; c < P.n; c += 32) acc = fma(a[c], x[c], acc);
    acc = dev::warp_sum_d(acc);
    if (lane == 0) {
      double v = acc * P.scale;
      for (int c = 0; c < cn; ++c) v -= coefs[c] * Qb[(int64_t)(c0 + c) * ldq + r];
      w[r] = v;
    }
  }
}

// this CTA's partial sums zp[c] = sum_{r in [r0, r1)} a_rc u_r for all columns.
// Every thread owns one 16-byte group of columns per sweep (E columns), walks
// the slice's rows eight at a time, sums f32 runs of kRunRows rows and combines
// them in f64; rows that are not 16-byte aligned take the scalar path.
// A^T u of the CTA's rows through the row ring: the thread owns 16-byte column groups
// tid, tid + 256, ...; u (f32) staged in S.xs; f32 runs of kRunRows rows combined in f64
// into S.zp; the columns of the partial last group from global memory
template <typename T>
__device__ bool ring_matvec_t(const BProb &P, Shm &S, int64_t r0, int64_t r1, const double *u) {
  if constexpr (std::is_same<T, double>::value) {
    return false;
  } else {
  RingGeom g;
  if (!ring_geom<T>(P, S, &g) || r1 - r0 > kNMax) return false;
  using VT = Vec<T>;
  constexpr int E = VT::E;
  constexpr int G = kNMax / (E * kBThreads);  // column groups per thread at most (4 f32, 2 bf16/f16)
  const T *A = (const T *)P.A;
  const int nvb = g.bulk / 16;
  const int64_t n = P.n;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) S.xs[r - r0] = (float)u[r];
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) S.zp[c] = 0.0;
  __syncthreads();
  float a32[G][E];
#pragma unroll
  for (int k = 0; k < G; ++k)
#pragma unroll
    for (int e = 0; e < E; ++e) a32[k][e] = 0.f;
  int run = 0;
  auto flush = [&]() {
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int gi = threadIdx.x + k * kBThreads;
      if (gi < nvb) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          S.zp[gi * E + e] += (double)a32[k][e];
          a32[k][e] = 0.f;
        }
      }
    }
  };
  bool to;
  ring_rows<T>(
      P, S, g, r0, r1,
      [&](const unsigned char *st, int64_t row0, int cnt) {
        for (int i = 0; i < cnt; ++i) {
          const typename VT::V *rv = reinterpret_cast<const typename VT::V *>(st + (size_t)i * g.pitch);
          const float ur = S.xs[row0 + i - r0];
#pragma unroll
          for (int k = 0; k < G; ++k) {
            const int gi = threadIdx.x + k * kBThreads;
            if (gi < nvb) {
              float f[E];
              VT::unpack(rv[gi], f);
#pragma unroll
              for (int e = 0; e < E; ++e) a32[k][e] = fmaf(f[e], ur, a32[k][e]);
            }
          }
          if (++run == kRunRows) {
            flush();
            run = 0;
          }
        }
      },
      &to);
  flush();
  // columns of the partial last group
  for (int64_t c = (int64_t)nvb * E + threadIdx.x; c < n; c += blockDim.x) {
    double acc = 0.0;
    float sr = 0.f;
    int rr = 0;
    for (int64_t r = r0; r < r1; ++r) {
      sr = fmaf(load_val<T>(A + r * P.ld + c), S.xs[r - r0], sr);
      if (++rr == kRunRows) {
        acc += (double)sr;
        sr = 0.f;
        rr = 0;
      }
    }
    S.zp[c] = acc + (double)sr;
  }
  if (to)
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) S.zp[c] = __longlong_as_double(0x7ff8000000000000ll);
  return true;
  }
}

// A^T u of the CTA's rows by row-streaming warps: the columns go in panels of 32 lanes x G
// 16-byte groups (512 f32 or bf16/f16 columns); warp w streams rows r0 + w, r0 + w + 8, ...
// two at a time (2 G loads of 16 bytes per lane in flight) and accumulates u_r a_r over its
// rows in f32 runs of 32 rows, combined in f64 per warp in the ring area; after each panel
// the eight warps' sums are added in warp order into S.zp.  u (f32) is staged in S.xs.
template <typename T>
__device__ bool warp_matvec_t(const BProb &P, Shm &S, int64_t r0, int64_t r1, const double *u) {
  if constexpr (std::is_same<T, double>::value) {
    return false;
  } else {
    using VT = Vec<T>;
    constexpr int E = VT::E;
    constexpr int G = 16 / E;         // groups per lane and panel: 4 (f32) or 2 (bf16/f16)
    constexpr int PG = 32 * G;        // groups per panel
    constexpr int PC = PG * E;        // columns per panel (512)
    const T *A = (const T *)P.A;
    if (((uintptr_t)A & 15) || ((P.ld * (int64_t)sizeof(T)) & 15) || r1 - r0 > kNMax) return false;
    static_assert(8 * PC * sizeof(double) <= (size_t)kRingStages * kRingStage, "panel sums fit the ring area");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t n = P.n, nv = n / E;
    const int64_t ldv = P.ld / E;
    double *acc = reinterpret_cast<double *>(S.ring) + (size_t)warp * PC;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) S.xs[r - r0] = (float)u[r];
    __syncthreads();
    for (int64_t g0 = 0; g0 < nv; g0 += PG) {
      for (int c = lane; c < PC; c += 32) acc[c] = 0.0;
      float a32[G][E];
#pragma unroll
      for (int q = 0; q < G; ++q)
#pragma unroll
        for (int e = 0; e < E; ++e) a32[q][e] = 0.f;
      int run = 0;
      auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < G; ++q)
#pragma unroll
          for (int e = 0; e < E; ++e) {
            acc[(lane + 32 * q) * E + e] += (double)a32[q][e];
            a32[q][e] = 0.f;
          }
      };
      const typename VT::V *base = reinterpret_cast<const typename VT::V *>(A) + g0 + lane;
      const int64_t pgroups = (nv - g0) < PG ? (nv - g0) : PG;
      for (int64_t r = r0 + warp; r < r1; r += 2 * nw) {
        const bool two = r + nw < r1;
        if (lane == 0) {  // the warp's rows two passes ahead into L2 (this panel's groups)
          const int64_t pr = r + 4 * nw;
          if (pr < r1) l2_prefetch(reinterpret_cast<const typename VT::V *>(A) + pr * ldv + g0, (unsigned)(pgroups * 16));
          if (pr + nw < r1)
            l2_prefetch(reinterpret_cast<const typename VT::V *>(A) + (pr + nw) * ldv + g0, (unsigned)(pgroups * 16));
        }
        typename VT::V b0[G] = {}, b1[G] = {};
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (g0 + lane + 32 * q < nv) {
            b0[q] = __ldcs(base + r * ldv + 32 * q);
            if (two) b1[q] = __ldcs(base + (r + nw) * ldv + 32 * q);
          }
        }
        const float u0 = S.xs[r - r0], u1 = two ? S.xs[r + nw - r0] : 0.f;
#pragma unroll
        for (int q = 0; q < G; ++q) {
          float f0[E], f1[E];
          VT::unpack(b0[q], f0);
          VT::unpack(b1[q], f1);
#pragma unroll
          for (int e = 0; e < E; ++e) a32[q][e] = fmaf(f1[e], u1, fmaf(f0[e], u0, a32[q][e]));
        }
        run += 2;
        if (run >= kRunRows) {
          flush();
          run = 0;
        }
      }
      flush();
      __syncthreads();
      // the warps' panel sums, added in warp order
      for (int c = threadIdx.x; c < PC; c += blockDim.x) {
        const int64_t col = g0 * E + c;
        if (col >= nv * E) break;
        const double *a0 = reinterpret_cast<const double *>(S.ring) + c;
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += a0[(size_t)w * PC];
        S.zp[col] = t;
      }
      __syncthreads();
    }
    // columns of the partial last group
    for (int64_t c = nv * E + threadIdx.x; c < n; c += blockDim.x) {
      double accd = 0.0;
      float sr = 0.f;
      int rr = 0;
      for (int64_t r = r0; r < r1; ++r) {
        sr = fmaf(load_val<T>(A + r * P.ld + c), S.xs[r - r0], sr);
        if (++rr == kRunRows) {
          accd += (double)sr;
          sr = 0.f;
          rr = 0;
        }
      }
      S.zp[c] = accd + (double)sr;
    }
    __syncthreads();
    return true;
  }
}

template <typename T>
__device__ void rows_matvec_t(const BProb &P, Shm &S, int64_t r0, int64_t r1, const double *u) {
  if (warp_matvec_t<T>(P, S, r0, r1, u)) return;
  if (ring_matvec_t<T>(P, S, r0, r1, u)) return;
  const T *A = (const T *)P.A;
  const int64_t n = P.n;
  if constexpr (std::is_same<T, double>::value) {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      double acc = 0.0;
      for (int64_t r = r0; r < r1; ++r) acc = fma(A[r * P.ld + c], u[r], acc);
      S.zp[c] = acc;
    }
  } else {
    using VT = Vec<T>;
    constexpr int E = VT::E;
    const bool vec = ((uintptr_t)A % 16) == 0 && ((P.ld * (int64_t)sizeof(T)) % 16) == 0;
    const int64_t nv = vec ? n / E : 0;  // whole 16-byte groups
    const int64_t ldv = P.ld / E;
    for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
      const typename VT::V *col = reinterpret_cast<const typename VT::V *>(A) + g;
      float a32[E];
      double a64[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        a32[e] = 0.f;
        a64[e] = 0.0;
      }
      int run = 0;
      int64_t r = r0;
      for (; r + 8 <= r1; r += 8) {
        typename VT::V buf[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) buf[q] = __ldcs(col + (r + q) * ldv);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float f[E];
          VT::unpack(buf[q], f);
          const float ur = (float)u[r + q];
#pragma unroll
          for (int e = 0; e < E; ++e) a32[e] = fmaf(f[e], ur, a32[e]);
        }
        run += 8;
        if (run >= kRunRows) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            a64[e] += (double)a32[e];
            a32[e] = 0.f;
          }
          run = 0;
        }
      }
      for (; r < r1; ++r) {
        float f[E];
        VT::unpack(__ldcs(col + r * ldv), f);
        const float ur = (float)u[r];
#pragma unroll
        for (int e = 0; e < E; ++e) a32[e] = fmaf(f[e], ur, a32[e]);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) S.zp[g * E + e] = a64[e] + (double)a32[e];
    }
    for (int64_t c = nv * E + threadIdx.x; c < n; c += blockDim.x) {
      double acc = 0.0;
      float s = 0.f;
      int run = 0;
      for (int64_t r = r0; r < r1; ++r) {
        s = fmaf(load_val<T>(A + r * P.ld + c), (float)u[r], s);
        if (++run == kRunRows) {
          acc += (double)s;
          s = 0.f;
          run = 0;
        }
      }
      S.zp[c] = acc + (double)s;
    }
  }
}

// z[i] = scale * sum over CTAs of zp[i] - coef * sub[i] for i in [v0, v1)
__device__ void reduce_matvec_t(cg::cluster_group &cl, const BProb &P, Shm &S, int64_t v0, int64_t v1, double *z,
                                const double *sub, double coef) {
  cl.sync();
  const unsigned cs = cl.num_blocks();
  for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
    double t = 0.0;
    for (unsigned c = 0; c < cs; ++c) t += cl.map_shared_rank(S.zp, c)[i];
    z[i] = t * P.scale - (sub ? coef * sub[i] : 0.0);
  }
  cl.sync();
}

// classical Gram-Schmidt of the slice [s0, s1) of vec against j columns of Qb,
// `passes` times, then the norm (the same value in every CTA)
// sum over the cluster of the squares of vec[s0, s1) (the same value in every CTA)
__device__ double cl_norm2(cg::cluster_group &cl, Shm &S, const double *vec, int64_t s0, int64_t s1, int slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double s = 0.0;
  for (int64_t r = s0 + threadIdx.x; r < s1; r += blockDim.x) s = fma(vec[r], vec[r], s);
  s = dev::warp_sum_d(s);
  __shared__ double wred[32];
  if (lane == 0) wred[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += wred[i];
    S.red[slot] = t;
  }
  __syncthreads();
  return 0.0;
}

// classical Gram-Schmidt of the slice [s0, s1) of vec against j columns of Qb, then the
// norm (the same value in every CTA).  passes >= 1: that many passes; passes = 0: one pass,
// a second only if the first left less than 1/sqrt(2) of the norm (Daniel-Gragg-Kaufman-
// Stewart); the norm before the first pass rides in the first pass's all-reduce.
__device__ double cl_cgs_norm(cg::cluster_group &cl, Shm &S, double *vec, int64_t s0, int64_t s1, const double *Qb,
                              int64_t ldq, int j, int passes) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool adaptive = passes == 0;
  const int maxp = adaptive ? 2 : passes;
  double n0 = 0.0;
  for (int p = 0; p < maxp && j > 0; ++p) {
    for (int c = warp; c < j; c += nw) {
      const double *q = Qb + (int64_t)c * ldq;
      double s0a = 0.0, s1a = 0.0, s2a = 0.0, s3a = 0.0;
      int64_t r = s0 + lane;
      for (; r + 96 < s1; r += 128) {
        s0a = fma(q[r], vec[r], s0a);
        s1a = fma(q[r + 32], vec[r + 32], s1a);
        s2a = fma(q[r + 64], vec[r + 64], s2a);
        s3a = fma(q[r + 96], vec[r + 96], s3a);
      }
      for (; r < s1; r += 32) s0a = fma(q[r], vec[r], s0a);
      double s = dev::warp_sum_d((s0a + s1a) + (s2a + s3a));
      if (lane == 0) S.red[c] = s;
    }
    const bool first_adaptive = adaptive && p == 0;
    if (first_adaptive) cl_norm2(cl, S, vec, s0, s1, j);
    cl_allreduce(cl, S, j + (first_adaptive ? 1 : 0));
    if (first_adaptive) n0 = S.hv[j];
    for (int64_t r = s0 + threadIdx.x; r < s1; r += blockDim.x) {
      double acc = vec[r];
      for (int c = 0; c < j; ++c) acc = fma(-Qb[(int64_t)c * ldq + r], S.hv[c], acc);
      vec[r] = acc;
    }
    __syncthreads();
    if (first_adaptive) {
      cl_norm2(cl, S, vec, s0, s1, 0);
      cl_allreduce(cl, S, 1);
      const double n1 = S.hv[0];
      if (n1 >= 0.5 * n0) return sqrt(n1);  // no cancellation: one pass is enough
    }
  }
  cl_norm2(cl, S, vec, s0, s1, 0);
  cl_allreduce(cl, S, 1);
  return sqrt(S.hv[0]);
}

__device__ void scale_slice(double *dst, const double *src, int64_t s0, int64_t s1, double f) {
  for (int64_t r = s0 + threadIdx.x; r < s1; r += blockDim.x) dst[r] = src[r] * f;
  __syncthreads();
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

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

// q1 entries ~ N(2,1) (same stream as the single-problem start vector)
__device__ double start_entry(uint64_t seed, int64_t i) {
  const uint64_t b = (uint64_t)i >> 1;
  const uint4 x = philox(make_uint4((unsigned)b, (unsigned)(b >> 32), 0u, 0u),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const double ua = ((double)(((uint64_t)(x.x >> 5) << 26) | (x.y >> 6)) + 0.5) * 0x1.0p-53;
  const double ub = ((double)(((uint64_t)(x.z >> 5) << 26) | (x.w >> 6)) + 0.5) * 0x1.0p-53;
  const double rr = sqrt(-2.0 * log(ua));
  const double two_pi = 6.283185307179586476925286766559;
  return 2.0 + ((i & 1) ? rr * sin(two_pi * ub) : rr * cos(two_pi * ub));
}

// replacement direction (SplitMix64) orthogonalized twice against j columns;
// writes the normalized vector (or zero) into column dst; returns 1 if kept
__device__ int cl_fresh(cg::cluster_group &cl, Shm &S, double *vec, int64_t s0, int64_t s1, const double *Qb,
                        int64_t ldq, int j, double *dst, uint64_t seed, int64_t dnum) {
  const uint64_t base = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(dnum + 1));
  for (int64_t r = s0 + threadIdx.x; r < s1; r += blockDim.x)
    vec[r] = (double)(splitmix64(base + (uint64_t)r) >> 11) * 0x1.0p-52 - 1.0;
  __syncthreads();
  const double n0 = cl_cgs_norm(cl, S, vec, s0, s1, Qb, ldq, 0, 0);
  const double n1 = cl_cgs_norm(cl, S, vec, s0, s1, Qb, ldq, j, 2);
  const bool keep = n1 > 1e-8 * n0;
  scale_slice(dst, vec, s0, s1, keep ? 1.0 / n1 : 0.0);
  return keep ? 1 : 0;
}

template <typename T>
__device__ void stage_x(const BProb &P, Shm &S, const double *v) {
  if constexpr (!std::is_same<T, double>::value) {
    for (int64_t i = threadIdx.x; i < P.n; i += blockDim.x) S.xs[i] = (float)v[i];
  }
  __syncthreads();
}

template <typename T>
__device__ void left_product(const BProb &P, Shm &S, int64_t r0, int64_t r1, const double *v, double *w,
                             const double *Qb, int64_t ldq, int c0, int cn, const double *coefs) {
  if constexpr (std::is_same<T, double>::value)
    rows_matvec_f64(P, r0, r1, v, w, Qb, ldq, c0, cn, coefs);
  else {
    // the register-streaming kernel measured faster than the row ring for A v on the batched
    // workload (two rows per warp, eight 16-byte loads per lane in flight); the ring serves A^T u
    stage_x<T>(P, S, v);
    rows_matvec<T>(P, S, r0, r1, w, Qb, ldq, c0, cn, coefs);
  }
  __syncthreads();
}

// One-sided Jacobi SVD of the K x K matrix held column-major in shared memory (sB), on
// the calling CTA alone: the rotations, the tournament ordering and the tolerance of the
// cluster version.  Each round: the pairs' sums by 8-lane groups, the rotations by one
// lane per pair (so each pair's f64 divisions and square roots run once, not on eight
// lanes), then the updates by 8-lane groups; block barriers between the phases.  rot:
// 4 doubles per pair in shared memory.  The skip test compares squares: c^2 <= tol^2 a b.  sY receives the accumulated
// rotations; outputs sigma (descending), X (normalized columns of the rotated B) and Y
// (rotations) in global memory, ordered by sigma.  Returns the sweeps (negative if the
// sweep limit was reached).
constexpr int kCtaJacobiMax = 78;  // K with 8 K^2 bytes within each of the two shared regions

// One-sided Jacobi sweeps (tournament ordering) on the K x K column-major sB with the
// rotations accumulated into sY.  A pair rotates unless c^2 <= tol^2 a b, or unless one of its
// columns has a squared norm at most `floor` (left to a later, more precise stage).
template <typename R>
__device__ int cta_sweeps(R *sB, R *sY, int K, R tol, R floor, int max_sweeps, R *rot, int *s_rot) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int grp = lane >> 3, gl = lane & 7;
  const int Kp = K + (K & 1);
  int sweep;
  for (sweep = 1; sweep <= max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    for (int r = 0; r < Kp - 1; ++r) {
      // (1) one pair per 8-lane group: its three sums a = |b_p|^2, b = |b_q|^2, c = b_p . b_q
      for (int pb = warp * 4; pb < Kp / 2; pb += nw * 4) {
        const int pi = pb + grp;
        int p = 0, q = K;
        if (pi < Kp / 2) {
          p = dev::player(r, pi, Kp);
          q = dev::player(r, Kp - 1 - pi, Kp);
          if (p > q) {
            const int t = p;
            p = q;
            q = t;
          }
        }
        const bool live = q < K;
        const R *bp = sB + p * K, *bq = sB + (live ? q : p) * K;
        R a = 0, b = 0, c = 0;
        if (live)
          for (int i = gl; i < K; i += 8) {
            const R x = bp[i], y = bq[i];
            a = fma(x, x, a);
            b = fma(y, y, b);
            c = fma(x, y, c);
          }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (gl == 0 && pi < Kp / 2) {
          rot[4 * pi] = a;
          rot[4 * pi + 1] = b;
          rot[4 * pi + 2] = live ? c : R(0);
        }
      }
      __syncthreads();
      // (2) the rotations, one lane per pair (the divisions and roots once per pair)
      if (warp == 0)
        for (int pi = lane; pi < Kp / 2; pi += 32) {
          const R a = rot[4 * pi], b = rot[4 * pi + 1], c = rot[4 * pi + 2];
          R cs = 1, sn = 0;
          if (!(c == R(0) || c * c <= tol * tol * a * b || a <= floor || b <= floor)) {
            *s_rot = 1;
            const R zeta = (b - a) / (R(2) * c);
            const R t = fabs(zeta) > R(1e30) ? R(0.5) / zeta
                                              : (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
            cs = R(1) / sqrt(R(1) + t * t);
            sn = cs * t;
          }
          rot[4 * pi] = cs;
          rot[4 * pi + 1] = sn;
          rot[4 * pi + 3] = (cs == R(1) && sn == R(0)) ? R(0) : R(1);
        }
      __syncthreads();
      // (3) apply them, one pair per 8-lane group
      for (int pb = warp * 4; pb < Kp / 2; pb += nw * 4) {
        const int pi = pb + grp;
        if (pi >= Kp / 2 || rot[4 * pi + 3] == R(0)) continue;
        int p = dev::player(r, pi, Kp), q = dev::player(r, Kp - 1 - pi, Kp);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const R cs = rot[4 * pi], sn = rot[4 * pi + 1];
        R *bp = sB + p * K, *bq = sB + q * K;
        for (int i = gl; i < K; i += 8) {
          const R x = bp[i], y = bq[i];
          bp[i] = cs * x - sn * y;
          bq[i] = sn * x + cs * y;
        }
        R *yp = sY + p * K, *yq = sY + q * K;
        for (int i = gl; i < K; i += 8) {
          const R x = yp[i], y = yq[i];
          yp[i] = cs * x - sn * y;
          yq[i] = sn * x + cs * y;
        }
      }
      __syncthreads();
    }
    const int any = *s_rot;
    __syncthreads();  // every thread has read the flag before it is cleared
    if (!any) return sweep;
  }
  return -(sweep - 1);
}

// the projected matrix's entry (i, c): kept Ritz values sigma_i and the coupling rho_i in
// column l for the first l rows, alpha_i on and beta_i above the diagonal below them
struct ProjB {
  const double *sigma, *rho, *alpha, *beta;
  int l, K;
  __device__ __forceinline__ double entry(int i, int c) const {
    if (i < l) return c == i ? __ldcg(sigma + i) : (c == l ? __ldcg(rho + i) : 0.0);
    return c == i ? __ldcg(alpha + i) : (c == i + 1 ? __ldcg(beta + i) : 0.0);
  }
  // (B Q)(i, c) for column-major Q: B has at most two entries per row
  __device__ __forceinline__ double times(const double *Q, int i, int c) const {
    const double *q = Q + (int64_t)c * K;
    if (i < l) return __ldcg(sigma + i) * q[i] + __ldcg(rho + i) * q[l];
    double v = __ldcg(alpha + i) * q[i];
    if (i + 1 < K) v += __ldcg(beta + i) * q[i + 1];
    return v;
  }
};

// SVD of the projected K x K matrix on the calling CTA alone, in shared memory (K <= 78):
// (1) one-sided Jacobi sweeps in f32 on B / max|B| until its columns are orthogonal to
// about 1e-5 (f32 work, 64x the FP64 rate); (2) the accumulated f32 rotations, made
// orthonormal in f64 by two Gram-Schmidt passes per column, give Q; (3) f64 one-sided
// Jacobi on B Q (formed directly from B's two entries per row) with Q as the starting
// rotation, to the tolerance of the cluster version; a few sweeps remain.  B V = U S with
// V = Q J exactly orthogonal in f64, so the outputs are those of a plain f64 Jacobi SVD:
// sigma descending, X the normalized columns of the rotated matrix, Y the rotations.
__device__ int cta_svd(double *sB, double *sY, const ProjB &Bp, double *sigma, double *X, double *Y, double *nrm,
                       int *pos, int *s_rot, double *rot) {
  const int K = Bp.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float *Bf = reinterpret_cast<float *>(sB), *Yf = Bf + K * K;
  // (1) f32 sweeps on the scaled matrix
  __shared__ double s_max;
  if (threadIdx.x == 0) s_max = 0.0;
  __syncthreads();
  double mloc = 0.0;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) mloc = fmax(mloc, fabs(Bp.entry(idx % K, idx / K)));
  mloc = dev::warp_max_d(mloc);
  if (lane == 0) atomicMax(reinterpret_cast<unsigned long long *>(&s_max), (unsigned long long)__double_as_longlong(mloc));
  __syncthreads();
  const double inv = s_max > 0.0 ? 1.0 / s_max : 1.0;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    Bf[idx] = (float)(Bp.entry(idx % K, idx / K) * inv);
    Yf[idx] = ((idx % K) == (idx / K)) ? 1.f : 0.f;
  }
  __syncthreads();
  // columns below 1e-10 of the Frobenius norm squared carry f32 rounding more than their
  // own direction: their rotations wait for the f64 stage
  double fro = 0.0;
  if (warp == 0) {
    for (int idx = lane; idx < K * K; idx += 32) fro = fma((double)Bf[idx], (double)Bf[idx], fro);
    fro = dev::warp_sum_d(fro);
    if (lane == 0) rot[0] = fro;
  }
  __syncthreads();
  const float floor32 = (float)(1e-10 * rot[0]);
  __syncthreads();
  const int sw32 = cta_sweeps<float>(Bf, Yf, K, 1e-5f, floor32, 40, reinterpret_cast<float *>(rot), s_rot);
  // (2) Q = Yf made orthonormal in f64, column by column (two passes each)
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) sY[idx] = (double)Yf[idx];
  __syncthreads();
  for (int c = 0; c < K; ++c) {
    double *qc = sY + (int64_t)c * K;
    for (int pass = 0; pass < 2 && c > 0; ++pass) {
      for (int k = warp; k < c; k += nw) {
        const double *qk = sY + (int64_t)k * K;
        double d = 0.0;
        for (int i = lane; i < K; i += 32) d = fma(qk[i], qc[i], d);
        d = dev::warp_sum_d(d);
        if (lane == 0) rot[k] = d;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < K; i += blockDim.x) {
        double v = qc[i];
        for (int k = 0; k < c; ++k) v = fma(-sY[(int64_t)k * K + i], rot[k], v);
        qc[i] = v;
      }
      __syncthreads();
    }
    if (warp == 0) {
      double d = 0.0;
      for (int i = lane; i < K; i += 32) d = fma(qc[i], qc[i], d);
      d = dev::warp_sum_d(d);
      if (lane == 0) rot[0] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
    __syncthreads();
    const double f = rot[0];
    for (int i = threadIdx.x; i < K; i += blockDim.x) qc[i] *= f;
    __syncthreads();
  }
  // (3) B Q in f64 (sB's f32 contents are no longer needed), then f64 sweeps
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) sB[idx] = Bp.times(sY, idx % K, idx / K);
  __syncthreads();
  const double tol = fmax(2.0 * sqrt((double)K) * 0x1.0p-52, (double)K * 0x1.0p-53);
  const int sw64 = cta_sweeps<double>(sB, sY, K, tol, 0.0, 80, rot, s_rot);
  // singular values = column norms, ordered descending (stable by index)
  for (int c = warp; c < K; c += nw) {
    const double *bc = sB + c * K;
    double sq = 0.0;
    for (int i = lane; i < K; i += 32) sq = fma(bc[i], bc[i], sq);
    sq = dev::warp_sum_d(sq);
    if (lane == 0) nrm[c] = sqrt(sq);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const double nc = nrm[c];
    int rk = 0;
    for (int o = 0; o < K; ++o) {
      const double no = nrm[o];
      rk += (no > nc) || (no == nc && o < c);
    }
    pos[c] = rk;
  }
  __syncthreads();
  for (int c = warp; c < K; c += nw) {
    const int pc = pos[c];
    const double nc = nrm[c];
    for (int i = lane; i < K; i += 32) {
      X[(int64_t)pc * K + i] = nc > 0.0 ? sB[c * K + i] / nc : 0.0;
      Y[(int64_t)pc * K + i] = sY[c * K + i];
    }
    if (lane == 0) sigma[pc] = nc;
  }
  __syncthreads();
  (void)sw32;
  return sw64;
}

// ---------------------------------------------------------------------------
// restarted partial SVD of one problem on the calling cluster
// ---------------------------------------------------------------------------
template <typename T>
__device__ void solve_psvd(cg::cluster_group &cl, const BProb &P, BWork W, const BDims &D, Shm &S, BRes &res) {
  const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
  const int64_t m = P.m, n = P.n, ldu = D.ldu, ldv = D.ldv;
  const int K = P.K, k = P.k, keep = P.keep;
  int64_t r0, r1, v0, v1;
  slice(m, rank, cs, &r0, &r1);
  slice(n, rank, cs, &v0, &v1);
  double sest = 0.0;
  int64_t nfresh = 0;
  PhaseClock pc(P.prof != 0 && rank == 0 && threadIdx.x == 0 ? S.cyc : nullptr);
  // start vector, normalized, in w
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) W.w[r] = P.start ? P.start[r] : start_entry(P.seed, r);
  __syncthreads();
  {
    const double q = cl_cgs_norm(cl, S, W.w, r0, r1, W.Ub, ldu, 0, 0);
    scale_slice(W.w, W.w, r0, r1, q > 0.0 ? 1.0 / q : 0.0);
  }
  // v1 = A^T q1 / ||A^T q1||
  rows_matvec_t<T>(P, S, r0, r1, W.w);
  reduce_matvec_t(cl, P, S, v0, v1, W.z, nullptr, 0.0);
  {
    const double nv = cl_cgs_norm(cl, S, W.z, v0, v1, W.Vb, ldv, 0, 0);
    if (nv > 0.0)
      scale_slice(W.Vb, W.z, v0, v1, 1.0 / nv);
    else {
      cl_fresh(cl, S, W.z, v0, v1, W.Vb, ldv, 0, W.Vb, P.seed, nfresh++);
      res.breakdowns++;
    }
  }
  res.matvecs = 1;
  int l = 0;
  pc.mark(4);
  for (int cycle = 0;; ++cycle) {
    double bprev = 0.0;
    for (int j = l; j < K; ++j) {
      cl.sync();  // v_j complete in every slice
      pc.mark(2);
      // left: w = A v_j - (beta_{j-1} u_{j-1} | sum_i rho_i u_i)
      if (j == l && l > 0)
        left_product<T>(P, S, r0, r1, W.Vb + (int64_t)j * ldv, W.w, W.Ub, ldu, 0, l, W.rho);
      else if (j > 0)
        left_product<T>(P, S, r0, r1, W.Vb + (int64_t)j * ldv, W.w, W.Ub, ldu, j - 1, 1, &bprev);
      else
        left_product<T>(P, S, r0, r1, W.Vb + (int64_t)j * ldv, W.w, W.Ub, ldu, 0, 0, nullptr);
      pc.mark(0);
      double a = cl_cgs_norm(cl, S, W.w, r0, r1, W.Ub, ldu, j, P.passes);
      sest = fmax(sest, a);
      if (!(a > 0x1.0p-46 * sest)) {
        if (!isfinite(a)) {
          res.status = GK_NUMERICAL;
          return;
        }
        a = 0.0;
        cl_fresh(cl, S, W.w, r0, r1, W.Ub, ldu, j, W.Ub + (int64_t)j * ldu, P.seed, nfresh++);
        res.breakdowns++;
      } else {
        scale_slice(W.Ub + (int64_t)j * ldu, W.w, r0, r1, 1.0 / a);
      }
      if (rank == 0 && threadIdx.x == 0) W.alpha[j] = a;
      pc.mark(2);
      // right: z = A^T u_j - alpha_j v_j
      rows_matvec_t<T>(P, S, r0, r1, W.Ub + (int64_t)j * ldu);
      reduce_matvec_t(cl, P, S, v0, v1, W.z, W.Vb + (int64_t)j * ldv, a);
      pc.mark(1);
      double b = cl_cgs_norm(cl, S, W.z, v0, v1, W.Vb, ldv, j + 1, P.passes);
      sest = fmax(sest, b);
      if (!(b > 0x1.0p-46 * sest)) {
        if (!isfinite(b)) {
          res.status = GK_NUMERICAL;
          return;
        }
        b = 0.0;
        cl_fresh(cl, S, W.z, v0, v1, W.Vb, ldv, j + 1, W.Vb + (int64_t)(j + 1) * ldv, P.seed, nfresh++);
        res.breakdowns++;
      } else {
        scale_slice(W.Vb + (int64_t)(j + 1) * ldv, W.z, v0, v1, 1.0 / b);
      }
      if (rank == 0 && threadIdx.x == 0) W.beta[j] = b;
      bprev = b;
      res.matvecs += 2;
      res.steps++;
    }
    // B of this cycle, its SVD, the Ritz residual test
    cl.sync();
    const bool small_on_cta = K <= kCtaJacobiMax;
    double *sB = reinterpret_cast<double *>(S.xs), *sYw = reinterpret_cast<double *>(S.ring);
    if (!small_on_cta) {
      for (int64_t idx = (int64_t)rank * blockDim.x + threadIdx.x; idx < (int64_t)K * K;
           idx += (int64_t)cs * blockDim.x) {
        const int r = (int)(idx % K), c = (int)(idx / K);
        double v = 0.0;
        if (r < l) {
          if (c == r) v = W.sigma[r];
          else if (c == l) v = W.rho[r];
        } else {
          if (c == r) v = W.alpha[r];
          else if (c == r + 1) v = W.beta[r];
        }
        W.Bm[idx] = v;
      }
    }
    if (small_on_cta) {
      // the leading CTA alone, in its shared memory (the vector and ring areas are idle now)
      int sw = 0;
      if (rank == 0) {
        const ProjB Bp{W.sigma, W.rho, W.alpha, W.beta, l, K};
        sw = cta_svd(sB, sYw, Bp, W.sigma, W.X, W.Y, S.red, S.redi, S.s_rot, S.hv);
      }
      cl.sync();  // sigma, X, Y visible to every CTA
      res.sweeps = sw;
    } else {
      res.sweeps = dev::cluster_jacobi(cl, W.Bm, W.Yw, K, W.sigma, W.X, W.Y, W.nrm, W.pos, S.s_rot, S.s_any);
    }
    const double bK = __ldcg(W.beta + (K - 1));
    const double s1 = __ldcg(W.sigma);
    double mx = 0.0;
    int above = 0;
    for (int i = 0; i < k; ++i) {
      const double ri = fabs(bK * __ldcg(W.X + (int64_t)i * K + (K - 1))), th = __ldcg(W.sigma + i);
      // below the rank cut (with its residual bound) the triplet is not part of the answer
      if (P.cut > 0.0 && th + ri <= P.cut * s1) continue;
      mx = fmax(mx, ri);
    }
    for (int i = 0; i < k; ++i) above += !(P.cut > 0.0) || __ldcg(W.sigma + i) > P.cut * s1;
    res.rank = above;
    res.cycles = cycle + 1;
    pc.mark(3);
    res.resid_est = s1 > 0.0 ? mx / s1 : 0.0;
    sest = fmax(sest, s1);
    const bool conv = mx <= P.tol * s1;
    if (conv || cycle >= P.max_restarts) {
      res.status = conv ? GK_OK : GK_NOT_CONVERGED;
      res.sigma_next = k < K ? __ldcg(W.sigma + k) : 0.0;
      break;
    }
    // thick restart: U' = U_K X_keep, V' = [V_K Y_keep, v_{K+1}], rho = beta_K X_{K,:}
    if (rank == 0)
      for (int i = threadIdx.x; i < K; i += blockDim.x) W.rho[i] = bK * __ldcg(W.X + (int64_t)i * K + (K - 1));
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
      for (int i = 0; i < keep; ++i) {
        double s = 0.0;
        for (int c = 0; c < K; ++c) s = fma(W.Ub[(int64_t)c * ldu + r], __ldcg(W.X + (int64_t)i * K + c), s);
        W.Ub2[(int64_t)i * ldu + r] = s;
      }
    for (int64_t r = v0 + threadIdx.x; r < v1; r += blockDim.x) {
      for (int i = 0; i < keep; ++i) {
        double s = 0.0;
        for (int c = 0; c < K; ++c) s = fma(W.Vb[(int64_t)c * ldv + r], __ldcg(W.Y + (int64_t)i * K + c), s);
        W.Vb2[(int64_t)i * ldv + r] = s;
      }
      W.Vb2[(int64_t)keep * ldv + r] = W.Vb[(int64_t)K * ldv + r];
    }
    double *t = W.Ub;
    W.Ub = W.Ub2;
    W.Ub2 = t;
    t = W.Vb;
    W.Vb = W.Vb2;
    W.Vb2 = t;
    l = keep;
    res.restarts++;
    cl.sync();
    pc.mark(4);
  }
  res.sigma_est = sest;
  // outputs: U = U_K X_k, V = V_K Y_k, S = sigma_k; sign of the largest |v_i| entry positive
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      for (int c = 0; c < K; ++c) s = fma(W.Ub[(int64_t)c * ldu + r], __ldcg(W.X + (int64_t)i * K + c), s);
      P.U[(int64_t)i * m + r] = s;
    }
  for (int64_t r = v0 + threadIdx.x; r < v1; r += blockDim.x)
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      for (int c = 0; c < K; ++c) s = fma(W.Vb[(int64_t)c * ldv + r], __ldcg(W.Y + (int64_t)i * K + c), s);
      P.V[(int64_t)i * n + r] = s;
    }
  if (rank == 0)
    for (int i = threadIdx.x; i < k; i += blockDim.x) P.S[i] = __ldcg(W.sigma + i);
  __syncthreads();
  // this CTA's largest |v_i| entry (first index on ties) for every column i
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < k; i += nw) {
    double best = -1.0;
    int64_t bi = v0;
    for (int64_t r = v0 + lane; r < v1; r += 32) {
      const double a = fabs(P.V[(int64_t)i * n + r]);
      if (a > best) {
        best = a;
        bi = r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double b2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (b2 > best || (b2 == best && i2 < bi)) {
        best = b2;
        bi = i2;
      }
    }
    if (lane == 0) {
      S.red[i] = best;
      S.redi[i] = (int)bi;
    }
  }
  cl.sync();
  // the cluster's choice: ranks hold consecutive slices, so the first maximum in rank order wins
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double best = -1.0;
    int bi = 0;
    for (unsigned c = 0; c < cs; ++c) {
      const double b2 = cl.map_shared_rank(S.red, c)[i];
      const int i2 = cl.map_shared_rank(S.redi, c)[i];
      if (b2 > best) {
        best = b2;
        bi = i2;
      }
    }
    S.hv[i] = (__ldcg(P.V + (int64_t)i * n + bi) < 0.0) ? -1.0 : 1.0;
  }
  cl.sync();
  for (int i = 0; i < k; ++i) {
    if (S.hv[i] > 0.0) continue;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) P.U[(int64_t)i * m + r] = -P.U[(int64_t)i * m + r];
    for (int64_t r = v0 + threadIdx.x; r < v1; r += blockDim.x) P.V[(int64_t)i * n + r] = -P.V[(int64_t)i * n + r];
  }
  cl.sync();
  pc.mark(4);
}

// ---------------------------------------------------------------------------
// Algorithm 3 (on Algorithm 1) of one problem on the calling cluster
// ---------------------------------------------------------------------------
template <typename T>
__device__ void solve_numrank(cg::cluster_group &cl, const BProb &P, BWork W, const BDims &D, Shm &S, BRes &res) {
  const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
  const int64_t m = P.m, ldu = D.ldu, ldv = D.ldv;
  const int kmax = P.K;
  int64_t r0, r1, v0, v1;
  slice(m, rank, cs, &r0, &r1);
  slice(P.n, rank, cs, &v0, &v1);
  const double eps = P.tol;
  PhaseClock pc(P.prof != 0 && rank == 0 && threadIdx.x == 0 ? S.cyc : nullptr);
  for (int i = rank * blockDim.x + threadIdx.x; i < kmax + 2; i += cs * blockDim.x) {
    W.alpha[i] = 0.0;
    W.beta[i] = 0.0;
  }
  // q1, normalized, is Q[:, 0]
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) W.w[r] = P.start ? P.start[r] : start_entry(P.seed, r);
  __syncthreads();
  {
    const double q = cl_cgs_norm(cl, S, W.w, r0, r1, W.Ub, ldu, 0, 0);
    scale_slice(W.Ub, W.w, r0, r1, q > 0.0 ? 1.0 / q : 0.0);
  }
  // p1 = A^T q1, alpha_1 = ||p1||
  rows_matvec_t<T>(P, S, r0, r1, W.Ub);
  reduce_matvec_t(cl, P, S, v0, v1, W.z, nullptr, 0.0);
  double a = cl_cgs_norm(cl, S, W.z, v0, v1, W.Vb, ldv, 0, 0);
  double sest = a;
  res.matvecs = 1;
  int kp = 0, reason = 0;
  if (rank == 0 && threadIdx.x == 0) W.alpha[0] = a;
  if (!isfinite(a)) {
    res.status = GK_NUMERICAL;
    return;
  }
  if (a <= (P.eps_rel ? eps * sest : eps)) {
    reason = 2;
  } else {
    scale_slice(W.Vb, W.z, v0, v1, 1.0 / a);
    int j;
    for (j = 1; j <= kmax; ++j) {
      cl.sync();  // p_j complete
      pc.mark(2);
      const double aj = a;
      left_product<T>(P, S, r0, r1, W.Vb + (int64_t)(j - 1) * ldv, W.w, W.Ub, ldu, j - 1, 1, &aj);
      pc.mark(0);
      const double b = cl_cgs_norm(cl, S, W.w, r0, r1, W.Ub, ldu, j, P.passes);
      res.matvecs++;
      if (rank == 0 && threadIdx.x == 0) W.beta[j] = b;
      if (!isfinite(b)) {
        res.status = GK_NUMERICAL;
        return;
      }
      sest = fmax(sest, hypot(aj, b));
      if (b <= (P.eps_rel ? eps * sest : eps)) {
        kp = j;
        reason = 1;
        break;
      }
      scale_slice(W.Ub + (int64_t)j * ldu, W.w, r0, r1, 1.0 / b);
      pc.mark(2);
      rows_matvec_t<T>(P, S, r0, r1, W.Ub + (int64_t)j * ldu);
      reduce_matvec_t(cl, P, S, v0, v1, W.z, W.Vb + (int64_t)(j - 1) * ldv, b);
      pc.mark(1);
      a = cl_cgs_norm(cl, S, W.z, v0, v1, W.Vb, ldv, j, P.passes);
      res.matvecs++;
      if (rank == 0 && threadIdx.x == 0) W.alpha[j] = a;
      if (!isfinite(a)) {
        res.status = GK_NUMERICAL;
        return;
      }
      sest = fmax(sest, hypot(b, a));
      if (a <= (P.eps_rel ? eps * sest : eps)) {
        kp = j;
        reason = 2;
        break;
      }
      scale_slice(W.Vb + (int64_t)j * ldv, W.z, v0, v1, 1.0 / a);
    }
    if (j > kmax) kp = kmax;
  }
  res.steps = kp;
  res.sigma_est = sest;
  cl.sync();
  // Algorithm 3's count on one CTA: the singular values of B_{k'+1,k'} above the threshold
  if (rank == 0) {
    __shared__ int s_rank;
    __shared__ double s_s1;
    dev::block_bidiag_rank(W.alpha, W.beta, kp, eps, P.eps_rel, &s_rank, &s_s1, P.S, S.zp);
    __syncthreads();
    res.rank = s_rank;
  }
  res.status = GK_OK;
  res.pad = reason;
  cl.sync();
  pc.mark(3);
}

template <typename T>
__global__ void __launch_bounds__(kBThreads, 2) k_batched(const BProb *__restrict__ probs, const int *__restrict__ order,
                                                       int count, int *next, char *ws, size_t ws_stride, BDims D,
                                                       BRes *results) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_rot, s_any, s_idx, s_dead;
  __shared__ long long s_cyc[5];
  __shared__ __align__(8) uint64_t s_bar[kRingStages];
  Shm S;
  S.xs = reinterpret_cast<float *>(smem);
  S.zp = reinterpret_cast<double *>(smem + sizeof(float) * kNMax);
  S.red = S.zp + kNMax;
  S.hv = S.red + kKMax + 8;
  S.redi = reinterpret_cast<int *>(S.hv + kKMax + 8);
  S.s_rot = &s_rot;
  S.s_any = &s_any;
  S.s_idx = &s_idx;
  S.cyc = s_cyc;
  S.ring = smem + kRingOffset;
  S.bar = s_bar;
  S.dead = &s_dead;
  S.err = next + 1;
  S.seq = 0;
  if (threadIdx.x == 0) {
    s_dead = 0;
    for (int i = 0; i < kRingStages; ++i) mbar_init(&s_bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const unsigned cid = blockIdx.x / cl.num_blocks();
  char *mine = ws + (size_t)cid * ws_stride;
  for (;;) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) s_idx = atomicAdd(next, 1);
    cl.sync();
    const int idx = *cl.map_shared_rank(&s_idx, 0);
    cl.sync();  // every CTA has read the index before the leader takes the next one
    if (idx >= count) break;
    const BProb P = probs[order[idx]];
    BWork W = carve(mine, D);
    BRes res;
    memset(&res, 0, sizeof(res));
    res.status = GK_OK;
    if (threadIdx.x < 5) s_cyc[threadIdx.x] = 0;
    __syncthreads();
    if (P.mode == 0)
      solve_psvd<T>(cl, P, W, D, S, res);
    else
      solve_numrank<T>(cl, P, W, D, S, res);
    cl.sync();
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      for (int i = 0; i < 5; ++i) res.cyc[i] = s_cyc[i];
      results[P.out] = res;
    }
  }
}

}  // namespace

// k_batched<T> for one storage type, compiled in a translation unit of its own
// (gk_batched_f64.cu, _f32, _bf16, _f16) so that the four instantiations build in parallel;
// the host driver launches them through these pointers
const void *batched_kernel_f64();
const void *batched_kernel_f32();
const void *batched_kernel_bf16();
const void *batched_kernel_f16();

}  // namespace gk
