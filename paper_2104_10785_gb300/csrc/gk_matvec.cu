// gk_matvec.cu -- the products A x and A^T x of the bidiagonalization sweep
// (Eq. 2.2: A p_i and A^T q_{i+1}; Algorithm 1).
//
// These passes stream the whole operator once per half-step and are bounded by
// HBM bandwidth.  Dense operators are row-major:
//  * A x   : one warp per row, 16-byte streaming loads (ld.global.cs) of A, the
//            f32 copy of x read through the L1 (it is reused by every row);
//            f32 products summed over short runs, runs combined in f64, f64
//            warp reduction.
//  * A^T x : a (row block) x (column tile) grid; every thread owns one 16-byte
//            group of consecutive columns, walks the rows of its block with
//            eight loads in flight, and writes f64 partial sums per row block;
//            a second kernel sums the partials in a fixed order (deterministic).
//  * CSR   : a group of lanes per row (sized from the mean row length), f64
//            products; A^T uses the caller's stored CSR of A^T.
#include "gk_internal.cuh"

namespace gk {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;   // 16-byte loads in flight per lane in the row kernel
constexpr int kRowUnroll = 8;  // rows in flight per thread in the column kernel
constexpr int kRun = 32;     // rows summed in f32 before an f64 combine (column kernel)

__device__ __forceinline__ bool halted(const Ctl *ctl) {
  return ctl != nullptr && *reinterpret_cast<const volatile int *>(&ctl->halt) != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// y = scale * A x - coef * sub, reduced-precision A (f32 / bf16 / f16)
// Persistent grid; each block iteration takes kRowsPerBlk rows, kWarpsPerRow
// warps per row: the row's 16-byte vectors are dealt to the row's 128 lanes
// (512 contiguous bytes per warp per load), each lane keeps kUnroll loads in
// flight, the lane sums in f32 per unrolled group and in f64 across groups,
// and the row's warp partials are added in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kWarpsPerRow = 4;
constexpr int kRowsPerBlk = (kThreads / 32) / kWarpsPerRow;

template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads) k_gemv_lp(const T *__restrict__ A, int64_t m, int64_t n, int64_t ld,
                                                      double scale, const float *__restrict__ x,
                                                      double *__restrict__ y, const double *__restrict__ sub,
                                                      const double *__restrict__ coef, const Ctl *ctl) {
  if (halted(ctl)) return;
  using VT = Vec<T>;
  constexpr int E = VT::E;
  constexpr int RT = kWarpsPerRow * 32;  // lanes per row
  __shared__ double red[kThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rsub = warp / kWarpsPerRow;
  const int tr = (warp % kWarpsPerRow) * 32 + lane;  // lane index within the row
  const double c = sub ? *coef : 0.0;
  const int64_t units = (m + kRowsPerBlk - 1) / kRowsPerBlk;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t r = u * kRowsPerBlk + rsub;
    double acc = 0.0;
    if (r < m) {
      const T *a = A + r * ld;
      int64_t tail0 = 0;
      if (VEC) {
        const int64_t nv = n / E;
        const typename VT::V *av = reinterpret_cast<const typename VT::V *>(a);
        int64_t i = tr;
        for (; i + RT * (kUnroll - 1) < nv; i += RT * kUnroll) {
          typename VT::V buf[kUnroll];
#pragma unroll
          for (int q = 0; q < kUnroll; ++q) buf[q] = __ldcs(av + i + RT * q);
          float sacc = 0.f;
#pragma unroll
          for (int q = 0; q < kUnroll; ++q) {
            float f[E];
            VT::unpack(buf[q], f);
            const float4 *xv = reinterpret_cast<const float4 *>(x + (i + RT * q) * E);
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
              const float4 xx = __ldg(xv + h);
              sacc = fmaf(f[4 * h + 0], xx.x, sacc);
              sacc = fmaf(f[4 * h + 1], xx.y, sacc);
              sacc = fmaf(f[4 * h + 2], xx.z, sacc);
              sacc = fmaf(f[4 * h + 3], xx.w, sacc);
            }
          }
          acc += (double)sacc;
        }
        for (; i < nv; i += RT) {
          float f[E];
          VT::unpack(__ldcs(av + i), f);
          const float4 *xv = reinterpret_cast<const float4 *>(x + i * E);
          float sacc = 0.f;
#pragma unroll
          for (int h = 0; h < E / 4; ++h) {
            const float4 xx = __ldg(xv + h);
            sacc = fmaf(f[4 * h + 0], xx.x, sacc);
            sacc = fmaf(f[4 * h + 1], xx.y, sacc);
            sacc = fmaf(f[4 * h + 2], xx.z, sacc);
            sacc = fmaf(f[4 * h + 3], xx.w, sacc);
          }
          acc += (double)sacc;
        }
        tail0 = nv * E;
      }
      float sacc = 0.f;
      int cnt = 0;
      for (int64_t cidx = tail0 + tr; cidx < n; cidx += RT) {
        sacc = fmaf(VT::one(a + cidx), __ldg(x + cidx), sacc);
        if (++cnt == 32) {
          acc += (double)sacc;
          sacc = 0.f;
          cnt = 0;
        }
      }
      acc += (double)sacc;
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x < kRowsPerBlk) {
      const int64_t rr = u * kRowsPerBlk + threadIdx.x;
      if (rr < m) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kWarpsPerRow; ++w) t += red[threadIdx.x * kWarpsPerRow + w];
        y[rr] = t * scale - (sub ? c * sub[rr] : 0.0);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// A x with the rows of A streamed by the bulk-copy (TMA) engine.
// Work unit = one column chunk (kPiece bytes of every row, kChunk columns) x
// kUnitRows rows.  Block = 8 consumer warps + 1 producer warp.  A stage holds
// the chunk's pieces of 8 consecutive rows (8 x kPiece bytes), copied by
// cp.async.bulk into a kStages-deep shared-memory ring: full[s] completes
// when the stage's bytes have landed (complete_tx), empty[s] when the 8
// consumer warps have read it.  Each lane keeps the chunk's x values it needs
// in registers for the whole unit, so x is read once per unit; consumer warp w
// takes row w of every stage, sums its lanes' products in f32 and writes the
// row's partial for this chunk in f64.  k_gemv_reduce then adds the chunks'
// partials of every row in chunk order (deterministic).  Every wait is bounded:
// on expiry the kernel records a timeout in the control block, halts the sweep
// and lets its own copies land before exiting.
// ---------------------------------------------------------------------------
constexpr int kBulkRows = 8;                 // rows per stage = consumer warps
constexpr int kBulkThreads = (kBulkRows + 1) * 32;
constexpr int kStages = 4;
constexpr int kPiece = 2048;                 // bytes of one row per stage
constexpr int kStageBytes = kPiece * kBulkRows;
constexpr int kUnitRows = 128;               // rows per work unit (16 stages)
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz before a wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}
// bounded wait for the phase with the given parity; false if it did not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  const uint32_t a = smem_addr(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ void record_timeout(Ctl *ctl, int where) {
  if (atomicCAS(&ctl->timeout, 0, where) == 0) {
    ctl->event = EV_TIMEOUT;
    __threadfence();
    atomicExch(&ctl->halt, 1);
  }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// part[c * m + r] = sum over the columns of chunk c of a_rc x_c (chunks of 16-byte pieces only)
template <typename T>
__global__ void __launch_bounds__(kBulkThreads) k_gemv_bulk(const T *__restrict__ A, int64_t m, int64_t n, int64_t ld,
                                                           const float *__restrict__ x, double *__restrict__ part,
                                                           Ctl *ctl) {
  if (halted(ctl)) return;
  using VT = Vec<T>;
  constexpr int E = VT::E;
  constexpr int64_t kChunk = kPiece / (int64_t)sizeof(T);  // columns per chunk
  constexpr int VPL = kPiece / 16 / 32;                       // 16-byte vectors per lane per row piece
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kBulkRows);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t vec_cols = (n * (int64_t)sizeof(T)) / 16 * 16 / (int64_t)sizeof(T);  // columns in 16-byte pieces
  const int64_t nchunk = (vec_cols + kChunk - 1) / kChunk;
  const int64_t ngroup = (m + kUnitRows - 1) / kUnitRows;
  const int64_t nunit = nchunk * ngroup;
  if (warp == kBulkRows) {
    // producer: one elected lane issues the stages of this block's units in order
    if (lane == 0) {
      int64_t s = 0;
      for (int64_t u = blockIdx.x; u < nunit; u += gridDim.x) {
        const int64_t c = u / ngroup, g = u % ngroup;
        const int64_t c0 = c * kChunk;
        const int64_t c1 = (c0 + kChunk < vec_cols) ? c0 + kChunk : vec_cols;
        const unsigned piece = (unsigned)((c1 - c0) * (int64_t)sizeof(T));
        const int64_t rg0 = g * kUnitRows;
        const int64_t rg1 = (rg0 + kUnitRows < m) ? rg0 + kUnitRows : m;
        for (int64_t r0 = rg0; r0 < rg1; r0 += kBulkRows, ++s) {
          const int slot = (int)(s % kStages);
          if (s >= kStages && !mbar_wait(&empty[slot], (unsigned)(((s / kStages) - 1) & 1))) {
            record_timeout(ctl, 2);
            return;
          }
          const int rows = (int)((rg1 - r0) < kBulkRows ? (rg1 - r0) : kBulkRows);
          mbar_arrive_expect_tx(&full[slot], piece * (unsigned)rows);
          for (int r = 0; r < rows; ++r)
            bulk_g2s(smem + (size_t)slot * kStageBytes + (size_t)r * kPiece, A + (r0 + r) * ld + c0, piece,
                     &full[slot]);
        }
      }
    }
    return;
  }
  // consumers
  int64_t s = 0;
  for (int64_t u = blockIdx.x; u < nunit; u += gridDim.x) {
    const int64_t c = u / ngroup, g = u % ngroup;
    const int64_t c0 = c * kChunk;
    const int64_t c1 = (c0 + kChunk < vec_cols) ? c0 + kChunk : vec_cols;
    const int nv = (int)((c1 - c0) / E);  // 16-byte vectors in this chunk's row piece
    // this lane's x values for the chunk (vectors lane, lane + 32, ...)
    float xr[VPL][E];
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
      const int v = lane + 32 * q;
#pragma unroll
      for (int h = 0; h < E / 4; ++h) {
        float4 xx = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v < nv) xx = __ldg(reinterpret_cast<const float4 *>(x + c0 + (int64_t)v * E) + h);
        xr[q][4 * h + 0] = xx.x;
        xr[q][4 * h + 1] = xx.y;
        xr[q][4 * h + 2] = xx.z;
        xr[q][4 * h + 3] = xx.w;
      }
    }
    const int64_t rg0 = g * kUnitRows;
    const int64_t rg1 = (rg0 + kUnitRows < m) ? rg0 + kUnitRows : m;
    for (int64_t r0 = rg0; r0 < rg1; r0 += kBulkRows, ++s) {
      const int slot = (int)(s % kStages);
      if (!mbar_wait(&full[slot], (unsigned)((s / kStages) & 1))) {
        // give up: record it, then let the copies the producer may still have in
        // flight (at most the next kStages - 1 stages) land before the block exits
        record_timeout(ctl, 1);
        for (int64_t t = s + 1; t < s + kStages; ++t) mbar_wait(&full[t % kStages], (unsigned)((t / kStages) & 1));
        return;
      }
      const int64_t r = r0 + warp;
      if (r < rg1) {
        const typename VT::V *tile =
            reinterpret_cast<const typename VT::V *>(smem + (size_t)slot * kStageBytes + (size_t)warp * kPiece);
        float sacc = 0.f;
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
          const int v = lane + 32 * q;
          if (v < nv) {
            float f[E];
            VT::unpack(tile[v], f);
#pragma unroll
            for (int e = 0; e < E; ++e) sacc = fmaf(f[e], xr[q][e], sacc);
          }
        }
        sacc = warp_sum_f(sacc);
        if (lane == 0) part[c * m + r] = (double)sacc;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
  }
}

// y[r] = scale * (sum_c part[c * m + r] + leftover columns) - coef * sub[r]
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gemv_reduce(const T *__restrict__ A, int64_t m, int64_t n, int64_t ld,
                                                          double scale, const float *__restrict__ x,
                                                          const double *__restrict__ part, int64_t nchunk,
                                                          double *__restrict__ y, const double *__restrict__ sub,
                                                          const double *__restrict__ coef, const Ctl *ctl) {
  if (halted(ctl)) return;
  const int64_t vec_cols = (n * (int64_t)sizeof(T)) / 16 * 16 / (int64_t)sizeof(T);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) t += part[c * m + r];
    for (int64_t cidx = vec_cols; cidx < n; ++cidx) t += (double)(Vec<T>::one(A + r * ld + cidx) * x[cidx]);
    y[r] = t * scale - (sub ? (*coef) * sub[r] : 0.0);
  }
}

// y = A x - coef * sub, f64 A (products in f64)
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_gemv_f64(const double *__restrict__ A, int64_t m, int64_t n, int64_t ld,
                                                       double scale, const double *__restrict__ x,
                                                       double *__restrict__ y, const double *__restrict__ sub,
                                                       const double *__restrict__ coef, const Ctl *ctl) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double c = sub ? *coef : 0.0;
  for (int64_t r = warp; r < m; r += nwarp) {
    const double *a = A + r * ld;
    double acc = 0.0;
    int64_t tail0 = 0;
    if (VEC) {
      const int64_t nv = n / 2;
      const double2 *av = reinterpret_cast<const double2 *>(a);
      const double2 *xv = reinterpret_cast<const double2 *>(x);
      int64_t i = lane;
      for (; i + 32 * (kUnroll - 1) < nv; i += 32 * kUnroll) {
        double2 buf[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) buf[u] = __ldcs(av + i + 32 * u);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const double2 xx = __ldg(xv + i + 32 * u);
          acc = fma(buf[u].x, xx.x, acc);
          acc = fma(buf[u].y, xx.y, acc);
        }
      }
      for (; i < nv; i += 32) {
        const double2 b = __ldcs(av + i), xx = __ldg(xv + i);
        acc = fma(b.x, xx.x, acc);
        acc = fma(b.y, xx.y, acc);
      }
      tail0 = nv * 2;
    }
    for (int64_t cidx = tail0 + lane; cidx < n; cidx += 32) acc = fma(a[cidx], __ldg(x + cidx), acc);
    acc = warp_sum(acc);
    if (lane == 0) y[r] = acc * scale - (sub ? c * sub[r] : 0.0);
  }
}

// ---------------------------------------------------------------------------
// A^T x, partial sums per row block: part[rb * n + col]
// ---------------------------------------------------------------------------
template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads) k_gemvt_lp(const T *__restrict__ A, int64_t m, int64_t n, int64_t ld,
                                                       int64_t RB, const float *__restrict__ x,
                                                       double *__restrict__ part, const Ctl *ctl) {
  if (halted(ctl)) return;
  using VT = Vec<T>;
  constexpr int E = VT::E;
  __shared__ float xs[1024];
  const int64_t r0 = (int64_t)blockIdx.y * RB;
  const int64_t r1 = (r0 + RB < m) ? r0 + RB : m;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) xs[r - r0] = x[r];
  __syncthreads();
  const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
  if (c0 >= n) return;
  float a32[E];
  double a64[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    a32[e] = 0.f;
    a64[e] = 0.0;
  }
  if (VEC && c0 + E <= n) {
    const int64_t ldv = ld / E;
    const typename VT::V *p = reinterpret_cast<const typename VT::V *>(A + r0 * ld + c0);
    int64_t r = r0;
    int run = 0;
    for (; r + kRowUnroll <= r1; r += kRowUnroll) {
      typename VT::V buf[kRowUnroll];
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) buf[u] = __ldcs(p + (r - r0 + u) * ldv);
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) {
        float f[E];
        VT::unpack(buf[u], f);
        const float xv = xs[r - r0 + u];
#pragma unroll
        for (int e = 0; e < E; ++e) a32[e] = fmaf(f[e], xv, a32[e]);
      }
      run += kRowUnroll;
      if (run >= kRun) {
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
      VT::unpack(__ldcs(p + (r - r0) * ldv), f);
      const float xv = xs[r - r0];
#pragma unroll
      for (int e = 0; e < E; ++e) a32[e] = fmaf(f[e], xv, a32[e]);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) a64[e] += (double)a32[e];
#pragma unroll
    for (int e = 0; e < E; ++e) part[(int64_t)blockIdx.y * n + c0 + e] = a64[e];
  } else {
    const int ne = (int)((n - c0) < E ? (n - c0) : E);
    for (int e = 0; e < ne; ++e) {
      double acc = 0.0;
      float s = 0.f;
      int run = 0;
      for (int64_t r = r0; r < r1; ++r) {
        s = fmaf(VT::one(A + r * ld + c0 + e), xs[r - r0], s);
        if (++run == kRun) {
          acc += (double)s;
          s = 0.f;
          run = 0;
        }
      }
      acc += (double)s;
      part[(int64_t)blockIdx.y * n + c0 + e] = acc;
    }
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_gemvt_f64(const double *__restrict__ A, int64_t m, int64_t n,
                                                        int64_t ld, int64_t RB, const double *__restrict__ x,
                                                        double *__restrict__ part, const Ctl *ctl) {
  if (halted(ctl)) return;
  __shared__ double xs[1024];
  const int64_t r0 = (int64_t)blockIdx.y * RB;
  const int64_t r1 = (r0 + RB < m) ? r0 + RB : m;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) xs[r - r0] = x[r];
  __syncthreads();
  const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (c0 >= n) return;
  if (VEC && c0 + 2 <= n) {
    const int64_t ldv = ld / 2;
    const double2 *p = reinterpret_cast<const double2 *>(A + r0 * ld + c0);
    double s0 = 0.0, s1 = 0.0;
    int64_t r = r0;
    for (; r + kRowUnroll <= r1; r += kRowUnroll) {
      double2 buf[kRowUnroll];
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) buf[u] = __ldcs(p + (r - r0 + u) * ldv);
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) {
        const double xv = xs[r - r0 + u];
        s0 = fma(buf[u].x, xv, s0);
        s1 = fma(buf[u].y, xv, s1);
      }
    }
    for (; r < r1; ++r) {
      const double2 b = __ldcs(p + (r - r0) * ldv);
      s0 = fma(b.x, xs[r - r0], s0);
      s1 = fma(b.y, xs[r - r0], s1);
    }
    part[(int64_t)blockIdx.y * n + c0] = s0;
    part[(int64_t)blockIdx.y * n + c0 + 1] = s1;
  } else {
    const int ne = (int)((n - c0) < 2 ? (n - c0) : 2);
    for (int e = 0; e < ne; ++e) {
      double s = 0.0;
      for (int64_t r = r0; r < r1; ++r) s = fma(A[r * ld + c0 + e], xs[r - r0], s);
      part[(int64_t)blockIdx.y * n + c0 + e] = s;
    }
  }
}

// y[c] = scale * sum_rb part[rb * n + c] - coef * sub[c]; block = 32 columns x 8 row-block groups,
// each group sums a contiguous range of row blocks, groups are combined in order.
__global__ void __launch_bounds__(kThreads) k_gemvt_reduce(const double *__restrict__ part, int64_t n, int nrb,
                                                           double scale, double *__restrict__ y,
                                                           const double *__restrict__ sub,
                                                           const double *__restrict__ coef, const Ctl *ctl) {
  if (halted(ctl)) return;
  __shared__ double red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + tx;
  const int per = (nrb + 7) / 8;
  const int b0 = ty * per, b1 = (b0 + per < nrb) ? b0 + per : nrb;
  double s = 0.0;
  if (c < n)
    for (int b = b0; b < b1; ++b) s += part[(int64_t)b * n + c];
  red[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && c < n) {
    double t = 0.0;
#pragma unroll
    for (int g = 0; g < 8; ++g) t += red[g][tx];
    y[c] = t * scale - (sub ? (*coef) * sub[c] : 0.0);
  }
}

// ---------------------------------------------------------------------------
// CSR: y = scale * A x - coef * sub, TPR lanes per row, f64 products
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double csr_val(const T *v, int64_t p);
template <>
__device__ __forceinline__ double csr_val<float>(const float *v, int64_t p) { return (double)__ldcs(v + p); }
template <>
__device__ __forceinline__ double csr_val<double>(const double *v, int64_t p) { return __ldcs(v + p); }
template <>
__device__ __forceinline__ double csr_val<__nv_bfloat16>(const __nv_bfloat16 *v, int64_t p) {
  return (double)__bfloat162float(v[p]);
}
template <>
__device__ __forceinline__ double csr_val<__half>(const __half *v, int64_t p) { return (double)__half2float(v[p]); }

template <typename T, int TPR>
__global__ void __launch_bounds__(kThreads) k_spmv(const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colind, const T *__restrict__ vals,
                                                   int64_t m, double scale, const double *__restrict__ x,
                                                   double *__restrict__ y, const double *__restrict__ sub,
                                                   const double *__restrict__ coef, const Ctl *ctl) {
  if (halted(ctl)) return;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sub_lane = threadIdx.x % TPR;
  constexpr int RPW = 32 / TPR;  // rows per warp per iteration
  const int64_t warp = tid >> 5, nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double c = sub ? *coef : 0.0;
  for (int64_t base = warp * RPW; base < m; base += nwarp * RPW) {
    const int64_t row = base + (threadIdx.x & 31) / TPR;
    double s = 0.0;
    if (row < m) {
      const int64_t p1 = rowptr[row + 1];
      for (int64_t p = rowptr[row] + sub_lane; p < p1; p += TPR) s = fma(csr_val<T>(vals, p), __ldg(x + colind[p]), s);
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
    if (row < m && sub_lane == 0) y[row] = s * scale - (sub ? c * sub[row] : 0.0);
  }
}

template <class K>
int resident_blocks(K kernel, const Dev &d) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * d.sms;
}

template <typename T>
cudaError_t launch_gemv(const Op &A, const float *x32, double *y, const double *sub, const double *coef,
                        double *part, const Ctl *ctl, cudaStream_t s, const Dev &d) {
  const bool vec = ((uintptr_t)A.vals % 16 == 0) && ((A.ld * (int64_t)sizeof(T)) % 16 == 0);
  if (vec && A.n * (int64_t)sizeof(T) >= 16 && part != nullptr) {
    // rows start on 16-byte boundaries: stream them with the bulk-copy engine
    static int per_sm = 0;
    const size_t dyn = (size_t)kStages * kStageBytes;
    if (!per_sm) {
      if (cudaFuncSetAttribute(k_gemv_bulk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv_bulk<T>, kBulkThreads, dyn) != cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
    }
    constexpr int64_t kChunk = kPiece / (int64_t)sizeof(T);
    const int64_t vec_cols = (A.n * (int64_t)sizeof(T)) / 16 * 16 / (int64_t)sizeof(T);
    const int64_t nchunk = (vec_cols + kChunk - 1) / kChunk;
    const int64_t nunit = nchunk * ((A.m + kUnitRows - 1) / kUnitRows);
    const int64_t full = (int64_t)per_sm * d.sms;
    const int blocks = (int)(nunit < full ? nunit : full);
    GK_LAUNCH(k_gemv_bulk<T><<<blocks, kBulkThreads, dyn, s>>>((const T *)A.vals, A.m, A.n, A.ld, x32, part,
                                                               const_cast<Ctl *>(ctl)));
    int64_t rb = (A.m + kThreads - 1) / kThreads;
    if (rb > 4096) rb = 4096;
    GK_LAUNCH(k_gemv_reduce<T><<<(int)rb, kThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, A.scale, x32, part,
                                                            nchunk, y, sub, coef, ctl));
    return cudaGetLastError();
  }
  const int64_t units = (A.m + kRowsPerBlk - 1) / kRowsPerBlk;
  static int full_vec = 0, full_sc = 0;  // resident blocks of each variant on this device
  if (vec) {
    if (!full_vec) full_vec = resident_blocks(k_gemv_lp<T, true>, d);
    const int blocks = (int)(units < full_vec ? units : full_vec);
    GK_LAUNCH(k_gemv_lp<T, true><<<blocks, kThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, A.scale, x32, y,
                                                              sub, coef, ctl));
  } else {
    if (!full_sc) full_sc = resident_blocks(k_gemv_lp<T, false>, d);
    const int blocks = (int)(units < full_sc ? units : full_sc);
    GK_LAUNCH(k_gemv_lp<T, false><<<blocks, kThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, A.scale, x32, y,
                                                               sub, coef, ctl));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmv(const int32_t *rp, const int32_t *ci, const void *v, int64_t rows, int64_t nnz, double scale,
                        const double *x, double *y, const double *sub, const double *coef, const Ctl *ctl,
                        cudaStream_t s, const Dev &d) {
  // lanes per row from the mean row length: 4 up to 24 entries, 8 up to 96, else 16
  const int blocks = d.sms * 8;
  const T *vals = (const T *)v;
  const double mean = rows > 0 && nnz > 0 ? (double)nnz / (double)rows : 32.0;
  if (mean <= 24.0)
    GK_LAUNCH(k_spmv<T, 4><<<blocks, kThreads, 0, s>>>(rp, ci, vals, rows, scale, x, y, sub, coef, ctl));
  else if (mean <= 96.0)
    GK_LAUNCH(k_spmv<T, 8><<<blocks, kThreads, 0, s>>>(rp, ci, vals, rows, scale, x, y, sub, coef, ctl));
  else
    GK_LAUNCH(k_spmv<T, 16><<<blocks, kThreads, 0, s>>>(rp, ci, vals, rows, scale, x, y, sub, coef, ctl));
  return cudaGetLastError();
}

}  // namespace

int64_t gemvt_row_block(const Op &A, const Dev &d) {
  const int E = (A.dtype == GK_F64) ? 2 : (A.dtype == GK_F32 ? 4 : 8);
  const int64_t cb = (int64_t)kThreads * E;
  const int64_t ntile = (A.n + cb - 1) / cb;
  const int64_t want = (int64_t)8 * d.sms;  // blocks to fill the machine
  int64_t rb = (A.m * ntile + want - 1) / want;
  rb = round_up(rb < 1 ? 1 : rb, 32);
  if (rb > 1024) rb = 1024;
  if (rb < 32) rb = 32;
  return rb;
}

int64_t gemvt_partials(const Op &A, const Dev &d) {
  if (A.kind != GK_DENSE) return 0;
  const int64_t rb = gemvt_row_block(A, d);
  const int64_t t = ((A.m + rb - 1) / rb) * A.n;
  // the bulk-copy A x kernel keeps one partial per row and column chunk
  const int64_t es = A.dtype == GK_F64 ? 8 : (A.dtype == GK_F32 ? 4 : 2);
  const int64_t chunk = kPiece / es;
  const int64_t g = ((A.n + chunk - 1) / chunk) * A.m;
  return t > g ? t : g;
}

cudaError_t matvec(const Op &A, const float *x32, const double *x64, double *y, const double *sub,
                   const double *coef, double *part, const Ctl *ctl, cudaStream_t s, const Dev &d) {
  if (A.kind == GK_CSR) {
    switch (A.dtype) {
      case GK_F64: return launch_spmv<double>(A.rowptr, A.colind, A.vals, A.m, A.nnz, A.scale, x64, y, sub, coef, ctl, s, d);
      case GK_F32: return launch_spmv<float>(A.rowptr, A.colind, A.vals, A.m, A.nnz, A.scale, x64, y, sub, coef, ctl, s, d);
      case GK_BF16:
        return launch_spmv<__nv_bfloat16>(A.rowptr, A.colind, A.vals, A.m, A.nnz, A.scale, x64, y, sub, coef, ctl, s, d);
      default: return launch_spmv<__half>(A.rowptr, A.colind, A.vals, A.m, A.nnz, A.scale, x64, y, sub, coef, ctl, s, d);
    }
  }
  switch (A.dtype) {
    case GK_F64: {
      const bool vec = ((uintptr_t)A.vals % 16 == 0) && ((A.ld * 8) % 16 == 0);
      int blocks = d.sms * 8;
      const int64_t need = (A.m + 7) / 8;
      if (blocks > need) blocks = (int)need;
      if (blocks < 1) blocks = 1;
      if (vec)
        GK_LAUNCH(k_gemv_f64<true><<<blocks, kThreads, 0, s>>>((const double *)A.vals, A.m, A.n, A.ld, A.scale, x64, y, sub,
                                                     coef, ctl));
      else
        GK_LAUNCH(k_gemv_f64<false><<<blocks, kThreads, 0, s>>>((const double *)A.vals, A.m, A.n, A.ld, A.scale, x64, y, sub,
                                                      coef, ctl));
      return cudaGetLastError();
    }
    case GK_F32: return launch_gemv<float>(A, x32, y, sub, coef, part, ctl, s, d);
    case GK_BF16: return launch_gemv<__nv_bfloat16>(A, x32, y, sub, coef, part, ctl, s, d);
    default: return launch_gemv<__half>(A, x32, y, sub, coef, part, ctl, s, d);
  }
}

namespace {
template <typename T>
cudaError_t launch_gemvt(const Op &A, const float *x32, double *part, const Ctl *ctl, cudaStream_t s, const Dev &d,
                         int64_t rb, int nrb) {
  constexpr int E = Vec<T>::E;
  const bool vec = ((uintptr_t)A.vals % 16 == 0) && ((A.ld * (int64_t)sizeof(T)) % 16 == 0);
  dim3 grid((unsigned)((A.n + (int64_t)kThreads * E - 1) / ((int64_t)kThreads * E)), (unsigned)nrb);
  if (vec)
    GK_LAUNCH(k_gemvt_lp<T, true><<<grid, kThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, rb, x32, part, ctl));
  else
    GK_LAUNCH(k_gemvt_lp<T, false><<<grid, kThreads, 0, s>>>((const T *)A.vals, A.m, A.n, A.ld, rb, x32, part, ctl));
  return cudaGetLastError();
}
}  // namespace

cudaError_t matvec_t(const Op &A, const float *x32, const double *x64, double *y, const double *sub,
                     const double *coef, double *part, const Ctl *ctl, cudaStream_t s, const Dev &d) {
  if (A.kind == GK_CSR) {
    switch (A.dtype) {
      case GK_F64:
        return launch_spmv<double>(A.t_rowptr, A.t_colind, A.t_vals, A.n, A.nnz, A.scale, x64, y, sub, coef, ctl, s, d);
      case GK_F32:
        return launch_spmv<float>(A.t_rowptr, A.t_colind, A.t_vals, A.n, A.nnz, A.scale, x64, y, sub, coef, ctl, s, d);
      case GK_BF16:
        return launch_spmv<__nv_bfloat16>(A.t_rowptr, A.t_colind, A.t_vals, A.n, A.nnz, A.scale, x64, y, sub, coef, ctl, s,
                                          d);
      default:
        return launch_spmv<__half>(A.t_rowptr, A.t_colind, A.t_vals, A.n, A.nnz, A.scale, x64, y, sub, coef, ctl, s, d);
    }
  }
  const int64_t rb = gemvt_row_block(A, d);
  const int nrb = (int)((A.m + rb - 1) / rb);
  cudaError_t e;
  switch (A.dtype) {
    case GK_F64: {
      const bool vec = ((uintptr_t)A.vals % 16 == 0) && ((A.ld * 8) % 16 == 0);
      dim3 grid((unsigned)((A.n + (int64_t)kThreads * 2 - 1) / ((int64_t)kThreads * 2)), (unsigned)nrb);
      if (vec)
        GK_LAUNCH(k_gemvt_f64<true><<<grid, kThreads, 0, s>>>((const double *)A.vals, A.m, A.n, A.ld, rb, x64, part, ctl));
      else
        GK_LAUNCH(k_gemvt_f64<false><<<grid, kThreads, 0, s>>>((const double *)A.vals, A.m, A.n, A.ld, rb, x64, part, ctl));
      e = cudaGetLastError();
      break;
    }
    case GK_F32: e = launch_gemvt<float>(A, x32, part, ctl, s, d, rb, nrb); break;
    case GK_BF16: e = launch_gemvt<__nv_bfloat16>(A, x32, part, ctl, s, d, rb, nrb); break;
    default: e = launch_gemvt<__half>(A, x32, part, ctl, s, d, rb, nrb); break;
  }
  if (e != cudaSuccess) return e;
  GK_LAUNCH(k_gemvt_reduce<<<(unsigned)((A.n + 31) / 32), kThreads, 0, s>>>(part, A.n, nrb, A.scale, y, sub, coef, ctl));
  return cudaGetLastError();
}

}  // namespace gk
