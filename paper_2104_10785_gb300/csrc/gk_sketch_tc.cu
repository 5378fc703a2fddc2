// gk_sketch_tc.cu -- the predictor's sketch Y = A Omega of one bf16 operator on the fifth-generation
// tensor cores: tiles staged by TMA (cp.async.bulk.tensor, 128-byte swizzle), the products by
// tcgen05.mma with the 128 x 32 accumulator of a row chunk in tensor memory, read back by
// tcgen05.ld for the chunk's Gram partials.  Opt-in (GK_FLAG_SKETCH_TC) beside k_sketch_mma,
// which forms the same products with mma.sync; the epilogue (the chunk's 528 Gram entries in
// f64 and its ||A_c||_F^2) is the same, so the features differ only by the order of the f32
// accumulation inside the tensor pipe.
//
// CTA = one 128-row chunk of A, 4 warps:
//   warp 0 (one lane): the producer -- per stage the 128 x 64 tile of A (16 KB) and the 32 x 64
//     tile of Omega^T (4 KB), both K-major with the 128-byte swizzle, on full[s];
//   warp 1: allocates 32 columns of tensor memory; one lane issues the stage's four
//     M128 x N32 x K16 MMAs (bf16 in, f32 accumulate) and commits them to empty[s], and after the
//     last stage to `done`;
//   warps 2-3: ||A_c||_F^2 from the staged tiles (zero outside A), then arrive on empty[s];
//   all warps: the accumulator's 32 lanes each (tcgen05.ld 32x32b), the Gram partials.
// Every wait is bounded; a wait that gives up raises a shared abort flag that ends the other
// roles' loops, records the kernel's error flag, and the kernel still waits (bounded) for its
// own copies and MMAs before it frees the tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "gk_internal.cuh"

namespace gk {

namespace {

constexpr int kTcRows = 128;     // rows of A per CTA: the MMA's M, one tensor-memory lane each
constexpr int kTcN = 32;         // sketch columns: the MMA's N, tensor-memory columns
constexpr int kTcK = 64;         // columns of A per stage: one 128-byte swizzle row of bf16
constexpr int kTcStages = 4;
constexpr int kTcThreads = 128;
constexpr uint32_t kTileA = kTcRows * kTcK * 2;  // 16384 bytes
constexpr uint32_t kTileB = kTcN * kTcK * 2;     // 4096 bytes
constexpr int kTcTri = kTcN * (kTcN + 1) / 2;    // 528 Gram entries
constexpr int kTcPitch = kTcN + 1;               // f32 pitch of the staged Y rows
constexpr long long kTcWaitCycles = 4000000000ll;  // ~2 s at 2 GHz before a wait gives up
constexpr size_t kTcBarOff = (size_t)kTcStages * (kTileA + kTileB);
constexpr size_t kTcYOff = kTcBarOff + 128;
constexpr size_t kTcRedOff = kTcYOff + sizeof(float) * kTcRows * kTcPitch;
constexpr size_t kTcSmem = kTcRedOff + 64 + 1024;  // + slack for the 1024-byte alignment

__device__ __forceinline__ uint32_t tc_saddr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void tc_bar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_expect_tx(uint32_t bar, unsigned bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
// bounded wait for the phase of the given parity; gives up (false) after kTcWaitCycles or
// when another role raised the abort flag (unless `ignore_abort`)
__device__ __forceinline__ bool tc_wait(uint32_t bar, unsigned parity, const volatile int *abort_flag,
                                        bool ignore_abort = false) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (!ignore_abort && *abort_flag) return false;
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
}
__device__ __forceinline__ void tc_tma_2d(uint32_t dst, const CUtensorMap *tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// shared-memory matrix descriptor: K-major tile with the 128-byte swizzle, 8-row groups 1024 bytes
// apart (stride byte offset), start address in 16-byte units, descriptor version 1, swizzle mode 2
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (16 B; not used by swizzled K-major tiles)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}
// instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both K-major, N = 32, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_abort(volatile int *abort_flag, int *err, int where) {
  *abort_flag = 1;
  atomicCAS(err, 0, where);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_sketch_tc(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmO, int64_t m,
                                                             int ksteps, double scale, double *__restrict__ gpart,
                                                             double *__restrict__ fpart, int *__restrict__ err) {
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ volatile int s_abort;
  const uint32_t raw = tc_saddr(tc_smem_raw);
  unsigned char *smem = tc_smem_raw + ((1024u - (raw & 1023u)) & 1023u);  // 1024-byte aligned tiles
  const uint32_t sbase = tc_saddr(smem);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kTcBarOff);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kTcBarOff + 8 * (2 * kTcStages + 1));
  float *sY = reinterpret_cast<float *>(smem + kTcYOff);
  double *sred = reinterpret_cast<double *>(smem + kTcRedOff);
  const uint32_t full0 = tc_saddr(bars), empty0 = full0 + 8 * kTcStages, done = full0 + 16 * kTcStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int it = blockIdx.x;
  const int64_t r0 = (int64_t)it * kTcRows;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kTcStages; ++s) {
      tc_bar_init(full0 + 8 * s, 1);
      tc_bar_init(empty0 + 8 * s, 3);  // the MMA commit and one arrive from each of warps 2 and 3
    }
    tc_bar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmO)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(tmem_slot)),
                 "r"(kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  double fro = 0.0;
  int issued = 0;  // stages the producer issued

  if (warp == 0) {
    if (lane == 0) {
      for (int k = 0; k < ksteps; ++k) {
        const int s = k % kTcStages;
        if (k >= kTcStages && !tc_wait(empty0 + 8 * s, ((k / kTcStages) & 1) ^ 1, &s_abort)) {
          tc_abort(&s_abort, err, 1);
          break;
        }
        if (s_abort) break;
        tc_expect_tx(full0 + 8 * s, kTileA + kTileB);
        tc_tma_2d(sbase + s * kTileA, &tmA, k * kTcK, (int)r0, full0 + 8 * s);
        tc_tma_2d(sbase + kTcStages * kTileA + s * kTileB, &tmO, k * kTcK, 0, full0 + 8 * s);
        issued = k + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int k = 0; k < ksteps; ++k) {
        const int s = k % kTcStages;
        if (!tc_wait(full0 + 8 * s, (k / kTcStages) & 1, &s_abort)) {
          tc_abort(&s_abort, err, 2);
          break;
        }
        tc_fence_after();
        const uint32_t a0 = sbase + s * kTileA, b0 = sbase + kTcStages * kTileA + s * kTileB;
#pragma unroll
        for (int kk = 0; kk < kTcK / 16; ++kk)  // K = 16 per MMA: 32 bytes along the swizzled row
          tc_mma(tmem, tc_desc(a0 + 32 * kk), tc_desc(b0 + 32 * kk), (k | kk) != 0 ? 1u : 0u);
        tc_commit(empty0 + 8 * s);
      }
      tc_commit(done);  // arrives once every MMA issued above has completed
    }
  } else {
    // ||A_c||_F^2 from the staged tile (the swizzle permutes 16-byte pieces, not their sum)
    for (int k = 0; k < ksteps; ++k) {
      const int s = k % kTcStages;
      if (!tc_wait(full0 + 8 * s, (k / kTcStages) & 1, &s_abort)) {
        if (lane == 0) tc_abort(&s_abort, err, 3);
        break;
      }
      const uint4 *t = reinterpret_cast<const uint4 *>(smem + (size_t)s * kTileA);
      float f = 0.f;
#pragma unroll 4
      for (int i = (warp - 2) * 32 + lane; i < (int)(kTileA / 16); i += 64) {
        const uint4 v = t[i];
        const unsigned w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float lo = __uint_as_float(w4[q] << 16), hi = __uint_as_float(w4[q] & 0xffff0000u);
          f = fmaf(lo, lo, f);
          f = fmaf(hi, hi, f);
        }
      }
      fro += (double)f;
      __syncwarp();
      if (lane == 0) tc_arrive(empty0 + 8 * s);
    }
  }

  // the accumulator: every MMA complete (or the kernel gave up)
  const bool ok = tc_wait(done, 0, &s_abort, true) && !s_abort;
  __syncwarp();  // the roles' lanes meet again before the warp-wide tensor-memory load
  tc_fence_after();
  {
    uint32_t r[kTcN];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const float sc = (float)scale;
    const int row = warp * 32 + lane;
#pragma unroll
    for (int j = 0; j < kTcN; ++j) sY[row * kTcPitch + j] = __uint_as_float(r[j]) * sc;
  }
  fro = warp >= 2 ? fro : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if (lane == 0) sred[warp] = fro;
  __syncthreads();
  if (ok) {
    const int rows = (int)((m - r0) < kTcRows ? (m - r0) : kTcRows);
    for (int e = threadIdx.x; e < kTcTri; e += kTcThreads) {
      int a = 0, rem = e;
      while (rem >= kTcN - a) {
        rem -= kTcN - a;
        ++a;
      }
      const int b = a + rem;
      double g = 0.0;
      for (int rr = 0; rr < rows; ++rr) g = fma((double)sY[rr * kTcPitch + a], (double)sY[rr * kTcPitch + b], g);
      gpart[(int64_t)it * kTcTri + e] = g;
    }
    if (threadIdx.x == 0) fpart[it] = (sred[0] + sred[1] + sred[2] + sred[3]) * scale * scale;
  }
  // the producer's copies must have landed before the CTA's shared memory goes away
  if (warp == 0 && lane == 0) {
    for (int k = issued - kTcStages > 0 ? issued - kTcStages : 0; k < issued; ++k)
      tc_wait(full0 + 8 * (k % kTcStages), (k / kTcStages) & 1, &s_abort, true);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tc_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// 2-D bf16 tensor map: rows x cols (row stride ld elements), box of 64 columns x box_rows rows,
// 128-byte swizzle, zero fill outside
bool tc_map(CUtensorMap *tm, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool sketch_tc_ok(const void *A, int64_t m, int64_t n, int64_t ld) {
  return A != nullptr && (uintptr_t)A % 16 == 0 && (ld * 2) % 16 == 0 && m > 0 && n > 0 && m <= INT32_MAX &&
         n <= INT32_MAX;
}

cudaError_t sketch_tc(const void *A, int64_t m, int64_t n, int64_t ld, double scale, const void *omT, int64_t nk,
                      double *gpart, double *fpart, int *err, cudaStream_t s) {
  if (!sketch_tc_ok(A, m, n, ld) || nk % kTcK != 0 || nk < n) return cudaErrorInvalidValue;
  CUtensorMap tmA, tmO;
  if (!tc_map(&tmA, A, m, n, ld, kTcRows) || !tc_map(&tmO, omT, kTcN, nk, nk, kTcN)) return cudaErrorNotSupported;
  static std::mutex attr_mu;
  static int attr_dev = -1;  // the device whose shared-memory limit for the kernel was raised
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(attr_mu);
    if (attr_dev != dev) {
      e = cudaFuncSetAttribute(k_sketch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
      if (e != cudaSuccess) return e;
      attr_dev = dev;
    }
  }
  const int nitems = (int)((m + kTcRows - 1) / kTcRows);
  GK_LAUNCH(k_sketch_tc<<<nitems, kTcThreads, kTcSmem, s>>>(tmA, tmO, m, (int)(nk / kTcK), scale, gpart, fpart, err));
  return cudaGetLastError();
}

}  // namespace gk
