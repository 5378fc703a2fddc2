// gk_fused.cu -- the fused sweep: one pass over a dense operator from HBM per
// bidiagonalization step produces both products of the step.
//
// A Golub-Kahan step (Eq. 2.2; Algorithm 1) needs w = A x - c sub (the left vector
// before reorthogonalization) and then A^T u with u = (w - U h) / ||w - U h|| (h the
// Gram-Schmidt coefficients).  A^T u = (A^T w - A^T U h) / ||.||, and A^T U lies in the
// span of the right basis (A^T u_i = alpha_i v_i + beta_i v_{i+1}), which the right
// Gram-Schmidt removes anyway; so the sweep can form A^T w from the rows that produced w,
// and divide by the norm afterwards.  The operator then streams from HBM once per step
// instead of twice.
//
// Layout: a thread-block cluster of Q CTAs owns batches of kSRows rows (batch b goes to
// cluster b mod #clusters); CTA q of the cluster owns one piece of columns (at most
// kSVPT 16-byte vectors per thread and row) for the whole launch.  Per batch i:
//   - thread 0 prefetches the CTA's pieces of the rows of batch i + kSAhead into L2
//     (cp.async.bulk.prefetch), so HBM keeps streaming while the CTA computes;
//   - (a) every thread forms its share of the dot product of each row with x (f32 over its
//     vectors -- held in registers since the previous batch -- with x from shared memory, then
//     a warp tree); after a block barrier warp 0 sums the 8 warp partials in double-f32 and
//     sends them to every CTA of the cluster (distributed shared memory and a remote mbarrier
//     arrive with release semantics); the next batch's rows are then loaded;
//   - (b) the A^T w update of batch i - 1, whose exchange has had a batch to land: the wait
//     (acquire, cluster scope), w_r summed over the Q CTA partials in a fixed order (every CTA
//     forms the same w_r), then the batch's rows are read again -- from L2, a few microseconds
//     after (a) read them -- and a_rc * w_r added to per-thread f32 accumulators that are
//     folded into f64 (shared memory) every kSRun rows.
// The exchanged partials live in kSGen generations: a CTA posts batch i only after every CTA
// of its cluster posted batch i - 2, hence finished the update of batch i - 4.  At the end
// every CTA writes its columns' f64 partial of A^T w for its cluster, and k_fused_finish sums
// the clusters' partials in a fixed order, divides by the new norm and subtracts the
// recurrence term: z = scale (A^T w) / alpha - alpha v.  Every reduction has a fixed order
// (bitwise reproducible).  Every wait is bounded; a wait that gives up records a timeout in
// the control block, every thread of the CTA learns of it at the next block barrier (a
// barrier with an OR reduction) and stops, and the CTAs meet at a final cluster barrier, so
// no CTA leaves while a peer may still write into its shared memory.
#include "gk_internal.cuh"

namespace gk {

namespace {

constexpr int kSThreads = 256;                  // threads per CTA (8 warps)
constexpr int kSRows = 4;                       // rows per batch
constexpr int kSWarps = kSThreads / 32;
constexpr int kSVPT = 5;                        // 16-byte vectors per thread and row (at most)
constexpr int kSMaxPiece = kSThreads * kSVPT;   // 16-byte vectors of one CTA's column piece
constexpr int kSGen = 8;                        // generations of the exchanged partial sums
constexpr int kSAhead = 2;                      // batches prefetched into L2 ahead of the dots
constexpr int kSRun = 64;                       // rows summed in f32 before an f64 combine (A^T w)
constexpr int kFMaxCluster = 16;
constexpr long long kFWaitCycles = 4000000000ll;  // ~2 s of SM clock before a wait gives up

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// address of the same shared-memory location in CTA `peer` of this cluster
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t peer) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(peer));
  return r;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar_addr) : "memory");
}
// bounded wait with cluster-scope acquire (the partial sums stored by the peers)
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, unsigned parity) {
  const uint32_t a = saddr(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kFWaitCycles) return false;
  }
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ bool halted(const Ctl *ctl) {
  return *reinterpret_cast<const volatile int *>(&ctl->halt) != 0;
}

__device__ void record_timeout(Ctl *ctl, int where) {
  if (atomicCAS(&ctl->timeout, 0, where) == 0) {
    ctl->event = EV_TIMEOUT;
    __threadfence();
    atomicExch(&ctl->halt, 1);
  }
}

// TwoSum (Knuth): s + e == a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += x with the rounding error of hi kept in lo (double-f32 accumulation)
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// w = scale * A x - coef * sub (rows of this cluster's batches; warp 0 of CTA 0 writes)
// zpart[cluster * n + col] = sum over those rows of a_{r,col} * f32(w_r)  (without scale)
// Dynamic shared memory: z64 [piece_vecs * E] f64, x of the piece as E / 4 planes of
// [piece_vecs] float4, then the exchanged partials [kSGen][Q][2 kSRows] f32 (the CTA partial
// of each row as hi, lo).
template <typename T>
__global__ void __launch_bounds__(kSThreads, 1)
    k_fused(const T *__restrict__ A, int64_t m, int64_t n, int64_t ld, double scale, const float *__restrict__ x,
            double *__restrict__ w, const double *__restrict__ sub, const double *__restrict__ coef,
            double *__restrict__ zpart, int piece_vecs, Ctl *ctl) {
  using VT = Vec<T>;
  using V = typename VT::V;
  constexpr int E = VT::E;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t xbar[kSGen];
  __shared__ float wsum[2][kSWarps][kSRows];
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t q = cluster_rank(), Q = cluster_size(), cid = cluster_id(), NC = cluster_count();
  const int64_t nvec = n / E;  // n * sizeof(T) is a multiple of 16 (checked on the host)
  const int64_t v0 = (int64_t)q * piece_vecs;
  const int nloc = (int)(v0 >= nvec ? 0 : (nvec - v0 < piece_vecs ? nvec - v0 : piece_vecs));
  double *z64 = reinterpret_cast<double *>(smem);
  float4 *xs = reinterpret_cast<float4 *>(z64 + (size_t)piece_vecs * E);  // [E / 4][piece_vecs]
  float *slots = reinterpret_cast<float *>(xs + (size_t)(E / 4) * piece_vecs);
  const int64_t nb = (m + kSRows - 1) / kSRows;
  const int64_t ns = nb > (int64_t)cid ? (nb - (int64_t)cid + NC - 1) / NC : 0;  // batches of this cluster

  for (int i = tid; i < piece_vecs * E; i += kSThreads) z64[i] = 0.0;
  // x of this CTA's columns, E / 4 float4 planes (conflict-free 16-byte reads)
  for (int v = tid; v < piece_vecs; v += kSThreads)
#pragma unroll
    for (int h = 0; h < E / 4; ++h) {
      float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (v < nloc) {
        const float *xp = x + (v0 + v) * E + 4 * h;
        t4 = make_float4(xp[0], xp[1], xp[2], xp[3]);
      }
      xs[(size_t)h * piece_vecs + v] = t4;
    }
  if (tid == 0) {
    for (int i = 0; i < kSGen; ++i) mbar_init(&xbar[i], Q);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // every CTA's barriers are initialized before any peer arrives on them
  cluster_sync_all();
  const bool skip = halted(ctl);  // the whole cluster reads the same flag: a halted sweep does nothing
  volatile int *abort_v = &abort_flag;

  if (!skip) {
    const T *Ab = A + v0 * E;  // this CTA's column piece
    auto row0 = [&](int64_t t) { return ((int64_t)cid + t * (int64_t)NC) * kSRows; };
    auto nrows = [&](int64_t r0) { return (int)(m - r0 < kSRows ? m - r0 : kSRows); };
    auto prefetch = [&](int64_t t) {
      if (t < ns && nloc > 0) {
        const int64_t r0 = row0(t);
        const int rows = nrows(r0);
        for (int r = 0; r < rows; ++r) prefetch_l2(Ab + (r0 + r) * ld, (unsigned)nloc * 16u);
      }
    };
    auto load = [&](int64_t t, V (&a)[kSRows][kSVPT]) {
      const int64_t r0 = row0(t);
      const int rows = nrows(r0);
#pragma unroll
      for (int r = 0; r < kSRows; ++r)
#pragma unroll
        for (int j = 0; j < kSVPT; ++j) {
          const int v = tid + kSThreads * j;
          if (r < rows && v < nloc)
            a[r][j] = __ldg(reinterpret_cast<const V *>(Ab + (r0 + r) * ld) + v);
          else
            a[r][j] = V{};
        }
    };
    float za[kSVPT][E];
#pragma unroll
    for (int j = 0; j < kSVPT; ++j)
#pragma unroll
      for (int e = 0; e < E; ++e) za[j][e] = 0.f;
    auto flush = [&]() {
#pragma unroll
      for (int j = 0; j < kSVPT; ++j) {
        const int v = tid + kSThreads * j;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (v < nloc) z64[v * E + e] += (double)za[j][e];
          za[j][e] = 0.f;
        }
      }
    };
    const double c = sub ? *coef : 0.0;
    if (tid == 0)
      for (int t = 0; t < kSAhead; ++t) prefetch(t);
    V a[kSRows][kSVPT];  // the rows of the next batch's dot products, loaded one batch ahead
    if (ns > 0) load(0, a);
    bool fail = false;
    int run = 0;
    for (int64_t i = 0; i <= ns; ++i) {
      if (i < ns) {
        if (tid == 0) prefetch(i + kSAhead);
        // (a) this thread's share of the dot product of each row of batch i with x
        float d[kSRows];
#pragma unroll
        for (int r = 0; r < kSRows; ++r) d[r] = 0.f;
#pragma unroll
        for (int j = 0; j < kSVPT; ++j) {
          const int v = tid + kSThreads * j;
          if (v < nloc) {
            float xv[E];
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
              const float4 t4 = xs[(size_t)h * piece_vecs + v];
              xv[4 * h] = t4.x;
              xv[4 * h + 1] = t4.y;
              xv[4 * h + 2] = t4.z;
              xv[4 * h + 3] = t4.w;
            }
#pragma unroll
            for (int r = 0; r < kSRows; ++r) {
              float f[E];
              VT::unpack(a[r][j], f);
#pragma unroll
              for (int e = 0; e < E; ++e) d[r] = fmaf(f[e], xv[e], d[r]);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < kSRows; ++r) d[r] = warp_sum_f(d[r]);
        if (lane == 0)
#pragma unroll
          for (int r = 0; r < kSRows; ++r) wsum[i & 1][warp][r] = d[r];
      }
      // every thread takes the same decision at the same barrier
      if (__syncthreads_or(fail || *abort_v)) {
        fail = true;
        break;
      }
      if (i < ns && warp == 0) {
        // the CTA partial of each row (double-f32 over the warps, fixed order), to every CTA
        float hi = 0.f, lo = 0.f;
        if (lane < kSRows)
          for (int ww = 0; ww < kSWarps; ++ww) df_add(hi, lo, wsum[i & 1][ww][lane]);
        float h[kSRows], l[kSRows];
#pragma unroll
        for (int r = 0; r < kSRows; ++r) {
          h[r] = __shfl_sync(0xffffffffu, hi, r);
          l[r] = __shfl_sync(0xffffffffu, lo, r);
        }
        if (lane < (int)Q) {
          const int gen = (int)(i % kSGen);
          const uint32_t dst = peer_addr(saddr(slots + ((size_t)gen * Q + q) * 2 * kSRows), (uint32_t)lane);
          asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "f"(h[0]), "f"(h[1]), "f"(h[2]),
                       "f"(h[3])
                       : "memory");
          asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst + 16), "f"(l[0]), "f"(l[1]),
                       "f"(l[2]), "f"(l[3])
                       : "memory");
          mbar_arrive_remote(peer_addr(saddr(&xbar[gen]), (uint32_t)lane));
        }
      }
      // the next batch's rows, in flight while the update below waits for its own
      if (i + 1 < ns) load(i + 1, a);
      // (b) the A^T w update of batch i - 1 (its rows read again, now from L2)
      if (i >= 1 && !fail) {
        const int64_t t = i - 1;
        V b2[kSRows][kSVPT];
        load(t, b2);
        const int gen = (int)(t % kSGen);
        if (!mbar_wait_cluster(&xbar[gen], (unsigned)((t / kSGen) & 1))) {
          fail = true;
        } else {
          const int64_t r0 = row0(t);
          const int rows = nrows(r0);
          float wv32 = 0.f;
          if (lane < rows) {
            float hi = 0.f, lo = 0.f;
            for (uint32_t p = 0; p < Q; ++p) {
              const float *sp = slots + ((size_t)gen * Q + p) * 2 * kSRows;
              df_add(hi, lo, sp[lane]);
              df_add(hi, lo, sp[kSRows + lane]);
            }
            const double wv = ((double)hi + (double)lo) * scale - (sub ? c * sub[r0 + lane] : 0.0);
            wv32 = (float)wv;
            if (q == 0 && warp == 0) w[r0 + lane] = wv;
          }
          float wr[kSRows];
#pragma unroll
          for (int r = 0; r < kSRows; ++r) wr[r] = __shfl_sync(0xffffffffu, wv32, r);
#pragma unroll
          for (int r = 0; r < kSRows; ++r)
#pragma unroll
            for (int j = 0; j < kSVPT; ++j) {
              float f[E];
              VT::unpack(b2[r][j], f);
#pragma unroll
              for (int e = 0; e < E; ++e) za[j][e] = fmaf(f[e], wr[r], za[j][e]);
            }
          run += rows;
          if (run >= kSRun) {
            flush();
            run = 0;
          }
        }
      }
    }
    if (!__syncthreads_or(fail || *abort_v)) {
      flush();
      // this thread's columns of the cluster's partial A^T w (its own z64 entries)
#pragma unroll
      for (int j = 0; j < kSVPT; ++j) {
        const int v = tid + kSThreads * j;
        if (v < nloc) {
          double *zp = zpart + (int64_t)cid * n + (v0 + v) * E;
#pragma unroll
          for (int e = 0; e < E; ++e) zp[e] = z64[v * E + e];
        }
      }
    } else {
      if (tid == 0) record_timeout(ctl, 1);
      *abort_v = 1;
    }
  }
  // no CTA leaves while a peer may still store into its shared memory
  __syncthreads();
  cluster_sync_all();
}

__global__ void __launch_bounds__(256) k_fused_finish(const double *__restrict__ zpart, int nc, int64_t n,
                                                      double scale, const double *__restrict__ coef,
                                                      const double *__restrict__ sub, double *__restrict__ z,
                                                      const Ctl *ctl) {
  if (halted(ctl)) return;
  const double a = *coef;
  const double f = scale / a;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int k = 0; k < nc; ++k) t += zpart[(int64_t)k * n + c];
    z[c] = t * f - (sub ? a * sub[c] : 0.0);
  }
}

struct FusedPlan {
  int Q = 0, NC = 0, piece_vecs = 0;
  size_t smem = 0;
};

template <typename T>
cudaError_t plan_for(const Op &A, const Dev &d, FusedPlan *pl) {
  constexpr int E = Vec<T>::E;
  const int64_t nvec = A.n / E;
  auto kern = k_fused<T>;
  auto smem_for = [&](int64_t pv, int Q) {
    return (size_t)pv * E * (sizeof(double) + sizeof(float)) + (size_t)kSGen * Q * 2 * kSRows * sizeof(float);
  };
  static int attr_dev = -1;
  if (attr_dev != d.id) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_for(kSMaxPiece, kFMaxCluster));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    attr_dev = d.id;
  }
  // among the cluster sizes whose column piece fits the threads' vectors, the one that keeps
  // the most SMs busy (clusters are placed within one GPC: sizes that do not divide a GPC
  // idle SMs); the smaller cluster on a tie
  int best_active = 0;
  for (int Q = 1; Q <= kFMaxCluster; Q *= 2) {
    const int64_t pv = (nvec + Q - 1) / Q;
    if (pv > kSMaxPiece) continue;
    const size_t smem = smem_for(pv, Q);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Q, 1, 1);
    cfg.blockDim = dim3(kSThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = Q;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      nc = 0;
    }
    if (nc * Q > best_active) {
      best_active = nc * Q;
      pl->Q = Q;
      pl->NC = nc;
      pl->piece_vecs = (int)pv;
      pl->smem = smem;
    }
  }
  return best_active > 0 ? cudaSuccess : cudaErrorNotSupported;
}

cudaError_t plan(const Op &A, const Dev &d, FusedPlan *pl) {
  switch (A.dtype) {
    case GK_F32: return plan_for<float>(A, d, pl);
    case GK_BF16: return plan_for<__nv_bfloat16>(A, d, pl);
    case GK_F16: return plan_for<__half>(A, d, pl);
    default: return cudaErrorNotSupported;
  }
}

// one plan per (device, dtype, n): the occupancy queries run once
struct PlanCache {
  int dev = -1, dtype = -1;
  int64_t n = -1;
  FusedPlan pl;
  bool valid = false;
};
thread_local PlanCache t_plan;

bool cached_plan(const Op &A, const Dev &d, FusedPlan *pl) {
  if (t_plan.dev == d.id && t_plan.dtype == A.dtype && t_plan.n == A.n) {
    *pl = t_plan.pl;
    return t_plan.valid;
  }
  FusedPlan p;
  const bool v = plan(A, d, &p) == cudaSuccess;
  cudaGetLastError();
  t_plan.dev = d.id;
  t_plan.dtype = A.dtype;
  t_plan.n = A.n;
  t_plan.pl = p;
  t_plan.valid = v;
  *pl = p;
  return v;
}

}  // namespace

bool fused_ok(const Op &A, const Dev &d) {
  if (A.kind != GK_DENSE || A.dtype == GK_F64) return false;
  const int64_t es = A.dtype == GK_F32 ? 4 : 2;
  if ((uintptr_t)A.vals % 16 != 0 || (A.ld * es) % 16 != 0 || (A.n * es) % 16 != 0) return false;
  if (A.m < 1 || A.n * es > (int64_t)kFMaxCluster * kSMaxPiece * 16) return false;
  FusedPlan pl;
  return cached_plan(A, d, &pl);
}

// the plan depends on the storage type and n only (not on where the operator lives)
int fused_cluster(const Op &A, const Dev &d) {
  FusedPlan pl;
  if (A.kind != GK_DENSE || A.dtype == GK_F64 || !cached_plan(A, d, &pl)) return 0;
  return pl.Q;
}

int64_t fused_partials(const Op &A, const Dev &d) {
  FusedPlan pl;
  if (A.kind != GK_DENSE || A.dtype == GK_F64 || !cached_plan(A, d, &pl)) return 0;
  return (int64_t)pl.NC * A.n;
}

cudaError_t fused_matvec(const Op &A, const float *x32, double *w, const double *sub, const double *coef,
                         double *zpart, Ctl *ctl, cudaStream_t s, const Dev &d) {
  FusedPlan pl;
  if (!fused_ok(A, d) || !cached_plan(A, d, &pl)) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.NC * pl.Q, 1, 1);
  cfg.blockDim = dim3(kSThreads, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pl.Q;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e;
  switch (A.dtype) {
    case GK_F32:
      e = cudaLaunchKernelEx(&cfg, k_fused<float>, (const float *)A.vals, A.m, A.n, A.ld, A.scale, x32, w, sub, coef,
                             zpart, pl.piece_vecs, ctl);
      break;
    case GK_BF16:
      e = cudaLaunchKernelEx(&cfg, k_fused<__nv_bfloat16>, (const __nv_bfloat16 *)A.vals, A.m, A.n, A.ld, A.scale,
                             x32, w, sub, coef, zpart, pl.piece_vecs, ctl);
      break;
    default:
      e = cudaLaunchKernelEx(&cfg, k_fused<__half>, (const __half *)A.vals, A.m, A.n, A.ld, A.scale, x32, w, sub,
                             coef, zpart, pl.piece_vecs, ctl);
      break;
  }
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

cudaError_t fused_finish(const Op &A, const double *zpart, const double *coef, const double *sub, double *z,
                         const Ctl *ctl, cudaStream_t s, const Dev &d) {
  FusedPlan pl;
  if (!fused_ok(A, d) || !cached_plan(A, d, &pl)) return cudaErrorNotSupported;
  int64_t blocks = (A.n + 255) / 256;
  if (blocks > 4 * (int64_t)d.sms) blocks = 4 * (int64_t)d.sms;
  GK_LAUNCH(k_fused_finish<<<(int)blocks, 256, 0, s>>>(zpart, pl.NC, A.n, A.scale, coef, sub, z, ctl));
  return cudaGetLastError();
}

}  // namespace gk
