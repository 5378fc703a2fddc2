// gk_fused.cu -- the fused sweep: one pass over a dense operator per bidiagonalization
// step produces both products of the step.
//
// A Golub-Kahan step (Eq. 2.2; Algorithm 1) needs w = A x - c sub (the left vector
// before reorthogonalization) and then A^T u with u = (w - U h) / ||w - U h|| (h the
// Gram-Schmidt coefficients).  A^T u = (A^T w - A^T U h) / ||.||, and A^T U lies in the
// span of the right basis (A^T u_i = alpha_i v_i + beta_i v_{i+1}), which the right
// Gram-Schmidt removes anyway; so the sweep can form A^T w while w is produced, from the
// same bytes of A, and divide by the norm afterwards.  That halves the operator traffic
// of a step (one pass instead of two).
//
// Layout: a thread-block cluster of Q CTAs owns a set of row blocks (rows kFRows at a
// time, row block b goes to cluster b mod #clusters); CTA q of the cluster owns one tile
// of columns (a contiguous run of 16-byte vectors) for the whole launch.
//   producer warp : cp.async.bulk of the CTA's piece of each row of a stage (row block) into
//                   a kFStages-deep shared-memory ring (mbarrier complete_tx), bounded waits
//                   for free slots;
//   8 consumer warps, each on its own (no block-wide barrier in the loop), per stage s:
//     (a) the warp's partial dot product of each row with x (f32 products over at most 24
//         columns per lane, a warp tree in f32), stored as one 16-byte remote store into every
//         CTA of the cluster and announced by a remote mbarrier arrive (release, cluster scope);
//     (b) the A^T w update of stage s - kFLag: the wait (acquire, cluster scope) for that stage's
//         8 Q warp partials -- posted a stage earlier, so the exchange hides behind (a) -- their
//         sum in a fixed order (every warp of every CTA forms the same w_r), then a_rc * w_r
//         added for the warp's columns (f32 runs of 64 rows, combined in f64 registers); the
//         last warp through releases the ring slot.
// The partial sums live in 2 kFStages generations: a CTA can post stage s + 2 kFStages only
// after every CTA of the cluster has released stage s + kFStages, hence finished stage s.
// At the end every CTA writes its columns' f64 partial of A^T w for its cluster, and
// k_fused_finish sums the clusters' partials in a fixed order, divides by the new norm and
// subtracts the recurrence term: z = scale (A^T w) / alpha - alpha v.  Every reduction has a
// fixed order (bitwise reproducible).  Every wait is bounded; on expiry the kernel records
// a timeout in the control block, halts the sweep, lets its own copies land and meets its
// peers at the final cluster barrier, so no CTA leaves while another may still write into
// its shared memory.
#include "gk_internal.cuh"

namespace gk {

namespace {

constexpr int kFThreads = 256;                  // consumer threads (8 warps)
constexpr int kFWarps = kFThreads / 32;
constexpr int kFBlock = kFThreads + 32;         // + one producer warp
constexpr int kFRows = 4;                       // rows per stage
constexpr int kFStages = 5;                     // ring depth
constexpr int kFGen = 2 * kFStages;             // generations of the exchanged partial sums
constexpr int kFLag = 1;                        // stages between a stage's dots and its A^T w update
constexpr int kFVec = 3;                        // 16-byte vectors per consumer lane per row piece (at most)
constexpr int kFMaxPiece = 10240;               // bytes of one row piece (one CTA's columns of one row)
constexpr int kFRunRows = 64;                   // rows summed in f32 before an f64 combine (A^T w)
constexpr int kFMaxCluster = 16;
constexpr long long kFWaitCycles = 4000000000ll;  // ~2 s of SM clock before a wait gives up
static_assert(kFMaxPiece <= kFThreads * kFVec * 16, "a row piece must fit the consumers' vectors");

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
__device__ __forceinline__ void mbar_arrive_local(uint64_t *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar_addr) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}
// bounded wait for phase `parity` (CTA scope: the ring of bulk copies)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  const uint32_t a = saddr(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kFWaitCycles) return false;
  }
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
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
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

// w = scale * A x - coef * sub (rows of this cluster's row blocks; warp 0 of CTA 0 writes)
// zpart[cluster * n + col] = sum over those rows of a_{r,col} * f32(w_r)  (without scale)
// Dynamic shared memory: the ring (kFStages x kFRows x piece_vecs x 16 bytes), then the
// exchanged partials [kFGen][Q][kFWarps][kFRows] f32.
template <typename T>
__global__ void __launch_bounds__(kFBlock, 1)
    k_fused(const T *__restrict__ A, int64_t m, int64_t n, int64_t ld, double scale, const float *__restrict__ x,
            double *__restrict__ w, const double *__restrict__ sub, const double *__restrict__ coef,
            double *__restrict__ zpart, int piece_vecs, Ctl *ctl) {
  using VT = Vec<T>;
  using V = typename VT::V;
  constexpr int E = VT::E;
  extern __shared__ __align__(128) unsigned char ring[];
  __shared__ __align__(8) uint64_t full[kFStages], empty[kFStages], xbar[kFGen];
  __shared__ int64_t last_issued[kFStages];
  __shared__ int abort_flag;

  const int tid = threadIdx.x;
  const uint32_t q = cluster_rank(), Q = cluster_size(), cid = cluster_id(), NC = cluster_count();
  const int64_t nvec = n / E;  // n * sizeof(T) is a multiple of 16 (checked on the host)
  const int64_t v0 = (int64_t)q * piece_vecs;
  const int nloc = (int)(v0 >= nvec ? 0 : (nvec - v0 < piece_vecs ? nvec - v0 : piece_vecs));
  const unsigned piece_bytes = (unsigned)nloc * 16u;
  const size_t stage_bytes = (size_t)kFRows * (size_t)piece_vecs * 16u;
  float *part = reinterpret_cast<float *>(ring + (size_t)kFStages * stage_bytes);  // [kFGen][Q][kFWarps][kFRows]
  const int64_t nrb = (m + kFRows - 1) / kFRows;
  const int64_t ns = nrb > (int64_t)cid ? (nrb - (int64_t)cid + NC - 1) / NC : 0;  // stages of this cluster

  if (tid == 0) {
    for (int i = 0; i < kFStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kFWarps);
      last_issued[i] = -1;
    }
    for (int i = 0; i < kFGen; ++i) mbar_init(&xbar[i], kFWarps * Q);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // every CTA's barriers are initialized before any peer arrives on them
  cluster_sync_all();
  const bool skip = halted(ctl);  // the whole cluster reads the same flag: a halted sweep does nothing
  volatile int *abort_v = &abort_flag;

  if (tid >= kFThreads) {
    // producer: one elected lane issues the stages in order, then waits for its last copies
    if (tid == kFThreads && !skip) {
      for (int64_t s = 0; s < ns; ++s) {
        const int sl = (int)(s % kFStages);
        if (s >= kFStages && !mbar_wait(&empty[sl], (unsigned)(((s / kFStages) - 1) & 1))) {
          record_timeout(ctl, 2);
          *abort_v = 1;
          break;
        }
        const int64_t r0 = ((int64_t)cid + s * (int64_t)NC) * kFRows;
        const int rows = (int)((m - r0) < kFRows ? (m - r0) : kFRows);
        mbar_expect_tx(&full[sl], piece_bytes * (unsigned)rows);
        last_issued[sl] = s;
        if (piece_bytes)
          for (int r = 0; r < rows; ++r)
            bulk_g2s(ring + (size_t)sl * stage_bytes + (size_t)r * piece_vecs * 16, A + (r0 + r) * ld + v0 * E,
                     piece_bytes, &full[sl]);
      }
      // no copy may still be landing when the CTA leaves (each slot's last phase is the only one
      // that can be pending: the next one was never issued)
      for (int i = 0; i < kFStages; ++i)
        if (last_issued[i] >= 0) mbar_wait(&full[i], (unsigned)((last_issued[i] / kFStages) & 1));
    }
  } else if (!skip) {
    const int warp = tid >> 5, lane = tid & 31;
    const double c = sub ? *coef : 0.0;
    // this lane's x values (vectors tid, tid + 256, tid + 512 of the CTA's piece)
    float xr[kFVec][E];
    float z32[kFVec][E];
    double z64[kFVec][E];
#pragma unroll
    for (int i = 0; i < kFVec; ++i) {
      const int vl = tid + i * kFThreads;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        z32[i][e] = 0.f;
        z64[i][e] = 0.0;
        xr[i][e] = 0.f;
      }
      if (vl < nloc) {
#pragma unroll
        for (int h = 0; h < E / 4; ++h) {
          const float4 xx = __ldg(reinterpret_cast<const float4 *>(x + (v0 + vl) * E) + h);
          xr[i][4 * h + 0] = xx.x;
          xr[i][4 * h + 1] = xx.y;
          xr[i][4 * h + 2] = xx.z;
          xr[i][4 * h + 3] = xx.w;
        }
      }
    }
    int run = 0;
    bool ok = true;
    // sub entry of row rr of the stage being summed next (prefetched one stage ahead)
    double sub_next = 0.0;
    {
      const int rr = lane >> 3;
      const int64_t r0n = (int64_t)cid * kFRows + rr;
      if (sub && (lane & 7) == 0 && r0n < m && ns > 0) sub_next = sub[r0n];
    }
    // (b) for stage t: the exchanged partials -> w_r, then the A^T w update; releases the slot
    auto zstage = [&](int64_t t) -> bool {
      const int sl = (int)(t % kFStages), g = (int)(t % kFGen);
      const int64_t r0 = ((int64_t)cid + t * (int64_t)NC) * kFRows;
      const int rows = (int)((m - r0) < kFRows ? (m - r0) : kFRows);
      const int rr = lane >> 3, src = lane & 7;  // this lane sums row rr's partials of source warp src
      const double sv = sub_next;
      {  // the next stage's entry of sub, loaded while this one is summed
        const int64_t rn = ((int64_t)cid + (t + 1) * (int64_t)NC) * kFRows + rr;
        sub_next = (sub && src == 0 && rr < kFRows && rn < m && t + 1 < ns) ? sub[rn] : 0.0;
      }
      if (!mbar_wait_cluster(&xbar[g], (unsigned)((t / kFGen) & 1))) return false;
      if (!mbar_wait(&full[sl], (unsigned)((t / kFStages) & 1))) return false;  // complete: orders the staged bytes
      // the row's 8 Q warp partials in double-f32 (every rounding error kept), fixed order: the
      // total is then rounded once, to f64
      float hi = 0.f, lo = 0.f;
      for (uint32_t p = 0; p < Q; ++p) df_add(hi, lo, part[(((size_t)g * Q + p) * kFWarps + src) * kFRows + rr]);
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        // combine so that both lanes of the pair compute the same sum (lower lane's value first)
        const bool first = (lane & o) == 0;
        float s, e;
        two_sum(first ? hi : h2, first ? h2 : hi, s, e);
        hi = s;
        lo = __fadd_rn(__fadd_rn(first ? lo : l2, first ? l2 : lo), e);
      }
      float wv32 = 0.f;
      if ((lane & 7) == 0 && rr < rows) {
        const double wv = ((double)hi + (double)lo) * scale - c * sv;
        wv32 = (float)wv;
        if (q == 0 && warp == 0) w[r0 + rr] = wv;
      }
      float wr[kFRows];
#pragma unroll
      for (int r = 0; r < kFRows; ++r) wr[r] = __shfl_sync(0xffffffffu, wv32, r * 8);
      const unsigned char *st = ring + (size_t)sl * stage_bytes;
#pragma unroll
      for (int r = 0; r < kFRows; ++r) {
        if (r < rows) {
          const V *row = reinterpret_cast<const V *>(st + (size_t)r * piece_vecs * 16);
#pragma unroll
          for (int i = 0; i < kFVec; ++i) {
            const int vl = tid + i * kFThreads;
            if (vl < nloc) {
              float f[E];
              VT::unpack(row[vl], f);
#pragma unroll
              for (int e = 0; e < E; ++e) z32[i][e] = fmaf(f[e], wr[r], z32[i][e]);
            }
          }
        }
      }
      run += rows;
      if (run >= kFRunRows) {
#pragma unroll
        for (int i = 0; i < kFVec; ++i)
#pragma unroll
          for (int e = 0; e < E; ++e) {
            z64[i][e] += (double)z32[i][e];
            z32[i][e] = 0.f;
          }
        run = 0;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&empty[sl]);
      return true;
    };

    int64_t zdone = 0;  // stages whose A^T w update is done
    for (int64_t s = 0; s < ns && ok; ++s) {
      if (*abort_v) {
        ok = false;
        break;
      }
      const int sl = (int)(s % kFStages), g = (int)(s % kFGen);
      if (!mbar_wait(&full[sl], (unsigned)((s / kFStages) & 1))) {
        ok = false;
        break;
      }
      const int64_t r0 = ((int64_t)cid + s * (int64_t)NC) * kFRows;
      const int rows = (int)((m - r0) < kFRows ? (m - r0) : kFRows);
      // (a) this warp's partial dot of each row of the stage with x
      float d[kFRows];
      const unsigned char *st = ring + (size_t)sl * stage_bytes;
#pragma unroll
      for (int r = 0; r < kFRows; ++r) {
        d[r] = 0.f;
        if (r < rows) {
          const V *row = reinterpret_cast<const V *>(st + (size_t)r * piece_vecs * 16);
#pragma unroll
          for (int i = 0; i < kFVec; ++i) {
            const int vl = tid + i * kFThreads;
            if (vl < nloc) {
              float f[E];
              VT::unpack(row[vl], f);
#pragma unroll
              for (int e = 0; e < E; ++e) d[r] = fmaf(f[e], xr[i][e], d[r]);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kFRows; ++r) d[r] = warp_sum_f(d[r]);
      // one 16-byte remote store and one remote arrive per peer (lane p serves CTA p)
      if (lane < (int)Q) {
        const uint32_t dst = peer_addr(saddr(part + (((size_t)g * Q + q) * kFWarps + warp) * kFRows), (uint32_t)lane);
        asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "f"(d[0]), "f"(d[1]), "f"(d[2]),
                     "f"(d[3])
                     : "memory");
        mbar_arrive_remote(peer_addr(saddr(&xbar[g]), (uint32_t)lane));
      }
      // (b) the update of the stage kFLag back, whose exchange has had a stage to complete
      if (s >= kFLag) {
        if (!zstage(s - kFLag)) {
          ok = false;
          break;
        }
        zdone = s - kFLag + 1;
      }
    }
    for (int64_t t = zdone; ok && t < ns; ++t) {
      if (*abort_v || !zstage(t)) ok = false;
    }
    if (ok) {
      // this CTA's columns of the cluster's partial A^T w (each warp its own vectors)
#pragma unroll
      for (int i = 0; i < kFVec; ++i) {
        const int vl = tid + i * kFThreads;
        if (vl < nloc) {
          double *zp = zpart + (int64_t)cid * n + (v0 + vl) * E;
#pragma unroll
          for (int e = 0; e < E; ++e) zp[e] = z64[i][e] + (double)z32[i][e];
        }
      }
    } else {
      if (lane == 0) record_timeout(ctl, 1);
      *abort_v = 1;
    }
  }
  // no CTA leaves while a peer may still store into its shared memory
  __syncwarp();
  cluster_sync_all();
}

// z[c] = scale * (sum over clusters of zpart[cl * n + c]) / alpha - alpha * sub[c], alpha = *coef
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
  const int64_t nvec = A.n * (int64_t)sizeof(T) / 16;
  auto kern = k_fused<T>;
  static int attr_dev = -1;
  if (attr_dev != d.id) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kFStages * kFRows * kFMaxPiece +
                                             kFGen * kFMaxCluster * kFWarps * kFRows * (int)sizeof(float));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    attr_dev = d.id;
  }
  // among the cluster sizes whose column tile fits a ring slot, the one that keeps the most
  // SMs busy (clusters are placed within one GPC: sizes that do not divide a GPC idle SMs)
  int best_active = 0;
  for (int Q = 1; Q <= kFMaxCluster; Q *= 2) {
    const int64_t pv = (nvec + Q - 1) / Q;
    if (pv * 16 > kFMaxPiece) continue;
    const size_t smem = (size_t)kFStages * kFRows * (size_t)pv * 16 +
                        (size_t)kFGen * Q * kFWarps * kFRows * sizeof(float);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Q, 1, 1);
    cfg.blockDim = dim3(kFBlock, 1, 1);
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
  if (A.m < 1 || A.n * es > (int64_t)kFMaxCluster * kFMaxPiece) return false;
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
  cfg.blockDim = dim3(kFBlock, 1, 1);
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
