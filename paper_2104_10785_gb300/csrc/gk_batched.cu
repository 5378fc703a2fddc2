// gk_batched.cu -- host driver of the batched persistent solver (the kernel and its device
// routines are in gk_batched_kernel.cuh, instantiated per storage type in gk_batched_<type>.cu),
// and the bounded-wait self-test kernel.
#include "gk_batched_kernel.cuh"

namespace gk {
namespace {

// The bounded wait on its own: one CTA waits on an mbarrier that nothing arrives at, with a
// limit of `limit` SM clock cycles, and records in *out whether it gave up (1) or saw the
// phase complete (0).  No copy is in flight, so returning after the limit is safe.
__global__ void k_wait_probe(long long limit, int *out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit);
  const int bad = __syncthreads_or(!ok);
  if (threadIdx.x == 0) *out = bad;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool dense_ok(const gk_matrix &A) {
  return A.kind == GK_DENSE && A.m > 0 && A.n > 0 && A.n <= kNMax && A.ld >= A.n && A.vals && A.dtype >= GK_F64 &&
         A.dtype <= GK_F16 && A.scale == A.scale && A.scale != 0.0 && A.m <= INT32_MAX;
}

size_t esz(int dtype) { return dtype == GK_F64 ? 8 : (dtype == GK_F32 ? 4 : 2); }

struct TuneKey {
  int count, mode, dtype;
  int64_t work;
  bool operator<(const TuneKey &o) const {
    return std::tie(count, mode, dtype, work) < std::tie(o.count, o.mode, o.dtype, o.work);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;  // cluster size chosen by the autotuner per batch signature

using BatchedKernel = void (*)(const BProb *, const int *, int, int *, char *, size_t, BDims, BRes *);

BatchedKernel kernel_for(int dtype) {
  const void *k = dtype == GK_F64    ? batched_kernel_f64()
                  : dtype == GK_F32  ? batched_kernel_f32()
                  : dtype == GK_BF16 ? batched_kernel_bf16()
                                     : batched_kernel_f16();
  return reinterpret_cast<BatchedKernel>(const_cast<void *>(k));
}

int launch_batched(BatchedKernel kern, int cs, const BProb *dprobs, const int *dorder, int count, int *dnext, char *dws,
                   size_t stride, const BDims &D, BRes *dres, int nclusters, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * cs, 1, 1);
  cfg.blockDim = dim3(kBThreads, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaMemsetAsync(dnext, 0, 2 * sizeof(int), s) != cudaSuccess) return GK_CUDA_ERROR;
  if (cudaLaunchKernelEx(&cfg, kern, dprobs, dorder, count, dnext, dws, stride, D, dres) != cudaSuccess)
    return GK_CUDA_ERROR;
  note_launch();
  return GK_OK;
}

int max_clusters(BatchedKernel kern, int cs, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kBThreads, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int batched_impl(gk_batch_item *items, int count, int mode, const gk_opts *oin, gk_info *info, int cs_force = 0) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launch_count();
  if (info) memset(info, 0, sizeof(*info));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return GK_NO_DEVICE;
  }
  if (!items || count <= 0) return GK_INVALID_ARG;
  gk_opts o;
  if (oin)
    o = *oin;
  else
    gk_default_opts(&o);
  if (o.reorth_passes < 0 || o.reorth_passes > 3 || o.max_restarts < 0) return GK_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)o.stream;
  const int dtype_all = items[0].A.dtype;
  for (int i = 0; i < count; ++i)
    if (items[i].A.dtype != dtype_all) return GK_INVALID_ARG;  // one storage type per batch
  if (dtype_all < GK_F64 || dtype_all > GK_F16) return GK_INVALID_ARG;
  const BatchedKernel kern = kernel_for(dtype_all);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return GK_CUDA_ERROR;
  }
  // problem table and the dimensions of the per-cluster workspace
  std::vector<BProb> probs(count);
  std::vector<double> cost(count);
  BDims D{32, 32, 2, 2};
  int dtype0 = items[0].A.dtype;
  int64_t work = 0;
  for (int i = 0; i < count; ++i) {
    const gk_batch_item &it = items[i];
    if (!dense_ok(it.A)) return GK_INVALID_ARG;
    if (!(it.tol >= 0.0)) return GK_INVALID_ARG;
    if (mode == 0 && !(it.rank_cut >= 0.0 && it.rank_cut < 1.0)) return GK_INVALID_ARG;
    const int64_t m = it.A.m, n = it.A.n, mn = m < n ? m : n;
    BProb &P = probs[i];
    memset(&P, 0, sizeof(P));
    P.A = it.A.vals;
    P.dtype = it.A.dtype;
    P.mode = mode;
    P.m = m;
    P.n = n;
    P.ld = it.A.ld;
    P.scale = it.A.scale;
    P.tol = it.tol;
    P.passes = o.reorth_passes;
    P.max_restarts = o.max_restarts;
    P.prof = (o.flags & GK_FLAG_PROFILE) ? 1 : 0;
    P.eps_rel = o.eps_absolute ? 0 : 1;
    P.start = it.start;
    P.cut = mode == 0 ? it.rank_cut : 0.0;
    P.seed = o.seed + (uint64_t)i;
    P.out = i;
    int cols;
    if (mode == 0) {
      const int k = it.k;
      if (k < 1 || k > mn || !it.U || !it.S || !it.V) return GK_INVALID_ARG;
      int K = it.krylov_dim;
      if (K <= 0) {
        int64_t d = 2 * (int64_t)k;
        if (d < k + 16) d = k + 16;
        if (d > mn) d = mn;
        K = (int)d;
      }
      if (K < k || K > mn || (K == k && K < mn) || K > kKMax - 2) return GK_INVALID_ARG;
      int keep = k + (K - k) / 2;
      if (keep >= K) keep = K - 1;
      if (keep < 0) keep = 0;
      P.k = k;
      P.K = K;
      P.keep = keep;
      P.U = it.U;
      P.S = it.S;
      P.V = it.V;
      cols = K + 1;
      D.K = std::max(D.K, K);
    } else {
      int km = it.k;
      if (km <= 0 || km > mn) km = (int)std::min<int64_t>(mn, 256);
      if (km > kKMax - 2) km = kKMax - 2;
      P.K = km;
      P.S = it.S;
      cols = km + 2;
      D.K = std::max(D.K, km + 2);
    }
    D.ldu = std::max<int64_t>(D.ldu, round_up(m, 32));
    D.ldv = std::max<int64_t>(D.ldv, round_up(n, 32));
    D.cols = std::max(D.cols, cols);
    // cost model: the passes over A dominate, plus f64 Gram-Schmidt over the basis
    const double kk = mode == 0 ? 2.0 * P.K : 1.2 * P.K;
    cost[i] = (double)m * n * esz(P.dtype) * kk + 8.0 * (m + n) * (double)P.K * P.K * 1.5;
    work += m * n;
    if (P.dtype != dtype0) dtype0 = -1;
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

  // cluster size: the caller's (a single solve takes the largest cluster that fits), the
  // autotuned choice for this batch signature, else 8
  const TuneKey key{count, mode, dtype0, work};
  int cs = 8;
  bool tune = (o.flags & GK_FLAG_AUTOTUNE) != 0;
  if (cs_force > 0) {
    for (int c = cs_force; c >= 2; c /= 2)
      if (max_clusters(kern, c, s) > 0) {
        cs = c;
        break;
      }
    tune = false;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto itk = g_tuned.find(key);
    if (cs_force <= 0 && itk != g_tuned.end()) {
      cs = itk->second;
      tune = false;
    }
  }
  const int cands[4] = {2, 4, 8, 16};
  int ncl_max = 0;
  for (int c : cands) ncl_max = std::max(ncl_max, max_clusters(kern, c, s));
  if (ncl_max <= 0) return GK_CUDA_ERROR;
  const size_t stride = al256(work_bytes(D));
  const int ncl_alloc = std::min(count, ncl_max);
  const size_t bytes = al256(sizeof(BProb) * count) + al256(sizeof(int) * count) + 256 +
                       al256(sizeof(BRes) * count) + stride * ncl_alloc;
  void *base = nullptr;
  if (o.workspace) {
    if (o.workspace_bytes < bytes) return GK_OUT_OF_MEMORY;
    base = o.workspace;
  } else if (cudaMallocAsync(&base, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  char *p = (char *)base;
  BProb *dprobs = (BProb *)p;
  p += al256(sizeof(BProb) * count);
  int *dorder = (int *)p;
  p += al256(sizeof(int) * count);
  int *dnext = (int *)p;
  p += 256;
  BRes *dres = (BRes *)p;
  p += al256(sizeof(BRes) * count);
  char *dws = p;
  int rc = GK_OK;
  int herr = 0, ncl_used = 0;
  std::vector<BRes> res(count);
  do {
    if (cudaMemcpyAsync(dprobs, probs.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dorder, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      rc = GK_CUDA_ERROR;
      break;
    }
    if (tune) {
      // autotuner: time the whole batch once per candidate cluster size, keep the fastest
      float best = 1e30f;
      int best_cs = cs;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int c : cands) {
        const int ncl = std::min(count, max_clusters(kern, c, s));
        if (ncl <= 0) continue;
        cudaEventRecord(e0, s);
        if (launch_batched(kern, c, dprobs, dorder, count, dnext, dws, stride, D, dres, ncl, s) != GK_OK) {
          cudaGetLastError();
          continue;
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_cs = c;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cs = best_cs;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tuned[key] = cs;
    }
    const int ncl = std::min(count, max_clusters(kern, cs, s));
    if (ncl <= 0) {
      rc = GK_CUDA_ERROR;
      break;
    }
    ncl_used = ncl;
    rc = launch_batched(kern, cs, dprobs, dorder, count, dnext, dws, stride, D, dres, ncl, s);
    if (rc) break;
    if (cudaMemcpyAsync(res.data(), dres, sizeof(BRes) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&herr, dnext + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = GK_CUDA_ERROR;
      break;
    }
  } while (0);
  if (!o.workspace) {
    cudaFreeAsync(base, s);
    cudaStreamSynchronize(s);
  }
  if (rc) return rc;
  if (herr) return GK_TIMEOUT;  // a bulk-copy wait gave up: results are not trustworthy
  int worst = GK_OK;
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  int clock_khz = 0, dev_id = 0;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev_id);
  const double ms_per_cycle = clock_khz > 0 ? 1.0 / clock_khz : 0.0;
  for (int i = 0; i < count; ++i) {
    gk_batch_item &it = items[i];
    const BRes &r = res[i];
    it.status = r.status;
    it.rank = r.rank;
    it.steps = r.steps;
    it.restarts = r.restarts;
    it.cycles = r.cycles;
    it.breakdowns = r.breakdowns;
    it.matvecs = r.matvecs;
    it.resid_est_max = r.resid_est;
    it.sigma_est = r.sigma_est;
    it.sigma_next = r.sigma_next;
    if (r.status < 0)
      worst = r.status;
    else if (worst == GK_OK && r.status != GK_OK)
      worst = r.status;
    inf.matvecs += r.matvecs;
    inf.steps += r.steps;
    inf.restarts += r.restarts;
    inf.cycles += r.cycles;
    inf.breakdowns += r.breakdowns;
    inf.svd_sweeps = std::max(inf.svd_sweeps, r.sweeps < 0 ? -r.sweeps : r.sweeps);
    inf.resid_est_max = std::max(inf.resid_est_max, r.resid_est);
    inf.ms_matvec += r.cyc[0] * ms_per_cycle;
    inf.ms_matvec_t += r.cyc[1] * ms_per_cycle;
    inf.ms_orth += r.cyc[2] * ms_per_cycle;
    inf.ms_small += r.cyc[3] * ms_per_cycle;
    inf.ms_restart += r.cyc[4] * ms_per_cycle;
  }
  inf.reserved = cs;    // cluster size used
  inf.kprime = ncl_used;  // clusters launched
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  inf.launches = launch_count() - l0;
  if (info) *info = inf;
  return worst;
}

}  // namespace

int psvd_persistent(gk_batch_item *item, const gk_opts *opts, gk_info *info) {
  return batched_impl(item, 1, 0, opts, info, 16);
}

}  // namespace gk

extern "C" int gk_wait_selftest(long long cycles) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return GK_NO_DEVICE;
  }
  if (cycles < 0 || cycles > 4000000000ll) return GK_INVALID_ARG;  // at most about 2 s
  int *d = nullptr, h = -1;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  gk::k_wait_probe<<<1, 64>>>(cycles, d);
  gk::note_launch();
  const cudaError_t e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GK_CUDA_ERROR;
  }
  return h ? GK_TIMEOUT : GK_OK;
}

extern "C" int gk_psvd_batched(gk_batch_item *items, int count, const gk_opts *opts, gk_info *info) {
  if (opts && opts->predictor) return gk::learned_batched(items, count, opts, info);
  return gk::batched_impl(items, count, 0, opts, info);
}

extern "C" int gk_numrank_batched(gk_batch_item *items, int count, const gk_opts *opts, gk_info *info) {
  return gk::batched_impl(items, count, 1, opts, info);
}
