// gk_predict.cu -- the learned predictor behind the C ABI: weights loaded once into device
// memory (gk_predictor_load), the network's (log r, log K) for a set of operators from their
// sketch features (gk_predictor_predict), the Krylov dimension of a single partial SVD, and the
// learned batched pipeline: predicted (rank, K), one batched partial SVD with the rank cut,
// each problem judged by its own spectrum, the rejected ones re-solved by the plain pipeline
// (Algorithm 3 for the rank, then the partial SVD).  The paper has no counterpart; the
// decisions here are host logic around the library's kernels (sketch, MLP forward in bf16
// weights, the batched solvers).
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "gk_internal.cuh"

struct gk_predictor {
  float *params;  // GK_MLP_PARAMS f32, device
  int device;
};

namespace gk {

void margins(double rf, double kf, int64_t mn, int cap, int *r_out, int *K_out);

namespace {

constexpr uint64_t kSketchSeed = 0x5E7C4;  // the seed the committed weights were trained with
constexpr int kKLimit = 500;               // largest Krylov dimension a prediction may ask for

__global__ void k_gather_first(const double *const *__restrict__ ptrs, int count, double *__restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = ptrs[i] ? ptrs[i][0] : 0.0;
}

}  // namespace

// r^ = ceil(1.05 rf) + 1, K^ = ceil(kf) + 2 shifted by the same margin, clamped to
// 1 <= r^ <= cap, r^ + 2 <= K^ <= min(mn, 500) where there is room (a non-finite estimate asks
// for the whole range)
void margins(double rf, double kf, int64_t mn, int cap, int *r_out, int *K_out) {
  const int64_t lim = mn < kKLimit ? mn : kKLimit;
  if (!isfinite(rf)) rf = (double)lim;
  if (!isfinite(kf)) kf = (double)lim;
  int64_t ri = (int64_t)ceil(1.05 * rf) + 1;
  if (ri < 1) ri = 1;
  const int64_t rmax = lim - 1 > 1 ? lim - 1 : 1;
  if (ri > rmax) ri = rmax;
  if (ri > cap) ri = cap;
  int64_t Ki = (int64_t)ceil(kf) + 2 + (ri - (int64_t)llround(rf));
  if (Ki < ri + 2) Ki = ri + 2;
  if (Ki > lim) Ki = lim;
  if (Ki < ri) Ki = ri;
  *r_out = (int)ri;
  *K_out = (int)Ki;
}

int predict_raw(const gk_predictor *p, const gk_matrix *A, int count, std::vector<float> &out, cudaStream_t s,
                int sketch_flags) {
  float *feat = nullptr;
  if (cudaMallocAsync((void **)&feat, sizeof(float) * (size_t)count * GK_FEATURES, s) != cudaSuccess) {
    cudaGetLastError();
    return GK_OUT_OF_MEMORY;
  }
  gk_opts o;
  gk_default_opts(&o);
  o.stream = s;
  // the tensor-core sketch where it applies (one bf16 operator whose rows the TMA can address)
  if ((sketch_flags & GK_FLAG_SKETCH_TC) && count == 1 && A[0].kind == GK_DENSE && A[0].dtype == GK_BF16 &&
      sketch_tc_ok(A[0].vals, A[0].m, A[0].n, A[0].ld))
    o.flags = GK_FLAG_SKETCH_TC;
  int rc = gk_sketch_batched(A, count, kSketchSeed, feat, &o);
  o.flags = 0;
  out.assign(2 * (size_t)count, 0.f);
  if (rc == GK_OK) rc = gk_mlp_forward(p->params, feat, count, out.data(), 1, &o);
  cudaFreeAsync(feat, s);
  cudaStreamSynchronize(s);
  return rc;
}

int predict_krylov(const gk_predictor *p, const gk_matrix *A, int k, cudaStream_t s, int *K, int sketch_flags) {
  std::vector<float> out;
  const int rc = predict_raw(p, A, 1, out, s, sketch_flags);
  if (rc) return rc;
  double kf = out[1];
  kf = kf < 0.0 ? 0.0 : (kf > 20.0 ? 20.0 : kf);
  int64_t Kp = (int64_t)ceil(exp(kf)) + 2;
  const int64_t mn = A->m < A->n ? A->m : A->n;
  if (Kp < k + 2) Kp = k + 2;
  if (Kp > mn) Kp = mn;
  if (Kp > kKLimit) Kp = kKLimit;
  if (Kp < k) Kp = k;
  *K = (int)Kp;
  return GK_OK;
}

// the learned batched partial SVD (see gk_psvd_batched with opts->predictor)
int learned_batched(gk_batch_item *items, int count, const gk_opts *oin, gk_info *info) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launch_count();
  if (info) memset(info, 0, sizeof(*info));
  gk_opts o = *oin;
  const gk_predictor *pred = o.predictor;
  o.predictor = nullptr;
  cudaStream_t s = (cudaStream_t)o.stream;
  for (int i = 0; i < count; ++i)
    if (items[i].k < 1 || !(items[i].rank_cut > 0.0 && items[i].rank_cut < 1.0) || !items[i].U || !items[i].S ||
        !items[i].V)
      return GK_INVALID_ARG;
  std::vector<gk_matrix> mats(count);
  for (int i = 0; i < count; ++i) mats[i] = items[i].A;
  std::vector<float> out;
  int rc = predict_raw(pred, mats.data(), count, out, s, 0);
  if (rc) return rc;
  // one batched partial SVD at the predicted (rank, K) with the rank cut
  std::vector<gk_batch_item> run(items, items + count);
  std::vector<int> rhat(count);
  for (int i = 0; i < count; ++i) {
    const double rf = exp(fmin(fmax((double)out[2 * i], -20.0), 20.0));
    const double kf = exp(fmin(fmax((double)out[2 * i + 1], -20.0), 20.0));
    const int64_t mn = items[i].A.m < items[i].A.n ? items[i].A.m : items[i].A.n;
    int r, K;
    margins(rf, kf, mn, items[i].k, &r, &K);
    rhat[i] = r;
    run[i].k = r;
    if (items[i].krylov_dim <= 0) run[i].krylov_dim = K;
  }
  gk_info i1;
  const int st1 = gk_psvd_batched(run.data(), count, &o, &i1);
  if (st1 < 0) return st1;
  // the judge: some Ritz value of the last projected matrix fell below the cut (rank < r^, or
  // theta_{r^+1} <= eps theta_1); otherwise r^ was too small and the plain pipeline re-solves it
  std::vector<double> s1(count, 0.0);
  {
    std::vector<const double *> ptrs(count);
    for (int i = 0; i < count; ++i) ptrs[i] = items[i].S;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, sizeof(double *) * count + sizeof(double) * count + 256, s) != cudaSuccess) {
      cudaGetLastError();
      return GK_OUT_OF_MEMORY;
    }
    const double **dp = (const double **)buf;
    double *dv = (double *)(buf + (sizeof(double *) * count + 255) / 256 * 256);
    cudaMemcpyAsync(dp, ptrs.data(), sizeof(double *) * count, cudaMemcpyHostToDevice, s);
    GK_LAUNCH(k_gather_first<<<(count + 255) / 256, 256, 0, s>>>(dp, count, dv));
    cudaMemcpyAsync(s1.data(), dv, sizeof(double) * count, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    if (e != cudaSuccess) return GK_CUDA_ERROR;
  }
  std::vector<int> redo;
  for (int i = 0; i < count; ++i) {
    const bool seen_below = run[i].rank < rhat[i] || run[i].sigma_next <= items[i].rank_cut * s1[i];
    if (run[i].status != GK_OK || !seen_below) redo.push_back(i);
  }
  gk_info i2, i3;
  memset(&i2, 0, sizeof(i2));
  memset(&i3, 0, sizeof(i3));
  int st2 = GK_OK, st3 = GK_OK;
  if (!redo.empty()) {
    // the plain pipeline: Algorithm 3 for the rank, then the partial SVD with the default K
    std::vector<gk_batch_item> nr(redo.size()), ps(redo.size());
    for (size_t j = 0; j < redo.size(); ++j) {
      const gk_batch_item &it = items[redo[j]];
      memset(&nr[j], 0, sizeof(gk_batch_item));
      nr[j].A = it.A;
      const int64_t mn = it.A.m < it.A.n ? it.A.m : it.A.n;
      nr[j].k = (int)(mn < 160 ? mn : 160);
      nr[j].tol = it.rank_cut;
      nr[j].start = it.start;
    }
    st2 = gk_numrank_batched(nr.data(), (int)nr.size(), &o, &i2);
    if (st2 < 0) return st2;
    for (size_t j = 0; j < redo.size(); ++j) {
      const gk_batch_item &it = items[redo[j]];
      ps[j] = it;
      int r = nr[j].rank > 1 ? nr[j].rank : 1;
      if (r > it.k) r = it.k;
      ps[j].k = r;
      ps[j].krylov_dim = 0;
      ps[j].rank_cut = 0.0;
    }
    st3 = gk_psvd_batched(ps.data(), (int)ps.size(), &o, &i3);
    if (st3 < 0) return st3;
    for (size_t j = 0; j < redo.size(); ++j) {
      const int i = redo[j];
      const int64_t mv = run[i].matvecs + nr[j].matvecs;
      run[i] = ps[j];
      run[i].rank = ps[j].k;
      run[i].matvecs += mv;
    }
  }
  int worst = GK_OK;
  for (int i = 0; i < count; ++i) {
    gk_batch_item &it = items[i];
    const gk_batch_item &r = run[i];
    it.status = r.status;
    it.rank = r.rank > 1 ? r.rank : 1;
    it.steps = r.steps;
    it.restarts = r.restarts;
    it.cycles = r.cycles;
    it.breakdowns = r.breakdowns;
    it.matvecs = r.matvecs + 1;  // + the sketch's pass over A
    it.resid_est_max = r.resid_est_max;
    it.sigma_est = r.sigma_est;
    it.sigma_next = r.sigma_next;
    if (r.status < 0)
      worst = r.status;
    else if (worst == GK_OK && r.status != GK_OK)
      worst = r.status;
  }
  if (info) {
    gk_info inf = i1;
    inf.matvecs = i1.matvecs + i2.matvecs + i3.matvecs + count;
    inf.steps = i1.steps + i3.steps;
    inf.restarts = i1.restarts + i3.restarts;
    inf.cycles = i1.cycles + i3.cycles;
    inf.fallbacks = (int32_t)redo.size();
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    inf.launches = launch_count() - l0;
    *info = inf;
  }
  return worst;
}

}  // namespace gk

extern "C" int gk_predictor_load(const void *weights, size_t bytes, gk_predictor **pred) {
  if (!pred) return GK_INVALID_ARG;
  *pred = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    return GK_NO_DEVICE;
  }
  if (!weights || bytes != sizeof(float) * GK_MLP_PARAMS) return GK_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GK_NO_DEVICE;
  gk_predictor *p = new gk_predictor;
  p->device = dev;
  p->params = nullptr;
  if (cudaMalloc((void **)&p->params, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return GK_OUT_OF_MEMORY;
  }
  if (cudaMemcpy(p->params, weights, bytes, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->params);
    delete p;
    return GK_CUDA_ERROR;
  }
  // every parameter must be finite (a truncated or foreign file is refused)
  std::vector<float> h(GK_MLP_PARAMS);
  if (cudaMemcpy(h.data(), p->params, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaFree(p->params);
    delete p;
    return GK_CUDA_ERROR;
  }
  for (float v : h)
    if (!isfinite(v)) {
      cudaFree(p->params);
      delete p;
      return GK_INVALID_ARG;
    }
  *pred = p;
  return GK_OK;
}

extern "C" int gk_predictor_margins(double rf, double kf, int64_t mn, int cap, int *r, int *K) {
  if (!r || !K || mn < 1 || cap < 1) return GK_INVALID_ARG;
  gk::margins(rf, kf, mn, cap, r, K);
  return GK_OK;
}

extern "C" int gk_predictor_free(gk_predictor *pred) {
  if (!pred) return GK_INVALID_ARG;
  cudaFree(pred->params);
  delete pred;
  return GK_OK;
}

extern "C" int gk_predictor_predict(const gk_predictor *pred, const gk_matrix *A, int count, float *out,
                                    const gk_opts *opts) {
  if (!pred || !A || count <= 0 || !out) return GK_INVALID_ARG;
  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  std::vector<float> h;
  const int rc = gk::predict_raw(pred, A, count, h, s, 0);
  if (rc) return rc;
  if (cudaMemcpy(out, h.data(), sizeof(float) * 2 * (size_t)count, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return GK_CUDA_ERROR;
  }
  return GK_OK;
}
