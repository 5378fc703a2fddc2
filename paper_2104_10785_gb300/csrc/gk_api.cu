// gk_api.cu -- the C ABI of libgk.so and the host drivers of the two methods.
//
// gk_numrank: Algorithm 1 (lower-bidiagonal Golub-Kahan with reorthogonalization
//   and the break test) followed by the rank count of Algorithm 3.
// gk_psvd:    the upper-bidiagonal Golub-Kahan process from v1 = A^T q1/||A^T q1||
//   with thick restarts: each cycle extends the basis to K columns, takes the SVD
//   of the K x K projected matrix, tests the Ritz residuals |beta_K X_{K,i}| and
//   either returns the leading Ritz triplets or keeps `keep` of them plus
//   v_{K+1} and continues.
//
// The host only enqueues kernels.  Data-dependent decisions (break, breakdown,
// convergence) are taken on the device and recorded in a control block; after
// an event every later kernel of the sweep returns at entry, and the host reads
// the block once per chunk of steps (numrank) or once per cycle (psvd).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <mutex>
#include <vector>

#include <utility>

#include "gk_internal.cuh"

using namespace gk;

namespace gk {
namespace {
thread_local int64_t t_launches = 0;
}
void note_launch() { ++t_launches; }
int64_t launch_count() { return t_launches; }
}  // namespace gk

namespace {

thread_local char g_err[512] = "";

struct Status {
  int code;
};

#define GK_CUDA(x)                                                                                          \
  do {                                                                                                      \
    cudaError_t e_ = (x);                                                                                   \
    if (e_ != cudaSuccess) {                                                                                \
      snprintf(g_err, sizeof(g_err), "%s -> %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__);   \
      return GK_CUDA_ERROR;                                                                                 \
    }                                                                                                       \
  } while (0)

bool get_device(Dev *d) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    return false;
  }
  int id = 0;
  if (cudaGetDevice(&id) != cudaSuccess) return false;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, id) != cudaSuccess) return false;
  d->sms = sms;
  d->id = id;
  return true;
}

// true if p is host memory (pageable or pinned) rather than device/managed memory
bool on_host(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

size_t esize(int dtype) { return dtype == GK_F64 ? 8 : (dtype == GK_F32 ? 4 : 2); }

// bump allocator over the workspace (a null base only measures)
struct Carve {
  char *base;
  size_t off;
  template <class T>
  T *take(size_t count) {
    off = (off + 255) / 256 * 256;
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T) + 256;
    return p;
  }
};

gk_opts defaults() {
  gk_opts o;
  memset(&o, 0, sizeof(o));
  o.krylov_dim = 0;
  o.keep = 0;
  o.max_restarts = 200;
  o.reorth_passes = 0;
  o.eps_absolute = 0;
  o.flags = 0;
  o.seed = 2104107ull;
  o.start = nullptr;
  o.stream = nullptr;
  o.workspace = nullptr;
  o.workspace_bytes = 0;
  return o;
}

int check_matrix(const gk_matrix *A) {
  if (!A || A->m <= 0 || A->n <= 0 || !A->vals) return GK_INVALID_ARG;
  if (A->dtype < GK_F64 || A->dtype > GK_F16) return GK_INVALID_ARG;
  if (!(A->scale == A->scale) || A->scale == 0.0) return GK_INVALID_ARG;
  if (A->m > INT32_MAX || A->n > INT32_MAX) return GK_INVALID_ARG;
  if (A->kind == GK_DENSE) {
    if (A->ld < A->n) return GK_INVALID_ARG;
  } else if (A->kind == GK_CSR) {
    if (!A->rowptr || !A->colind || !A->t_vals || !A->t_rowptr || !A->t_colind) return GK_INVALID_ARG;
  } else {
    return GK_INVALID_ARG;
  }
  return GK_OK;
}

// number of stored entries of a CSR array (reads rowptr[rows])
int csr_nnz(const int32_t *rowptr, int64_t rows, int64_t *nnz) {
  int32_t v = 0;
  if (on_host(rowptr)) {
    v = rowptr[rows];
  } else {
    GK_CUDA(cudaMemcpy(&v, rowptr + rows, sizeof(int32_t), cudaMemcpyDeviceToHost));
  }
  if (v < 0) return GK_INVALID_ARG;
  *nnz = v;
  return GK_OK;
}

// Device copy of a host operator inside the workspace.
struct OpStage {
  bool host = false;
  int64_t nnz = 0, tnnz = 0;
  size_t vals_bytes = 0;
};

int stage_plan(const gk_matrix *A, OpStage *st) {
  st->host = on_host(A->vals);
  if (A->kind == GK_DENSE) {
    st->vals_bytes = (size_t)((A->m - 1) * A->ld + A->n) * esize(A->dtype);
  } else {
    int rc = csr_nnz(A->rowptr, A->m, &st->nnz);
    if (rc) return rc;
    rc = csr_nnz(A->t_rowptr, A->n, &st->tnnz);
    if (rc) return rc;
    if (st->nnz != st->tnnz) return GK_INVALID_ARG;
  }
  return GK_OK;
}

void stage_carve(const gk_matrix *A, const OpStage &st, Carve &cv, Op *op, char **dense_dst, void **v, int32_t **rp,
                 int32_t **ci, void **tv, int32_t **trp, int32_t **tci) {
  *dense_dst = nullptr;
  if (!st.host) return;
  if (A->kind == GK_DENSE) {
    *dense_dst = cv.take<char>(st.vals_bytes);
    op->vals = *dense_dst;
  } else {
    *v = cv.take<char>((size_t)st.nnz * esize(A->dtype));
    *rp = cv.take<int32_t>((size_t)A->m + 1);
    *ci = cv.take<int32_t>((size_t)st.nnz);
    *tv = cv.take<char>((size_t)st.nnz * esize(A->dtype));
    *trp = cv.take<int32_t>((size_t)A->n + 1);
    *tci = cv.take<int32_t>((size_t)st.nnz);
    op->vals = *v;
    op->rowptr = *rp;
    op->colind = *ci;
    op->t_vals = *tv;
    op->t_rowptr = *trp;
    op->t_colind = *tci;
  }
}

int stage_copy(const gk_matrix *A, const OpStage &st, const Op &op, cudaStream_t s) {
  if (!st.host) return GK_OK;
  if (A->kind == GK_DENSE) {
    GK_CUDA(cudaMemcpyAsync(const_cast<void *>(op.vals), A->vals, st.vals_bytes, cudaMemcpyHostToDevice, s));
  } else {
    const size_t es = esize(A->dtype);
    GK_CUDA(cudaMemcpyAsync(const_cast<void *>(op.vals), A->vals, st.nnz * es, cudaMemcpyHostToDevice, s));
    GK_CUDA(cudaMemcpyAsync(const_cast<int32_t *>(op.rowptr), A->rowptr, (A->m + 1) * 4, cudaMemcpyHostToDevice, s));
    GK_CUDA(cudaMemcpyAsync(const_cast<int32_t *>(op.colind), A->colind, st.nnz * 4, cudaMemcpyHostToDevice, s));
    GK_CUDA(cudaMemcpyAsync(const_cast<void *>(op.t_vals), A->t_vals, st.nnz * es, cudaMemcpyHostToDevice, s));
    GK_CUDA(
        cudaMemcpyAsync(const_cast<int32_t *>(op.t_rowptr), A->t_rowptr, (A->n + 1) * 4, cudaMemcpyHostToDevice, s));
    GK_CUDA(cudaMemcpyAsync(const_cast<int32_t *>(op.t_colind), A->t_colind, st.nnz * 4, cudaMemcpyHostToDevice, s));
  }
  return GK_OK;
}

// the fused sweep's conditions, judged on the operator the kernels will read: a host
// operator is staged into the 256-byte-aligned workspace, so only its row stride matters
bool fused_ok_staged(const Op &op, const OpStage &st, const Dev &d) {
  if (!st.host) return fused_ok(op, d);
  Op probe = op;
  probe.vals = reinterpret_cast<const void *>((uintptr_t)256);
  return fused_ok(probe, d);
}

Op make_op(const gk_matrix *A) {
  Op op;
  op.kind = A->kind;
  op.dtype = A->dtype;
  op.m = A->m;
  op.n = A->n;
  op.ld = A->kind == GK_DENSE ? A->ld : 0;
  op.nnz = 0;
  if (A->kind == GK_CSR && A->rowptr) {
    int64_t nz = 0;
    if (csr_nnz(A->rowptr, A->m, &nz) == GK_OK) op.nnz = nz;
  }
  op.scale = A->scale;
  op.vals = A->vals;
  op.rowptr = A->rowptr;
  op.colind = A->colind;
  op.t_vals = A->t_vals;
  op.t_rowptr = A->t_rowptr;
  op.t_colind = A->t_colind;
  return op;
}

// Workspace owner: caller memory or a stream-ordered allocation freed on exit.
struct Workspace {
  char *base = nullptr;
  bool owned = false;
  cudaStream_t s = nullptr;
  ~Workspace() {
    if (owned && base) {
      cudaFreeAsync(base, s);
      cudaStreamSynchronize(s);
    }
  }
};

// The library's own stream-ordered pool per device.  Its release threshold is
// unbounded, so workspace freed at the end of a call stays mapped and the next
// call reuses it instead of mapping fresh memory (which costs tens of
// milliseconds for multi-GB operator staging buffers).
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {nullptr};

int library_pool(int dev, cudaMemPool_t *out) {
  if (dev < 0 || dev >= 64) return GK_NO_DEVICE;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    GK_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t thr = UINT64_MAX;
    GK_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
    g_pool[dev] = p;
  }
  *out = g_pool[dev];
  return GK_OK;
}

int acquire(Workspace &ws, size_t bytes, const gk_opts &o, cudaStream_t s) {
  ws.s = s;
  if (o.workspace) {
    if (o.workspace_bytes < bytes) return GK_OUT_OF_MEMORY;
    if ((uintptr_t)o.workspace % 256 != 0) return GK_INVALID_ARG;
    ws.base = (char *)o.workspace;
    return GK_OK;
  }
  int dev = 0;
  GK_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  const int rc = library_pool(dev, &pool);
  if (rc) return rc;
  void *p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_err, sizeof(g_err), "cudaMallocFromPoolAsync(%zu) -> %s", bytes, cudaGetErrorString(e));
    return GK_OUT_OF_MEMORY;
  }
  ws.base = (char *)p;
  ws.owned = true;
  return GK_OK;
}

// CUDA-event timing of kernel groups (GK_FLAG_PROFILE); events are pooled per thread
enum ProfCat { PC_MATVEC = 0, PC_MATVEC_T = 1, PC_ORTH = 2, PC_SMALL = 3, PC_RESTART = 4, PC_COPY = 5, PC_N = 6 };
thread_local std::vector<cudaEvent_t> t_event_pool;

struct Prof {
  bool on = false;
  cudaStream_t s = nullptr;
  size_t used = 0;
  struct Rec {
    int cat;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  int cur = -1;
  cudaEvent_t cur_ev = nullptr;
  cudaEvent_t get() {
    if (used == t_event_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        on = false;
        return nullptr;
      }
      t_event_pool.push_back(e);
    }
    return t_event_pool[used++];
  }
  void begin(int cat) {
    if (!on) return;
    cur_ev = get();
    if (!on) return;
    cudaEventRecord(cur_ev, s);
    cur = cat;
  }
  void end() {
    if (!on || cur < 0) return;
    cudaEvent_t e = get();
    if (!on) return;
    cudaEventRecord(e, s);
    recs.push_back({cur, cur_ev, e});
    cur = -1;
  }
  void finish(gk_info *inf) {
    if (!on) return;
    cudaStreamSynchronize(s);
    double ms[PC_N] = {0, 0, 0, 0, 0, 0};
    int64_t cnt[PC_N] = {0, 0, 0, 0, 0, 0};
    for (const Rec &r : recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.cat] += t;
        cnt[r.cat]++;
      }
    }
    inf->ms_matvec = ms[PC_MATVEC];
    inf->ms_matvec_t = ms[PC_MATVEC_T];
    inf->ms_orth = ms[PC_ORTH];
    inf->ms_small = ms[PC_SMALL];
    inf->ms_restart = ms[PC_RESTART];
    inf->ms_copy = ms[PC_COPY];
    inf->n_matvec = cnt[PC_MATVEC];
    inf->n_matvec_t = cnt[PC_MATVEC_T];
  }
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// ---------------------------------------------------------------------------
// gk_psvd
// ---------------------------------------------------------------------------
struct PsvdPlan {
  int64_t m, n, ldu, ldv;
  int k, K, keep, passes, max_restarts;
  bool fused;   // one pass over A per step (gk_fused.cu)
  bool refine;  // FP64-grade check of the returned triplets (GK_FLAG_REFINE)
  bool df;      // Gram-Schmidt on the bases' double-f32 shadows (not GK_FLAG_ORTH_F64)
  bool bdsvd;   // cycles without kept vectors: the bidiagonal B by Golub-Kahan SVD steps (GK_FLAG_BDSVD)
  bool ritz_df; // Ritz vectors from the bases' double-f32 copies (GK_FLAG_RITZ_DF, needs df)
};

struct PsvdBufs {
  Ctl *ctl;
  double *Ub, *Ub2, *Vb, *Vb2, *w, *z, *t, *part, *h, *alpha, *beta, *Bm, *Yw, *X, *Y, *sigma, *rho, *out;
  float *x32;
  int *sweeps;
  double *Uo, *So, *Vo, *q1, *svd_nrm, *zpart, *rY, *rZ, *rr1, *rr2;
  float *rsplit;
  int *svd_pos;
  float2 *Us, *Us2, *Vs, *Vs2, *ws2;  // double-f32 shadows of Ub, Ub2, Vb, Vb2; split of w (or null)
};

size_t psvd_layout(const gk_matrix *A, const PsvdPlan &p, const Dev &d, const OpStage &st, bool host_out,
                   bool host_start, char *base, PsvdBufs *b, Op *op) {
  Carve cv{base, 0};
  const int K = p.K;
  b->ctl = cv.take<Ctl>(1);
  b->Ub = cv.take<double>((size_t)p.ldu * K);
  b->Ub2 = cv.take<double>((size_t)p.ldu * K);
  b->Vb = cv.take<double>((size_t)p.ldv * (K + 1));
  b->Vb2 = cv.take<double>((size_t)p.ldv * (K + 1));
  b->w = cv.take<double>(p.ldu);
  b->t = cv.take<double>(p.ldu);
  b->z = cv.take<double>(p.ldv);
  b->x32 = cv.take<float>(p.ldu > p.ldv ? p.ldu : p.ldv);
  const int64_t gmax = cgs_blocks(p.m, d) > cgs_blocks(p.n, d) ? cgs_blocks(p.m, d) : cgs_blocks(p.n, d);
  int64_t pcount = gmax * (K + 2) + gmax;
  if (coop_partials(K, d) > pcount) pcount = coop_partials(K, d);
  const int64_t gp = gemvt_partials(*op, d);
  if (gp > pcount) pcount = gp;
  b->part = cv.take<double>(pcount);
  b->h = cv.take<double>(2 * (size_t)K + 4);  // two passes' coefficients and norms (adaptive rule)
  b->alpha = cv.take<double>(K + 2);
  b->beta = cv.take<double>(K + 2);
  b->Bm = cv.take<double>((size_t)K * K);
  b->Yw = cv.take<double>((size_t)K * K);
  b->X = cv.take<double>((size_t)K * K);
  b->Y = cv.take<double>((size_t)K * K);
  b->sigma = cv.take<double>(K);
  b->rho = cv.take<double>(K);
  b->out = cv.take<double>(8);
  b->sweeps = cv.take<int>(4);
  b->svd_nrm = cv.take<double>(K);
  b->svd_pos = cv.take<int>(K);
  b->Uo = host_out ? cv.take<double>((size_t)p.m * p.k) : nullptr;
  b->Vo = host_out ? cv.take<double>((size_t)p.n * p.k) : nullptr;
  b->So = host_out ? cv.take<double>(p.k) : nullptr;
  b->q1 = host_start ? cv.take<double>(p.ldu) : nullptr;
  b->zpart = p.fused ? cv.take<double>(fused_partials(*op, d)) : nullptr;
  b->Us = p.df ? cv.take<float2>((size_t)p.ldu * K) : nullptr;
  b->Us2 = p.df ? cv.take<float2>((size_t)p.ldu * K) : nullptr;
  b->Vs = p.df ? cv.take<float2>((size_t)p.ldv * (K + 1)) : nullptr;
  b->Vs2 = p.df ? cv.take<float2>((size_t)p.ldv * (K + 1)) : nullptr;
  b->ws2 = p.df ? cv.take<float2>(p.ldu > p.ldv ? p.ldu : p.ldv) : nullptr;
  b->rY = b->rZ = b->rr1 = b->rr2 = nullptr;
  b->rsplit = nullptr;
  if (p.refine) {
    b->rr1 = cv.take<double>(p.k);
    b->rr2 = cv.take<double>(p.k);
    if (accurate_ok(*op)) {
      b->rY = cv.take<double>((size_t)p.m * p.k);
      b->rZ = cv.take<double>((size_t)p.n * p.k);
      b->rsplit = cv.take<float>(accurate_floats(*op, p.k));
    }
  }
  char *dd;
  void *v, *tv;
  int32_t *rp, *ci, *trp, *tci;
  stage_carve(A, st, cv, op, &dd, &v, &rp, &ci, &tv, &trp, &tci);
  return cv.off + 256;
}

int psvd_plan(const gk_matrix *A, int k, const gk_opts &o, PsvdPlan *p) {
  const int64_t mn = A->m < A->n ? A->m : A->n;
  if (k < 1 || k > mn) return GK_INVALID_ARG;
  int K = o.krylov_dim;
  if (K <= 0) {
    int64_t d = 2 * (int64_t)k;
    if (d < k + 16) d = k + 16;
    if (d > mn) d = mn;
    K = (int)d;
  }
  if (K < k || K > mn) return GK_INVALID_ARG;
  if (K == k && K < mn) return GK_INVALID_ARG;  // a restart needs room beyond the wanted vectors
  if (K > 1024) return GK_INVALID_ARG;
  int keep = o.keep > 0 ? o.keep : k + (K - k) / 2;
  if (keep < k) keep = k;
  if (keep >= K) keep = K - 1;
  if (keep < 0) keep = 0;
  if (o.reorth_passes < 0 || o.reorth_passes > 3) return GK_INVALID_ARG;
  if (o.max_restarts < 0) return GK_INVALID_ARG;
  p->m = A->m;
  p->n = A->n;
  p->ldu = round_up(A->m, 32);
  p->ldv = round_up(A->n, 32);
  p->k = k;
  p->K = K;
  p->keep = keep;
  p->passes = o.reorth_passes;
  p->max_restarts = o.max_restarts;
  p->fused = false;
  p->refine = (o.flags & GK_FLAG_REFINE) != 0;
  p->df = (o.flags & GK_FLAG_ORTH_F64) == 0;
  p->bdsvd = (o.flags & GK_FLAG_BDSVD) != 0 && K <= kBdMaxK;
  p->ritz_df = (o.flags & GK_FLAG_RITZ_DF) != 0 && p->df;
  return GK_OK;
}

struct HostCtl {
  Ctl ctl;
  double out[8];
};

int read_ctl(const Ctl *dctl, const double *dout, HostCtl *hc, cudaStream_t s) {
  GK_CUDA(cudaMemcpyAsync(&hc->ctl, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  if (dout) GK_CUDA(cudaMemcpyAsync(hc->out, dout, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaStreamSynchronize(s));
  return GK_OK;
}

int clear_halt(Ctl *ctl, cudaStream_t s) {
  GK_CUDA(cudaMemsetAsync(ctl, 0, 2 * sizeof(int), s));  // halt and event
  return GK_OK;
}

// replacement direction for a basis column: fresh values, orthogonalized twice
// against the first `jcols` columns, normalized (or zero if the basis is full)
int fresh_column(double *wbuf, int64_t len, const double *Qb, int64_t ld, int jcols, double *dst, float *x32,
                 uint64_t seed, int64_t *nfresh, PsvdBufs &b, cudaStream_t s, const Dev &d, const float2 *Qs,
                 float2 *dsts) {
  GK_CUDA(draw_fresh(wbuf, len, seed, (*nfresh)++, s));
  GK_CUDA(orthonormalize(wbuf, len, Qb, ld, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 0, nullptr, nullptr, s, d));
  GK_CUDA(orthonormalize(wbuf, len, Qb, ld, jcols, 2, b.part, b.h, b.ctl, NM_FRESH, -1, 0, nullptr, nullptr, s, d,
                         Qs, b.ws2));
  GK_CUDA(normalize_append(wbuf, len, dst, x32, b.ctl, s, d, dsts));
  return GK_OK;
}

// True residuals of the k output triplets (device Uo m x k, So, Vo n x k): FP64-grade products
// (double-f32 for reduced-precision dense operators, f64 otherwise); returns
// max_i max(r_av, r_atu) / s_1 in *rel.
int refine_check(const Op &op, int64_t m, int64_t n, int k, const double *Uo, const double *So, const double *Vo,
                 PsvdBufs &b, double *rel, double *err_rel, cudaStream_t s, const Dev &d) {
  if (accurate_ok(op)) {
    GK_CUDA(accurate_products(op, false, Vo, k, b.rY, b.rsplit, s));
    GK_CUDA(resid_norms(b.rY, Uo, So, m, k, b.rr1, s));
    GK_CUDA(accurate_products(op, true, Uo, k, b.rZ, b.rsplit, s));
    GK_CUDA(resid_norms(b.rZ, Vo, So, n, k, b.rr2, s));
  } else {
    for (int i = 0; i < k; ++i) {
      const double *ui = Uo + (int64_t)i * m, *vi = Vo + (int64_t)i * n;
      GK_CUDA(copy_vec(nullptr, b.x32, vi, n, s));
      GK_CUDA(matvec(op, b.x32, vi, b.w, ui, So + i, b.part, b.ctl, s, d));
      GK_CUDA(orthonormalize(b.w, m, nullptr, m, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 0, b.rr1 + i, nullptr, s, d));
      GK_CUDA(copy_vec(nullptr, b.x32, ui, m, s));
      GK_CUDA(matvec_t(op, b.x32, ui, b.z, vi, So + i, b.part, b.ctl, s, d));
      GK_CUDA(orthonormalize(b.z, n, nullptr, n, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 1, b.rr2 + i, nullptr, s, d));
    }
  }
  std::vector<double> h(3 * (size_t)k);
  GK_CUDA(cudaMemcpyAsync(h.data(), b.rr1, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaMemcpyAsync(h.data() + k, b.rr2, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaMemcpyAsync(h.data() + 2 * k, So, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaStreamSynchronize(s));
  double mx = 0.0, r2 = 0.0, s2 = 0.0;
  for (int i = 0; i < 2 * k; ++i) mx = fmax(mx, h[i]);
  for (int i = 0; i < k; ++i) {
    r2 += h[k + i] * h[k + i];
    s2 += h[2 * k + i] * h[2 * k + i];
  }
  *rel = h[2 * k] > 0.0 ? mx / h[2 * k] : 0.0;
  // the paper's err_rel (Section 5): ||A^T U - V Sigma||_F / ||Sigma||_F
  *err_rel = s2 > 0.0 ? sqrt(r2 / s2) : 0.0;
  return GK_OK;
}

// With GK_FLAG_PERSISTENT a small dense device operator goes to the batched solver as a single
// problem: one persistent launch (one cluster) runs the whole thick-restart solve.
constexpr size_t kPersistentBytes = 24u << 20;

bool persistent_ok(const gk_matrix *A, const PsvdPlan &p, const gk_opts &o, const gk_opts *oin, const OpStage &st,
                   bool host_out, bool host_start) {
  if (A->kind != GK_DENSE || st.host || host_out || host_start) return false;
  if (!(o.flags & GK_FLAG_PERSISTENT) || (o.flags & (GK_FLAG_FUSED | GK_FLAG_REFINE))) return false;
  if (o.workspace || o.predictor || (oin && oin->keep > 0)) return false;
  if (A->n > 4096 || A->ld < A->n || p.K > 500 || A->m > INT32_MAX) return false;
  return st.vals_bytes <= kPersistentBytes;
}

int psvd_persistent_call(const gk_matrix *A, int k, double tol, const PsvdPlan &p, const gk_opts &o, double *U,
                         double *S, double *V, gk_info *info, std::chrono::steady_clock::time_point t0, int64_t l0) {
  gk_batch_item it;
  memset(&it, 0, sizeof(it));
  it.A = *A;
  it.k = k;
  it.krylov_dim = p.K;
  it.tol = tol;
  it.U = U;
  it.S = S;
  it.V = V;
  it.start = o.start;
  gk_opts ob = o;
  ob.flags = o.flags & GK_FLAG_PROFILE;
  gk_info bi;
  memset(&bi, 0, sizeof(bi));
  int rc = psvd_persistent(&it, &ob, &bi);
  if (rc < 0) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;
  // the multi-kernel path's conventions: the sign of each v, and a zero s_k reported
  GK_CUDA(sign_normalize(U, A->m, A->m, V, A->n, A->n, k, s));
  double sk = 0.0;
  GK_CUDA(cudaMemcpyAsync(&sk, S + (k - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaStreamSynchronize(s));
  int status = it.status;
  if (status == GK_OK && sk == 0.0) status = GK_RANK_DEFICIENT;
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.steps = it.steps;
  inf.restarts = it.restarts;
  inf.cycles = it.cycles;
  inf.breakdowns = it.breakdowns;
  inf.matvecs = it.matvecs;
  inf.resid_est_max = it.resid_est_max;
  inf.sigma_est = it.sigma_est;
  inf.svd_sweeps = bi.svd_sweeps;
  inf.ms_matvec = bi.ms_matvec;
  inf.ms_matvec_t = bi.ms_matvec_t;
  inf.ms_orth = bi.ms_orth;
  inf.ms_small = bi.ms_small;
  inf.ms_restart = bi.ms_restart;
  inf.kprime = p.K;
  inf.reserved = 0;
  inf.seconds = seconds_since(t0);
  inf.launches = launch_count() - l0;
  if (info) *info = inf;
  return status;
}

int psvd_impl(const gk_matrix *Ain, int k, double tol, const gk_opts *oin, double *U, double *S, double *V,
              gk_info *info) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launch_count();
  g_err[0] = 0;
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  if (info) *info = inf;
  Dev d;
  if (!get_device(&d)) return GK_NO_DEVICE;
  int rc = check_matrix(Ain);
  if (rc) return rc;
  if (!U || !S || !V || !(tol >= 0.0) || !isfinite(tol)) return GK_INVALID_ARG;
  gk_opts o = oin ? *oin : defaults();
  cudaStream_t s = (cudaStream_t)o.stream;
  // the learned Krylov dimension: from the sketch of a device operator now, of a host operator
  // once it is staged (the workspace is laid out for the largest dimension a prediction allows)
  bool predict_after_stage = false;
  if (o.predictor && o.krylov_dim <= 0) {
    if (Ain->kind != GK_DENSE || k < 1) return GK_INVALID_ARG;
    const int64_t mn = Ain->m < Ain->n ? Ain->m : Ain->n;
    if (!on_host(Ain->vals)) {
      int Kp = 0;
      rc = predict_krylov(o.predictor, Ain, k, s, &Kp, o.flags);
      if (rc) return rc;
      o.krylov_dim = Kp;
    } else {
      const int64_t kmax = mn < 500 ? mn : 500;
      o.krylov_dim = (int)(kmax > k ? kmax : mn);
      predict_after_stage = true;
    }
  }
  PsvdPlan p;
  rc = psvd_plan(Ain, k, o, &p);
  if (rc) return rc;
  OpStage st;
  rc = stage_plan(Ain, &st);
  if (rc) return rc;
  const bool host_out = on_host(U) || on_host(S) || on_host(V);
  const bool host_start = o.start && on_host(o.start);
  if (persistent_ok(Ain, p, o, oin, st, host_out, host_start))
    return psvd_persistent_call(Ain, k, tol, p, o, U, S, V, info, t0, l0);
  Op op = make_op(Ain);
  p.fused = (o.flags & GK_FLAG_FUSED) && fused_ok_staged(op, st, d);
  PsvdBufs b;
  const size_t bytes = psvd_layout(Ain, p, d, st, host_out, host_start, nullptr, &b, &op);
  Workspace ws;
  rc = acquire(ws, bytes, o, s);
  if (rc) return rc;
  op = make_op(Ain);
  psvd_layout(Ain, p, d, st, host_out, host_start, ws.base, &b, &op);
  Prof prof;
  prof.on = (o.flags & GK_FLAG_PROFILE) != 0;
  prof.s = s;
  prof.begin(PC_COPY);
  rc = stage_copy(Ain, st, op, s);
  prof.end();
  if (rc) return rc;
  if (predict_after_stage) {
    gk_matrix Astaged = *Ain;
    Astaged.vals = op.vals;
    Astaged.ld = op.ld;
    int Kp = 0;
    rc = predict_krylov(o.predictor, &Astaged, k, s, &Kp, o.flags);
    if (rc) return rc;
    o.krylov_dim = Kp;
    PsvdPlan p2;
    rc = psvd_plan(Ain, k, o, &p2);
    if (rc) return rc;
    p.K = p2.K;  // within the layout: the workspace holds the largest dimension
    p.keep = p2.keep;
  }

  const int64_t m = p.m, n = p.n, ldu = p.ldu, ldv = p.ldv;
  const int K = p.K;
  GK_CUDA(reset_ctl(b.ctl, 0.0, 1, s));
  GK_CUDA(cudaMemsetAsync(b.alpha, 0, sizeof(double) * (K + 2), s));
  GK_CUDA(cudaMemsetAsync(b.beta, 0, sizeof(double) * (K + 2), s));
  if (p.df) {  // the shadows' padding rows (past m, n) are read beside the last odd row: keep them 0
    GK_CUDA(cudaMemsetAsync(b.Us, 0, sizeof(float2) * ldu * K, s));
    GK_CUDA(cudaMemsetAsync(b.Us2, 0, sizeof(float2) * ldu * K, s));
    GK_CUDA(cudaMemsetAsync(b.Vs, 0, sizeof(float2) * ldv * (K + 1), s));
    GK_CUDA(cudaMemsetAsync(b.Vs2, 0, sizeof(float2) * ldv * (K + 1), s));
  }
  // start vector q1 (Algorithm 1) and v1 = A^T q1 / ||A^T q1||
  if (o.start) {
    const double *src = o.start;
    if (host_start) {
      GK_CUDA(cudaMemcpyAsync(b.q1, o.start, sizeof(double) * m, cudaMemcpyHostToDevice, s));
      src = b.q1;
    }
    GK_CUDA(copy_vec(b.t, nullptr, src, m, s));
  } else {
    GK_CUDA(draw_start(b.t, m, o.seed, s));
  }
  GK_CUDA(orthonormalize(b.t, m, nullptr, ldu, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 0, nullptr, nullptr, s, d));
  GK_CUDA(normalize_append(b.t, m, b.t, b.x32, b.ctl, s, d));
  GK_CUDA(matvec_t(op, b.x32, b.t, b.z, nullptr, nullptr, b.part, b.ctl, s, d));
  GK_CUDA(orthonormalize(b.z, n, b.Vb, ldv, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 1, nullptr, nullptr, s, d));
  GK_CUDA(normalize_append(b.z, n, b.Vb, b.x32, b.ctl, s, d, b.Vs));
  inf.matvecs = 1;
  HostCtl hc;
  rc = read_ctl(b.ctl, nullptr, &hc, s);
  if (rc) return rc;
  if (!isfinite(hc.ctl.norm)) return GK_NUMERICAL;
  int64_t nfresh = 0;
  if (hc.ctl.norm == 0.0) {  // A^T q1 = 0
    rc = fresh_column(b.z, n, b.Vb, ldv, 0, b.Vb, b.x32, o.seed, &nfresh, b, s, d, b.Vs, b.Vs);
    if (rc) return rc;
    inf.breakdowns++;
  }
  GK_CUDA(reset_ctl(b.ctl, 0.0, 1, s));

  int l = 0;
  int status = GK_NOT_CONVERGED;
  double tol_ritz = tol;      // the Ritz test's tolerance (tightened by failed refinement checks)
  bool outputs_ready = false;  // Uo, So, Vo already hold the final triplets
  double *Uo = host_out ? b.Uo : U, *Vo = host_out ? b.Vo : V, *So = host_out ? b.So : S;
  // outputs: U = U_K X_k, V = V_K Y_k, S = sigma_k, sign convention on v
  // Ritz vectors C = Q X: in f64, or from the basis's double-f32 copy (b.Yw, free after the small
  // SVD, holds X's split)
  auto ritz = [&](const double *Qb, const float2 *Qsh, int64_t ld, int64_t len, const double *Xm, int ncol,
                  double *C, int64_t ldc) -> cudaError_t {
    if (p.ritz_df && Qsh) return ritz_gemm_df(Qsh, ld, len, K, Xm, K, ncol, C, ldc, reinterpret_cast<float2 *>(b.Yw), s);
    return ritz_gemm(Qb, ld, len, K, Xm, K, ncol, C, ldc, s, d);
  };
  auto form_outputs = [&]() -> int {
    prof.begin(PC_RESTART);
    GK_CUDA(ritz(b.Ub, b.Us, ldu, m, b.X, k, Uo, m));
    GK_CUDA(ritz(b.Vb, b.Vs, ldv, n, b.Y, k, Vo, n));
    prof.end();
    GK_CUDA(cudaMemcpyAsync(So, b.sigma, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
    GK_CUDA(sign_normalize(Uo, m, m, Vo, n, n, k, s));
    return GK_OK;
  };
  bool refine_failed = false;
  for (int cycle = 0;; ++cycle) {
    int j0 = l, side0 = 0;
    for (;;) {
      for (int j = j0; j < K; ++j) {
        bool fused_step = false;
        if (!(j == j0 && side0 == 1)) {
          // left half-step: A v_j minus its component along the previous u's
          const double *vj = b.Vb + (int64_t)j * ldv;
          prof.begin(PC_MATVEC);
          if (j == l && l > 0) {
            GK_CUDA(matvec(op, b.x32, vj, b.w, nullptr, nullptr, b.part, b.ctl, s, d));
            prof.end();
            prof.begin(PC_ORTH);
            GK_CUDA(sub_combination(b.w, m, b.Ub, ldu, l, b.rho, b.ctl, s, d));
          } else if (p.fused) {
            // one pass: w = A v_j - beta_{j-1} u_{j-1} and the partial sums of A^T w
            GK_CUDA(fused_matvec(op, b.x32, b.w, j > 0 ? b.Ub + (int64_t)(j - 1) * ldu : nullptr,
                                 j > 0 ? b.beta + (j - 1) : nullptr, b.zpart, b.ctl, s, d));
            fused_step = true;
            prof.end();
            prof.begin(PC_ORTH);
          } else if (j > 0) {
            GK_CUDA(matvec(op, b.x32, vj, b.w, b.Ub + (int64_t)(j - 1) * ldu, b.beta + (j - 1), b.part, b.ctl, s, d));
            prof.end();
            prof.begin(PC_ORTH);
          } else {
            GK_CUDA(matvec(op, b.x32, vj, b.w, nullptr, nullptr, b.part, b.ctl, s, d));
            prof.end();
            prof.begin(PC_ORTH);
          }
          GK_CUDA(orth_append(b.w, m, b.Ub, ldu, j, p.passes, b.part, b.h, b.ctl, NM_BREAKDOWN, j, 0, b.alpha + j,
                              nullptr, b.Ub + (int64_t)j * ldu, fused_step ? nullptr : b.x32, s, d, b.Us, b.ws2,
                              b.Us ? b.Us + (int64_t)j * ldu : nullptr));
          prof.end();
          inf.matvecs++;
        }
        // right half-step: A^T u_j - alpha_j v_j, orthogonalized against V_{j+1}; after a fused
        // pass A^T u_j is A^T w / alpha_j up to span(V_j), which the Gram-Schmidt removes
        prof.begin(PC_MATVEC_T);
        if (fused_step)
          GK_CUDA(fused_finish(op, b.zpart, b.alpha + j, b.Vb + (int64_t)j * ldv, b.z, b.ctl, s, d));
        else
          GK_CUDA(matvec_t(op, b.x32, b.Ub + (int64_t)j * ldu, b.z, b.Vb + (int64_t)j * ldv, b.alpha + j, b.part,
                           b.ctl, s, d));
        prof.end();
        prof.begin(PC_ORTH);
        GK_CUDA(orth_append(b.z, n, b.Vb, ldv, j + 1, p.passes, b.part, b.h, b.ctl, NM_BREAKDOWN, j, 1, b.beta + j,
                            nullptr, b.Vb + (int64_t)(j + 1) * ldv, b.x32, s, d, b.Vs, b.ws2,
                            b.Vs ? b.Vs + (int64_t)(j + 1) * ldv : nullptr));
        prof.end();
        inf.matvecs++;
        inf.steps++;
      }
      prof.begin(PC_SMALL);
      if (l == 0 && p.bdsvd) {  // B is upper bidiagonal (alpha on the diagonal, beta above it)
        GK_CUDA(bd_svd(b.alpha, b.beta, K, b.sigma, b.X, b.Y, b.Bm, b.Yw, b.sweeps, b.ctl, s));
      } else {
        GK_CUDA(assemble_B(b.Bm, K, l, b.sigma, b.rho, b.alpha, b.beta, b.ctl, s));
        GK_CUDA(small_svd(b.Bm, b.Yw, K, b.sigma, b.X, b.Y, b.svd_nrm, b.svd_pos, b.sweeps, b.ctl, s));
      }
      GK_CUDA(ritz_check(b.sigma, b.X, K, k, b.beta + (K - 1), tol_ritz, b.rho, b.out, b.ctl, s));
      prof.end();
      rc = read_ctl(b.ctl, b.out, &hc, s);
      if (rc) return rc;
      if (hc.ctl.event == EV_NUMERICAL) return GK_NUMERICAL;
      if (hc.ctl.event == EV_TIMEOUT) return GK_TIMEOUT;
      if (hc.ctl.event != EV_BREAKDOWN) break;
      // exact breakdown: replace the vanished vector and resume the cycle after it
      const int jb = hc.ctl.step, sb = hc.ctl.side;
      rc = clear_halt(b.ctl, s);
      if (rc) return rc;
      inf.breakdowns++;
      if (sb == 0) {
        rc = fresh_column(b.w, m, b.Ub, ldu, jb, b.Ub + (int64_t)jb * ldu, b.x32, o.seed, &nfresh, b, s, d, b.Us,
                          b.Us ? b.Us + (int64_t)jb * ldu : nullptr);
        j0 = jb;
        side0 = 1;
      } else {
        rc = fresh_column(b.z, n, b.Vb, ldv, jb + 1, b.Vb + (int64_t)(jb + 1) * ldv, b.x32, o.seed, &nfresh, b, s,
                          d, b.Vs, b.Vs ? b.Vs + (int64_t)(jb + 1) * ldv : nullptr);
        j0 = jb + 1;
        side0 = 0;
      }
      if (rc) return rc;
    }
    inf.cycles = cycle + 1;
    inf.resid_est_max = hc.out[1] > 0.0 ? hc.out[0] / hc.out[1] : 0.0;
    const bool conv = hc.out[2] != 0.0;
    if (p.refine && (conv || cycle >= p.max_restarts)) {
      // the returned triplets' true residuals with FP64-grade products
      rc = form_outputs();
      if (rc) return rc;
      outputs_ready = true;
      const auto tr = std::chrono::steady_clock::now();
      double rel = 0.0, erel = 0.0;
      rc = refine_check(op, m, n, k, Uo, So, Vo, b, &rel, &erel, s, d);
      if (rc) return rc;
      inf.ms_refine += seconds_since(tr) * 1e3;
      inf.refine_checks++;
      inf.resid_true_max = rel;
      inf.err_rel = erel;
      refine_failed = rel > tol;
      if (refine_failed && conv && cycle < p.max_restarts) {
        tol_ritz *= 0.25;  // the Ritz residuals must shrink further: restart and test again
        outputs_ready = false;
      } else {
        status = (conv && !refine_failed) ? GK_OK : GK_NOT_CONVERGED;
        break;
      }
    } else if (conv || cycle >= p.max_restarts) {
      status = conv ? GK_OK : GK_NOT_CONVERGED;
      break;
    }
    // thick restart: U' = U_K X_keep, V' = [V_K Y_keep, v_{K+1}]
    prof.begin(PC_RESTART);
    GK_CUDA(ritz(b.Ub, b.Us, ldu, m, b.X, p.keep, b.Ub2, ldu));
    GK_CUDA(ritz(b.Vb, b.Vs, ldv, n, b.Y, p.keep, b.Vb2, ldv));
    GK_CUDA(copy_vec(b.Vb2 + (int64_t)p.keep * ldv, b.x32, b.Vb + (int64_t)K * ldv, n, s));
    if (p.df) {  // the kept columns' shadows
      GK_CUDA(split_cols(b.Ub2, m, ldu, p.keep, b.Us2, s));
      GK_CUDA(split_cols(b.Vb2, n, ldv, p.keep + 1, b.Vs2, s));
    }
    prof.end();
    double *tmp = b.Ub;
    b.Ub = b.Ub2;
    b.Ub2 = tmp;
    tmp = b.Vb;
    b.Vb = b.Vb2;
    b.Vb2 = tmp;
    std::swap(b.Us, b.Us2);
    std::swap(b.Vs, b.Vs2);
    l = p.keep;
    inf.restarts++;
  }

  if (!outputs_ready) {
    rc = form_outputs();
    if (rc) return rc;
  }
  double sk = 0.0;
  int sweeps = 0;
  GK_CUDA(cudaMemcpyAsync(&sk, b.sigma + (k - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaMemcpyAsync(&sweeps, b.sweeps, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (host_out) {
    prof.begin(PC_COPY);
    GK_CUDA(cudaMemcpyAsync(U, Uo, sizeof(double) * m * k, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(V, Vo, sizeof(double) * n * k, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(S, So, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    prof.end();
  }
  GK_CUDA(cudaMemcpyAsync(&hc.ctl, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaStreamSynchronize(s));
  if (status == GK_OK && sk == 0.0) status = GK_RANK_DEFICIENT;
  prof.finish(&inf);
  inf.sigma_est = hc.ctl.sest;
  inf.svd_sweeps = sweeps;
  inf.reserved = p.fused ? fused_cluster(op, d) : 0;
  inf.kprime = K;  // the Krylov dimension used
  inf.seconds = seconds_since(t0);
  inf.launches = launch_count() - l0;
  if (info) *info = inf;
  if (hc.ctl.timeout) return GK_TIMEOUT;
  return status;
}

// ---------------------------------------------------------------------------
// gk_numrank
// ---------------------------------------------------------------------------
struct RankBufs {
  Ctl *ctl;
  double *Q, *P, *w, *z, *t, *part, *h, *alpha, *beta, *sig, *sigma1, *q1, *zpart;
  float *x32;
  int *rank;
  bool fused;  // one pass over A per step (gk_fused.cu)
  bool df;     // Gram-Schmidt on the bases' double-f32 shadows (not GK_FLAG_ORTH_F64)
  float2 *Qs, *Ps, *ws2;
};

size_t numrank_layout(const gk_matrix *A, int64_t kmax, const Dev &d, const OpStage &st, bool host_sigma,
                      bool host_start, char *base, RankBufs *b, Op *op) {
  Carve cv{base, 0};
  const int64_t ldu = round_up(A->m, 32), ldv = round_up(A->n, 32);
  b->ctl = cv.take<Ctl>(1);
  b->Q = cv.take<double>((size_t)ldu * (kmax + 1));
  b->P = cv.take<double>((size_t)ldv * (kmax + 1));
  b->w = cv.take<double>(ldu);
  b->t = cv.take<double>(ldu);
  b->z = cv.take<double>(ldv);
  b->x32 = cv.take<float>(ldu > ldv ? ldu : ldv);
  const int64_t gmax = cgs_blocks(A->m, d) > cgs_blocks(A->n, d) ? cgs_blocks(A->m, d) : cgs_blocks(A->n, d);
  int64_t pcount = gmax * (kmax + 2) + gmax;
  if (coop_partials((int)kmax, d) > pcount) pcount = coop_partials((int)kmax, d);
  const int64_t gp = gemvt_partials(*op, d);
  if (gp > pcount) pcount = gp;
  b->part = cv.take<double>(pcount);
  b->h = cv.take<double>(2 * (size_t)kmax + 4);  // two passes' coefficients and norms (adaptive rule)
  b->alpha = cv.take<double>(kmax + 2);
  b->beta = cv.take<double>(kmax + 2);
  b->sig = host_sigma ? cv.take<double>(kmax + 1) : nullptr;
  b->sigma1 = cv.take<double>(1);
  b->rank = cv.take<int>(1);
  b->q1 = host_start ? cv.take<double>(ldu) : nullptr;
  b->zpart = b->fused ? cv.take<double>(fused_partials(*op, d)) : nullptr;
  b->Qs = b->df ? cv.take<float2>((size_t)ldu * (kmax + 1)) : nullptr;
  b->Ps = b->df ? cv.take<float2>((size_t)ldv * (kmax + 1)) : nullptr;
  b->ws2 = b->df ? cv.take<float2>(ldu > ldv ? ldu : ldv) : nullptr;
  char *dd;
  void *v, *tv;
  int32_t *rp, *ci, *trp, *tci;
  stage_carve(A, st, cv, op, &dd, &v, &rp, &ci, &tv, &trp, &tci);
  return cv.off + 256;
}

int64_t clamp_kmax(const gk_matrix *A, int kmax) {
  const int64_t mn = A->m < A->n ? A->m : A->n;
  return (kmax <= 0 || kmax > mn) ? mn : kmax;
}

// Algorithm 1 on the staged operator: q1 (given or drawn), then up to kmax steps of the
// lower bidiagonalization with the break test (threshold eps, relative to the running
// sigma estimate when eps_rel), in chunks of 8 steps between reads of the control block.
// Leaves Q (k'+1 columns), P, alpha, beta in b; *kp_out = k'; fills matvecs, stop_reason.
int lower_sweep(const gk_matrix *Ain, const gk_opts &o, const Op &op, RankBufs &b, int64_t kmax, double eps,
                int eps_rel, bool host_start, Prof &prof, gk_info &inf, HostCtl &hc, int *kp_out, cudaStream_t s,
                const Dev &d) {
  const int64_t m = Ain->m, n = Ain->n, ldu = round_up(m, 32), ldv = round_up(n, 32);
  const int passes = o.reorth_passes;
  int rc = GK_OK;
  GK_CUDA(reset_ctl(b.ctl, eps, eps_rel, s));
  GK_CUDA(cudaMemsetAsync(b.alpha, 0, sizeof(double) * (kmax + 2), s));
  GK_CUDA(cudaMemsetAsync(b.beta, 0, sizeof(double) * (kmax + 2), s));
  // q1 ~ N(2,1)^m, q1 = q1 / ||q1||, Q_1 = q1
  if (o.start) {
    const double *src = o.start;
    if (host_start) {
      GK_CUDA(cudaMemcpyAsync(b.q1, o.start, sizeof(double) * m, cudaMemcpyHostToDevice, s));
      src = b.q1;
    }
    GK_CUDA(copy_vec(b.t, nullptr, src, m, s));
  } else {
    GK_CUDA(draw_start(b.t, m, o.seed, s));
  }
  if (b.df) {  // the shadows' padding rows (past m, n) are read beside the last odd row: keep them 0
    GK_CUDA(cudaMemsetAsync(b.Qs, 0, sizeof(float2) * ldu * (kmax + 1), s));
    GK_CUDA(cudaMemsetAsync(b.Ps, 0, sizeof(float2) * ldv * (kmax + 1), s));
  }
  GK_CUDA(orthonormalize(b.t, m, nullptr, ldu, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 0, nullptr, nullptr, s, d));
  GK_CUDA(normalize_append(b.t, m, b.Q, b.x32, b.ctl, s, d, b.Qs));
  // p1 = A^T q1, alpha_1 = ||p1||, p1 = p1 / alpha_1
  GK_CUDA(matvec_t(op, b.x32, b.Q, b.z, nullptr, nullptr, b.part, b.ctl, s, d));
  GK_CUDA(orthonormalize(b.z, n, b.P, ldv, 0, 0, b.part, b.h, b.ctl, NM_BREAK, 0, 1, b.alpha, nullptr, s, d));
  GK_CUDA(normalize_append(b.z, n, b.P, b.x32, b.ctl, s, d, b.Ps));
  inf.matvecs = 1;
  rc = read_ctl(b.ctl, nullptr, &hc, s);
  if (rc) return rc;
  // the remaining steps, in chunks between reads of the control block
  const int chunk = 8;
  int64_t j = 1;
  while (!hc.ctl.halt && j <= kmax) {
    const int64_t jend = (j + chunk - 1 < kmax) ? j + chunk - 1 : kmax;
    for (; j <= jend; ++j) {
      const int jj = (int)j;
      // beta_{j+1} q_{j+1} = A p_j - alpha_j q_j, reorthogonalized against Q_j
      prof.begin(PC_MATVEC);
      if (b.fused)  // one pass: w and the partial sums of A^T w
        GK_CUDA(fused_matvec(op, b.x32, b.w, b.Q + (j - 1) * ldu, b.alpha + (j - 1), b.zpart, b.ctl, s, d));
      else
        GK_CUDA(matvec(op, b.x32, b.P + (j - 1) * ldv, b.w, b.Q + (j - 1) * ldu, b.alpha + (j - 1), b.part, b.ctl,
                       s, d));
      prof.end();
      prof.begin(PC_ORTH);
      GK_CUDA(orth_append(b.w, m, b.Q, ldu, jj, passes, b.part, b.h, b.ctl, NM_BREAK, jj, 0, b.beta + j,
                          b.alpha + (j - 1), b.Q + j * ldu, b.fused ? nullptr : b.x32, s, d, b.Qs, b.ws2,
                          b.Qs ? b.Qs + j * ldu : nullptr));
      prof.end();
      // alpha_{j+1} p_{j+1} = A^T q_{j+1} - beta_{j+1} p_j, reorthogonalized against P_j; after a
      // fused pass A^T q_{j+1} is A^T w / beta_{j+1} up to span(P_j), removed by the Gram-Schmidt
      prof.begin(PC_MATVEC_T);
      if (b.fused)
        GK_CUDA(fused_finish(op, b.zpart, b.beta + j, b.P + (j - 1) * ldv, b.z, b.ctl, s, d));
      else
        GK_CUDA(matvec_t(op, b.x32, b.Q + j * ldu, b.z, b.P + (j - 1) * ldv, b.beta + j, b.part, b.ctl, s, d));
      prof.end();
      prof.begin(PC_ORTH);
      GK_CUDA(orth_append(b.z, n, b.P, ldv, jj, passes, b.part, b.h, b.ctl, NM_BREAK, jj, 1, b.alpha + j,
                          b.beta + j, b.P + j * ldv, b.x32, s, d, b.Ps, b.ws2, b.Ps ? b.Ps + j * ldv : nullptr));
      prof.end();
    }
    rc = read_ctl(b.ctl, nullptr, &hc, s);
    if (rc) return rc;
  }
  if (hc.ctl.event == EV_NUMERICAL) return GK_NUMERICAL;
  if (hc.ctl.event == EV_TIMEOUT) return GK_TIMEOUT;
  int kp;
  if (hc.ctl.halt) {
    kp = hc.ctl.step;
    inf.stop_reason = hc.ctl.event == EV_BETA_BREAK ? 1 : 2;
    inf.matvecs += 2 * (int64_t)kp + (hc.ctl.side == 0 ? 1 : 2) - (kp > 0 ? 0 : 1);
  } else {
    kp = (int)kmax;
    inf.stop_reason = 0;
    inf.matvecs += 2 * (int64_t)kp;
  }
  *kp_out = kp;
  return GK_OK;
}

int numrank_impl(const gk_matrix *Ain, double eps, int kmax_in, const gk_opts *oin, int *rank, double *sigma,
                 gk_info *info) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launch_count();
  g_err[0] = 0;
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  if (info) *info = inf;
  Dev d;
  if (!get_device(&d)) return GK_NO_DEVICE;
  int rc = check_matrix(Ain);
  if (rc) return rc;
  if (!rank || !(eps >= 0.0) || !isfinite(eps)) return GK_INVALID_ARG;
  const gk_opts o = oin ? *oin : defaults();
  if (o.reorth_passes < 0 || o.reorth_passes > 3) return GK_INVALID_ARG;
  const int64_t kmax = clamp_kmax(Ain, kmax_in);
  cudaStream_t s = (cudaStream_t)o.stream;
  OpStage st;
  rc = stage_plan(Ain, &st);
  if (rc) return rc;
  const bool host_sigma = sigma && on_host(sigma);
  const bool host_start = o.start && on_host(o.start);
  Op op = make_op(Ain);
  RankBufs b;
  b.fused = (o.flags & GK_FLAG_FUSED) && fused_ok_staged(op, st, d);
  b.df = (o.flags & GK_FLAG_ORTH_F64) == 0;
  const size_t bytes = numrank_layout(Ain, kmax, d, st, host_sigma, host_start, nullptr, &b, &op);
  Workspace ws;
  rc = acquire(ws, bytes, o, s);
  if (rc) return rc;
  op = make_op(Ain);
  numrank_layout(Ain, kmax, d, st, host_sigma, host_start, ws.base, &b, &op);
  rc = stage_copy(Ain, st, op, s);
  if (rc) return rc;

  const int eps_rel = o.eps_absolute ? 0 : 1;
  Prof prof;
  prof.on = (o.flags & GK_FLAG_PROFILE) != 0;
  prof.s = s;
  HostCtl hc;
  int kp = 0;
  rc = lower_sweep(Ain, o, op, b, kmax, eps, eps_rel, host_start, prof, inf, hc, &kp, s, d);
  if (rc) return rc;
  inf.kprime = kp;
  inf.steps = kp;
  // Algorithm 3: singular values of B_{k'+1,k'} above the threshold
  double *sig_dev = sigma ? (host_sigma ? b.sig : sigma) : nullptr;
  prof.begin(PC_SMALL);
  GK_CUDA(bidiag_rank(b.alpha, b.beta, kp, eps, eps_rel, b.rank, b.sigma1, sig_dev, s));
  prof.end();
  int r = 0;
  GK_CUDA(cudaMemcpyAsync(&r, b.rank, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (host_sigma && kp > 0) GK_CUDA(cudaMemcpyAsync(sigma, b.sig, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaStreamSynchronize(s));
  *rank = r;
  prof.finish(&inf);
  inf.reserved = b.fused ? fused_cluster(op, d) : 0;
  inf.sigma_est = hc.ctl.sest;
  inf.seconds = seconds_since(t0);
  inf.launches = launch_count() - l0;
  if (info) *info = inf;
  return GK_OK;
}

// ---------------------------------------------------------------------------
// gk_block_numrank: Algorithm 1 and Algorithm 3 on blocks of s start vectors
// ---------------------------------------------------------------------------
constexpr int kBlockMaxOrder = 1024;  // (block steps + 1) * s: the order of B's square (small SVD)

struct BlockBufs {
  Ctl *ctl;
  BlockCtl *bc;
  double *Q, *P, *W, *w, *Xc, *part, *h, *dpart, *raw, *Bf, *Bm, *Yw, *X, *Y, *sigma, *nrm, *q0;
  float *x32, *split;
  float2 *Qs, *Ps, *ws2;
  double *npart;                 // the narrow block products' contraction-slice partials
  double *gW, *gC, *gH, *gpart;  // block Gram-Schmidt: projected block, Q H, H, Q^T X partials
  float2 *gWs, *gHs;             // and the double-f32 copies of the source block and of H
  int *pos, *sweeps, *rank;
  bool df;   // Gram-Schmidt on the bases' double-f32 shadows (not GK_FLAG_ORTH_F64)
  bool bgs;  // with df: the block Gram-Schmidt (GK_FLAG_BLOCK_GS)
  bool acc;  // dense reduced-precision operator: block products in one pass (double-f32)
  bool f32;  // with acc: the f32 form of that pass (GK_FLAG_BLOCK_F32)
};

size_t block_layout(const gk_matrix *A, int s, int64_t kb, const Dev &d, const OpStage &st, char *base, BlockBufs *b,
                    Op *op) {
  Carve cv{base, 0};
  const int64_t m = A->m, n = A->n, ldu = round_up(m, 32), ldv = round_up(n, 32), mx = m > n ? m : n;
  const int64_t lmax = ldu > ldv ? ldu : ldv;
  const int64_t cols = (kb + 1) * s;  // basis columns, and the order of B's square
  b->ctl = cv.take<Ctl>(1);
  b->bc = cv.take<BlockCtl>(1);
  b->Q = cv.take<double>((size_t)ldu * cols);
  b->P = cv.take<double>((size_t)ldv * cols);
  b->W = cv.take<double>((size_t)mx * s);
  b->w = cv.take<double>(lmax);
  b->Xc = b->acc ? cv.take<double>((size_t)mx * s) : nullptr;
  b->x32 = cv.take<float>(lmax);
  const int64_t gmax = cgs_blocks(m, d) > cgs_blocks(n, d) ? cgs_blocks(m, d) : cgs_blocks(n, d);
  int64_t pcount = gmax * (cols + 2) + gmax;
  if (coop_partials((int)cols, d) > pcount) pcount = coop_partials((int)cols, d);
  const int64_t gp = gemvt_partials(*op, d);
  if (gp > pcount) pcount = gp;
  b->part = cv.take<double>(pcount);
  b->h = cv.take<double>(2 * (size_t)cols + 4);
  b->dpart = cv.take<double>((size_t)s * s * block_dot_chunks(mx));
  b->raw = cv.take<double>((size_t)s * s);
  b->Bf = cv.take<double>((size_t)cols * cols);
  b->Bm = cv.take<double>((size_t)cols * cols);
  b->Yw = cv.take<double>((size_t)cols * cols);
  b->X = cv.take<double>((size_t)cols * cols);
  b->Y = cv.take<double>((size_t)cols * cols);
  b->sigma = cv.take<double>(cols);
  b->nrm = cv.take<double>(cols);
  b->pos = cv.take<int>(cols);
  b->sweeps = cv.take<int>(1);
  b->rank = cv.take<int>(1);
  b->split = b->acc ? cv.take<float>(accurate_floats(*op, s)) : nullptr;
  const size_t nparts = b->acc ? accurate_narrow_doubles(*op, s) : 0;
  b->npart = nparts ? cv.take<double>(nparts) : nullptr;
  b->q0 = cv.take<double>((size_t)m * s);  // staging of a host start block
  b->Qs = b->df ? cv.take<float2>((size_t)ldu * cols) : nullptr;
  b->Ps = b->df ? cv.take<float2>((size_t)ldv * cols) : nullptr;
  b->ws2 = b->df ? cv.take<float2>(lmax) : nullptr;
  b->gW = b->bgs ? cv.take<double>((size_t)mx * s) : nullptr;
  b->gC = b->bgs ? cv.take<double>((size_t)mx * s) : nullptr;
  b->gH = b->bgs ? cv.take<double>((size_t)cols * s) : nullptr;
  b->gpart = b->bgs ? cv.take<double>((size_t)bgs_dot_chunks(mx) * cols * s) : nullptr;
  b->gWs = b->bgs ? cv.take<float2>((size_t)mx * s) : nullptr;
  b->gHs = b->bgs ? cv.take<float2>((size_t)cols * s) : nullptr;
  char *dd;
  void *v, *tv;
  int32_t *rp, *ci, *trp, *tci;
  stage_carve(A, st, cv, op, &dd, &v, &rp, &ci, &tv, &trp, &tci);
  return cv.off + 256;
}

// block steps: kmax <= 0 means until the blocks fill min(m, n), within the small SVD's order
int block_steps(const gk_matrix *A, int s, int kmax, int64_t *kb) {
  const int64_t mn = A->m < A->n ? A->m : A->n;
  const int64_t cap = kBlockMaxOrder / s - 1;
  if (kmax <= 0) {
    int64_t k = mn / s;
    if (k > cap) k = cap;
    *kb = k < 1 ? 1 : k;
    return GK_OK;
  }
  if (kmax > cap) return GK_INVALID_ARG;
  *kb = kmax;
  return GK_OK;
}

// W[:, c] = op(A) src[:, c], c < s (W column-major with ld = the output length)
int block_product(const Op &op, BlockBufs &b, bool trans, const double *src, int64_t ldsrc, int s, cudaStream_t st,
                  const Dev &d) {
  const int64_t lin = trans ? op.m : op.n, lout = trans ? op.n : op.m;
  if (b.acc) {  // one pass over A for the whole block, products exact to ~2^-47
    GK_CUDA(cudaMemcpy2DAsync(b.Xc, sizeof(double) * lin, src, sizeof(double) * ldsrc, sizeof(double) * lin, s,
                              cudaMemcpyDeviceToDevice, st));
    GK_CUDA(accurate_products(op, trans, b.Xc, s, b.W, b.split, st, b.f32, true, b.npart));
    return GK_OK;
  }
  for (int c = 0; c < s; ++c) {
    const double *x = src + (int64_t)c * ldsrc;
    double *y = b.W + (int64_t)c * lout;
    GK_CUDA(copy_vec(nullptr, b.x32, x, lin, st));
    if (trans)
      GK_CUDA(matvec_t(op, b.x32, x, y, nullptr, nullptr, b.part, b.ctl, st, d));
    else
      GK_CUDA(matvec(op, b.x32, x, y, nullptr, nullptr, b.part, b.ctl, st, d));
  }
  return GK_OK;
}

// a column that the Gram-Schmidt reduced to rounding (the block is numerically rank deficient)
// is replaced by a fresh direction orthogonalized twice against the jc columns before it and
// normalized: an orthonormal completion, as a Householder QR of the block would give
int block_fresh(BlockBufs &b, int64_t len, double *Bas, int64_t ld, float2 *Bs, int jc, uint64_t seed, int64_t *nfresh,
                cudaStream_t st, const Dev &d) {
  GK_CUDA(draw_fresh(b.w, len, seed, (*nfresh)++, st));
  GK_CUDA(orthonormalize(b.w, len, Bas, ld, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 0, nullptr, nullptr, st, d));
  GK_CUDA(orthonormalize(b.w, len, Bas, ld, jc, 2, b.part, b.h, b.ctl, NM_FRESH, -1, 0, nullptr, nullptr, st, d, Bs,
                         b.ws2));
  GK_CUDA(normalize_append(b.w, len, Bas + (int64_t)jc * ld, nullptr, b.ctl, st, d, Bs ? Bs + (int64_t)jc * ld : nullptr));
  return GK_OK;
}

// columns jc0 .. jc0 + s - 1 of the basis Bas (ld; double-f32 shadow Bs or null): column c of
// Wsrc (ld ldw) orthonormalized by classical Gram-Schmidt, two passes, against the columns jlo ..
// before it -- with jlo = 0 the reorthogonalization and the QR of the block in one; with jlo = jc0
// the block's own QR (the block Gram-Schmidt projects against the earlier basis first).  With
// mode NM_BREAKDOWN a column whose norm after the passes is at most 2^-46 of the largest norm so
// far halts the launches that follow (an exact breakdown); the host then puts a fresh direction,
// orthogonalized against every column before it, in its place and goes on with the next column.
// NM_PLAIN only normalizes.
int block_orth(BlockBufs &b, int64_t len, double *Bas, int64_t ld, float2 *Bs, int jc0, int s, const double *Wsrc,
               int64_t ldw, int side, uint64_t seed, int64_t *nfresh, int *breakdowns, cudaStream_t st,
               const Dev &d, int jlo = 0, int mode = NM_BREAKDOWN) {
  int c0 = 0;
  double *Blo = Bas + (int64_t)jlo * ld;
  float2 *Bslo = Bs ? Bs + (int64_t)jlo * ld : nullptr;
  while (c0 < s) {
    for (int c = c0; c < s; ++c) {
      const int jc = jc0 + c;
      double *qcol = Bas + (int64_t)jc * ld;
      float2 *qs = Bs ? Bs + (int64_t)jc * ld : nullptr;
      GK_CUDA(copy_vec(b.w, nullptr, Wsrc + (int64_t)c * ldw, len, st));
      if (jc == jlo) {
        GK_CUDA(orthonormalize(b.w, len, nullptr, ld, 0, 0, b.part, b.h, b.ctl, mode, jc, side, nullptr, nullptr, st,
                               d));
        GK_CUDA(normalize_append(b.w, len, qcol, nullptr, b.ctl, st, d, qs));
      } else {
        GK_CUDA(orth_append(b.w, len, Blo, ld, jc - jlo, 2, b.part, b.h, b.ctl, mode, jc, side, nullptr, nullptr,
                            qcol, nullptr, st, d, Bslo, b.ws2, qs));
      }
    }
    HostCtl hc;
    int rc = read_ctl(b.ctl, nullptr, &hc, st);
    if (rc) return rc;
    if (hc.ctl.timeout || hc.ctl.event == EV_TIMEOUT) return GK_TIMEOUT;
    if (!hc.ctl.halt) return GK_OK;
    if (hc.ctl.event != EV_BREAKDOWN) return GK_NUMERICAL;
    const int jb = hc.ctl.step;  // the column the passes reduced to rounding
    if (jb < jc0 + c0 || jb >= jc0 + s) return GK_NUMERICAL;
    rc = clear_halt(b.ctl, st);
    if (rc) return rc;
    rc = block_fresh(b, len, Bas, ld, Bs, jb, seed, nfresh, st, d);
    if (rc) return rc;
    ++*breakdowns;
    c0 = jb - jc0 + 1;
  }
  return GK_OK;
}

// the block's columns by the block Gram-Schmidt (reorthogonalized block classical Gram-Schmidt,
// Barlow and Smoktunowicz 2013): W1 = W - Q (Q^T W) against the jc0 columns before the block, the
// block's own QR (with the breakdown test and fresh completions), W2 = W1' - Q (Q^T W1') for the
// orthonormal block W1' (removing what the QR's rounding brought back of Q's directions where a
// column cancelled), and the QR of W2 (plain normalization: its norms are ~1).  The column-wise
// flow where there is no earlier basis or no double-f32 copy of it.
int block_orth_bgs(BlockBufs &b, int64_t len, double *Bas, int64_t ld, float2 *Bs, int jc0, int s,
                   const double *Wsrc, int64_t ldw, int side, uint64_t seed, int64_t *nfresh, int *breakdowns,
                   cudaStream_t st, const Dev &d) {
  if (!b.bgs || jc0 == 0 || !Bs)
    return block_orth(b, len, Bas, ld, Bs, jc0, s, Wsrc, ldw, side, seed, nfresh, breakdowns, st, d);
  GK_CUDA(split_cols(Wsrc, len, ldw, s, b.gWs, st));
  GK_CUDA(bgs_project(Bs, ld, len, jc0, Wsrc, ldw, b.gWs, ldw, s, b.gpart, b.gH, b.gHs, b.gC, b.gW, st));
  int rc = block_orth(b, len, Bas, ld, Bs, jc0, s, b.gW, len, side, seed, nfresh, breakdowns, st, d, jc0,
                      NM_BREAKDOWN);
  if (rc) return rc;
  GK_CUDA(bgs_project(Bs, ld, len, jc0, Bas + (int64_t)jc0 * ld, ld, Bs + (int64_t)jc0 * ld, ld, s, b.gpart, b.gH,
                      b.gHs, b.gC, b.gW, st));
  return block_orth(b, len, Bas, ld, Bs, jc0, s, b.gW, len, side, seed, nfresh, breakdowns, st, d, jc0, NM_PLAIN);
}

int read_block(const BlockBufs &b, BlockCtl *hb, HostCtl *hc, cudaStream_t st) {
  GK_CUDA(cudaMemcpyAsync(hb, b.bc, sizeof(BlockCtl), cudaMemcpyDeviceToHost, st));
  GK_CUDA(cudaMemcpyAsync(&hc->ctl, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  GK_CUDA(cudaStreamSynchronize(st));
  if (hc->ctl.event == EV_TIMEOUT || hc->ctl.timeout) return GK_TIMEOUT;
  if (hc->ctl.event == EV_NUMERICAL || hb->brk == 2) return GK_NUMERICAL;
  return GK_OK;
}

// One block sweep's state (block_impl, block_fsvd_impl): options, operator, buffers and counts.
struct BlockRun {
  gk_opts o;
  cudaStream_t st = nullptr;
  Dev d;
  OpStage stg;
  Op op;
  BlockBufs b{};
  Workspace ws;
  int64_t m = 0, n = 0, ldu = 0, ldv = 0, cols = 0, kb = 0;
  int s = 0;
  int64_t nfresh = 0, matvecs = 0;
  int breakdowns = 0;
  Prof prof;  // GK_FLAG_PROFILE: products (A P, A^T Q), Gram-Schmidt, small kernels and SVD, Ritz vectors
};

// The workspace and the staged operator; Q_1 R_0 = Q0 (the given block, or column c drawn as
// Algorithm 1's start vector with seed + c); P_1 R_1 = A^T Q_1 and sigma~ = ||R_1|| (the first
// right block judged with eps).
int block_begin(BlockRun &R, const gk_matrix *Ain, int s, const double *Q0, int64_t kb, const gk_opts &o,
                const Dev &d, double eps) {
  R.o = o;
  R.st = (cudaStream_t)o.stream;
  R.d = d;
  R.s = s;
  R.kb = kb;
  R.m = Ain->m;
  R.n = Ain->n;
  R.prof.on = (o.flags & GK_FLAG_PROFILE) != 0;
  R.prof.s = R.st;
  const cudaStream_t st = R.st;
  int rc = stage_plan(Ain, &R.stg);
  if (rc) return rc;
  const bool host_q0 = Q0 && on_host(Q0);
  BlockBufs &b = R.b;
  R.op = make_op(Ain);
  b.df = (o.flags & GK_FLAG_ORTH_F64) == 0;
  b.acc = accurate_ok(R.op);
  b.f32 = (o.flags & GK_FLAG_BLOCK_F32) != 0;
  b.bgs = b.df && (o.flags & GK_FLAG_BLOCK_GS) != 0;
  const size_t bytes = block_layout(Ain, s, kb, d, R.stg, nullptr, &b, &R.op);
  rc = acquire(R.ws, bytes, o, st);
  if (rc) return rc;
  R.op = make_op(Ain);
  block_layout(Ain, s, kb, d, R.stg, R.ws.base, &b, &R.op);
  rc = stage_copy(Ain, R.stg, R.op, st);
  if (rc) return rc;
  const int64_t m = R.m, n = R.n;
  R.ldu = round_up(m, 32);
  R.ldv = round_up(n, 32);
  R.cols = (kb + 1) * s;
  const int64_t ldu = R.ldu, ldv = R.ldv, cols = R.cols;
  GK_CUDA(reset_ctl(b.ctl, 0.0, 1, st));
  GK_CUDA(cudaMemsetAsync(b.bc, 0, sizeof(BlockCtl), st));
  GK_CUDA(cudaMemsetAsync(b.Bf, 0, sizeof(double) * cols * cols, st));
  if (b.df) {  // the shadows' padding rows (past m, n) are read beside the last odd row: keep them 0
    GK_CUDA(cudaMemsetAsync(b.Qs, 0, sizeof(float2) * ldu * cols, st));
    GK_CUDA(cudaMemsetAsync(b.Ps, 0, sizeof(float2) * ldv * cols, st));
  }
  const double *q0 = Q0;
  if (host_q0) {
    GK_CUDA(cudaMemcpyAsync(b.q0, Q0, sizeof(double) * m * s, cudaMemcpyHostToDevice, st));
    q0 = b.q0;
  }
  if (!q0) {
    for (int c = 0; c < s; ++c) GK_CUDA(draw_start(b.W + (int64_t)c * m, m, o.seed + (uint64_t)c, st));
    q0 = b.W;
  }
  R.prof.begin(PC_ORTH);
  rc = block_orth_bgs(b, m, b.Q, ldu, b.Qs, 0, s, q0, m, 0, o.seed, &R.nfresh, &R.breakdowns, st, d);
  if (rc) return rc;
  R.prof.end();
  GK_CUDA(reset_ctl(b.ctl, 0.0, 1, st));  // the breakdown scale follows the blocks' norms from here
  R.prof.begin(PC_MATVEC_T);
  rc = block_product(R.op, b, true, b.Q, ldu, s, st, d);
  if (rc) return rc;
  R.prof.end();
  R.prof.begin(PC_ORTH);
  rc = block_orth_bgs(b, n, b.P, ldv, b.Ps, 0, s, b.W, n, 1, o.seed, &R.nfresh, &R.breakdowns, st, d);
  if (rc) return rc;
  R.prof.end();
  R.prof.begin(PC_SMALL);
  GK_CUDA(block_dots(b.P, ldv, b.W, n, n, s, b.dpart, b.raw, st));
  GK_CUDA(block_judge(b.raw, s, b.Bf, cols, 0, 0, 2, eps, b.bc, st));
  R.prof.end();
  R.matvecs = s;
  return GK_OK;
}

// Q_{j+1} S_{j+1} = A P_j - Q_j R_j^T, reorthogonalized, judged (left side) and read back (j = steps)
int block_left_step(BlockRun &R, int steps, double eps, BlockCtl *hb, HostCtl *hc) {
  BlockBufs &b = R.b;
  const int s = R.s;
  const int64_t pj = (int64_t)(steps - 1) * s, qn = (int64_t)steps * s;
  R.prof.begin(PC_MATVEC);
  int rc = block_product(R.op, b, false, b.P + pj * R.ldv, R.ldv, s, R.st, R.d);
  if (rc) return rc;
  R.prof.end();
  R.prof.begin(PC_ORTH);
  rc = block_orth_bgs(b, R.m, b.Q, R.ldu, b.Qs, (int)qn, s, b.W, R.m, 0, R.o.seed, &R.nfresh, &R.breakdowns, R.st,
                      R.d);
  if (rc) return rc;
  R.prof.end();
  R.prof.begin(PC_SMALL);
  GK_CUDA(block_dots(b.Q + qn * R.ldu, R.ldu, b.W, R.m, R.m, s, b.dpart, b.raw, R.st));
  GK_CUDA(block_judge(b.raw, s, b.Bf, R.cols, (int)qn, (int)pj, 0, eps, b.bc, R.st));
  R.prof.end();
  R.matvecs += s;
  return read_block(b, hb, hc, R.st);
}

// P_{j+1} R_{j+1} = A^T Q_{j+1} - P_j S_{j+1}^T, reorthogonalized, judged (right side) and read back
int block_right_step(BlockRun &R, int steps, double eps, BlockCtl *hb, HostCtl *hc) {
  BlockBufs &b = R.b;
  const int s = R.s;
  const int64_t qn = (int64_t)steps * s;
  R.prof.begin(PC_MATVEC_T);
  int rc = block_product(R.op, b, true, b.Q + qn * R.ldu, R.ldu, s, R.st, R.d);
  if (rc) return rc;
  R.prof.end();
  R.prof.begin(PC_ORTH);
  rc = block_orth_bgs(b, R.n, b.P, R.ldv, b.Ps, (int)qn, s, b.W, R.n, 1, R.o.seed, &R.nfresh, &R.breakdowns, R.st,
                      R.d);
  if (rc) return rc;
  R.prof.end();
  R.prof.begin(PC_SMALL);
  GK_CUDA(block_dots(b.P + qn * R.ldv, R.ldv, b.W, R.n, R.n, s, b.dpart, b.raw, R.st));
  GK_CUDA(block_judge(b.raw, s, b.Bf, R.cols, (int)qn, (int)qn, 1, eps, b.bc, R.st));
  R.prof.end();
  R.matvecs += s;
  return read_block(b, hb, hc, R.st);
}

int block_impl(const gk_matrix *Ain, int s, const double *Q0, double eps, int kmax, const gk_opts *oin, int *rank,
               double *sigma, int *steps_out, gk_info *info) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launch_count();
  g_err[0] = 0;
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  if (info) *info = inf;
  // the arguments first: a bad request is refused with or without a device
  int rc = check_matrix(Ain);
  if (rc) return rc;
  const int64_t mn = Ain->m < Ain->n ? Ain->m : Ain->n;
  if (!rank || s < 1 || s > kBlockMaxS || s > mn || !(eps >= 0.0) || !isfinite(eps)) return GK_INVALID_ARG;
  const gk_opts o = oin ? *oin : defaults();
  if (o.eps_absolute) return GK_INVALID_ARG;
  int64_t kb = 0;
  rc = block_steps(Ain, s, kmax, &kb);
  if (rc) return rc;
  Dev d;
  if (!get_device(&d)) return GK_NO_DEVICE;
  const bool host_sigma = sigma && on_host(sigma);
  BlockRun R;
  rc = block_begin(R, Ain, s, Q0, kb, o, d, eps);
  if (rc) return rc;
  BlockBufs &b = R.b;
  const cudaStream_t st = R.st;
  int steps = 1, stop = 0;
  BlockCtl hb;
  HostCtl hc;
  for (;;) {
    rc = block_left_step(R, steps, eps, &hb, &hc);
    if (rc) return rc;
    if (hb.brk) {
      stop = 1;
      break;
    }
    if (steps >= kb) {
      stop = 0;
      break;
    }
    if ((int64_t)(steps + 1) * s > mn) {
      stop = 3;
      break;
    }
    rc = block_right_step(R, steps, eps, &hb, &hc);
    if (rc) return rc;
    if (hb.brk) {
      stop = 2;
      break;
    }
    ++steps;
  }
  // Algorithm 3 on B ((steps + 1) s x steps s), padded with zero columns to its square
  const int K = (steps + 1) * s, nsig = steps * s;
  R.prof.begin(PC_SMALL);
  GK_CUDA(cudaMemcpy2DAsync(b.Bm, sizeof(double) * K, b.Bf, sizeof(double) * R.cols, sizeof(double) * K, K,
                            cudaMemcpyDeviceToDevice, st));
  GK_CUDA(small_svd(b.Bm, b.Yw, K, b.sigma, b.X, b.Y, b.nrm, b.pos, b.sweeps, b.ctl, st));
  GK_CUDA(block_count(b.sigma, nsig, eps, b.rank, st));
  R.prof.end();
  if (sigma) {
    if (host_sigma)
      GK_CUDA(cudaMemcpyAsync(sigma, b.sigma, sizeof(double) * nsig, cudaMemcpyDeviceToHost, st));
    else
      GK_CUDA(cudaMemcpyAsync(sigma, b.sigma, sizeof(double) * nsig, cudaMemcpyDeviceToDevice, st));
  }
  int r = 0, sweeps = 0;
  GK_CUDA(cudaMemcpyAsync(&r, b.rank, sizeof(int), cudaMemcpyDeviceToHost, st));
  GK_CUDA(cudaMemcpyAsync(&sweeps, b.sweeps, sizeof(int), cudaMemcpyDeviceToHost, st));
  GK_CUDA(cudaStreamSynchronize(st));
  *rank = r;
  if (steps_out) *steps_out = steps;
  inf.steps = steps;
  inf.kprime = nsig;
  inf.stop_reason = stop;
  inf.matvecs = R.matvecs;
  inf.svd_sweeps = sweeps;
  inf.breakdowns = R.breakdowns;
  inf.sigma_est = hb.sest;
  R.prof.finish(&inf);
  inf.seconds = seconds_since(t0);
  inf.launches = launch_count() - l0;
  if (info) *info = inf;
  return sweeps < 0 ? GK_NOT_CONVERGED : GK_OK;
}

// One cycle of the block form of Algorithm 2 (route 1): `steps` block steps without a break
// test, the SVD of B (padded with zero columns to its square), U = Q X_r, V = P Y_r, and each
// triplet's right residual ||R_{k+1} x_i'|| from the next right block (formed, never kept).
int block_fsvd_impl(const gk_matrix *Ain, int s, const double *Q0, int steps_in, int r, const gk_opts *oin, double *U,
                    double *S, double *V, double *resid, gk_info *info) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launch_count();
  g_err[0] = 0;
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  if (info) *info = inf;
  int rc = check_matrix(Ain);
  if (rc) return rc;
  const int64_t m = Ain->m, n = Ain->n, mn = m < n ? m : n;
  if (s < 1 || s > kBlockMaxS || s > mn || steps_in < 1 || r < 1 || !U || !S || !V || !resid) return GK_INVALID_ARG;
  int64_t kb = 0;
  rc = block_steps(Ain, s, steps_in, &kb);
  if (rc) return rc;
  if ((int64_t)r > kb * s) return GK_INVALID_ARG;
  Dev d;
  if (!get_device(&d)) return GK_NO_DEVICE;
  if (on_host(U) || on_host(S) || on_host(V) || on_host(resid)) return GK_INVALID_ARG;  // device outputs only
  const gk_opts o = oin ? *oin : defaults();
  BlockRun R;
  rc = block_begin(R, Ain, s, Q0, kb, o, d, 0.0);
  if (rc) return rc;
  BlockBufs &b = R.b;
  const cudaStream_t st = R.st;
  const int64_t ldu = R.ldu, ldv = R.ldv;
  int steps = 1;
  BlockCtl hb;
  HostCtl hc;
  for (;;) {  // eps = 0: no block ends the sweep; it runs kb steps or until the blocks fill min(m, n)
    rc = block_left_step(R, steps, 0.0, &hb, &hc);
    if (rc) return rc;
    if (steps >= kb || (int64_t)(steps + 1) * s > mn) break;
    rc = block_right_step(R, steps, 0.0, &hb, &hc);
    if (rc) return rc;
    ++steps;
  }
  const int K = (steps + 1) * s, ks = steps * s;
  const int rr = r < ks ? r : ks;
  if (rr < r) {  // the blocks filled the space first: the trailing triplets are zero
    GK_CUDA(cudaMemsetAsync(U, 0, sizeof(double) * (size_t)m * r, st));
    GK_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)n * r, st));
    GK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * (size_t)r, st));
    GK_CUDA(cudaMemsetAsync(resid, 0, sizeof(double) * (size_t)r, st));
  }
  // the next right block P_{k+1} R_{k+1} = A^T Q_{k+1} - P_k S_{k+1}^T (reorthogonalized): R_{k+1}
  // in b.raw for the residuals
  {
    const int64_t qn = (int64_t)steps * s;
    R.prof.begin(PC_MATVEC_T);
    rc = block_product(R.op, b, true, b.Q + qn * ldu, ldu, s, st, d);
    if (rc) return rc;
    R.prof.end();
    R.prof.begin(PC_ORTH);
    rc = block_orth_bgs(b, n, b.P, ldv, b.Ps, (int)qn, s, b.W, n, 1, o.seed, &R.nfresh, &R.breakdowns, st, d);
    if (rc) return rc;
    R.prof.end();
    GK_CUDA(block_dots(b.P + qn * ldv, ldv, b.W, n, n, s, b.dpart, b.raw, st));
    R.matvecs += s;
  }
  R.prof.begin(PC_SMALL);
  GK_CUDA(cudaMemcpy2DAsync(b.Bm, sizeof(double) * K, b.Bf, sizeof(double) * R.cols, sizeof(double) * K, K,
                            cudaMemcpyDeviceToDevice, st));
  GK_CUDA(small_svd(b.Bm, b.Yw, K, b.sigma, b.X, b.Y, b.nrm, b.pos, b.sweeps, b.ctl, st));
  R.prof.end();
  R.prof.begin(PC_RESTART);
  // U = Q X_r (all K rows of X), V = P_{1..k} Y_r (the first ks rows: the padding columns of B
  // never enter the right vectors of nonzero values); with GK_FLAG_RITZ_DF from the bases'
  // double-f32 copies (b.Yw, free after the small SVD, holds X's and then Y's split)
  if ((o.flags & GK_FLAG_RITZ_DF) && b.df) {
    GK_CUDA(ritz_gemm_df(b.Qs, ldu, m, K, b.X, K, rr, U, m, reinterpret_cast<float2 *>(b.Yw), st));
    GK_CUDA(ritz_gemm_df(b.Ps, ldv, n, ks, b.Y, K, rr, V, n, reinterpret_cast<float2 *>(b.Yw), st));
  } else {
    GK_CUDA(ritz_gemm(b.Q, ldu, m, K, b.X, K, rr, U, m, st, d));
    GK_CUDA(ritz_gemm(b.P, ldv, n, ks, b.Y, K, rr, V, n, st, d));
  }
  R.prof.end();
  GK_CUDA(block_resid(b.raw, s, b.X, K, ks, rr, resid, st));
  GK_CUDA(cudaMemcpyAsync(S, b.sigma, sizeof(double) * rr, cudaMemcpyDeviceToDevice, st));
  GK_CUDA(sign_normalize(U, m, m, V, n, n, rr, st));
  int sweeps = 0;
  GK_CUDA(cudaMemcpyAsync(&sweeps, b.sweeps, sizeof(int), cudaMemcpyDeviceToHost, st));
  GK_CUDA(cudaStreamSynchronize(st));
  inf.steps = steps;
  inf.kprime = ks;
  inf.matvecs = R.matvecs;
  inf.svd_sweeps = sweeps;
  inf.breakdowns = R.breakdowns;
  inf.sigma_est = hb.sest;
  R.prof.finish(&inf);
  inf.seconds = seconds_since(t0);
  inf.launches = launch_count() - l0;
  if (info) *info = inf;
  if (sweeps < 0) return GK_NOT_CONVERGED;
  return rr < r ? GK_RANK_DEFICIENT : GK_OK;
}

// ---------------------------------------------------------------------------
// gk_fsvd: Algorithm 2 as printed (k steps of Algorithm 1, the SVD of B_{k'+1,k'}, no restart)
// ---------------------------------------------------------------------------
struct FsvdBufs {
  double *Bm, *Yw, *X, *Y, *sigma, *nrm, *Uo, *So, *Vo;
  float *split;
  int *pos, *sweeps;
};

size_t fsvd_layout(char *base, int k, int r, int64_t m, int64_t n, bool host_out, size_t split_floats, FsvdBufs *f) {
  Carve cv{base, 0};
  const size_t K = (size_t)k + 1;
  f->Bm = cv.take<double>(K * K);
  f->Yw = cv.take<double>(K * K);
  f->X = cv.take<double>(K * K);
  f->Y = cv.take<double>(K * K);
  f->sigma = cv.take<double>(K);
  f->nrm = cv.take<double>(K);
  f->pos = cv.take<int>(K);
  f->sweeps = cv.take<int>(1);
  f->Uo = host_out ? cv.take<double>((size_t)m * r) : nullptr;
  f->So = host_out ? cv.take<double>((size_t)r) : nullptr;
  f->Vo = host_out ? cv.take<double>((size_t)n * r) : nullptr;
  f->split = split_floats ? cv.take<float>(split_floats) : nullptr;
  return cv.off + 256;
}

int fsvd_impl(const gk_matrix *Ain, int k, int r, int route, const gk_opts *oin, double *U, double *S, double *V,
              gk_info *info) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launch_count();
  g_err[0] = 0;
  gk_info inf;
  memset(&inf, 0, sizeof(inf));
  if (info) *info = inf;
  Dev d;
  if (!get_device(&d)) return GK_NO_DEVICE;
  int rc = check_matrix(Ain);
  if (rc) return rc;
  const int64_t m = Ain->m, n = Ain->n, ldu = round_up(m, 32), ldv = round_up(n, 32);
  const int64_t mn = m < n ? m : n;
  if (k < 1 || k > mn || k > 1023 || r < 1 || r > k || (route != 0 && route != 1) || !U || !S || !V)
    return GK_INVALID_ARG;
  const gk_opts o = oin ? *oin : defaults();
  if (o.reorth_passes < 0 || o.reorth_passes > 3) return GK_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)o.stream;
  OpStage st;
  rc = stage_plan(Ain, &st);
  if (rc) return rc;
  const bool host_start = o.start && on_host(o.start);
  const bool host_out = on_host(U) || on_host(S) || on_host(V);
  Op op = make_op(Ain);
  RankBufs b;
  b.fused = (o.flags & GK_FLAG_FUSED) && fused_ok_staged(op, st, d);
  b.df = (o.flags & GK_FLAG_ORTH_F64) == 0;
  FsvdBufs f;
  const size_t nb = (numrank_layout(Ain, k, d, st, false, host_start, nullptr, &b, &op) + 255) / 256 * 256;
  const size_t split_floats = (route == 0 && accurate_ok(op)) ? accurate_floats(op, r) : 0;
  const size_t fb = fsvd_layout(nullptr, k, r, m, n, host_out, split_floats, &f);
  Workspace ws;
  rc = acquire(ws, nb + fb, o, s);
  if (rc) return rc;
  op = make_op(Ain);
  numrank_layout(Ain, k, d, st, false, host_start, ws.base, &b, &op);
  fsvd_layout(ws.base + nb, k, r, m, n, host_out, split_floats, &f);
  rc = stage_copy(Ain, st, op, s);
  if (rc) return rc;
  Prof prof;
  prof.on = (o.flags & GK_FLAG_PROFILE) != 0;
  prof.s = s;
  HostCtl hc;
  int kp = 0;
  // k steps of Algorithm 1; with the absolute threshold 0 only an exact zero ends them early
  rc = lower_sweep(Ain, o, op, b, k, 0.0, 0, host_start, prof, inf, hc, &kp, s, d);
  if (rc) return rc;
  inf.kprime = kp;
  inf.steps = kp;
  double *Uo = host_out ? f.Uo : U, *Vo = host_out ? f.Vo : V, *So = host_out ? f.So : S;
  GK_CUDA(cudaMemsetAsync(Uo, 0, sizeof(double) * (size_t)m * r, s));
  GK_CUDA(cudaMemsetAsync(Vo, 0, sizeof(double) * (size_t)n * r, s));
  GK_CUDA(cudaMemsetAsync(So, 0, sizeof(double) * (size_t)r, s));
  const int rr = r < kp ? r : kp;
  int sweeps = 0;
  if (kp > 0) {
    // a break on the left side appended no q_{k'+1}: its column of Q is zero (beta_{k'+1} = 0)
    if (hc.ctl.halt && hc.ctl.side == 0) GK_CUDA(cudaMemsetAsync(b.Q + (int64_t)kp * ldu, 0, sizeof(double) * m, s));
    rc = clear_halt(b.ctl, s);
    if (rc) return rc;
    if (route == 1) {
      // the SVD of B_{k'+1,k'} itself (padded with a zero column to a square): V = P Y, U = Q X
      const int K = kp + 1;
      prof.begin(PC_SMALL);
      if ((o.flags & GK_FLAG_BDSVD) && K <= kBdMaxK) {
        // Golub-Kahan SVD steps on the transpose: the padded B^T is upper bidiagonal with
        // alpha_1..alpha_k' on the diagonal (the padding's 0 last), beta_2..beta_{k'+1} above it;
        // B^T = X' S Y'^T gives B = Y' S X'^T, so X' is B's right and Y' its left vectors
        GK_CUDA(cudaMemsetAsync(b.alpha + kp, 0, sizeof(double), s));
        GK_CUDA(bd_svd(b.alpha, b.beta + 1, K, f.sigma, f.Y, f.X, f.Bm, f.Yw, f.sweeps, b.ctl, s));
      } else {
        GK_CUDA(assemble_lower(f.Bm, kp, b.alpha, b.beta, s));
        GK_CUDA(small_svd(f.Bm, f.Yw, K, f.sigma, f.X, f.Y, f.nrm, f.pos, f.sweeps, b.ctl, s));
      }
      prof.end();
      prof.begin(PC_RESTART);
      // V = P Y: the first kp rows of Y (the zero padding column is never rotated)
      GK_CUDA(ritz_gemm(b.P, ldv, n, kp, f.Y, K, rr, Vo, n, s, d));
      GK_CUDA(ritz_gemm(b.Q, ldu, m, K, f.X, K, rr, Uo, m, s, d));
      prof.end();
    } else {
      // Algorithm 2 as printed: the eigendecomposition of B^T B (formed, tridiagonal; its one-sided
      // Jacobi SVD is its eigendecomposition since it is positive semidefinite), sigma = sqrt(theta),
      // V = P Y, and u_i = A v_i / sigma_i for all r triplets in one blocked pass over A
      prof.begin(PC_SMALL);
      GK_CUDA(assemble_btb(f.Bm, kp, b.alpha, b.beta, s));
      GK_CUDA(small_svd(f.Bm, f.Yw, kp, f.sigma, f.X, f.Y, f.nrm, f.pos, f.sweeps, b.ctl, s));
      GK_CUDA(sqrt_vals(f.sigma, kp, s));
      prof.end();
      prof.begin(PC_RESTART);
      GK_CUDA(ritz_gemm(b.P, ldv, n, kp, f.Y, kp, rr, Vo, n, s, d));
      if (accurate_ok(op)) {
        GK_CUDA(accurate_products(op, false, Vo, rr, Uo, f.split, s));
      } else {
        for (int i = 0; i < rr; ++i) {
          double *vi = Vo + (int64_t)i * n, *ui = Uo + (int64_t)i * m;
          GK_CUDA(copy_vec(nullptr, b.x32, vi, n, s));
          GK_CUDA(matvec(op, b.x32, vi, ui, nullptr, nullptr, b.part, b.ctl, s, d));
        }
      }
      GK_CUDA(scale_cols(Uo, m, rr, f.sigma, s));
      prof.end();
      inf.matvecs += rr;
    }
    GK_CUDA(cudaMemcpyAsync(So, f.sigma, sizeof(double) * rr, cudaMemcpyDeviceToDevice, s));
    GK_CUDA(sign_normalize(Uo, m, m, Vo, n, n, rr, s));
    GK_CUDA(cudaMemcpyAsync(&sweeps, f.sweeps, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  if (host_out) {
    prof.begin(PC_COPY);
    GK_CUDA(cudaMemcpyAsync(U, Uo, sizeof(double) * (size_t)m * r, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(V, Vo, sizeof(double) * (size_t)n * r, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(S, So, sizeof(double) * (size_t)r, cudaMemcpyDeviceToHost, s));
    prof.end();
  }
  GK_CUDA(cudaMemcpyAsync(&hc.ctl, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  GK_CUDA(cudaStreamSynchronize(s));
  prof.finish(&inf);
  inf.svd_sweeps = sweeps;
  inf.reserved = b.fused ? fused_cluster(op, d) : 0;
  inf.sigma_est = hc.ctl.sest;
  inf.seconds = seconds_since(t0);
  inf.launches = launch_count() - l0;
  if (info) *info = inf;
  if (hc.ctl.timeout) return GK_TIMEOUT;
  if (sweeps < 0) return GK_NOT_CONVERGED;
  return rr < r ? GK_RANK_DEFICIENT : GK_OK;
}

// ---------------------------------------------------------------------------
// gk_matvec / gk_residuals
// ---------------------------------------------------------------------------
struct VecBufs {
  Ctl *ctl;
  double *x, *y, *part, *h, *U, *S, *V, *r1, *r2, *Y, *Z;
  float *x32, *split;
};

size_t vec_layout(const gk_matrix *A, const Dev &d, const OpStage &st, int k, char *base, VecBufs *b, Op *op) {
  Carve cv{base, 0};
  const int64_t ld = round_up(A->m > A->n ? A->m : A->n, 32);
  b->ctl = cv.take<Ctl>(1);
  b->x = cv.take<double>(ld);
  b->y = cv.take<double>(ld);
  b->x32 = cv.take<float>(ld);
  const int64_t g = cgs_blocks(A->m > A->n ? A->m : A->n, d);
  int64_t pc = 2 * g + 8;
  const int64_t gp = gemvt_partials(*op, d);
  if (gp > pc) pc = gp;
  b->part = cv.take<double>(pc);
  b->h = cv.take<double>(4);
  b->Y = b->Z = nullptr;
  b->split = nullptr;
  if (k > 0) {
    b->U = cv.take<double>((size_t)A->m * k);
    b->V = cv.take<double>((size_t)A->n * k);
    b->S = cv.take<double>(k);
    b->r1 = cv.take<double>(k);
    b->r2 = cv.take<double>(k);
    if (accurate_ok(*op)) {
      b->Y = cv.take<double>((size_t)A->m * k);
      b->Z = cv.take<double>((size_t)A->n * k);
      b->split = cv.take<float>(accurate_floats(*op, k));
    }
  }
  char *dd;
  void *v, *tv;
  int32_t *rp, *ci, *trp, *tci;
  stage_carve(A, st, cv, op, &dd, &v, &rp, &ci, &tv, &trp, &tci);
  return cv.off + 256;
}

int matvec_impl(const gk_matrix *Ain, int trans, const double *x, double *y, const gk_opts *oin) {
  g_err[0] = 0;
  Dev d;
  if (!get_device(&d)) return GK_NO_DEVICE;
  int rc = check_matrix(Ain);
  if (rc) return rc;
  if (!x || !y || (trans != 0 && trans != 1)) return GK_INVALID_ARG;
  const gk_opts o = oin ? *oin : defaults();
  cudaStream_t s = (cudaStream_t)o.stream;
  OpStage st;
  rc = stage_plan(Ain, &st);
  if (rc) return rc;
  Op op = make_op(Ain);
  VecBufs b;
  const size_t bytes = vec_layout(Ain, d, st, 0, nullptr, &b, &op);
  Workspace ws;
  rc = acquire(ws, bytes, o, s);
  if (rc) return rc;
  op = make_op(Ain);
  vec_layout(Ain, d, st, 0, ws.base, &b, &op);
  rc = stage_copy(Ain, st, op, s);
  if (rc) return rc;
  const int64_t nin = trans ? Ain->m : Ain->n, nout = trans ? Ain->n : Ain->m;
  GK_CUDA(reset_ctl(b.ctl, 0.0, 1, s));
  GK_CUDA(cudaMemcpyAsync(b.x, x, sizeof(double) * nin, cudaMemcpyDefault, s));
  GK_CUDA(copy_vec(nullptr, b.x32, b.x, nin, s));
  if (trans)
    GK_CUDA(matvec_t(op, b.x32, b.x, b.y, nullptr, nullptr, b.part, b.ctl, s, d));
  else
    GK_CUDA(matvec(op, b.x32, b.x, b.y, nullptr, nullptr, b.part, b.ctl, s, d));
  GK_CUDA(cudaMemcpyAsync(y, b.y, sizeof(double) * nout, cudaMemcpyDefault, s));
  HostCtl hc;
  rc = read_ctl(b.ctl, nullptr, &hc, s);
  if (rc) return rc;
  return hc.ctl.event == EV_TIMEOUT ? GK_TIMEOUT : GK_OK;
}

int residuals_impl(const gk_matrix *Ain, int k, const double *U, const double *S, const double *V, double *r_av,
                   double *r_atu, const gk_opts *oin) {
  g_err[0] = 0;
  Dev d;
  if (!get_device(&d)) return GK_NO_DEVICE;
  int rc = check_matrix(Ain);
  if (rc) return rc;
  if (!U || !S || !V || !r_av || !r_atu || k < 1) return GK_INVALID_ARG;
  const gk_opts o = oin ? *oin : defaults();
  cudaStream_t s = (cudaStream_t)o.stream;
  OpStage st;
  rc = stage_plan(Ain, &st);
  if (rc) return rc;
  Op op = make_op(Ain);
  VecBufs b;
  const size_t bytes = vec_layout(Ain, d, st, k, nullptr, &b, &op);
  Workspace ws;
  rc = acquire(ws, bytes, o, s);
  if (rc) return rc;
  op = make_op(Ain);
  vec_layout(Ain, d, st, k, ws.base, &b, &op);
  rc = stage_copy(Ain, st, op, s);
  if (rc) return rc;
  const int64_t m = Ain->m, n = Ain->n;
  GK_CUDA(reset_ctl(b.ctl, 0.0, 1, s));
  GK_CUDA(cudaMemcpyAsync(b.U, U, sizeof(double) * m * k, cudaMemcpyDefault, s));
  GK_CUDA(cudaMemcpyAsync(b.V, V, sizeof(double) * n * k, cudaMemcpyDefault, s));
  GK_CUDA(cudaMemcpyAsync(b.S, S, sizeof(double) * k, cudaMemcpyDefault, s));
  if (accurate_ok(op)) {
    // all k triplets per pass over A, FP64-grade (double-f32) products
    GK_CUDA(accurate_products(op, false, b.V, k, b.Y, b.split, s));
    GK_CUDA(resid_norms(b.Y, b.U, b.S, m, k, b.r1, s));
    GK_CUDA(accurate_products(op, true, b.U, k, b.Z, b.split, s));
    GK_CUDA(resid_norms(b.Z, b.V, b.S, n, k, b.r2, s));
  } else {
  for (int i = 0; i < k; ++i) {
    const double *ui = b.U + (int64_t)i * m, *vi = b.V + (int64_t)i * n;
    GK_CUDA(copy_vec(nullptr, b.x32, vi, n, s));
    GK_CUDA(matvec(op, b.x32, vi, b.y, ui, b.S + i, b.part, b.ctl, s, d));
    GK_CUDA(orthonormalize(b.y, m, nullptr, m, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 0, b.r1 + i, nullptr, s, d));
    GK_CUDA(copy_vec(nullptr, b.x32, ui, m, s));
    GK_CUDA(matvec_t(op, b.x32, ui, b.y, vi, b.S + i, b.part, b.ctl, s, d));
    GK_CUDA(orthonormalize(b.y, n, nullptr, n, 0, 0, b.part, b.h, b.ctl, NM_PLAIN, -1, 1, b.r2 + i, nullptr, s, d));
  }
  }
  GK_CUDA(cudaMemcpyAsync(r_av, b.r1, sizeof(double) * k, cudaMemcpyDefault, s));
  GK_CUDA(cudaMemcpyAsync(r_atu, b.r2, sizeof(double) * k, cudaMemcpyDefault, s));
  GK_CUDA(cudaStreamSynchronize(s));
  return GK_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// exported C ABI
// ---------------------------------------------------------------------------
extern "C" {

void gk_default_opts(gk_opts *opts) {
  if (opts) *opts = defaults();
}

size_t gk_psvd_workspace(const gk_matrix *A, int k, const gk_opts *oin) {
  Dev d;
  if (!get_device(&d) || check_matrix(A) != GK_OK) return 0;
  const gk_opts o = oin ? *oin : defaults();
  PsvdPlan p;
  if (psvd_plan(A, k, o, &p) != GK_OK) return 0;
  OpStage st;
  if (stage_plan(A, &st) != GK_OK) return 0;
  PsvdBufs b;
  Op op = make_op(A);
  p.fused = (o.flags & GK_FLAG_FUSED) && fused_ok_staged(op, st, d);
  return psvd_layout(A, p, d, st, false, false, nullptr, &b, &op);
}

// NVTX ranges name each entry point's span for profilers (no cost without one attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int gk_psvd(const gk_matrix *A, int k, double tol, const gk_opts *opts, double *U, double *S, double *V,
            gk_info *info) {
  NvtxRange r("gk_psvd");
  return psvd_impl(A, k, tol, opts, U, S, V, info);
}

size_t gk_numrank_workspace(const gk_matrix *A, int kmax, const gk_opts *oin) {
  Dev d;
  if (!get_device(&d) || check_matrix(A) != GK_OK) return 0;
  const gk_opts o = oin ? *oin : defaults();
  OpStage st;
  if (stage_plan(A, &st) != GK_OK) return 0;
  RankBufs b;
  Op op = make_op(A);
  b.fused = (o.flags & GK_FLAG_FUSED) && fused_ok_staged(op, st, d);
  b.df = (o.flags & GK_FLAG_ORTH_F64) == 0;
  return numrank_layout(A, clamp_kmax(A, kmax), d, st, false, false, nullptr, &b, &op);
}

int gk_numrank(const gk_matrix *A, double eps, int kmax, const gk_opts *opts, int *rank, double *sigma,
               gk_info *info) {
  NvtxRange r("gk_numrank");
  return numrank_impl(A, eps, kmax, opts, rank, sigma, info);
}

int gk_block_fsvd(const gk_matrix *A, int s, const double *Q0, int steps, int r, const gk_opts *opts, double *U,
                  double *S, double *V, double *resid, gk_info *info) {
  NvtxRange nv("gk_block_fsvd");
  return block_fsvd_impl(A, s, Q0, steps, r, opts, U, S, V, resid, info);
}

size_t gk_block_numrank_workspace(const gk_matrix *A, int s, int kmax, const gk_opts *oin) {
  Dev d;
  if (check_matrix(A) != GK_OK || s < 1 || s > kBlockMaxS || s > A->m || s > A->n) return 0;
  int64_t kb = 0;
  if (block_steps(A, s, kmax, &kb) != GK_OK || !get_device(&d)) return 0;
  const gk_opts o = oin ? *oin : defaults();
  OpStage st;
  if (stage_plan(A, &st) != GK_OK) return 0;
  Op op = make_op(A);
  BlockBufs b{};
  b.df = (o.flags & GK_FLAG_ORTH_F64) == 0;
  b.acc = accurate_ok(op);
  b.f32 = (o.flags & GK_FLAG_BLOCK_F32) != 0;
  b.bgs = b.df && (o.flags & GK_FLAG_BLOCK_GS) != 0;
  return block_layout(A, s, kb, d, st, nullptr, &b, &op);
}

int gk_block_numrank(const gk_matrix *A, int s, const double *Q0, double eps, int kmax, const gk_opts *opts, int *rank,
                     double *sigma, int *steps, gk_info *info) {
  NvtxRange r("gk_block_numrank");
  return block_impl(A, s, Q0, eps, kmax, opts, rank, sigma, steps, info);
}

int gk_fsvd(const gk_matrix *A, int k, int r, int route, const gk_opts *opts, double *U, double *S, double *V,
            gk_info *info) {
  NvtxRange nv("gk_fsvd");
  return fsvd_impl(A, k, r, route, opts, U, S, V, info);
}

int gk_matvec(const gk_matrix *A, int trans, const double *x, double *y, const gk_opts *opts) {
  NvtxRange r(trans ? "gk_matvec_t" : "gk_matvec");
  return matvec_impl(A, trans, x, y, opts);
}

int gk_residuals(const gk_matrix *A, int k, const double *U, const double *S, const double *V, double *res_av,
                 double *res_atu, const gk_opts *opts) {
  return residuals_impl(A, k, U, S, V, res_av, res_atu, opts);
}

const char *gk_status_string(int status) {
  switch (status) {
    case GK_OK: return "GK_OK";
    case GK_NOT_CONVERGED: return "GK_NOT_CONVERGED";
    case GK_RANK_DEFICIENT: return "GK_RANK_DEFICIENT";
    case GK_INVALID_ARG: return "GK_INVALID_ARG";
    case GK_CUDA_ERROR: return "GK_CUDA_ERROR";
    case GK_NUMERICAL: return "GK_NUMERICAL";
    case GK_TIMEOUT: return "GK_TIMEOUT";
    case GK_OUT_OF_MEMORY: return "GK_OUT_OF_MEMORY";
    case GK_NOT_IMPLEMENTED: return "GK_NOT_IMPLEMENTED";
    case GK_NO_DEVICE: return "GK_NO_DEVICE";
    default: return "GK_UNKNOWN_STATUS";
  }
}

const char *gk_last_cuda_error(void) { return g_err; }

const char *gk_version(void) { return "gk-gb300 0.1 (sm_103a)"; }

int64_t gk_launch_count(void) { return gk::launch_count(); }

}  // extern "C"
