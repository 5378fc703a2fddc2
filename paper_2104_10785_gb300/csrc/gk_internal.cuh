// gk_internal.cuh -- declarations shared by the translation units of libgk.so.
//
// Layout in device memory (all f64 unless noted):
//   basis U: ldu x (cols) column-major, one Lanczos/Ritz vector per column;
//   basis V: ldv x (cols) column-major; ldu, ldv are m, n rounded up to 32.
//   x32:     f32 copy of the vector the next product reads (n or m entries).
//   part:    partial sums, [column][block] layout so reductions read rows
//            of contiguous memory.
// Reduced-precision operators (f32/bf16/f16) are multiplied in f32 with the
// input vector rounded to f32, summed in f32 over short runs and combined in
// f64; f64 operators are multiplied in f64.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gk.h"

namespace gk {

// ---- launch accounting: every kernel launch of the library goes through GK_LAUNCH
void note_launch();
int64_t launch_count();
#define GK_LAUNCH(...)    \
  do {                    \
    __VA_ARGS__;          \
    ::gk::note_launch();  \
  } while (0)

// ---- control block written by device kernels, read by the host driver ----
enum Event { EV_NONE = 0, EV_BETA_BREAK = 1, EV_ALPHA_BREAK = 2, EV_BREAKDOWN = 3, EV_NUMERICAL = 4, EV_TIMEOUT = 5 };
// how a norm kernel judges the new vector
enum NormMode {
  NM_BREAK = 0,      // Algorithm 1 break test: norm <= eps * sigma_est (or eps)
  NM_BREAKDOWN = 1,  // restarted SVD: norm <= 2^-46 * sigma_est counts as an exact breakdown
  NM_PLAIN = 2,      // just normalize (start vectors)
  NM_FRESH = 3,      // replacement direction: kept unless the projection removed all but 1e-8 of the norm
                     // measured by the preceding NM_PLAIN call; otherwise the column becomes zero
};

struct Ctl {
  int halt;          // nonzero: every step kernel returns at entry
  int event;         // Event
  int step;          // step index of the event
  int side;          // 0 left (u/q), 1 right (v/p)
  unsigned cnt[4];   // arrival counters of last-block reductions (kept zero between uses)
  double sest;       // running lower bound on sigma_1
  double norm;       // last norm computed
  double inv_norm;   // 1 / last accepted norm (0 if rejected)
  double eps;        // Algorithm 1 threshold parameter
  int eps_rel;       // 1: threshold eps * sest; 0: eps
  int timeout;       // a bounded device wait gave up (the kernel recorded where: 1 full, 2 empty barrier)
  int pass2;         // adaptive Gram-Schmidt: the first pass cancelled, the second pass runs
};

// device view of the operator
struct Op {
  int kind, dtype;
  int64_t m, n, ld;
  int64_t nnz;  // CSR: stored entries (0 if unknown); dense: 0
  double scale;
  const void *vals;
  const int32_t *rowptr;
  const int32_t *colind;
  const void *t_vals;
  const int32_t *t_rowptr;
  const int32_t *t_colind;
};

struct Dev {
  int sms;
  int id;
};

// ---- 16-byte vector of stored values -> floats (device helpers) ------------
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int E = 4;
  using V = float4;
  __device__ __forceinline__ static void unpack(const V &v, float *o) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ __forceinline__ static float one(const float *p) { return *p; }
};
template <>
struct Vec<__nv_bfloat16> {
  static constexpr int E = 8;
  using V = uint4;
  __device__ __forceinline__ static void unpack(const V &v, float *o) {
    // bf16 is the high half of an f32 word; element 0 sits in the low half of v.x
    o[0] = __uint_as_float(v.x << 16); o[1] = __uint_as_float(v.x & 0xffff0000u);
    o[2] = __uint_as_float(v.y << 16); o[3] = __uint_as_float(v.y & 0xffff0000u);
    o[4] = __uint_as_float(v.z << 16); o[5] = __uint_as_float(v.z & 0xffff0000u);
    o[6] = __uint_as_float(v.w << 16); o[7] = __uint_as_float(v.w & 0xffff0000u);
  }
  __device__ __forceinline__ static float one(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
};
template <>
struct Vec<__half> {
  static constexpr int E = 8;
  using V = uint4;
  __device__ __forceinline__ static void unpack(const V &v, float *o) {
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h = *reinterpret_cast<const __half2 *>(&w[i]);
      float2 f = __half22float2(h);
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
  __device__ __forceinline__ static float one(const __half *p) { return __half2float(*p); }
};

// ---- sizing helpers ------------------------------------------------------
inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
int64_t gemvt_row_block(const Op &A, const Dev &d);        // rows per block of the A^T product
int64_t gemvt_partials(const Op &A, const Dev &d);         // doubles of partial storage it needs
int cgs_chunk(int64_t len, const Dev &d);                  // rows per block of the CGS kernels
int cgs_blocks(int64_t len, const Dev &d);

// ---- products (gk_matvec.cu) -------------------------------------------
// y = A x - (*coef) * sub   (sub may be null).  x32: f32 copy of x (f32/bf16/f16 A), x64: f64 x (f64 A).
// part: scratch for partial sums (gemvt_partials() doubles); with part == null a dense
// reduced-precision A x runs the row-streaming kernel, which needs none.
cudaError_t matvec(const Op &A, const float *x32, const double *x64, double *y, const double *sub,
                   const double *coef, double *part, const Ctl *ctl, cudaStream_t s, const Dev &d);
// y = A^T x - (*coef) * sub
cudaError_t matvec_t(const Op &A, const float *x32, const double *x64, double *y, const double *sub,
                     const double *coef, double *part, const Ctl *ctl, cudaStream_t s, const Dev &d);

// ---- fused sweep (gk_fused.cu) --------------------------------------------
// Dense f32/bf16/f16 operators with 16-byte rows and n * sizeof(T) a multiple of 16, up
// to 160 KB per row: one pass over A gives w = scale A x - coef * sub and the partial
// sums of A^T w per cluster (zpart, fused_partials() doubles); fused_finish then forms
// z = scale (A^T w) / (*alpha) - (*alpha) * sub.
bool fused_ok(const Op &A, const Dev &d);
int64_t fused_partials(const Op &A, const Dev &d);
int fused_cluster(const Op &A, const Dev &d);  // CTAs per cluster of the fused kernel (0: not fused)
cudaError_t fused_matvec(const Op &A, const float *x32, double *w, const double *sub, const double *coef,
                         double *zpart, Ctl *ctl, cudaStream_t s, const Dev &d);
cudaError_t fused_finish(const Op &A, const double *zpart, const double *alpha, const double *sub, double *z,
                         const Ctl *ctl, cudaStream_t s, const Dev &d);

// ---- FP64-grade block products (gk_accurate.cu) ----------------------------
// Dense f32/bf16/f16 operators: out (column-major, ld = output length) = scale op(A) X for
// the k f64 vectors X (column-major, ld = input length), every product and sum carried in
// double-f32 (exact to ~2^-47 sum |a x|); split holds accurate_floats() floats.
bool accurate_ok(const Op &A);
size_t accurate_floats(const Op &A, int k);
// fast = true: f32 products (x rounded to f32, 16- or 32-term f32 chunk sums combined in
// double-f32), the precision of matvec, at about a tenth of the arithmetic.  narrow = true (the
// block calls): blocks of up to 8 or 16 vectors take tiles of that width instead of 32, the
// contraction split over slices when npart (accurate_narrow_doubles() doubles) is given
size_t accurate_narrow_doubles(const Op &A, int k);
cudaError_t accurate_products(const Op &A, bool trans, const double *X, int k, double *out, float *split,
                              cudaStream_t s, bool fast = false, bool narrow = false, double *npart = nullptr);
// res[j] = || Y[:, j] - S[j] W[:, j] ||, columns of length len (ld = len)
cudaError_t resid_norms(const double *Y, const double *W, const double *S, int64_t len, int k, double *res,
                        cudaStream_t s);

// ---- the sketch on the tensor cores (gk_sketch_tc.cu) ------------------------
// bf16 operator whose rows start on 16-byte boundaries (the TMA's requirement)
bool sketch_tc_ok(const void *A, int64_t m, int64_t n, int64_t ld);
// per 128-row chunk c of A: gpart[c * 528 + e] = the chunk's Gram entries of Y = scale A Omega
// (upper triangle, row-major order), fpart[c] = its ||A_c||_F^2; omT = Omega^T in bf16,
// 32 x nk (nk a multiple of 64, zero past n); *err (zeroed by the caller) != 0 when a bounded
// wait gave up
cudaError_t sketch_tc(const void *A, int64_t m, int64_t n, int64_t ld, double scale, const void *omT, int64_t nk,
                      double *gpart, double *fpart, int *err, cudaStream_t s);

// ---- learned predictor (gk_predict.cu) -------------------------------------
// Krylov dimension for the top-k partial SVD of the dense device operator A from its sketch
// features: ceil(exp(out_K)) + 2, clamped to [k + 2, min(m, n, 500)].
// sketch_flags: GK_FLAG_SKETCH_TC selects the tensor-core sketch (other bits are ignored).
int predict_krylov(const gk_predictor *p, const gk_matrix *A, int k, cudaStream_t s, int *K, int sketch_flags);
// gk_psvd_batched with opts->predictor set
int learned_batched(gk_batch_item *items, int count, const gk_opts *opts, gk_info *info);

// ---- Gram-Schmidt and vector kernels (gk_orth.cu) -------------------------
// Classical Gram-Schmidt of w (len) against the first j columns of Q (ld):
// passes = 1..3 passes, or 0 = one pass and a second only if the first left less
// than 1/sqrt(2) of the norm; then the norm and its judgement; see NormMode.
// coef_out receives the accepted norm (0 on breakdown); prev is the previous
// recurrence coefficient (for the sigma_est update of Algorithm 1).
// Qs, ws2 (optional): the basis's double-f32 shadow (Qs[c * ld + i] = (hi, lo) of Q) and a
// len-entry buffer for w's split; with both, vectors past the one-CTA size run the
// double-f32 kernels.
cudaError_t orthonormalize(double *w, int64_t len, const double *Q, int64_t ld, int j, int passes, double *part,
                           double *h, Ctl *ctl, int mode, int step, int side, double *coef_out, const double *prev,
                           cudaStream_t s, const Dev &d, const float2 *Qs = nullptr, float2 *ws2 = nullptr);
// Q[:, col] = w * ctl->inv_norm, x32 = f32 copy (skipped when halted)
cudaError_t normalize_append(const double *w, int64_t len, double *qcol, float *x32, const Ctl *ctl, cudaStream_t s,
                             const Dev &d, float2 *qs = nullptr);
// orthonormalize followed by normalize_append into qcol (and its copy qscol, and x32): with a
// double-f32 copy of the basis and a vector past the one-CTA size whose slabs fit shared
// memory, one cooperative launch does all of it (gk_orth.cu, k_orth_coop)
cudaError_t orth_append(double *w, int64_t len, const double *Q, int64_t ld, int j, int passes, double *part,
                        double *h, Ctl *ctl, int mode, int step, int side, double *coef_out, const double *prev,
                        double *qcol, float *x32, cudaStream_t s, const Dev &d, const float2 *Qs, float2 *ws2,
                        float2 *qscol);
// one partial SVD of a small dense device operator in one persistent launch of the batched
// solver (gk_batched.cu; the largest cluster that fits), for gk_psvd
int psvd_persistent(gk_batch_item *item, const gk_opts *opts, gk_info *info);
// doubles of `part` the cooperative orthonormalization needs for Krylov dimension K
int64_t coop_partials(int K, const Dev &d);
// Qs[c * ld + i] = (hi, lo) of Q[c * ld + i] for the first `cols` columns (the shadow of a basis)
cudaError_t split_cols(const double *Q, int64_t len, int64_t ld, int cols, float2 *Qs, cudaStream_t s);
// w = (start vector q1 ~ N(2,1), Philox4x32-10 + Box-Muller), len entries
cudaError_t draw_start(double *w, int64_t len, uint64_t seed, cudaStream_t s);
// w = replacement direction number dnum (SplitMix64, uniform [-1,1))
cudaError_t draw_fresh(double *w, int64_t len, uint64_t seed, int64_t dnum, cudaStream_t s);
// dst = src (f64) and x32 = f32(src)
cudaError_t copy_vec(double *dst, float *x32, const double *src, int64_t len, cudaStream_t s);
// y -= Q[:, 0:l] * coef[0:l]
cudaError_t sub_combination(double *y, int64_t len, const double *Q, int64_t ld, int l, const double *coef,
                            const Ctl *ctl, cudaStream_t s, const Dev &d);
cudaError_t reset_ctl(Ctl *ctl, double eps, int eps_rel, cudaStream_t s);

// ---- block Golub-Kahan (gk_block.cu) -----------------------------------------
constexpr int kBlockMaxS = 32;  // largest block (start vectors per block)
// state of the block sweep's tests, written by block_judge
struct BlockCtl {
  double sest;  // running estimate of sigma_1: the largest block 2-norm so far
  double nrm;   // 2-norm of the last judged block
  int brk;      // 1: the last judged block ends the sweep; 2: its norm was not finite
  int sweeps;   // Jacobi sweeps of the last norm
};
// partial sums block_dots needs: s * s * block_dot_chunks(len) doubles
int block_dot_chunks(int64_t len);
// raw[a + b s] = X[:, a] . Y[:, b] (a, b < s <= kBlockMaxS; len rows; f64)
cudaError_t block_dots(const double *X, int64_t ldx, const double *Y, int64_t ldy, int64_t len, int s, double *part,
                       double *raw, cudaStream_t st);
// T = triu(raw) (s x s): its 2-norm, the running estimate and the break test of `side`
// (0: a left block S_{j+1}, placed as T at (row0, col0) of Bf; 1: a right block R_{j+1},
// placed as T^T unless it ends the sweep; 2: the first right block, no test), into *bc
cudaError_t block_judge(const double *raw, int s, double *Bf, int64_t ldb, int row0, int col0, int side, double eps,
                        BlockCtl *bc, cudaStream_t st);
// est[i] = ||triu(raw) X[row0 .. row0 + s, i]|| for i < r (X column-major, ld ldx; device)
cudaError_t block_resid(const double *raw, int s, const double *X, int ldx, int row0, int r, double *est,
                        cudaStream_t st);
// *rank = #{i < n : sigma[i] > eps sigma[0]} (device)
cudaError_t block_count(const double *sigma, int n, double eps, int *rank, cudaStream_t st);
// the block Gram-Schmidt's projection out (len x s, ld len) = X - Q (Q^T X) for the first j
// columns of Q, from the double-f32 copies Qs (ld ldq) and Xs (ld ldxs) of Q and X: Q^T X in
// double-f32 per thread, f64 across threads and row chunks (part: bgs_dot_chunks(len) j s
// doubles), H (j x s) and its split Hs, C = Q H in double-f32 (len x s)
int bgs_dot_chunks(int64_t len);
cudaError_t bgs_project(const float2 *Qs, int64_t ldq, int64_t len, int j, const double *X, int64_t ldx,
                        const float2 *Xs, int64_t ldxs, int s, double *part, double *H, float2 *Hs, double *C,
                        double *out, cudaStream_t st);

// ---- small dense kernels (gk_small.cu) ----------------------------------
// B (K x K, column-major) of one restart cycle: kept Ritz values on the
// diagonal of the first l rows, the coupling column rho in column l, and the
// new recurrence coefficients alpha_j (diagonal) and beta_j (superdiagonal)
// for j >= l.
cudaError_t assemble_B(double *Bm, int K, int l, const double *sigma, const double *rho, const double *alpha,
                       const double *beta, const Ctl *ctl, cudaStream_t s);
// Bm = the lower-bidiagonal B_{kp+1,kp} (alpha[0..kp-1] on the diagonal, beta[1..kp] below it)
// padded with a zero column to (kp+1) x (kp+1), column-major
cudaError_t assemble_lower(double *Bm, int kp, const double *alpha, const double *beta, cudaStream_t s);
// Bm = B^T B (kp x kp, tridiagonal) of the lower-bidiagonal B_{kp+1,kp}
cudaError_t assemble_btb(double *Bm, int kp, const double *alpha, const double *beta, cudaStream_t s);
// theta[0:n] = sqrt(max(theta, 0))
cudaError_t sqrt_vals(double *theta, int n, cudaStream_t s);
// column i of U (len x ncol) /= sigma[i] (unchanged when sigma[i] <= 0)
cudaError_t scale_cols(double *U, int64_t len, int ncol, const double *sigma, cudaStream_t s);
// y[0:len] /= *d (unchanged when *d <= 0)
cudaError_t scale_inv(double *y, int64_t len, const double *d, cudaStream_t s);
// One-sided Jacobi SVD of the K x K matrix Bm (overwritten; Yw is K x K work,
// nrm/pos K-entry work) on one thread-block cluster: sigma (K, descending),
// X (K x K left vectors), Y (K x K right vectors), sweeps (negative if the
// sweep limit was reached).
cudaError_t small_svd(double *Bm, double *Yw, int K, double *sigma, double *X, double *Y, double *nrm, int *pos,
                      int *sweeps, const Ctl *ctl, cudaStream_t s);
// The same outputs for an upper-bidiagonal B (alpha on the diagonal, beta[0..K-1) above it) by
// Golub-Kahan SVD steps on one CTA (gk_bdsvd.cuh); Xw, Yw: K x K work.  K <= kBdMaxK.
constexpr int kBdMaxK = 1024;
cudaError_t bd_svd(const double *alpha, const double *beta, int K, double *sigma, double *X, double *Y, double *Xw,
                   double *Yw, int *sweeps, const Ctl *ctl, cudaStream_t s);
// Restart bookkeeping: rho_i = betaK X_{K,i} (all i < K), and
// out[0] = max_{i<k} |rho_i|, out[1] = sigma_1, out[2] = converged (0/1).
cudaError_t ritz_check(const double *sigma, const double *X, int K, int k, const double *betaK, double tol,
                       double *rho, double *out, Ctl *ctl, cudaStream_t s);
// C[:, 0:ncol] = Q[:, 0:K] * X[:, 0:ncol]   (C may alias nothing in Q)
cudaError_t ritz_gemm(const double *Q, int64_t ldq, int64_t len, int K, const double *X, int ldx, int ncol,
                      double *C, int64_t ldc, cudaStream_t s, const Dev &d);
// the same product from the double-f32 copy Qs of Q (gk_ritz_df.cuh) on the FP32 pipes, exact to
// ~2^-46 of sum |q x|; Xs: K * ncol float2 of scratch for X's split
cudaError_t ritz_gemm_df(const float2 *Qs, int64_t ldq, int64_t len, int K, const double *X, int ldx, int ncol,
                         double *C, int64_t ldc, float2 *Xs, cudaStream_t s);
// sign convention: largest-|v_i| entry positive (flips u_i and v_i)
cudaError_t sign_normalize(double *U, int64_t ldu, int64_t m, double *V, int64_t ldv, int64_t n, int k,
                           cudaStream_t s);
// rank of the lower-bidiagonal B_{kp+1,kp} (alpha[0..kp-1], beta[1..kp]) by
// Sturm counts on its Golub-Kahan tridiagonal; sigma (optional, kp values)
cudaError_t bidiag_rank(const double *alpha, const double *beta, int kp, double eps, int eps_rel, int *rank,
                        double *sigma1, double *sigma, cudaStream_t s);

}  // namespace gk
