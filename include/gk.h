/*
 * gk.h -- C ABI of the GB300 Golub-Kahan partial-SVD / numerical-rank library
 * (libgk.so).  Method: "Accurate and fast matrix factorization for low-rank
 * learning", arXiv 2104.10785.
 *
 * Conventions shared by every entry point
 *  - All matrices are read-only and caller-owned.  Dense operators are
 *    row-major with leading dimension ld (elements between consecutive rows).
 *    Vectors and output factors are column-major (each vector contiguous).
 *  - Pointers may be device pointers or host pointers (pageable or pinned):
 *    the library detects host memory with cudaPointerGetAttributes, copies
 *    host inputs to its device workspace before computing and copies results
 *    back to host outputs before returning.
 *  - Calls are synchronous: they return after the result is final, because the
 *    method's control flow (break test, convergence test) depends on device
 *    results.  Work is issued on opts->stream (0 = the legacy default stream).
 *  - Every call returns a gk_status; nothing aborts or throws across the ABI.
 *  - The library never falls back to host computation: without a usable CUDA
 *    device every call returns GK_NO_DEVICE.
 *  - Workspace: if opts->workspace is NULL the library allocates its device
 *    workspace (plus a staging copy of a host operator) on the call's stream
 *    from its own stream-ordered memory pool and frees it before returning;
 *    the pool keeps freed memory mapped for the next call (until the process
 *    exits).  Otherwise opts->workspace must point to at least
 *    gk_*_workspace() bytes of device memory, 256-byte aligned.
 *  - Calls on different streams with different workspaces may run
 *    concurrently; two calls sharing one workspace must not overlap.
 */
#ifndef GK_H
#define GK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GK_OK = 0,
  GK_NOT_CONVERGED = 1,    /* restart budget spent; outputs hold the best Ritz triplets */
  GK_RANK_DEFICIENT = 2,   /* fewer than k nonzero singular values exist; outputs padded */
  GK_INVALID_ARG = -1,     /* bad sizes, null pointers, unsupported dtype/kind combination */
  GK_CUDA_ERROR = -2,      /* a CUDA runtime call failed (see gk_last_cuda_error) */
  GK_NUMERICAL = -3,       /* NaN or Inf appeared in a norm */
  GK_TIMEOUT = -4,         /* a bounded device wait gave up */
  GK_OUT_OF_MEMORY = -5,   /* workspace allocation failed or caller workspace too small */
  GK_NOT_IMPLEMENTED = -6,
  GK_NO_DEVICE = -7        /* no CUDA device usable by this library */
} gk_status;

typedef enum { GK_F64 = 0, GK_F32 = 1, GK_BF16 = 2, GK_F16 = 3 } gk_dtype;

/* opts->flags bits */
#define GK_FLAG_PROFILE 1  /* time kernel groups with CUDA events on opts->stream (gk_info.ms_*) */
#define GK_FLAG_AUTOTUNE 2 /* batched calls: time each candidate cluster size on this batch, keep the fastest */
#define GK_FLAG_FUSED 4    /* gk_psvd, gk_numrank, gk_fsvd: the fused sweep, one pass over A per step
                              (see gk_psvd), where the operator qualifies; default: two passes */
#define GK_FLAG_REFINE 8   /* gk_psvd: check the returned triplets' true residuals with FP64-grade
                              products (as gk_residuals) and keep restarting, with the Ritz test
                              tightened 4x each time, while one exceeds tol * s_1 */
#define GK_FLAG_ORTH_F64 16 /* gk_psvd, gk_numrank, gk_fsvd: Gram-Schmidt with f64 arithmetic on the f64
                              bases.  Without it, vectors longer than the one-CTA size (8192 entries)
                              are orthogonalized against a double-f32 copy of each basis (every entry
                              as two f32, written beside the f64 column; the basis products in
                              double-f32 arithmetic, ~2^-46 of |q w| per term, w and the norms f64):
                              the same passes and rules (Algorithm 1 reorthogonalization), on the
                              FP32 pipes, with the workspace holding the copies (8 bytes per basis
                              entry) */
#define GK_FLAG_PERSISTENT 32 /* gk_psvd: solve a small dense device operator (at most 4096 columns and
                              24 MB, device outputs, no caller workspace, no fixed keep count, none of
                              the FUSED/REFINE/predictor options) in one persistent launch of the
                              batched solver (gk_psvd_batched's method on one problem, one cluster of
                              16 CTAs) instead of the multi-kernel sweep: the same algorithm in 2
                              launches instead of ~225 (f64 2000 x 1000, top 10).  Opt-in: measured
                              6.7 ms against 6.0 ms for the multi-kernel sweep, both bound by f64
                              arithmetic latency rather than launches.  gk_info then reports its
                              counters; reserved = 0. */
#define GK_FLAG_SKETCH_TC 64 /* gk_sketch_batched, one bf16 operator with rows on 16-byte boundaries:
                              Y = A Omega on the tcgen05 tensor cores with TMA-staged tiles and the
                              accumulator in tensor memory, instead of mma.sync (GK_INVALID_ARG for
                              any other request with this flag); gk_psvd with a predictor: the same
                              for the sketch of such an operator (others keep the default sketch).  Experimental: not yet run on a GPU;
                              returns GK_TIMEOUT if one of its bounded waits gives up. */
#define GK_FLAG_BDSVD 128 /* gk_psvd: in a cycle without kept Ritz vectors (the first, or every cycle when
                              the Krylov dimension is reached without a restart) the projected matrix is
                              upper bidiagonal: its SVD by implicitly shifted Golub-Kahan SVD steps on one
                              CTA instead of the cluster Jacobi (K <= 1024); gk_fsvd route 1: the same for
                              B_{k'+1,k'} (through its transpose, upper bidiagonal).  Experimental: the
                              step and rotation code is tested on the host; the kernel has not yet run
                              on a GPU. */
#define GK_FLAG_RITZ_DF 256 /* gk_psvd (with the double-f32 basis copies, i.e. without GK_FLAG_ORTH_F64): the
                              Ritz vectors U_K X and V_K Y (restarts and outputs) from the copies in
                              double-f32 arithmetic on the FP32 pipes (exact to ~2^-46 of sum |q x|)
                              instead of f64 products.  Experimental: the product code is tested on the
                              host; the kernel has not yet run on a GPU. */
#define GK_FLAG_BLOCK_F32 512 /* gk_block_numrank, gk_block_fsvd on a dense f32/bf16/f16 operator: the block
                              products in f32 (x rounded to f32, 16- or 32-term f32 sums combined in
                              double-f32: the precision of gk_matvec) instead of double-f32, about a
                              tenth of the arithmetic per product.  Experimental: not yet run on a GPU. */
#define GK_FLAG_BLOCK_GS 1024 /* gk_block_numrank, gk_block_fsvd (with the double-f32 basis copies, i.e.
                              without GK_FLAG_ORTH_F64): each block orthogonalized against the earlier
                              basis as a block (reorthogonalized block classical Gram-Schmidt: the block
                              projected, its own QR column by column, projected again, QR again), the
                              basis read twice per projection of s columns instead of four times per
                              column.  Experimental: not yet run on a GPU. */
typedef enum { GK_DENSE = 0, GK_CSR = 1 } gk_kind;

/* The operator A (m x n).
 *  dense: vals points to m*ld values of dtype (row-major); rowptr/colind unused.
 *  CSR:   vals/rowptr/colind hold A (rowptr: m+1 int32 offsets, colind: int32,
 *         nnz = rowptr[m]); t_vals/t_rowptr/t_colind hold the CSR of A^T (n
 *         rows).  Both are required for CSR: the library never transposes.
 *  scale multiplies every stored value (use 1.0; for f16 storage a power of two
 *  that keeps the stored values in the normal range). */
typedef struct {
  int32_t kind;
  int32_t dtype;
  int64_t m, n, ld;
  double scale;
  const void *vals;
  const int32_t *rowptr;
  const int32_t *colind;
  const void *t_vals;
  const int32_t *t_rowptr;
  const int32_t *t_colind;
} gk_matrix;

/* A loaded learned predictor (gk_predictor_load); opaque. */
typedef struct gk_predictor gk_predictor;

typedef struct {
  int32_t krylov_dim;    /* K, the Krylov dimension of one restart cycle (0 = default min(max(2k, k+16), min(m,n)),
                            or the predictor's choice when opts->predictor is set) */
  int32_t keep;          /* Ritz vectors kept at a restart (0 = k + (K-k)/2) */
  int32_t max_restarts;  /* restart budget of gk_psvd (default 200) */
  int32_t reorth_passes; /* classical Gram-Schmidt per vector: 0 (default) = one pass, and a second
                            only if the first left less than 1/sqrt(2) of the norm (the
                            Daniel-Gragg-Kaufman-Stewart test); 1 = one pass (as printed in the
                            paper); 2 or 3 = that many passes */
  int32_t eps_absolute;  /* gk_numrank: 0 = eps relative to sigma_1 (default), 1 = absolute threshold */
  int32_t flags;         /* GK_FLAG_* bits (0 = none) */
  uint64_t seed;         /* seed of the start vector and of replacement directions */
  const double *start;   /* optional m-vector q1 (device or host); NULL = draw q1 ~ N(2,1)^m from seed */
  void *stream;          /* cudaStream_t, NULL = legacy default stream */
  void *workspace;       /* optional caller-owned device workspace */
  size_t workspace_bytes;
  const gk_predictor *predictor; /* optional learned predictor (NULL = none): gk_psvd takes K from it
                                    when krylov_dim is 0; gk_psvd_batched runs the learned pipeline */
} gk_opts;

typedef struct {
  int32_t steps;         /* bidiagonalization steps taken (left+right half-steps count as one) */
  int32_t restarts;
  int32_t cycles;
  int32_t kprime;        /* gk_numrank, gk_fsvd: k' of Algorithm 1 (columns of B_{k'+1,k'}); gk_psvd: the
                            Krylov dimension used */
  int32_t stop_reason;   /* gk_numrank: 0 reached kmax, 1 beta break, 2 alpha break */
  int32_t breakdowns;    /* exact breakdowns replaced by fresh directions */
  int32_t svd_sweeps;    /* gk_psvd: Jacobi sweeps of the last small SVD (negative: sweep limit reached);
                            batched: the most sweeps any problem's last small SVD took */
  int32_t reserved;      /* batched calls: cluster size used; gk_psvd, gk_numrank, gk_fsvd: CTAs per
                            cluster of the fused sweep (0 = two passes over A per step) */
  int64_t matvecs;       /* products with A or A^T */
  double resid_est_max;  /* gk_psvd: max_i<k |beta_K X_{K,i}| / sigma_1 (Ritz residual estimate) */
  double sigma_est;      /* running lower bound on sigma_1 used by the break test */
  double seconds;        /* wall time of the call */
  /* with GK_FLAG_PROFILE: device milliseconds and launch counts of kernel
   * groups, from CUDA events recorded on opts->stream around each group */
  double ms_matvec;      /* A x products (with the fused sweep: the passes that form both products) */
  double ms_matvec_t;    /* A^T x products (partial sums + their reduction; with the fused sweep the
                            reduction of its A^T w partial sums, and the unfused steps) */
  double ms_orth;        /* Gram-Schmidt passes, norms, normalization */
  double ms_small;       /* small SVD, Ritz residual test, rank count */
  double ms_restart;     /* Ritz vectors U_K X, V_K Y (restarts and outputs) */
  int64_t n_matvec;
  int64_t n_matvec_t;
  int64_t launches;      /* kernels this call launched (all of them the library's own) */
  double ms_copy;        /* with GK_FLAG_PROFILE: host<->device copies of host operands and outputs */
  double resid_true_max; /* gk_psvd with GK_FLAG_REFINE: max_i max(||A v_i - s_i u_i||, ||A^T u_i - s_i v_i||)
                            / s_1 of the returned triplets, FP64-grade (0 when not checked) */
  double ms_refine;      /* gk_psvd with GK_FLAG_REFINE: wall milliseconds of those checks */
  int32_t refine_checks; /* gk_psvd with GK_FLAG_REFINE: checks run (1 = the first passed) */
  int32_t fallbacks;     /* gk_psvd_batched with a predictor: problems re-solved by the plain pipeline */
  double err_rel;        /* gk_psvd with GK_FLAG_REFINE: the paper's err_rel (Section 5),
                            ||A^T U - V S||_F / ||S||_F of the returned triplets (0 when not checked) */
} gk_info;

/* Fill *opts with the defaults above. */
void gk_default_opts(gk_opts *opts);

/* Device workspace (bytes) gk_psvd needs for this operator, k and opts. */
size_t gk_psvd_workspace(const gk_matrix *A, int k, const gk_opts *opts);

/* Partial SVD: the k largest singular triplets of A.
 * Method: Golub-Kahan bidiagonalization (Section 2.2, Eqs. 2.1-2.4) in the
 * upper-bidiagonal form started from v1 = A^T q1 / ||A^T q1|| (Algorithm 1),
 * full reorthogonalization by classical Gram-Schmidt (Algorithm 1; a second
 * pass where the first cancels, by default), Ritz pairs from the SVD of the
 * small projected matrix (Eq. 2.13, Algorithm 2), and thick restarts that
 * keep the leading Ritz vectors (the paper cites augmented restarting; the
 * restart itself is this library's choice).
 * Fused sweep (opts->flags GK_FLAG_FUSED; dense f32/bf16/f16 operators with 16-byte
 * rows, n * element size a multiple of 16 bytes and at most 160 KB per row): each step
 * reads A once.  The pass forms w = A v_j - beta_{j-1} u_{j-1} and, from the same bytes,
 * A^T w; after the left Gram-Schmidt (coefficients h, norm alpha_j) the right step takes
 * A^T w / alpha_j in place of A^T u_j.  The two differ by A^T U_{j-1} h / alpha_j, which
 * lies in span(V_j) (A^T u_i = alpha_i v_i + beta_i v_{i+1}, Eq. 2.2 in the upper form)
 * and is removed by the right Gram-Schmidt, so the recurrence is unchanged in exact
 * arithmetic.  The first step after a restart and a step after an exact breakdown run
 * the two passes.  gk_numrank and gk_fsvd (Algorithm 1) use the same ordering.
 *  tol: a triplet is converged when ||A^T u_i - s_i v_i|| (the Ritz residual,
 *       = |beta_K X_{K,i}|; A v_i = s_i u_i holds by construction) is at most
 *       tol * s_1.
 *  U:   m x k, column-major, f64 (device or host).
 *  S:   k singular values, f64, descending.
 *  V:   n x k, column-major, f64.
 * Each pair (u_i, v_i) is signed so that the largest-magnitude entry of v_i is
 * positive.  Returns GK_OK, GK_NOT_CONVERGED (outputs hold the last Ritz
 * triplets), or an error.  1 <= k <= min(m,n). */
int gk_psvd(const gk_matrix *A, int k, double tol, const gk_opts *opts, double *U, double *S, double *V,
            gk_info *info);

/* Device workspace (bytes) gk_numrank needs. */
size_t gk_numrank_workspace(const gk_matrix *A, int kmax, const gk_opts *opts);

/* Numerical rank (Algorithm 3): run Algorithm 1 (lower-bidiagonal GK with
 * reorthogonalization) for at most kmax iterations (kmax <= 0 or > min(m,n)
 * means min(m,n), as Algorithm 3 sets it), stopping when the new left norm
 * beta_{j+1} (or right norm alpha_{j+1}) is <= eps * sigma_est (relative
 * reading; opts->eps_absolute = 1 compares with eps itself), then count the
 * singular values of B_{k'+1,k'} (square roots of the eigenvalues of
 * B^T B, Algorithm 3) that exceed eps * sigma_1(B) (or eps).
 *  rank:  host int, written on success.
 *  sigma: optional (may be NULL) output of the k' singular values of B,
 *         descending (device or host, f64, capacity kmax).
 * The workspace holds two bases of kmax+1 columns: pass a realistic kmax
 * for large matrices. */
int gk_numrank(const gk_matrix *A, double eps, int kmax, const gk_opts *opts, int *rank, double *sigma,
               gk_info *info);

/* Numerical rank from a block of s start vectors: Algorithm 1 and Algorithm 3
 * with each vector replaced by a block (the paper has the single-vector form;
 * one start vector's Krylov space holds one direction per distinct singular
 * value, so Algorithm 1 counts a singular value of multiplicity > 1 once, and a
 * block of s counts multiplicities up to s).  The recurrence, with each block
 * orthonormalized by QR (diag >= 0) after two classical Gram-Schmidt passes
 * against the earlier blocks:
 *   Q_1 R_0 = Q0,  P_1 R_1 = A^T Q_1,
 *   Q_{j+1} S_{j+1} = A P_j - Q_j R_j^T,  P_{j+1} R_{j+1} = A^T Q_{j+1} - P_j S_{j+1}^T,
 * so A [P_1..P_k] = [Q_1..Q_{k+1}] B with B block lower bidiagonal (R_j^T on the
 * diagonal, S_{j+1} below it; the block form of Eq. 2.2).  The sweep stops when
 * ||S_{j+1}||_2 <= eps * sigma~ (sigma~: the largest block 2-norm so far), when
 * ||R_{j+1}||_2 <= eps * max(sigma~, ||R_{j+1}||_2) (that block is not kept),
 * after kmax block steps, or when one more block would exceed min(m, n)
 * columns; the rank is the number of singular values of B above eps * sigma_1(B).
 *  s:     block size, 1 <= s <= 32 and s <= min(m, n).
 *  Q0:    m x s start block, column-major (ld = m), f64, device or host; NULL draws
 *         column c as Algorithm 1's start vector with seed opts->seed + c.
 *  eps:   relative threshold (opts->eps_absolute must be 0).
 *  kmax:  block steps; <= 0 means min(m, n) / s, capped so that (kmax + 1) s <= 1024
 *         (the order of B's square for the small SVD); a larger explicit kmax is
 *         GK_INVALID_ARG.
 *  rank:  host int, written on success.
 *  sigma: optional (may be NULL): the steps * s singular values of B, descending
 *         (device or host, f64, capacity kmax * s).
 *  steps: optional host int: block steps taken.
 * Dense f32/bf16/f16 operators form each block product in one pass over A with
 * double-f32 products (as gk_residuals); f64 and CSR operators run one product
 * per column.  info: steps = block steps, kprime = columns of B, stop_reason 0
 * kmax, 1 left block break, 2 right block break, 3 the blocks filled min(m, n);
 * matvecs counts single-vector products.  With GK_FLAG_PROFILE: ms_matvec (the A P block
 * products), ms_matvec_t (A^T Q), ms_orth (the blocks' Gram-Schmidt), ms_small (the triangular
 * factors, their judges and the SVD of B) and, for gk_block_fsvd, ms_restart (U and V).  Returns GK_OK, GK_NOT_CONVERGED when
 * the small SVD hit its sweep limit, GK_NUMERICAL on a non-finite norm, or an
 * error. */
int gk_block_numrank(const gk_matrix *A, int s, const double *Q0, double eps, int kmax, const gk_opts *opts, int *rank,
                     double *sigma, int *steps, gk_info *info);

/* One cycle of the block form of Algorithm 2 (route 1): `steps` block steps of the recurrence
 * above from Q0 (or drawn as in gk_block_numrank) without a break test (fewer only when the
 * blocks fill min(m, n)), the SVD of the block lower bidiagonal B = X S Y^T, and the r largest
 * triplets U = Q X_r, V = P Y_r (A V = U S holds by construction), with each triplet's right
 * residual ||A^T u_i - s_i v_i|| = ||R_{k+1} x_i'|| read from the next right block (x_i' the
 * last s entries of x_i).  No restart: the accuracy is what the steps give.
 *  steps: block steps, (steps + 1) s <= 1024;  r: 1 <= r <= steps * s.
 *  U: m x r, S: r, V: n x r, resid: r -- device memory, column-major, f64; signs as gk_psvd.
 * GK_FLAG_BLOCK_F32 applies (the block products in f32), and GK_FLAG_RITZ_DF (U and V from the
 * bases' double-f32 copies; not with GK_FLAG_ORTH_F64).  A caller workspace (opts->workspace)
 * needs gk_block_numrank_workspace(A, s, steps, opts) bytes.  Returns GK_OK, GK_RANK_DEFICIENT
 * when the blocks filled the space with fewer than r columns (the trailing triplets zero), GK_NOT_CONVERGED when the small
 * SVD hit its sweep limit, or an error.  Experimental: not yet run on a GPU. */
int gk_block_fsvd(const gk_matrix *A, int s, const double *Q0, int steps, int r, const gk_opts *opts, double *U,
                  double *S, double *V, double *resid, gk_info *info);

/* Device workspace (bytes) gk_block_numrank needs for this operator, s, kmax and opts, and
 * gk_block_fsvd with steps = kmax (0 for invalid arguments or without a device). */
size_t gk_block_numrank_workspace(const gk_matrix *A, int s, int kmax, const gk_opts *opts);

/* F-SVD as printed (Algorithm 2): k steps of Algorithm 1 (lower-bidiagonal GK
 * with reorthogonalization; only an exact zero norm ends them early), then for
 * the r largest:
 *  route 0 (the printed algorithm): the eigendecomposition of B^T B (formed;
 *           tridiagonal) = Y Theta Y^T by one-sided Jacobi (its SVD, as it is
 *           positive semidefinite), sigma_i = sqrt(theta_i), V = P Y, and
 *           u_i = A v_i / sigma_i for all r triplets in one blocked pass over A
 *           (FP64-grade products, as gk_residuals);
 *  route 1: the SVD of B_{k'+1,k'} = X Sigma Y^T itself (one-sided Jacobi,
 *           without squaring B's condition number), V = P Y, u_i = Q x_i (the
 *           left Ritz vectors, Eq. 2.13), equal to A v_i / sigma_i in exact
 *           arithmetic.
 * No restart: the accuracy is what k steps give (compare gk_psvd).
 *  k:   Krylov steps, 1 <= k <= min(m, n), k <= 1023.
 *  r:   triplets wanted, 1 <= r <= k.
 *  U:   m x r, column-major, f64 (device or host); S: r values, descending;
 *  V:   n x r, column-major, f64.  Signs as in gk_psvd.
 * Returns GK_OK, GK_RANK_DEFICIENT when Algorithm 1 stopped at k' < r (the
 * trailing triplets are zero), GK_NOT_CONVERGED when the Jacobi sweeps hit
 * their limit, or an error.  info->kprime = k'. */
int gk_fsvd(const gk_matrix *A, int k, int r, int route, const gk_opts *opts, double *U, double *S, double *V,
            gk_info *info);

/* y = A x (trans = 0; x: n, y: m) or y = A^T x (trans = 1; x: m, y: n), f64
 * vectors (device or host).  These are the products of Eq. 2.2 (Algorithm 1)
 * run by the same kernels as the sweep: f32/bf16/f16 operators
 * multiply in f32 with x rounded to f32 and combine short f32 runs in f64;
 * f64 and CSR operators multiply in f64. */
int gk_matvec(const gk_matrix *A, int trans, const double *x, double *y, const gk_opts *opts);

/* True residuals of k triplets (columns of U m x k, V n x k, column-major,
 * f64; S k values): res_av[i] = ||A v_i - s_i u_i||, res_atu[i] =
 * ||A^T u_i - s_i v_i|| (the quantities behind the paper's err_rel of
 * Section 5 and the tolerance of gk_psvd).  Outputs f64, device or host.
 * The products are FP64-grade: f64 and CSR operators multiply in f64; f32,
 * bf16 and f16 operators multiply in double-f32 arithmetic (every product
 * and partial sum carried exactly to about 2^-47 of sum |a_ij x_j|, the
 * vectors split into two f32 parts), all k vectors per pass over A. */
int gk_residuals(const gk_matrix *A, int k, const double *U, const double *S, const double *V, double *res_av,
                 double *res_atu, const gk_opts *opts);

/* One problem of a batched call.  The operator is dense, in device memory,
 * with n <= 4096 columns; all problems of one call share one storage type;
 * outputs are device pointers.  The call writes the result fields.
 * Performance: the products read 16-byte vectors when the operator's address
 * and its row stride (ld times the element size) are multiples of 16 bytes;
 * otherwise they read one element at a time, several times slower (pad ld to
 * a multiple of 4 f32, 8 bf16/f16 or 2 f64 elements). */
typedef struct {
  gk_matrix A;
  int32_t k;             /* gk_psvd_batched: triplets wanted; gk_numrank_batched: kmax (0 = min(m, n, 256)) */
  int32_t krylov_dim;    /* gk_psvd_batched: K (0 = the gk_psvd default), at most 510 */
  double tol;            /* gk_psvd_batched: tolerance; gk_numrank_batched: eps */
  double *U, *S, *V;     /* psvd: U m x k, S k, V n x k (column-major, f64); numrank: S optional sigma(B), kmax+1 */
  const double *start;   /* optional start vector q1 (m, device) */
  double rank_cut;       /* gk_psvd_batched: relative rank cut eps (0 = none): a Ritz triplet with
                            theta_i + |residual estimate_i| <= eps * sigma_1 lies below the numerical
                            rank (Algorithm 3's threshold) and is left out of the convergence test */
  int32_t status;        /* result: per-problem status */
  int32_t rank;          /* result: numrank: estimated rank; psvd: #{i <= k : theta_i > rank_cut * sigma_1}
                            (k when rank_cut is 0) */
  int32_t steps;         /* result: bidiagonalization steps (numrank: k') */
  int32_t restarts;      /* result (psvd) */
  int32_t cycles;        /* result (psvd) */
  int32_t breakdowns;    /* result (psvd) */
  int64_t matvecs;       /* result: products with A or A^T */
  double resid_est_max;  /* result (psvd): max Ritz residual estimate / sigma_1 */
  double sigma_est;      /* result: running lower bound on sigma_1 */
  double sigma_next;     /* result (psvd): sigma_{k+1} of the last projected matrix B (a lower bound on sigma_{k+1}(A)) */
} gk_batch_item;

/* Many independent partial SVDs (the method of gk_psvd) in ONE persistent
 * launch.  The grid is a set of thread-block clusters; each cluster takes
 * problems from a device queue ordered longest-first by a cost model (bytes of
 * A times the expected passes, plus the Gram-Schmidt work) and solves each one
 * entirely on the device, its CTAs splitting the rows and combining partial
 * sums through distributed shared memory.  Cluster size: the autotuned choice
 * for this batch signature (opts->flags GK_FLAG_AUTOTUNE times 2, 4, 8 and 16
 * on the batch itself and remembers the fastest), else 8.  opts->seed + i
 * seeds problem i's start vector when no start is given.  Returns GK_OK, or the
 * worst per-problem status (errors first); gk_info sums the problems' counters
 * and reports the cluster size used in its `reserved` field and the number of
 * clusters launched in `kprime`.  With
 * GK_FLAG_PROFILE the ms_* fields hold cluster-milliseconds summed over the
 * problems (the leading CTA's SM clock at the max clock rate): ms_matvec the
 * A v products, ms_matvec_t the A^T u products with their cluster reduction,
 * ms_orth Gram-Schmidt and normalization, ms_small the projected matrix, its
 * SVD and the test, ms_restart setup, restarts and the output vectors.
 *
 * Learned pipeline (opts->predictor set; the paper has no counterpart): each
 * problem's numerical rank and Krylov dimension come from the network on its
 * sketch features instead of a separate rank pass.  Per item: k = the capacity
 * of U, S, V (columns available, >= 1), rank_cut = Algorithm 3's relative
 * threshold eps (0 < eps < 1, required), tol as usual, krylov_dim 0 (or a
 * fixed K).  The call predicts (r^, K^) = (ceil(1.05 r) + 1, ceil(K) + 2 + the
 * same margin, clamped to r^ <= k and r^ + 2 <= K^ <= min(m, n, 500)), solves
 * every problem for r^ triplets at K^ with the rank cut in one launch, and
 * judges each by its own spectrum: accepted when some Ritz value of the last
 * projected matrix fell below the cut (rank < r^, or sigma_next <= eps s_1);
 * otherwise (r^ too small, or a solve that did not converge) that problem is
 * re-solved by the plain pipeline -- Algorithm 3 for its rank r (kmax
 * min(m, n, 160)), then min(r, k) triplets at the default K.  Results: rank
 * (the numerical rank; above k when the capacity truncated the output), the
 * last solve's counters, matvecs including the sketch's pass;
 * gk_info.fallbacks counts the re-solved problems.  A Krylov dimension that
 * is too small costs restarts; a rank that is too small costs the re-solve. */
int gk_psvd_batched(gk_batch_item *items, int count, const gk_opts *opts, gk_info *info);

/* Many independent rank estimates (Algorithm 3 on Algorithm 1, as in
 * gk_numrank) in one persistent launch, scheduled as gk_psvd_batched. */
int gk_numrank_batched(gk_batch_item *items, int count, const gk_opts *opts, gk_info *info);

/* ---- Algorithm 4: fast Riemannian mini-batch gradient descent ---------- */
/* P independent similarity-learning problems of one shape (Section 4, Algorithm 4), each
 * minimizing the mini-batch objective over the manifold of rank-r d1 x d2 matrices.  Every
 * step, for every problem p at once:
 *   Gr = (1/b) sum_{i in batch} y_i x_i v_i^T - lam W      (the mini-batch gradient, printed sign)
 *   U_r, V_r = the rank-r SVD of Gr by Algorithm 2
 *   Z = U U^T Gr V V^T + (I - U U^T) Gr V V^T + U U^T Gr (I - V V^T)   (the Riemannian gradient)
 *   W = U S V^T, the rank-r SVD of W - eta Z by Algorithm 2  (the SVD retraction)
 * Each inner SVD ("Algorithm 2") is k_inner Golub-Kahan steps from q1_p without restart, the
 * SVD of the projected bidiagonal matrix and the Ritz vectors; the P inner SVDs of a step
 * run in one gk_psvd_batched launch (its statuses GK_NOT_CONVERGED are expected: no restart
 * is taken), the gradient, the projection and the retraction in this library's kernels.
 * All pointers are device memory owned by the caller; matrices are f64:
 *   X       P x N x d1: sample i of problem p is x = X + (p N + i) d1
 *   Vd      P x N x d2: its partner v = Vd + (p N + i) d2
 *   y       P x N labels (any real weights)
 *   batches steps x P x b sample indices in [0, N): step t's batch of problem p starts at
 *           batches + (t P + p) b (may be NULL when steps is 0)
 *   q1      P x d1 start vectors of the inner SVDs (nonzero)
 *   W       P x d1 x d2, row-major per problem: W0 on entry, the iterate after `steps` steps on
 *           return (the algorithm draws W0 ~ N(0, 1); the caller supplies it)
 * Limits: P >= 1, N >= b >= 1, 2 <= d1, 2 <= d2 <= 4096, 1 <= r <= 16,
 * r + 2 <= k_inner <= min(d1, d2, 510), steps >= 0.  opts: stream, reorth_passes of the
 * inner solves, GK_FLAG_AUTOTUNE for them; seed, start, krylov_dim and predictor are not
 * used.  info: matvecs and steps summed over the inner solves, cycles = RSGD steps done,
 * seconds.  Returns GK_OK, GK_INVALID_ARG (limits, null pointers, host pointers),
 * GK_OUT_OF_MEMORY, GK_CUDA_ERROR, GK_TIMEOUT or GK_NUMERICAL (from an inner solve; W then
 * holds the last completed step). */
typedef struct {
  int32_t P, N, d1, d2; /* problems, samples per problem, W is d1 x d2 */
  int32_t r;            /* rank of the manifold */
  int32_t k_inner;      /* Golub-Kahan steps of each inner SVD */
  int32_t steps, b;     /* iterations, mini-batch size */
  double eta, lam;      /* training rate, the coefficient of the -lam W term */
  const double *X, *Vd, *y;
  const int32_t *batches;
  const double *q1;
  double *W;
} gk_rsgd_args;
int gk_rsgd_batched(const gk_rsgd_args *a, const gk_opts *opts, gk_info *info);

/* ---- learned predictor of the rank and the Krylov dimension ----------- */
/* The paper has no counterpart: a small network that maps cheap sketch
 * features of A to (log r, log K) so the batched solver can skip the separate
 * rank pass and size its Krylov space; the solver's own convergence test
 * judges the prediction and its restart loop is the fallback. */
#define GK_SKETCH_COLS 32
#define GK_FEATURES 35
#define GK_MLP_TRAINABLE 75522 /* W1 256x35, b1 256, W2 256x256, b2 256, W3 2x256, b3 2 */
#define GK_MLP_PARAMS 75596    /* trainable, then input mean/std (35+35), target mean/std (2+2) */

/* Sketch features of `count` dense operators (device memory): Y = A Omega with
 * Omega (n x 32) drawn N(0,1) from Philox4x32-10 + Box-Muller (entry (j,c) is
 * draw 32j+c of the stream seeded with `seed`), the 32 singular values of Y
 * (square roots of the eigenvalues of Y^T Y, f64 Jacobi), ||A||_F, m and n:
 * features[p*35 + i] = log(sigma_i(Y) / (sqrt(32) ||A||_F)) for i < 32, then
 * log ||A||_F, log m, log n (f32, device). */
int gk_sketch_batched(const gk_matrix *A, int count, uint64_t seed, float *features, const gk_opts *opts);

/* Predictions out[b*2 + {0,1}] (de-standardized targets, f32, device or host)
 * for B feature rows x (device), with the f32 parameters or their bf16
 * rounding (bf16_weights != 0; sums stay f32). */
int gk_mlp_forward(const float *params, const float *x, int B, float *out, int bf16_weights, const gk_opts *opts);

/* Gradient of the training loss (0.5 * mean over rows of the squared error
 * of the standardized outputs) w.r.t. the GK_MLP_TRAINABLE parameters, and the
 * loss; all device pointers except loss (device or host). */
int gk_mlp_grad(const float *params, const float *x, const float *y, int B, float *grad, float *loss,
                const gk_opts *opts);

/* Adam training (lr, betas 0.9/0.999, eps 1e-8) of the trainable parameters on
 * n rows (x: n x 35, y: n x 2 targets, device) for `epochs` passes of
 * minibatches of `batch` rows in a seeded order; adam_m/adam_v (device,
 * GK_MLP_TRAINABLE each) carry the moments, t0 the step count so far;
 * losses (device or host, `epochs` floats, optional) get each epoch's last
 * minibatch loss. */
int gk_mlp_train(float *params, float *adam_m, float *adam_v, int t0, const float *x, const float *y, int n,
                 int batch, int epochs, float lr, uint64_t seed, float *losses, const gk_opts *opts);

/* Size of the device array behind gk_matvec_static (bytes). */
#define GK_STATIC_SCRATCH_BYTES (32u << 20)

/* gk_matvec_static: y = A x (trans = 0) or y = A^T x (trans = 1), the product
 * gk_matvec computes (up to the f32 summation order: A x runs the
 * row-streaming kernel), but without allocating any device memory.  The
 * paper has no counterpart; this entry point exists for callers that cannot
 * call cudaMalloc: code whose device memory is all owned by another
 * allocator (a framework's caching allocator that has reserved the GPU, so a
 * raw allocation would fail or fragment its pool), and latency-critical loops
 * where an allocation could block or synchronize the device.
 *  - Its scratch is a static device array of GK_STATIC_SCRATCH_BYTES (32 MiB)
 *    that every GPU loading this library holds until the process exits.
 *    A x needs 256 + 4*max(m,n) bytes of it (it runs the row-streaming
 *    kernel, which keeps no partial sums); dense A^T x also needs its partial
 *    sums, 8*n*(row blocks) bytes, where a row block has at most 1024 rows
 *    (about m*n/128 bytes for large m: up to m*n of about 4.1e9 elements).
 *    A problem that needs more returns GK_OUT_OF_MEMORY and computes nothing.
 *  - A, x and y must be device memory of the current device (host pointers or
 *    another GPU's memory give GK_INVALID_ARG: staging them would need an
 *    allocation).  x: n (or m) f64, y: m (or n) f64; x and y must not overlap
 *    (GK_INVALID_ARG).
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (with that device current); make that first call
 *    before any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents;
 *    the call clears what must start at zero.  Calls that overlap on the GPU
 *    (concurrent calls on different streams or host threads) race on it.
 *  - Synchronous like the other entry points; work runs on opts->stream
 *    (opts may be NULL: legacy default stream). */
int gk_matvec_static(const gk_matrix *A, int trans, const double *x, double *y, const gk_opts *opts);

/* Human-readable name of a status code. */
const char *gk_status_string(int status);

/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char *gk_last_cuda_error(void);

/* Library version string. */
const char *gk_version(void);

/* Pinned host memory for host operands and results (the calls above accept
 * any host pointer; copies from this memory stay at the link's full rate).
 * gk_host_alloc maps at least `bytes` of anonymous memory aligned to the
 * transparent-huge-page size (the mapping is rounded up to it: 512 MB with
 * 64 KB base pages, 2 MB with 4 KB ones, so carve many small operands from one
 * buffer), asks the kernel to back it with huge pages, zero-fills it, asks
 * the kernel to collapse any part the first touch left in small pages (Linux
 * 6.1+, best effort) and registers it with CUDA (cudaHostRegister); *ptr receives
 * the address (owned by the library until gk_host_free).  Errors:
 * GK_INVALID_ARG (null ptr, zero bytes, or an address gk_host_alloc did not
 * return), GK_NO_DEVICE, GK_OUT_OF_MEMORY (mmap), GK_CUDA_ERROR (registration). */
int gk_host_alloc(size_t bytes, void **ptr);
int gk_host_free(void *ptr);

/* Load the learned predictor's weights (GK_MLP_PARAMS f32 values: the layout of
 * gk_mlp_train's parameters, host or device memory, `bytes` =
 * 4 * GK_MLP_PARAMS) into device memory of the current device; *pred receives
 * a handle for opts->predictor, owned by the caller until gk_predictor_free.
 * Inference uses the bf16 rounding of the weights with f32 sums, on sketch
 * features drawn with the seed the committed weights were trained with.
 * Errors: GK_INVALID_ARG (null pointers, wrong size, a non-finite weight),
 * GK_NO_DEVICE, GK_OUT_OF_MEMORY, GK_CUDA_ERROR. */
int gk_predictor_load(const void *weights, size_t bytes, gk_predictor **pred);
int gk_predictor_free(gk_predictor *pred);

/* The (r^, K^) the learned batched pipeline derives from the network's rank and
 * Krylov estimates rf = exp(out_r), kf = exp(out_K) for an operator with
 * min(m, n) = mn and output capacity cap: r^ = min(ceil(1.05 rf) + 1,
 * min(mn, 500) - 1, cap) (at least 1), K^ = ceil(kf) + 2 + (r^ - round(rf))
 * within [r^ + 2, min(mn, 500)] where there is room (never below r^); a
 * non-finite estimate asks for min(mn, 500).  Host-only (no device needed). */
int gk_predictor_margins(double rf, double kf, int64_t mn, int cap, int *r, int *K);

/* The network's de-standardized outputs (log r, log K) for `count` dense
 * device operators: out[2 i], out[2 i + 1] (f32, host or device). */
int gk_predictor_predict(const gk_predictor *pred, const gk_matrix *A, int count, float *out, const gk_opts *opts);

/* Self-test of the device-side bounded wait that every spin of the library
 * uses (mbarrier waits of the bulk-copy pipelines): one CTA waits on an
 * mbarrier that nothing arrives at, for at most `cycles` SM clock cycles, and
 * returns.  Returns GK_TIMEOUT when the wait gave up (the expected result),
 * GK_OK if the phase completed, GK_NO_DEVICE, GK_INVALID_ARG (cycles < 0 or
 * above 4e9, about 2 s),
 * GK_OUT_OF_MEMORY or GK_CUDA_ERROR.  The context stays usable either way. */
int gk_wait_selftest(long long cycles);

/* Kernels the calling host thread has launched through this library so far
 * (every entry point counts its own launches; the counter never resets). */
int64_t gk_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* GK_H */
