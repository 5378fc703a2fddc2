/*
 * gk_oracle.h -- plain FP64 CPU oracle for the Golub-Kahan partial SVD and
 * numerical-rank method of "Accurate and fast matrix factorization for
 * low-rank learning" (arXiv 2104.10785).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code; only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library: the two are independent implementations of the same paper.
 *
 * Every routine is a slow, literal restatement of one passage of the paper (or
 * of a textbook definition the paper relies on) in double precision, with no
 * BLAS/LAPACK and no blocking or reordering beyond what the definition states.
 *
 * Matrix operands are read from the caller's stored bytes and promoted exactly
 * to double (f32, bf16 and f16 values are all exactly representable in f64).
 */
#ifndef GK_ORACLE_H
#define GK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* storage types of the operator's values */
enum { GKO_F64 = 0, GKO_F32 = 1, GKO_BF16 = 2, GKO_F16 = 3 };
/* operator kinds */
enum { GKO_DENSE = 0, GKO_CSR = 1 };

typedef struct {
  int kind;             /* GKO_DENSE (row-major, leading dimension ld) or GKO_CSR */
  int dtype;            /* GKO_F64 / F32 / BF16 / F16 */
  int64_t m, n;         /* rows, columns */
  int64_t ld;           /* dense: elements between consecutive rows (>= n) */
  double scale;         /* every stored value is multiplied by this (1.0 unless f16-scaled) */
  const void *vals;     /* dense: m*ld values; CSR: nnz values */
  const int32_t *rowptr;/* CSR: m+1 offsets */
  const int32_t *colind;/* CSR: nnz column indices */
} gko_op;

/* ---- helpers exposed for tests ---------------------------------------- */
double gko_elem_value(const gko_op *A, int64_t idx);            /* stored value #idx promoted to f64 */
void   gko_apply(const gko_op *A, const double *x, double *y);   /* y = A x  (x: n, y: m) */
void   gko_apply_t(const gko_op *A, const double *x, double *y); /* y = A^T x (x: m, y: n) */
void   gko_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void   gko_start_vector(uint64_t seed, int64_t m, double *q);   /* q_i ~ N(2,1) from the seed */
uint64_t gko_splitmix64(uint64_t x);
void   gko_set_threads(int nthreads);                            /* 0 = library default */

/* One-sided (Hestenes) Jacobi SVD of a dense rows x cols matrix M
 * (column-major, ld = rows, rows >= cols).  Outputs sigma[cols] descending,
 * Uc (rows x cols, column-major) and Vc (cols x cols, column-major).
 * Returns the number of sweeps used (negative if it did not converge). */
int gko_jacobi_svd(int64_t rows, int64_t cols, const double *M,
                   double *sigma, double *Uc, double *Vc);

/* Cyclic two-sided Jacobi eigen-decomposition of a symmetric n x n matrix S
 * (column-major).  theta[n] descending, G (n x n, column-major) eigenvectors. */
int gko_jacobi_eig(int64_t n, const double *S, double *theta, double *G);

/* ---- Algorithm 1: GK bidiagonalization with reorthogonalization -------- */
typedef struct {
  int kprime;           /* k' (number of completed columns of B_{k'+1,k'}) */
  int stop_reason;      /* 0 ran k iterations, 1 beta break, 2 alpha break */
  double sigma_est;     /* running lower bound on sigma_1 used by the break test */
} gko_gk_info;

/* Inputs: A, k (iterations, 1 <= k <= min(m,n)), eps and eps_relative (the
 * break threshold is eps*sigma_est if eps_relative != 0, else eps), passes (1 =
 * one classical Gram-Schmidt pass as printed in the paper, 2 = two passes,
 * 0 = a second pass only when the first left less than 1/sqrt(2) of the norm),
 * q1 (m start values, not necessarily normalized).
 * Outputs: alpha[k+1], beta[k+2] (beta[0] = ||q1||, beta[i] = beta_{i+1} of the
 * paper's 1-based notation is stored at index i), Q (m x (k+1), column-major),
 * P (n x (k+1), column-major).  Entries past k' are left zero.
 * fused != 0 runs the fused-sweep ordering (A^T w / beta_{j+1} in place of
 * A^T q_{j+1}, see gk_oracle.c); 0 is Algorithm 1 as printed. */
/* Classical Gram-Schmidt of w (len) against the j columns of Q (column-major,
 * leading dimension ld) with the pass rule of gko_gk_lower's `passes`. */
void gko_cgs(int passes, double *w, const double *Q, int64_t len, int64_t ld, int j);

int gko_gk_lower(const gko_op *A, int k, double eps, int eps_relative, int passes,
                 const double *q1, double *alpha, double *beta, double *Q, double *P,
                 gko_gk_info *info, int fused);

/* ---- Algorithm 3: rank determination ------------------------------------ */
/* r = #{ sigma_i(B_{k'+1,k'}) > eps * sigma_1(B) } (relative reading) or, with
 * literal != 0, #{ theta_i(B^T B) > eps } (the printed eigenvalue count). */
int gko_numrank(const gko_op *A, int kmax, double eps, int eps_relative, int literal,
                int passes, const double *q1, int *rank, gko_gk_info *info,
                double *sigma_out /* optional, kmax+1 */, int fused);

/* ---- Algorithm 2: F-SVD ------------------------------------------------- */
/* route 0: eig(B^T B) then U = A V / sigma (as printed);
 * route 1: one-sided Jacobi SVD of B, V = P Y, U = Q X.
 * Outputs U (m x r), S (r), V (n x r); returns k' through info. */
int gko_fsvd(const gko_op *A, int k, int r, int route, int passes, const double *q1,
             double *U, double *S, double *V, gko_gk_info *info, int fused);

/* ---- thick-restart partial SVD (upper-bidiagonal form) ---------------- */
typedef struct {
  int cycles;           /* bidiagonalization cycles run */
  int restarts;
  int64_t matvecs;      /* products with A or A^T */
  int converged;
  int kdim_used;        /* Krylov dimension actually used (<= K) */
  double resid_est_max; /* max_i<=k beta_K |X_{K,i}| / sigma_1 at exit */
} gko_psvd_info;

/* Partial SVD of A: the k largest singular triplets, Krylov dimension K
 * (k < K <= min(m,n), or K == k == min(m,n)), keep = number of Ritz vectors
 * kept at a restart (k <= keep < K; pass 0 for k + (K-k)/2), tol relative to
 * sigma_1, max_restarts, passes (Gram-Schmidt passes), q1 (m start values),
 * seed (for replacement directions after an exact breakdown).
 * Outputs U (m x k), S (k), V (n x k), all column-major, sign-normalized so
 * the largest-magnitude entry of each v_i is positive.  Returns 0 if
 * converged, 1 if not converged within max_restarts, <0 on bad arguments. */
int gko_psvd(const gko_op *A, int k, int K, int keep, double tol, int max_restarts,
             int passes, const double *q1, uint64_t seed,
             double *U, double *S, double *V, gko_psvd_info *info, int fused);

/* One cycle of the restart-free upper-bidiagonal process from v1 = A^T q1 /
 * ||A^T q1||: K steps, returns alpha[K], beta[K] (beta[K-1] couples v_{K+1}),
 * Ub (m x K), Vb (n x (K+1)).  Used by tests that check the bidiagonal
 * relations of the upper form. */
int gko_gk_upper(const gko_op *A, int K, int passes, const double *q1, uint64_t seed,
                 double *alpha, double *beta, double *Ub, double *Vb, int fused);

/* ---- error metrics ------------------------------------------------------ */
/* per-triplet residuals res[i] = max(||A v_i - s_i u_i||, ||A^T u_i - s_i v_i||) */
void gko_residuals(const gko_op *A, int k, const double *U, const double *S,
                   const double *V, double *res_av, double *res_atu);
/* the paper's relative error ||A^T U - V S||_F / ||S||_F */
double gko_err_rel(const gko_op *A, int k, const double *U, const double *S, const double *V);
/* the paper's residual error ||A - U S V^T||_F (dense operators only) */
double gko_err_res(const gko_op *A, int k, const double *U, const double *S, const double *V);

#ifdef __cplusplus
}
#endif
#endif
