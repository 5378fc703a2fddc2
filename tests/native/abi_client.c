/* A plain C client of the library's C ABI (include/gk.h): every entry point is referenced with
 * its declared signature, so compiling this file as C11 checks that the header is valid C and
 * that the declarations agree with their uses; linking it against libgk.so checks that every
 * referenced symbol is exported.  It runs without a GPU: the calls it makes return
 * GK_NO_DEVICE (or GK_INVALID_ARG) before touching any pointer. */
#include <stdio.h>
#include <string.h>

#include "../../include/gk.h"

typedef void (*any_fn)(void);

int main(void) {
  gk_opts o;
  gk_default_opts(&o);
  double A[12];
  memset(A, 0, sizeof(A));
  gk_matrix M;
  memset(&M, 0, sizeof(M));
  M.kind = GK_DENSE;
  M.dtype = GK_F64;
  M.m = 4;
  M.n = 3;
  M.ld = 3;
  M.scale = 1.0;
  M.vals = A;
  gk_info info;
  int r = -1, steps = 0;
  double U[12], S[3], V[9];
  int st[6];
  st[0] = gk_psvd(&M, 1, 1e-8, &o, U, S, V, &info);
  st[1] = gk_numrank(&M, 1e-8, 0, &o, &r, NULL, &info);
  st[2] = gk_fsvd(&M, 2, 1, 1, &o, U, S, V, &info);
  st[3] = gk_block_numrank(&M, 2, NULL, 1e-8, 0, &o, &r, NULL, &steps, &info);
  st[4] = gk_block_numrank(&M, 0, NULL, 1e-8, 0, &o, &r, NULL, &steps, &info); /* s = 0: refused */
  st[5] = gk_matvec(&M, 0, S, U, &o);
  /* referenced for the link check only (not called) */
  any_fn refs[] = {(any_fn)gk_psvd_workspace, (any_fn)gk_numrank_workspace, (any_fn)gk_block_numrank_workspace, (any_fn)gk_block_fsvd,
                  (any_fn)gk_residuals, (any_fn)gk_psvd_batched, (any_fn)gk_numrank_batched,
                  (any_fn)gk_rsgd_batched, (any_fn)gk_sketch_batched, (any_fn)gk_mlp_forward, (any_fn)gk_mlp_grad,
                  (any_fn)gk_mlp_train, (any_fn)gk_matvec_static, (any_fn)gk_predictor_load,
                  (any_fn)gk_predictor_free, (any_fn)gk_predictor_predict, (any_fn)gk_predictor_margins,
                  (any_fn)gk_host_alloc, (any_fn)gk_host_free, (any_fn)gk_wait_selftest, (any_fn)gk_launch_count,
                  (any_fn)gk_last_cuda_error, (any_fn)gk_version};
  printf("%d %d %d %d %d %d %s %d\n", st[0], st[1], st[2], st[3], st[4], st[5], gk_status_string(GK_NO_DEVICE),
         (int)(sizeof(refs) / sizeof(refs[0])));
  return 0;
}
