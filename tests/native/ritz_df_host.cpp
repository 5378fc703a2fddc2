// Host build of the double-f32 Ritz-vector product (gk_ritz_df.cuh) for the CPU tests: the
// per-thread function run for every row and column group, as the GPU grid runs it.
#include <vector>

#include "../../paper_2104_10785_gb300/csrc/gk_ritz_df.cuh"

extern "C" void ritz_df_host(const double *Q, long long ldq, long long len, int K, const double *X, long long ldx,
                             int ncol, double *C, long long ldc) {
  std::vector<gk::DfPair> Qs((size_t)ldq * K), Xs((size_t)ldx * ncol);
  for (long long k = 0; k < K; ++k)
    for (long long i = 0; i < ldq; ++i) Qs[(size_t)(k * ldq + i)] = gk::df_split(i < len ? Q[k * ldq + i] : 0.0);
  for (long long c = 0; c < ncol; ++c)
    for (long long k = 0; k < ldx; ++k) Xs[(size_t)(c * ldx + k)] = gk::df_split(X[c * ldx + k]);
  for (int c0 = 0; c0 < ncol; c0 += gk::kRitzCols) {
    const int nc = ncol - c0 < gk::kRitzCols ? ncol - c0 : gk::kRitzCols;
    for (long long i = 0; i < len; ++i) gk::ritz_df_row(Qs.data(), ldq, i, K, Xs.data(), ldx, c0, nc, C, ldc);
  }
}
