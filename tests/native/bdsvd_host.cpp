// Host build of the bidiagonal SVD's step and row functions (gk_bdsvd.cuh), driven the way the
// GPU kernel drives them, for the CPU tests: X, Y start as the identity, every step's left
// rotations go to every row of X and its right rotations to every row of Y, then the signs are
// made positive and the values sorted descending (stable by index).
#include <algorithm>
#include <numeric>
#include <vector>

#include "../../paper_2104_10785_gb300/csrc/gk_bdsvd.cuh"

extern "C" int bd_svd_host(const double *d_in, const double *e_in, int n, double *sigma, double *X, double *Y,
                           int *steps, int *chases) {
  chases[0] = chases[1] = 0;  // Golub-Kahan steps, zero-diagonal chases
  if (n <= 0) return -2;
  std::vector<double> d(d_in, d_in + n), e(n > 1 ? n - 1 : 1, 0.0);
  for (int k = 0; k + 1 < n; ++k) e[k] = e_in[k];
  std::vector<double> Xw((size_t)n * n, 0.0), Yw((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Xw[(size_t)i * n + i] = Yw[(size_t)i * n + i] = 1.0;
  std::vector<gk::BdRot> rl(n), rr(n);
  gk::BdState st;
  gk::bd_init(&st, d.data(), e.data(), n);
  int rc;
  for (;;) {
    int nl = 0, nr = 0;
    rc = gk::bd_step(d.data(), e.data(), &st, rl.data(), &nl, rr.data(), &nr);
    if (rc <= 0) break;
    if (nl < 0 || nl > n || nr < 0 || nr > n) return -3;  // the kernel has room for n rotations a side
    ++chases[rc == 1 ? 0 : 1];
    for (int i = 0; i < n; ++i) {
      if (rc == 1) {  // a Golub-Kahan step: adjacent pairs, the carried-register form
        gk::bd_apply_chase(Xw.data() + i, n, rl.data(), nl);
        gk::bd_apply_chase(Yw.data() + i, n, rr.data(), nr);
      } else {
        gk::bd_apply_row(Xw.data() + i, n, rl.data(), nl);
        gk::bd_apply_row(Yw.data() + i, n, rr.data(), nr);
      }
    }
  }
  *steps = st.steps;
  for (int k = 0; k < n; ++k)
    if (d[k] < 0.0) {
      d[k] = -d[k];
      for (int i = 0; i < n; ++i) Yw[(size_t)k * n + i] = -Yw[(size_t)k * n + i];
    }
  std::vector<int> p(n);
  std::iota(p.begin(), p.end(), 0);
  std::stable_sort(p.begin(), p.end(), [&](int a, int b) { return d[a] > d[b]; });
  for (int t = 0; t < n; ++t) {
    sigma[t] = d[p[t]];
    for (int i = 0; i < n; ++i) {
      X[(size_t)t * n + i] = Xw[(size_t)p[t] * n + i];
      Y[(size_t)t * n + i] = Yw[(size_t)p[t] * n + i];
    }
  }
  return rc;
}
