// Seeded driver of bd_svd_host (bdsvd_host.cpp) for a build with AddressSanitizer and
// UndefinedBehaviorSanitizer: bidiagonals of orders 1..max_n with zero diagonal entries, zero
// off-diagonal entries, graded and clustered values; every call must finish (status 0) with
// nonnegative descending values, and the sanitizers fail the run on any access outside the
// buffers the GPU kernel also sizes (n entries of d and e, n rotations a side).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

extern "C" int bd_svd_host(const double *d_in, const double *e_in, int n, double *sigma, double *X, double *Y,
                           int *steps, int *chases);

int main(int argc, char **argv) {
  const int max_n = argc > 1 ? atoi(argv[1]) : 64;
  std::mt19937_64 g(12345);
  std::normal_distribution<double> nd(0.0, 1.0);
  int calls = 0;
  for (int n = 1; n <= max_n; ++n) {
    for (int kind = 0; kind < 5; ++kind) {
      std::vector<double> d(n), e(n > 1 ? n - 1 : 1, 0.0);
      for (int i = 0; i < n; ++i) d[i] = nd(g);
      for (int i = 0; i + 1 < n; ++i) e[i] = nd(g);
      if (kind == 1)
        for (int i = 0; i < n; i += 3) d[i] = 0.0;  // zero diagonal entries: the chases
      if (kind == 2)
        for (int i = 1; i + 1 < n; i += 4) e[i] = 0.0;  // splits from the start
      if (kind == 3)
        for (int i = 0; i < n; ++i) {  // graded
          d[i] = std::pow(10.0, -i / 8.0);
          if (i + 1 < n) e[i] = std::pow(10.0, -i / 8.0);
        }
      if (kind == 4)
        for (int i = 0; i < n; ++i) {  // a tight cluster
          d[i] = 1.0;
          if (i + 1 < n) e[i] = 1e-9;
        }
      std::vector<double> s(n), X((size_t)n * n), Y((size_t)n * n);
      int steps = 0, chases[2];
      const int rc = bd_svd_host(d.data(), e.data(), n, s.data(), X.data(), Y.data(), &steps, chases);
      if (rc != 0) {
        printf("n=%d kind=%d status %d\n", n, kind, rc);
        return 1;
      }
      for (int i = 0; i < n; ++i)
        if (!(s[i] >= 0.0) || (i > 0 && s[i] > s[i - 1])) {
          printf("n=%d kind=%d: values not nonnegative and descending\n", n, kind);
          return 1;
        }
      ++calls;
    }
  }
  printf("%d\n", calls);
  return 0;
}
