// Host build of the block judge's arithmetic (gk_block_judge.cuh), run the way k_block_judge runs
// it on one warp: the lanes' updates of each phase one lane after another (the entries a phase
// touches are distinct per lane), for the CPU tests.
#include <math.h>

#include <vector>

#include "../../paper_2104_10785_gb300/csrc/gk_block_judge.cuh"

// status (0, 1, 2) of the judge of raw (s x s, column-major) on `side` with eps; *sest updated,
// *nrm = ||triu(raw)||_2, *sweeps = Jacobi sweeps; B (ld ldb) receives the placed entries at
// (row0, col0) when the kernel would place them
extern "C" int block_judge_host(const double *raw, int s, int side, double eps, double *sest, double *nrm,
                                int *sweeps, double *B, long long ldb, int row0, int col0) {
  const int ss = s * s;
  std::vector<double> T(ss), G(ss);
  double mu = 0.0;
  for (int e = 0; e < ss; ++e) {
    T[e] = gk::bj_triu(raw, s, e);
    mu = gk::bj_absmax(mu, fabs(T[e]));
  }
  const double rmu = gk::bj_rscale(mu);
  for (int e = 0; e < ss; ++e) G[e] = gk::bj_gram(T.data(), s, rmu, e);
  int sw = 0;
  if (rmu > 0.0) {
    for (; sw < gk::kBlockSweeps; ++sw) {
      bool rotated = false;
      for (int p = 0; p < s - 1; ++p)
        for (int q = p + 1; q < s; ++q) {
          double c, sn;
          if (!gk::bj_rotation(G.data(), s, p, q, &c, &sn)) continue;
          rotated = true;
          for (int lane = 0; lane < s; ++lane) gk::bj_col(G.data(), s, p, q, c, sn, lane);
          for (int lane = 0; lane < s; ++lane) gk::bj_row(G.data(), s, p, q, c, sn, lane);
        }
      if (!rotated) break;
    }
  }
  *sweeps = sw;
  const int brk = gk::bj_decide(G.data(), s, mu, side, eps, sest, nrm);
  if (B && (brk == 0 || (side == 0 && brk == 1)))
    for (int e = 0; e < ss; ++e)
      if (e % s <= e / s) B[gk::bj_place(side, row0, col0, e % s, e / s, ldb)] = T[e];
  return brk;
}
