"""Algorithm 4 on the GPU (gk_rsgd_batched: the gradient, projection and retraction kernels,
the inner SVDs on the batched solver) against the oracle (oracle/rsgd.py) on the same seeded
data, batches and start vectors.

Both sides run the inner SVD as the same restart-free cycle in f64; their iterates differ by
rounding only (the GPU's gradient multiplies y into x before the sum, its projection uses the
expanded form (Gr V - U C) V^T + U (U^T Gr) instead of explicit projectors), ~1e-13 per step,
and the retraction is smooth while the r-th and (r+1)-th Ritz values are apart, which holds
for these seeds.  Tolerance: 1e-8 of ||W||_F after the steps."""
import numpy as np
import pytest
import torch

import synth
from oracle import rsgd as ors

pytestmark = pytest.mark.gpu


def gk():
    import paper_2104_10785_gb300 as m

    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_gpu(X, Vd, y, W0, batches, q1, eta, lam, r, k_inner):
    W = cuda(W0.copy())
    st, info = gk().gk_rsgd_batched(cuda(X), cuda(Vd), cuda(y), W, cuda(batches), cuda(q1), eta, lam, r, k_inner)
    return st, info, W.cpu().numpy()


@pytest.mark.parametrize("P,N,d1,d2,r,k_inner,steps,b", [(3, 512, 784, 256, 5, 20, 3, 64),
                                                         (2, 512, 784, 256, 5, 35, 2, 64),
                                                         (4, 300, 100, 70, 3, 16, 4, 33)])
def test_rsgd_matches_oracle(P, N, d1, d2, r, k_inner, steps, b):
    X, Vd, y, W0, batches, q1, _ = synth.rsgd_data(P, N, d1, d2, r, steps, b, seed=d1 + k_inner)
    eta, lam = 2.0, 0.05
    st, info, W = run_gpu(X, Vd, y, W0, batches, q1, eta, lam, r, k_inner)
    assert st == 0 and info["cycles"] == steps and info["matvecs"] > 0
    for p in range(P):
        Wo = ors.rsgd(X[p], Vd[p], y[p], W0[p], batches[:, p], eta, lam, r, k_inner, q1[p])
        err = np.linalg.norm(W[p] - Wo) / np.linalg.norm(Wo)
        assert err <= 1e-8, (p, err)
        assert np.linalg.matrix_rank(W[p], tol=1e-9 * np.linalg.norm(W[p], 2)) == r


def test_rsgd_full_krylov_step_in_closed_form():
    """k_inner = min(d1, d2): the inner SVDs are exact, so one step is
    W1 = trunc_r(W0 - eta trunc_r(Gr)) -- checked with LAPACK, independently of the oracle."""
    X, Vd, y, W0, batches, q1, _ = synth.rsgd_data(2, 200, 40, 24, 3, 1, 50, seed=11)
    eta, lam, r = 0.7, 0.1, 3
    st, info, W = run_gpu(X, Vd, y, W0, batches, q1, eta, lam, r, 24)
    assert st == 0

    def trunc(M, r):
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        return (U[:, :r] * S[:r]) @ Vt[:r]

    for p in range(2):
        idx = batches[0, p]
        G = sum(y[p][i] * np.outer(X[p][i], Vd[p][i]) for i in idx) / len(idx) - lam * W0[p]
        np.testing.assert_allclose(W[p], trunc(W0[p] - eta * trunc(G, r), r), atol=1e-9)


def test_rsgd_zero_steps_leaves_w():
    X, Vd, y, W0, batches, q1, _ = synth.rsgd_data(2, 64, 30, 20, 2, 0, 8, seed=12)
    batches = np.zeros((0, 2, 8), dtype=np.int32)
    st, info, W = run_gpu(X, Vd, y, W0, batches, q1, 1.0, 0.0, 2, 10)
    assert st == 0 and info["cycles"] == 0
    np.testing.assert_array_equal(W, W0)


def test_rsgd_learns_the_planted_similarity():
    """Sixteen problems at the paper's shape: the sign agreement of x^T W v with the planted
    x^T W* v rises from chance."""
    P, N, d1, d2, r = 16, 2048, 784, 256, 5
    X, Vd, y, W0, batches, q1, Ws = synth.rsgd_data(P, N, d1, d2, r, 30, 256, seed=13)
    st, info, W = run_gpu(X, Vd, y, W0, batches, q1, 50.0, 0.0, r, 20)
    assert st == 0
    agree = [np.mean(np.sign(np.einsum("ni,ij,nj->n", X[p], W[p], Vd[p])) ==
                     np.sign(np.einsum("ni,ij,nj->n", X[p], Ws[p], Vd[p]))) for p in range(P)]
    assert min(agree) > 0.6, agree
