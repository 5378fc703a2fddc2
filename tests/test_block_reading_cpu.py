"""The block QR reading the GPU path of block Golub-Kahan takes, checked on the CPU.

gk_block_numrank does not factor a block by Householder QR as the oracle (oracle/block_gk.py)
does: it orthonormalizes the block's columns one at a time by two classical Gram-Schmidt passes
against every earlier basis column, puts a fresh direction (orthogonalized twice) in place of a
column the passes reduce to <= 2^-46 of the largest norm so far, and takes each triangular
factor as Q_{j+1}^T (A P_j) (resp. P_{j+1}^T (A^T Q_{j+1})).  This module restates that flow in
numpy and checks that it gives the oracle's block steps, rank and singular values of B, with
rank-deficient blocks (the fresh completions) included -- the reading the GPU parity tests rely
on, pinned independently of the GPU."""
import numpy as np
import pytest

import synth
from oracle import block_gk as bgk


def tri_norm(T):
    return float(np.sqrt(max(np.linalg.eigvalsh(T.T @ T).max(), 0.0)))


def column_block_gk(A, Q0, eps, kmax, fresh_seed=0):
    """(rank, sigma(B), block steps, replaced columns) by the library's column-wise flow."""
    m, n = A.shape
    s = Q0.shape[1]
    mn = min(m, n)
    kb = kmax if kmax > 0 else max(1, min(mn // s, 1024 // s - 1))
    cols = (kb + 1) * s
    Q, P, B = np.zeros((m, cols)), np.zeros((n, cols)), np.zeros((cols, cols))
    g = np.random.default_rng(fresh_seed)
    scale = [0.0]
    replaced = [0]

    def orth(Bas, jc0, W):
        for c in range(W.shape[1]):
            jc = jc0 + c
            w = W[:, c].copy()
            for _ in range(2 if jc > 0 else 0):
                w -= Bas[:, :jc] @ (Bas[:, :jc].T @ w)
            nrm = np.linalg.norm(w)
            scale[0] = max(scale[0], nrm)
            if nrm <= 2.0**-46 * scale[0]:
                replaced[0] += 1
                f = g.uniform(-1.0, 1.0, Bas.shape[0])
                f0 = np.linalg.norm(f)
                for _ in range(2):
                    f -= Bas[:, :jc] @ (Bas[:, :jc].T @ f)
                nf = np.linalg.norm(f)
                Bas[:, jc] = f / nf if nf > 1e-8 * f0 else 0.0
            else:
                Bas[:, jc] = w / nrm

    orth(Q, 0, Q0)
    scale[0] = 0.0
    W = A.T @ Q[:, :s]
    orth(P, 0, W)
    T = np.triu(P[:, :s].T @ W)
    sest = tri_norm(T)
    B[:s, :s] = T.T
    steps = 1
    while True:
        pj, qn = (steps - 1) * s, steps * s
        W = A @ P[:, pj:pj + s]
        orth(Q, qn, W)
        T = np.triu(Q[:, qn:qn + s].T @ W)
        nr = tri_norm(T)
        sest = max(sest, nr)
        B[qn:qn + s, pj:pj + s] = T
        if (eps > 0 and nr <= eps * sest) or steps >= kb or (steps + 1) * s > mn:
            break
        W = A.T @ Q[:, qn:qn + s]
        orth(P, qn, W)
        T = np.triu(P[:, qn:qn + s].T @ W)
        nr = tri_norm(T)
        if eps > 0 and nr <= eps * max(sest, nr):
            break
        sest = max(sest, nr)
        B[qn:qn + s, qn:qn + s] = T.T
        steps += 1
    K = (steps + 1) * s
    sig = np.linalg.svd(B[:K, :K], compute_uv=False)[: steps * s]
    return int(np.sum(sig > eps * sig[0])), sig, steps, replaced[0]


@pytest.mark.parametrize("case", ["repeated_s3", "repeated_s1", "product_s3", "product_s8", "noisy_s4"])
def test_column_wise_block_qr_gives_the_oracles_B(case):
    if case.startswith("repeated"):
        A, _, _ = synth.prescribed_spectrum(70, 40, np.array([5.0, 5.0, 5.0, 3.0, 3.0, 1.0, 1.0, 1.0]), seed=4,
                                            dtype=np.float64)
    elif case.startswith("product"):
        A = synth.gaussian_product(300, 200, 20, 0.0, seed=5, dtype=np.float64)
    else:
        A = synth.gaussian_product(400, 250, 16, 1e-7, seed=6, dtype=np.float64)
    s = int(case.split("_s")[1])
    eps = 1e-5 if case.startswith("noisy") else 1e-8
    Q0 = np.random.default_rng(s).standard_normal((A.shape[0], s))
    r_or, sig_or, k_or = bgk.block_numrank(A, Q0, eps=eps)
    for fresh_seed in (0, 1):  # whichever completion replaces a dependent column
        r, sig, k, replaced = column_block_gk(A, Q0, eps, 0, fresh_seed)
        assert (r, k) == (r_or, k_or)
        np.testing.assert_allclose(sig, sig_or[: k * s], rtol=0, atol=1e-13 * sig_or[0])
    if case in ("repeated_s3", "product_s3", "product_s8"):
        assert replaced > 0  # the rank-deficient blocks were exercised
