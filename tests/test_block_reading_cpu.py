"""The block QR reading the GPU path of block Golub-Kahan takes, checked on the CPU.

gk_block_numrank does not factor a block by Householder QR as the oracle (oracle/block_gk.py)
does: it orthonormalizes the block's columns one at a time by two classical Gram-Schmidt passes
against every earlier basis column, puts a fresh direction (orthogonalized twice) in place of a
column the passes reduce to <= 2^-46 of the largest norm so far, and takes each triangular
factor as Q_{j+1}^T (A P_j) (resp. P_{j+1}^T (A^T Q_{j+1})).  This module restates that flow in
numpy and checks that it gives the oracle's block steps, rank and singular values of B, with
rank-deficient blocks (the fresh completions) included -- the reading the GPU parity tests rely
on, pinned independently of the GPU.  The same for gk_block_fsvd's flow (the next right block's
R_{k+1} as inner products, U from all rows of X, V from the first ks rows of Y, the residuals
from rows ks .. ks + s of X), for blocks that run past the space (zero completions), and for the
block Gram-Schmidt of GK_FLAG_BLOCK_GS (reorthogonalized block classical Gram-Schmidt)."""
import numpy as np
import pytest

import synth
from oracle import block_gk as bgk


def tri_norm(T):
    return float(np.sqrt(max(np.linalg.eigvalsh(T.T @ T).max(), 0.0)))


def column_block_gk(A, Q0, eps, kmax, fresh_seed=0, block_gs=False, second=True):
    """(rank, sigma(B), block steps, replaced columns) by the library's column-wise flow, or with
    block_gs by its block Gram-Schmidt (GK_FLAG_BLOCK_GS; reorthogonalized block classical
    Gram-Schmidt, Barlow and Smoktunowicz 2013): W1 = W - Q (Q^T W); the block's QR column by
    column (two passes against its own earlier columns, the breakdown test and fresh completions
    as above); then (`second`) that orthonormal block projected once more, W2 = W1' - Q (Q^T W1'),
    and its QR again (plain normalization: its norms are ~1)."""
    m, n = A.shape
    s = Q0.shape[1]
    mn = min(m, n)
    kb = kmax if kmax > 0 else max(1, min(mn // s, 1024 // s - 1))
    cols = (kb + 1) * s
    Q, P, B = np.zeros((m, cols)), np.zeros((n, cols)), np.zeros((cols, cols))
    g = np.random.default_rng(fresh_seed)
    scale = [0.0]
    replaced = [0]

    def orth(Bas, jc0, W, judge=True):
        if block_gs and jc0 > 0 and judge:
            W1 = W - Bas[:, :jc0] @ (Bas[:, :jc0].T @ W)
            orth(Bas, jc0, W1, judge=None)  # the block's own QR, with the breakdown test
            if second:
                W1p = Bas[:, jc0:jc0 + W.shape[1]].copy()
                orth(Bas, jc0, W1p - Bas[:, :jc0] @ (Bas[:, :jc0].T @ W1p), judge=False)
            return
        for c in range(W.shape[1]):
            jc = jc0 + c
            w = W[:, c].copy()
            lo = jc0 if judge is not True else 0  # in-block only (block Gram-Schmidt) or every column
            for _ in range(2 if jc > lo else 0):
                w -= Bas[:, lo:jc] @ (Bas[:, lo:jc].T @ w)
            if judge is False:
                nw = np.linalg.norm(w)
                Bas[:, jc] = w / nw if nw > 0 else 0.0
                continue
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


def operator_case(case):
    if case.startswith("repeated"):
        return synth.prescribed_spectrum(70, 40, np.array([5.0, 5.0, 5.0, 3.0, 3.0, 1.0, 1.0, 1.0]), seed=4,
                                         dtype=np.float64)[0]
    if case.startswith("product"):
        return synth.gaussian_product(300, 200, 20, 0.0, seed=5, dtype=np.float64)
    return synth.gaussian_product(400, 250, 16, 1e-7, seed=6, dtype=np.float64)


@pytest.mark.parametrize("case", ["repeated_s3", "repeated_s1", "product_s3", "product_s8", "noisy_s4"])
def test_block_gram_schmidt_gives_the_oracles_B(case):
    """The block Gram-Schmidt flow (BCGS2) gives the oracle's steps, rank and sigma(B); with one
    projection only, a column that cancels in the block's own QR keeps the earlier basis'
    directions its rounding brought in, and the rank-deficient blocks of product_s8 go wrong."""
    A = operator_case(case)
    s = int(case.split("_s")[1])
    eps = 1e-5 if case.startswith("noisy") else 1e-8
    Q0 = np.random.default_rng(s).standard_normal((A.shape[0], s))
    r_or, sig_or, k_or = bgk.block_numrank(A, Q0, eps=eps)
    for fresh_seed in (0, 1):
        r, sig, k, _ = column_block_gk(A, Q0, eps, 0, fresh_seed, block_gs=True)
        assert (r, k) == (r_or, k_or)
        np.testing.assert_allclose(sig, sig_or[: k * s], rtol=0, atol=1e-13 * sig_or[0])
    if case == "product_s8":
        r, sig, k, _ = column_block_gk(A, Q0, eps, 0, 0, block_gs=True, second=False)
        assert (r, k) != (r_or, k_or) or np.abs(sig - sig_or[: k * s]).max() > 1e-8 * sig_or[0]


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


def column_block_fsvd(A, Q0, steps, r, fresh_seed=0):
    """gk_block_fsvd's flow in numpy: `steps` block steps without a break test by the column-wise
    QR above, the next right block's R_{k+1} as the inner products P_{k+1}^T (A^T Q_{k+1}), the SVD
    of B padded with zero columns to its square, U = Q X_r (all (k+1)s rows of X), V = P Y_r (the
    first ks rows of Y) and residuals ||R_{k+1} x_i'|| (x_i' = rows ks .. ks + s of x_i)."""
    m, n = A.shape
    s = Q0.shape[1]
    mn = min(m, n)
    cols = (steps + 1) * s
    Q, P, B = np.zeros((m, cols)), np.zeros((n, cols)), np.zeros((cols, cols))
    g = np.random.default_rng(fresh_seed)
    scale = [0.0]

    def orth(Bas, jc0, W):
        for c in range(W.shape[1]):
            jc = jc0 + c
            w = W[:, c].copy()
            for _ in range(2 if jc > 0 else 0):
                w -= Bas[:, :jc] @ (Bas[:, :jc].T @ w)
            nrm = np.linalg.norm(w)
            scale[0] = max(scale[0], nrm)
            if nrm <= 2.0**-46 * scale[0]:
                # a fresh direction; zero when the basis already spans the space (NM_FRESH)
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
    B[:s, :s] = np.triu(P[:, :s].T @ W).T
    k = 1
    while True:
        pj, qn = (k - 1) * s, k * s
        W = A @ P[:, pj:pj + s]
        orth(Q, qn, W)
        B[qn:qn + s, pj:pj + s] = np.triu(Q[:, qn:qn + s].T @ W)
        if k >= steps or (k + 1) * s > mn:
            break
        W = A.T @ Q[:, qn:qn + s]
        orth(P, qn, W)
        B[qn:qn + s, qn:qn + s] = np.triu(P[:, qn:qn + s].T @ W).T
        k += 1
    qn = k * s
    W = A.T @ Q[:, qn:qn + s]
    orth(P, qn, W)
    R = np.triu(P[:, qn:qn + s].T @ W)
    K, ks = (k + 1) * s, k * s
    rr = min(r, ks)
    X, S, Yt = np.linalg.svd(B[:K, :K])
    U = Q[:, :K] @ X[:, :rr]
    V = P[:, :ks] @ Yt[:rr, :ks].T
    res = np.linalg.norm(R @ X[ks:ks + s, :rr], axis=0)
    return U, S[:rr], V, res, k


def angle_err(X, Y):
    sg = np.sign(np.sum(X * Y, axis=0))
    sg[sg == 0] = 1
    return np.linalg.norm(X - Y * sg[None, :], axis=0).max()


@pytest.mark.parametrize("m,n,s,steps,r,rank", [(400, 300, 4, 10, 12, 0), (300, 200, 1, 30, 5, 0),
                                                (500, 240, 8, 6, 30, 0), (260, 180, 4, 5, 8, 12)])
def test_column_wise_block_fsvd_gives_the_oracles_triplets(m, n, s, steps, r, rank):
    """The flow gk_block_fsvd runs gives oracle/block_gk.block_fsvd's triplets and residuals: values
    to 1e-12 relative, vectors to 1e-9, residuals to 1e-10 relative (1e-13 sigma_1 absolute for the
    converged ones); with rank > 0 the operator has that rank, the blocks run past it (fresh
    completions, whichever stream draws them) and the r < rank leading triplets are exact."""
    if rank:
        A = synth.gaussian_product(m, n, rank, 0.0, seed=m + s, dtype=np.float64)
    else:
        A = synth.gaussian_product(m, n, min(m, n), 1e-3, seed=m + s, dtype=np.float64)
    Q0 = np.random.default_rng(m + steps).standard_normal((m, s))
    Uo, So, Vo, reso = bgk.block_fsvd(A, Q0, steps, r)
    for fresh_seed in (0, 1):
        U, S, V, res, k = column_block_fsvd(A, Q0, steps, r, fresh_seed)
        assert k == steps
        np.testing.assert_allclose(S, So, rtol=1e-12)
        assert angle_err(U, Uo) < 1e-9 and angle_err(V, Vo) < 1e-9
        np.testing.assert_allclose(res, reso, rtol=1e-10, atol=1e-13 * So[0])
        if rank:
            np.testing.assert_allclose(S, np.linalg.svd(A, compute_uv=False)[:r], rtol=1e-12)
            assert res.max() <= 1e-12 * So[0]


def test_block_fsvd_when_the_blocks_fill_the_space():
    """min(m, n) = 40 columns filled after 5 blocks of 8 (of the 10 asked for): the sweep stops, the
    values are A's (LAPACK), every residual is at rounding level (the next right block lies in
    the filled space), and the oracle agrees."""
    A = np.random.default_rng(3).standard_normal((60, 40))
    Q0 = np.random.default_rng(4).standard_normal((60, 8))
    U, S, V, res, k = column_block_fsvd(A, Q0, 10, 40)
    assert k == 5
    np.testing.assert_allclose(S, np.linalg.svd(A, compute_uv=False), rtol=1e-12)
    assert res.max() <= 1e-12 * S[0]
    np.testing.assert_allclose(A @ V, U * S, rtol=0, atol=1e-12 * S[0])
    Uo, So, Vo, reso = bgk.block_fsvd(A, Q0, 10, 40)
    np.testing.assert_allclose(S, So, rtol=1e-12)
    assert reso.max() <= 1e-12 * S[0]


@pytest.mark.parametrize("m,n,s", [(20, 30, 4), (21, 20, 4), (30, 20, 4), (24, 24, 8)])
def test_blocks_past_the_left_space_are_zero(m, n, s):
    """When the last left block Q_{k+1} has more columns than R^m has room for (a wide operator, or
    m < (k + 1) s), the fresh completions of its excess columns are zero (NM_FRESH), so their
    entries of S_{k+1} = Q_{k+1}^T (A P_k) are zero and sigma(B) = sigma(A) (LAPACK) once the right
    blocks fill min(m, n); the oracle (Householder QR of the reorthogonalized block) agrees."""
    A = np.random.default_rng(m * n).standard_normal((m, n))
    Q0 = np.random.default_rng(s).standard_normal((m, s))
    r_or, sig_or, k_or = bgk.block_numrank(A, Q0, eps=1e-8)
    for gs in (False, True):  # the column-wise flow and the block Gram-Schmidt
        r, sig, k, _ = column_block_gk(A, Q0, 1e-8, 0, block_gs=gs)
        assert k * s == min(m, n) and r == min(m, n)
        np.testing.assert_allclose(sig, np.linalg.svd(A, compute_uv=False), rtol=1e-12)
        assert (r_or, k_or) == (r, k)
        np.testing.assert_allclose(sig, sig_or[: k * s], rtol=1e-12)


@pytest.mark.parametrize("noise,eps,s", [(1e-12, 1e-14, 4), (1e-12, 1e-14, 8), (1e-11, 1e-13, 8)])
def test_block_gram_schmidt_through_near_breakdowns(noise, eps, s):
    """Past the planted rank the blocks' new directions come from a noise floor 1e-12 or 1e-11 of
    sigma_1: the projections cancel to just above the 2^-46 breakdown test, the hardest case for a
    block Gram-Schmidt; with eps below the floor the sweep runs through them for 12 steps, and the
    block flow gives the oracle's rank and sigma(B) as the column-wise flow does."""
    A = synth.gaussian_product(300, 200, 20, noise, seed=5, dtype=np.float64)
    Q0 = np.random.default_rng(s).standard_normal((300, s))
    r_or, sig_or, k_or = bgk.block_numrank(A, Q0, eps=eps, kmax=12)
    for gs in (False, True):
        r, sig, k, _ = column_block_gk(A, Q0, eps, 12, 0, block_gs=gs)
        assert (r, k) == (r_or, k_or) == (12 * s, 12)
        np.testing.assert_allclose(sig, sig_or[: k * s], rtol=0, atol=1e-13 * sig_or[0])
