"""Pins of the block Golub-Kahan oracle (oracle/block_gk.py): the block recurrence's relations
(A P = Q B, A^T Q = P B^T on the leading blocks, orthonormal bases), LAPACK's singular values
when the blocks fill the space, the single-vector oracle of Algorithm 1 when s = 1, and the
reason for blocks -- singular values of multiplicity > 1 are counted once by one start vector
and fully by a block of s >= the multiplicity."""
import numpy as np

import oracle
import synth
from oracle import block_gk as bgk


def test_block_relations_and_orthonormal_bases():
    g = np.random.default_rng(1)
    A = g.standard_normal((60, 40))
    Q0 = g.standard_normal((60, 3))
    Q, P, B, steps = bgk.block_gk(A, Q0, 6)
    s = 3
    assert steps == 6 and Q.shape == (60, 21) and P.shape == (40, 18) and B.shape == (21, 18)
    na = np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ P - Q @ B) <= 1e-12 * na
    ks = steps * s
    assert np.linalg.norm(A.T @ Q[:, :ks] - P @ B[:ks, :ks].T) <= 1e-12 * na
    assert np.linalg.norm(Q.T @ Q - np.eye(Q.shape[1])) <= 1e-13
    assert np.linalg.norm(P.T @ P - np.eye(P.shape[1])) <= 1e-13
    # block lower bidiagonal: nothing outside the diagonal and subdiagonal blocks, the
    # diagonal blocks lower triangular (R_j^T), the subdiagonal blocks upper triangular (S_j)
    for i in range(steps + 1):
        for j in range(steps):
            blk = B[i * s:(i + 1) * s, j * s:(j + 1) * s]
            if i == j:
                assert np.allclose(np.triu(blk, 1), 0.0)
            elif i == j + 1:
                assert np.allclose(np.tril(blk, -1), 0.0)
            else:
                assert np.all(blk == 0.0)


def test_blocks_filling_the_space_give_lapack_singular_values():
    g = np.random.default_rng(2)
    A = g.standard_normal((30, 20))
    Q, P, B, steps = bgk.block_gk(A, g.standard_normal((30, 2)), 10)
    assert steps * 2 == 20
    np.testing.assert_allclose(np.linalg.svd(B, compute_uv=False)[:20], np.linalg.svd(A, compute_uv=False),
                               rtol=1e-12)


def test_single_vector_block_is_algorithm_1():
    """s = 1 is Algorithm 1: the same bidiagonal as the single-vector oracle (up to signs), so the
    same singular values of B, over the same number of steps."""
    A = synth.gaussian_product(80, 50, 50, 0.0, seed=3, dtype=np.float64)
    q1 = synth.start_vector(80, 3)
    _, sig, steps = bgk.block_numrank(A, q1[:, None], eps=1e-8, kmax=15)
    r_or, kp_or, sig_or = oracle.numrank(oracle.Operator.dense(A), q1, eps=1e-8, kmax=15)
    assert steps == kp_or == 15
    np.testing.assert_allclose(sig[:15], np.sort(sig_or)[::-1][:15], rtol=1e-10)


def test_blocks_count_repeated_singular_values():
    """sigma = (5, 5, 5, 3, 3, 1, 1, 1): rank 8 with three distinct values.  One start vector's
    Krylov space holds one direction per distinct value (3), a block of 3 holds them all (8)."""
    sigma = np.array([5.0, 5.0, 5.0, 3.0, 3.0, 1.0, 1.0, 1.0])
    A, _, _ = synth.prescribed_spectrum(70, 40, sigma, seed=4, dtype=np.float64)
    g = np.random.default_rng(4)
    r1, _, _ = bgk.block_numrank(A, g.standard_normal((70, 1)), eps=1e-8)
    r3, sig3, _ = bgk.block_numrank(A, g.standard_normal((70, 3)), eps=1e-8)
    assert r1 == 3
    assert r3 == 8
    np.testing.assert_allclose(sig3[:8], sigma, rtol=1e-10)
    # Algorithm 1's oracle agrees with the single-vector count
    r_or, _, _ = oracle.numrank(oracle.Operator.dense(A), synth.start_vector(70, 4), eps=1e-8)
    assert r_or == 3


def test_block_rank_of_a_planted_product():
    A = synth.gaussian_product(300, 200, 20, 1e-9, seed=5, dtype=np.float64)
    r, sig, steps = bgk.block_numrank(A, np.random.default_rng(5).standard_normal((300, 4)), eps=1e-6)
    assert r == 20


def test_recurrence_terms_without_reorthogonalization():
    """With no reorthogonalization the recurrence's own terms (-Q_j R_j^T, -P_j S_{j+1}^T) carry the
    orthogonality: over a few steps the relations and the bases hold to rounding.  (With full
    reorthogonalization the Gram-Schmidt would remove those components whatever their
    coefficients, so only this form pins them.)"""
    g = np.random.default_rng(6)
    A = g.standard_normal((50, 35))
    Q, P, B, steps = bgk.block_gk(A, g.standard_normal((50, 2)), 4, passes=0)
    na = np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ P - Q @ B) <= 1e-12 * na
    ks = steps * 2
    assert np.linalg.norm(A.T @ Q[:, :ks] - P @ B[:ks, :ks].T) <= 1e-12 * na
    assert np.linalg.norm(Q.T @ Q - np.eye(Q.shape[1])) <= 1e-9
    assert np.linalg.norm(P.T @ P - np.eye(P.shape[1])) <= 1e-9


def test_block_fsvd_relations_and_residuals():
    """block_fsvd: A V = U diag(sigma) exactly (A P = Q B), orthonormal U and V, and the residual
    from the recurrence (||R_{k+1} x_i'||) equal to ||A^T u_i - sigma_i v_i|| computed directly."""
    A = synth.gaussian_product(400, 300, 60, 1e-3, seed=21, dtype=np.float64)
    Q0 = np.random.default_rng(21).standard_normal((400, 4))
    U, S, V, est = bgk.block_fsvd(A, Q0, 10, 12)
    assert U.shape == (400, 12) and V.shape == (300, 12) and np.all(np.diff(S) <= 0)
    assert np.linalg.norm(A @ V - U * S) <= 1e-12 * S[0]
    assert np.linalg.norm(U.T @ U - np.eye(12)) <= 1e-12 and np.linalg.norm(V.T @ V - np.eye(12)) <= 1e-12
    direct = np.linalg.norm(A.T @ U - V * S, axis=0)
    assert est.max() > 1e-6 * S[0]  # not converged: the residuals are real numbers to compare
    np.testing.assert_allclose(est, direct, rtol=1e-8, atol=1e-13 * S[0])


def test_block_fsvd_single_vector_is_algorithm_2():
    """s = 1 is Algorithm 2 (route 1): the same Ritz values and vectors as the single-vector oracle
    after the same number of steps."""
    A = synth.gaussian_product(300, 200, 200, 0.0, seed=22, dtype=np.float64)
    q1 = synth.start_vector(300, 22)
    U, S, V, est = bgk.block_fsvd(A, q1[:, None], 30, 5)
    Uo, So, Vo, kp = oracle.fsvd(oracle.Operator.dense(A), 30, 5, q1, route=1)
    assert kp == 30
    np.testing.assert_allclose(S, So, rtol=1e-10)
    sgn = np.sign(np.sum(V * Vo, axis=0))
    assert np.linalg.norm(V - Vo * sgn, axis=0).max() <= 1e-8
    assert np.linalg.norm(U - Uo * sgn, axis=0).max() <= 1e-8


def test_block_fsvd_full_space_and_multiplicities():
    """Blocks filling the column space give A's SVD with zero residuals; a block of 3 finds the
    triple singular value 5 three times where one start vector finds it once."""
    g = np.random.default_rng(23)
    A = g.standard_normal((30, 20))
    U, S, V, est = bgk.block_fsvd(A, g.standard_normal((30, 2)), 10, 20)
    np.testing.assert_allclose(S, np.linalg.svd(A, compute_uv=False), rtol=1e-12)
    assert est.max() <= 1e-12 * S[0]
    sigma = np.array([5.0, 5.0, 5.0, 3.0, 3.0, 1.0, 1.0, 1.0])
    B8, _, _ = synth.prescribed_spectrum(70, 40, sigma, seed=24, dtype=np.float64)
    _, S3, _, _ = bgk.block_fsvd(B8, g.standard_normal((70, 3)), 3, 3)
    np.testing.assert_allclose(S3, [5.0, 5.0, 5.0], rtol=1e-10)
    # one vector: three steps exhaust its Krylov space (one direction per distinct value)
    _, S1, _, _ = bgk.block_fsvd(B8, g.standard_normal((70, 1)), 3, 3)
    np.testing.assert_allclose(S1, [5.0, 3.0, 1.0], rtol=1e-10)
