"""Gram-Schmidt on the bases' double-f32 copies (the default for vectors past the one-CTA
size) against the f64 kernels (GK_FLAG_ORTH_F64) and the oracle.

The double-f32 products carry ~2^-46 of |q w| per term (TwoProd of the high words, both cross
terms, TwoSum accumulation), so the coefficients h = Q^T w agree with f64 ones to ~1e-14 of
||w||; over a solve the two paths' singular values agree to ~1e-13 relative on an f64
operator, far inside the FP64 path's 1e-10 bound against the oracle.  The shapes have odd
lengths (the last row of a column pairs with a padding row of the copy), thick restarts (the
kept columns are copied again), an exact breakdown (replacement directions written through
the copy), every reorthogonalization rule, the rank estimate and Algorithm 2."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def gk():
    import paper_2104_10785_gb300 as m

    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def angle_err(X, Y):
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return np.linalg.norm(X - Y * s[None, :], axis=0).max()


@pytest.mark.parametrize("m,n,k,K,passes", [(20011, 501, 10, 30, 0), (611, 16385, 8, 24, 1),
                                            (30001, 401, 12, 40, 2), (16385, 903, 6, 20, 3)])
def test_psvd_df_orth_matches_f64_orth_and_oracle(m, n, k, K, passes):
    """f64 operator, small Krylov dimension: several restarts, so the kept columns' copies are
    rebuilt; each rule against the f64 kernels (1e-12) and the oracle (the FP64 bounds).  One
    side is past the one-CTA size (its basis takes the double-f32 kernels), the other not."""
    sig = synth.sigma_geometric(min(m, n), 0.98)  # slow decay: 2-4 restarts at these K
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=m + passes, dtype=np.float64)
    At = cuda(A)
    q1 = synth.start_vector(m, k)
    M = gk()
    U1, S1, V1, st1, i1 = M.gk_psvd(At, k, 1e-10, krylov_dim=K, start=cuda(q1), reorth_passes=passes,
                                    max_restarts=300)
    U2, S2, V2, st2, i2 = M.gk_psvd(At, k, 1e-10, krylov_dim=K, start=cuda(q1), reorth_passes=passes,
                                    max_restarts=300, orth_f64=True)
    assert st1 == st2 == 0 and i1["restarts"] >= 1
    np.testing.assert_allclose(S1.cpu().numpy(), S2.cpu().numpy(), rtol=1e-12)
    assert angle_err(V1.cpu().numpy(), V2.cpu().numpy()) < 1e-9
    op = oracle.Operator.dense(A)
    Uo, So, Vo, io = oracle.psvd(op, k, K, q1, tol=1e-12, max_restarts=500, passes=passes)
    np.testing.assert_allclose(S1.cpu().numpy(), So, rtol=1e-10)
    assert angle_err(V1.cpu().numpy(), Vo) < 1e-8
    assert angle_err(U1.cpu().numpy(), Uo) < 1e-8


def test_psvd_df_orth_bf16_operator_residuals():
    """bf16 operator (the benchmark's storage): the true residuals stay at the f64 path's level."""
    m, n, k = 20001, 4001, 16
    sig = synth.sigma_power(n, 1.5)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=4, dtype=np.float64)
    bits = synth.to_bf16_bits(np.asarray(A, dtype=np.float32))
    At = cuda(bits.view(np.int16)).view(torch.bfloat16)
    op = oracle.Operator.dense(None, dtype="bf16", bits=bits)
    q1 = cuda(synth.start_vector(m, 4))
    M = gk()
    res = []
    for f64 in (False, True):
        U, S, V, st, info = M.gk_psvd(At, k, 1e-8, krylov_dim=44, start=q1, orth_f64=f64)
        assert st == 0
        r1, r2 = oracle.residuals(op, U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy())
        res.append(max(r1.max(), r2.max()) / float(S[0]))
    assert res[0] <= 1e-8 and res[0] <= 1.5 * res[1] + 1e-10, res


def test_psvd_df_orth_breakdown_replacement_directions():
    """Rank 5 with k = 8: exact breakdowns; the replacement directions are orthogonalized against
    the copies and written through them.  Same triplets as the f64 kernels."""
    m, n, r, k = 12001, 700, 5, 8
    g = np.random.default_rng(7)
    L = g.standard_normal((m, r)) * np.array([5.0, 4.0, 3.0, 2.0, 1.0])
    R = g.standard_normal((r, n)) / np.sqrt(n)
    A = L @ R
    At = cuda(A)
    q1 = cuda(synth.start_vector(m, 7))
    M = gk()
    U1, S1, V1, st1, i1 = M.gk_psvd(At, k, 1e-10, krylov_dim=20, start=q1)
    U2, S2, V2, st2, i2 = M.gk_psvd(At, k, 1e-10, krylov_dim=20, start=q1, orth_f64=True)
    assert i1["breakdowns"] >= 1 and i2["breakdowns"] >= 1
    s1, s2 = S1.cpu().numpy(), S2.cpu().numpy()
    np.testing.assert_allclose(s1[:r], s2[:r], rtol=1e-12)
    # A = Q1 (R1 R2^T) Q2^T with L = Q1 R1, R^T = Q2 R2: the singular values of the r x r core
    sv = np.linalg.svd(np.linalg.qr(L)[1] @ np.linalg.qr(R.T)[1].T, compute_uv=False)
    np.testing.assert_allclose(s1[:r], sv[:r], rtol=1e-10)
    assert np.all(np.abs(s1[r:]) <= 1e-10 * s1[0])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_numrank_df_orth_matches_f64_orth_and_oracle(dtype):
    m, n, r = 20001, 1200, 150
    A = synth.gaussian_product(m, n, r, 1e-7, seed=r, dtype=np.float64 if dtype == "f64" else np.float32)
    At = cuda(A)
    q1 = synth.start_vector(m, 3)
    M = gk()
    r1, s1, st1, i1 = M.gk_numrank(At, 1e-5, 400, start=cuda(q1), want_sigma=True)
    r2, s2, st2, i2 = M.gk_numrank(At, 1e-5, 400, start=cuda(q1), want_sigma=True, orth_f64=True)
    assert r1 == r2 == r and i1["kprime"] == i2["kprime"]
    # f64 operator: the two paths differ only by the Gram-Schmidt rounding (~1e-14); f32
    # operator: the products take v rounded to f32, and vectors that differ by ~1e-14 round
    # differently in a few entries, so the two runs agree to the f32 products' precision
    np.testing.assert_allclose(s1.cpu().numpy()[:r], s2.cpu().numpy()[:r], rtol=1e-11 if dtype == "f64" else 1e-6)
    op = oracle.Operator.dense(np.asarray(A, dtype=np.float64) if dtype == "f64" else np.asarray(A))
    r_or, kp_or, sig_or = oracle.numrank(op, q1, eps=1e-5, kmax=400)
    assert r_or == r1


def test_fsvd_df_orth_matches_oracle():
    m, n, k, r = 16001, 800, 40, 10
    sig = synth.sigma_geometric(n, 0.85)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=12, dtype=np.float64)
    q1 = synth.start_vector(m, 12)
    U, S, V, st, info = gk().gk_fsvd(cuda(A), k, r, route=1, start=cuda(q1))
    assert st == 0
    Uo, So, Vo, kp = oracle.fsvd(oracle.Operator.dense(A), k, r, q1, route=1)
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-10)
    assert angle_err(V.cpu().numpy(), Vo) < 1e-8
