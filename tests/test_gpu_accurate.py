"""FP64-grade true residuals (gk_residuals on f32/bf16/f16 operators: double-f32 products of
all k vectors per pass) against the oracle's FP64 residuals, and the refinement loop of
gk_psvd (GK_FLAG_REFINE).

Bound: every output of the double-f32 products is exact to about 2^-47 sum_j |a_ij x_j|
(TwoProd and TwoSum keep each rounding error; the vectors are split into two f32 parts exact
to 2^-48), so a residual norm over m rows agrees with the FP64 one to ~1e-14 sigma_1; the
tests allow 1e-12 sigma_1.  The sweep's own f32-accumulated products (the old check) sit at
~2^-24 sum |a x| instead, a floor near 1e-9 sigma_1."""
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


def stored(A, dtype):
    if dtype == "f32":
        A32 = np.asarray(A, dtype=np.float32)
        return oracle.Operator.dense(A32), cuda(A32)
    if dtype == "bf16":
        bits = synth.to_bf16_bits(np.asarray(A, dtype=np.float32))
        return oracle.Operator.dense(None, dtype="bf16", bits=bits), cuda(bits.view(np.int16)).view(torch.bfloat16)
    h = np.asarray(A, dtype=np.float16)
    return oracle.Operator.dense(None, dtype="f16", bits=h.view(np.uint16)), cuda(h)


@pytest.mark.parametrize("dtype,m,n,k", [("bf16", 3001, 1499, 37), ("f32", 1029, 2111, 33), ("f16", 517, 130, 5),
                                         ("bf16", 20011, 2048, 64)])
def test_accurate_residuals_of_converged_triplets_match_oracle(dtype, m, n, k):
    """Converged triplets (residuals ~1e-9 sigma_1 or below): the GPU's residuals agree with the
    oracle's FP64 residuals to 1e-12 sigma_1 -- tiles of 128 outputs x 32 vectors with ragged edges
    in both directions."""
    sig = synth.sigma_power(min(m, n), 1.5)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=m + k, dtype=np.float64)
    op, At = stored(A, dtype)
    q1 = synth.start_vector(m, k)
    U, S, V, st, info = gk().gk_psvd(At, k, 1e-10, krylov_dim=min(2 * k + 10, min(m, n)), start=cuda(q1),
                                     max_restarts=300)
    r1, r2 = gk().gk_residuals(At, U, S, V)
    o1, o2 = oracle.residuals(op, U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy())
    s1 = float(S[0])
    assert np.all(np.abs(r1.cpu().numpy() - o1) <= 1e-12 * s1), np.abs(r1.cpu().numpy() - o1).max() / s1
    assert np.all(np.abs(r2.cpu().numpy() - o2) <= 1e-12 * s1), np.abs(r2.cpu().numpy() - o2).max() / s1


def test_accurate_residuals_of_arbitrary_vectors_match_oracle():
    """Arbitrary (unconverged) triplets: residuals of order ||A||, relative agreement 1e-13."""
    g = np.random.default_rng(3)
    m, n, k = 777, 1234, 40
    A = g.standard_normal((m, n))
    op, At = stored(A, "bf16")
    U = g.standard_normal((m, k))
    V = g.standard_normal((n, k))
    S = np.abs(g.standard_normal(k)) * 10
    r1, r2 = gk().gk_residuals(At, cuda(U), cuda(S), cuda(V))
    o1, o2 = oracle.residuals(op, U, S, V)
    np.testing.assert_allclose(r1.cpu().numpy(), o1, rtol=1e-13)
    np.testing.assert_allclose(r2.cpu().numpy(), o2, rtol=1e-13)


def test_refine_accepts_converged_triplets_and_reports_the_true_residual():
    sig = synth.sigma_power(1500, 1.5)
    A, _, _ = synth.prescribed_spectrum(3000, 1500, sig, seed=9, dtype=np.float64)
    op, At = stored(A, "bf16")
    q1 = cuda(synth.start_vector(3000, 9))
    U, S, V, st, info = gk().gk_psvd(At, 12, 1e-8, krylov_dim=40, start=q1, refine=True)
    assert st == 0 and info["refine_checks"] >= 1 and info["ms_refine"] > 0
    o1, o2 = oracle.residuals(op, U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy())
    true_rel = max(o1.max(), o2.max()) / float(S[0])
    assert true_rel <= 1e-8
    assert abs(info["resid_true_max"] - true_rel) <= 1e-12
    # the paper's err_rel from the same check: each residual within 1e-12 sigma_1 of the oracle's,
    # so err_rel within sqrt(k) 1e-12
    err_or = oracle.err_rel(op, U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy())
    assert 0.0 < info["err_rel"] and abs(info["err_rel"] - err_or) <= 1e-11


def test_refine_keeps_restarting_while_the_true_residual_exceeds_tol():
    """tol = 1e-13 on a bf16 operator: the Ritz estimate can reach it, but the f32 products' floor
    (~1e-9 sigma_1) keeps the true residual above it, so each check fails, the Ritz test is tightened
    and the solve restarts until the budget is spent; the status says so and the reported true
    residual is the oracle's."""
    sig = synth.sigma_power(800, 1.5)
    A, _, _ = synth.prescribed_spectrum(2000, 800, sig, seed=10, dtype=np.float64)
    op, At = stored(A, "bf16")
    U, S, V, st, info = gk().gk_psvd(At, 6, 1e-13, krylov_dim=30, start=cuda(synth.start_vector(2000, 10)),
                                     max_restarts=6, refine=True)
    assert st == gk().gk.GK_NOT_CONVERGED
    assert info["refine_checks"] >= 2
    o1, o2 = oracle.residuals(op, U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy())
    true_rel = max(o1.max(), o2.max()) / float(S[0])
    assert true_rel > 1e-13
    assert abs(info["resid_true_max"] - true_rel) <= 1e-12
