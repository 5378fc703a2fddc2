"""F-SVD as printed (Algorithm 2: k steps of Algorithm 1, the SVD of B_{k'+1,k'}, no restart)
through the C ABI, against the oracle's Algorithm 2 on the same stored bytes and start vector.

Both sides build the same Krylov space, so for f64 operators the Ritz values agree to rounding
(1e-10 relative is generous) and the leading Ritz vectors to rounding over their gaps; f32
operators are multiplied in f32 with the vector rounded to f32, a relative perturbation of
order 1e-7 of each product (bounds 1e-6 and 1e-5 below).
"""
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
    """max_i || x_i - sign * y_i || for unit columns (sign-invariant)."""
    X = np.asarray(X)
    Y = np.asarray(Y)
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return np.linalg.norm(X - Y * s[None, :], axis=0).max()


@pytest.mark.parametrize("route", [0, 1])
@pytest.mark.parametrize("shape", [(800, 350), (300, 700)])
def test_fsvd_matches_oracle_f64(route, shape):
    m, n = shape
    sig = synth.sigma_geometric(min(m, n), 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=51)
    q1 = synth.start_vector(m, 51)
    U, S, V, st, info = gk().gk_fsvd(cuda(A), 40, 8, route=route, start=cuda(q1))
    Uo, So, Vo, kp = oracle.fsvd(oracle.Operator.dense(A), 40, 8, q1, route=route)
    assert st == gk().gk.GK_OK and info["kprime"] == kp == 40
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-10)
    assert angle_err(V.cpu().numpy(), Vo) <= 1e-8
    assert angle_err(U.cpu().numpy(), Uo) <= 1e-8
    # the leading Ritz values are the top singular values to the accuracy 40 steps give
    np.testing.assert_allclose(S.cpu().numpy()[:4], sig[:4], rtol=1e-8)


def test_fsvd_f32_storage_and_both_routes():
    m, n = 1200, 500
    sig = synth.sigma_geometric(n, 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=52)
    A32 = A.astype(np.float32)
    q1 = synth.start_vector(m, 52)
    M = gk()
    U1, S1, V1, st1, _ = M.gk_fsvd(cuda(A32), 40, 8, route=1, start=cuda(q1))
    U0, S0, V0, st0, info0 = M.gk_fsvd(cuda(A32), 40, 8, route=0, start=cuda(q1))
    Uo, So, Vo, kp = oracle.fsvd(oracle.Operator.dense(A32), 40, 8, q1, route=1)
    assert st1 == st0 == 0
    np.testing.assert_allclose(S1.cpu().numpy(), So, rtol=1e-6)
    # route 0's sqrt(eig(B^T B)) against route 1's SVD of B: equal up to the squared condition number
    np.testing.assert_allclose(S0.cpu().numpy(), S1.cpu().numpy(), rtol=1e-12)
    Uo0, So0, Vo0, _ = oracle.fsvd(oracle.Operator.dense(A32), 40, 8, q1, route=0)
    np.testing.assert_allclose(S0.cpu().numpy(), So0, rtol=1e-6)
    assert angle_err(V0.cpu().numpy(), Vo0) <= 1e-5
    assert angle_err(U0.cpu().numpy(), Uo0) <= 1e-5
    assert angle_err(V1.cpu().numpy(), Vo) <= 1e-5
    assert angle_err(U1.cpu().numpy(), Uo) <= 1e-5
    # u_i = A v_i / sigma_i equals Q x_i in exact arithmetic (A P Y = Q B Y = Q X Sigma)
    assert angle_err(U0.cpu().numpy(), U1.cpu().numpy()) <= 1e-5
    # the printed route computes one product per triplet on top of the sweep (one blocked pass)
    assert info0["matvecs"] >= 2 * 40 + 8


def test_fsvd_host_outputs_match_device_outputs():
    sig = synth.sigma_geometric(200, 0.8)
    A, _, _ = synth.prescribed_spectrum(500, 200, sig, seed=53)
    q1 = synth.start_vector(500, 53)
    M = gk()
    Ud, Sd, Vd, st, _ = M.gk_fsvd(cuda(A), 30, 5, start=cuda(q1))
    Uh, Sh, Vh, st2, _ = M.gk_fsvd(torch.from_numpy(A), 30, 5, start=torch.from_numpy(q1))
    assert st == st2 == 0
    np.testing.assert_allclose(Sh.numpy(), Sd.cpu().numpy(), rtol=1e-12)
    assert angle_err(Uh.numpy(), Ud.cpu().numpy()) <= 1e-10
    assert angle_err(Vh.numpy(), Vd.cpu().numpy()) <= 1e-10


def test_fsvd_zero_matrix_is_rank_deficient():
    U, S, V, st, info = gk().gk_fsvd(torch.zeros(50, 30, dtype=torch.float64, device="cuda"), 10, 3)
    assert st == gk().gk.GK_RANK_DEFICIENT and info["kprime"] == 0
    assert not S.abs().sum().item() and not U.abs().sum().item() and not V.abs().sum().item()


def test_fsvd_rejects_bad_arguments():
    M = gk()
    A = torch.ones(50, 30, dtype=torch.float64, device="cuda")
    for k, r in ((10, 11), (31, 3), (0, 1), (10, 0)):
        with pytest.raises(M.GKError):
            M.gk_fsvd(A, k, r)
    with pytest.raises(M.GKError):
        M.gk_fsvd(A, 10, 3, route=2)


def test_fsvd_printed_route_bf16_blocked_products():
    """Route 0 on a bf16 operator (the blocked double-f32 pass U = A V_r / Sigma): every u_i against
    the oracle's u_i = A v_i / sigma_i and the true residual A v_i - s_i u_i vanishing to FP64 grade."""
    m, n, k, r = 3001, 1400, 60, 33
    sig = synth.sigma_geometric(n, 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=54)
    bits = synth.to_bf16_bits(A.astype(np.float32))
    op = oracle.Operator.dense(None, dtype="bf16", bits=bits)
    q1 = synth.start_vector(m, 54)
    U, S, V, st, info = gk().gk_fsvd(cuda(bits.view(np.int16)).view(torch.bfloat16), k, r, route=0, start=cuda(q1))
    Uo, So, Vo, kp = oracle.fsvd(op, k, r, q1, route=0)
    assert st == 0
    S, U, V = S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()
    np.testing.assert_allclose(S[:12], So[:12], rtol=1e-6)
    r1, _ = oracle.residuals(op, U, S, V)
    # A v_i - s_i u_i = 0 by construction; left to the rounding of the blocked products
    assert r1.max() <= 1e-12 * S[0]
