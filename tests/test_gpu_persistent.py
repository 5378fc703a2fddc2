"""gk_psvd with GK_FLAG_PERSISTENT on a small dense device operator: one persistent launch of the
batched solver (one cluster) instead of the multi-kernel sweep.  Same method, so the results meet
the FP64 path's bounds against the oracle (sigma 1e-10 relative, vectors 1e-8) and agree with the
multi-kernel path to the same bounds; the launch count drops from hundreds to a few."""
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


@pytest.mark.parametrize("m,n,k,K", [(2000, 1000, 10, 30), (1501, 999, 6, 20), (700, 2048, 8, 24)])
def test_persistent_f64_matches_oracle_and_multi_kernel_path(m, n, k, K):
    sig = synth.sigma_geometric(min(m, n), 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=m + n, dtype=np.float64)
    q1 = synth.start_vector(m, k)
    M = gk()
    U1, S1, V1, st1, i1 = M.gk_psvd(cuda(A), k, 1e-10, krylov_dim=K, start=cuda(q1), persistent=True)
    U2, S2, V2, st2, i2 = M.gk_psvd(cuda(A), k, 1e-10, krylov_dim=K, start=cuda(q1))
    assert st1 == st2 == 0
    assert i1["launches"] < 20 < i2["launches"], (i1["launches"], i2["launches"])
    Uo, So, Vo, io = oracle.psvd(oracle.Operator.dense(A), k, K, q1, tol=1e-12, max_restarts=500)
    for U, S, V in ((U1, S1, V1), (U2, S2, V2)):
        np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-10)
        assert angle_err(V.cpu().numpy(), Vo) < 1e-8
        assert angle_err(U.cpu().numpy(), Uo) < 1e-8
    # the same sign convention on both paths
    np.testing.assert_allclose(V1.cpu().numpy(), V2.cpu().numpy(), atol=1e-8)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_persistent_reduced_storage_agrees_with_multi_kernel_path(dtype):
    m, n, k = 3000, 1200, 12
    sig = synth.sigma_power(n, 1.5)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=5, dtype=np.float64)
    A32 = np.asarray(A, dtype=np.float32)
    At = cuda(A32) if dtype == "f32" else cuda(synth.to_bf16_bits(A32).view(np.int16)).view(torch.bfloat16)
    q1 = cuda(synth.start_vector(m, 5))
    M = gk()
    U1, S1, V1, st1, i1 = M.gk_psvd(At, k, 1e-8, start=q1, persistent=True)
    U2, S2, V2, st2, i2 = M.gk_psvd(At, k, 1e-8, start=q1)
    assert st1 == st2 == 0 and i1["launches"] < i2["launches"]
    np.testing.assert_allclose(S1.cpu().numpy(), S2.cpu().numpy(), rtol=1e-7)
    assert angle_err(V1.cpu().numpy(), V2.cpu().numpy()) < 1e-5


def test_persistent_rank_deficient_status():
    g = np.random.default_rng(9)
    A = g.standard_normal((800, 3)) @ g.standard_normal((3, 500))
    q1 = cuda(synth.start_vector(800, 9))
    M = gk()
    U1, S1, V1, st1, i1 = M.gk_psvd(cuda(A), 5, 1e-10, krylov_dim=20, start=q1, persistent=True)
    U2, S2, V2, st2, i2 = M.gk_psvd(cuda(A), 5, 1e-10, krylov_dim=20, start=q1)
    sv = np.linalg.svd(A, compute_uv=False)[:3]
    np.testing.assert_allclose(S1.cpu().numpy()[:3], sv, rtol=1e-10)
    np.testing.assert_allclose(S2.cpu().numpy()[:3], sv, rtol=1e-10)
    assert np.all(np.abs(S1.cpu().numpy()[3:]) <= 1e-10 * sv[0])


def test_host_outputs_take_the_multi_kernel_path_even_when_asked():
    sig = synth.sigma_geometric(500, 0.9)
    A, _, _ = synth.prescribed_spectrum(1000, 500, sig, seed=3, dtype=np.float64)
    M = gk()
    U = torch.empty(5, 1000, dtype=torch.float64).pin_memory()
    S = torch.empty(5, dtype=torch.float64).pin_memory()
    V = torch.empty(5, 500, dtype=torch.float64).pin_memory()
    _, S1, _, st, info = M.gk_psvd(cuda(A), 5, 1e-10, krylov_dim=20, out=(U, S, V), persistent=True)
    assert st == 0 and info["launches"] > 20
    np.testing.assert_allclose(S1.numpy(), sig[:5], rtol=1e-10)
