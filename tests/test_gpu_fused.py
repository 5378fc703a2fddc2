"""The fused sweep (one pass over A from HBM per bidiagonalization step: w = A v - beta u and
A^T w from the same rows, the second read from L2; the right step takes A^T w / alpha for
A^T u) against the oracle's restatement of the same ordering (oracle: fused=True), through the
C ABI.

Shapes span the cluster sizes the kernel picks (column pieces of up to 1280 16-byte vectors
per CTA, the last CTA's piece short and threads with a partial fifth vector), ragged row
counts (the last batch of 4 rows short), clusters that own no batch (m < 4 x clusters), and
enough rows that every cluster wraps its 8 exchange generations many times.  Tolerances are
those of the two-pass path (tests/test_gpu_parity.py): the fused kernel's sums are f32 over
at most 40 products per thread (a warp tree after them, double-f32 across warps and CTAs) or
64 rows (A^T w), combined in f64, within 2^-24 (64 + 2) sum |a x| of the exact products like
the two-pass kernels."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

U32 = 2.0**-24


def gk():
    import paper_2104_10785_gb300 as m

    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def stored(A, dtype):
    """(oracle operator on the stored bytes, device tensor, f64 values)."""
    if dtype == "f32":
        A32 = np.asarray(A, dtype=np.float32)
        return oracle.Operator.dense(A32), cuda(A32), A32.astype(np.float64)
    if dtype == "bf16":
        bits = synth.to_bf16_bits(np.asarray(A, dtype=np.float32))
        return (oracle.Operator.dense(None, dtype="bf16", bits=bits), cuda(bits.view(np.int16)).view(torch.bfloat16),
                synth.bf16_bits_to_f32(bits).astype(np.float64))
    h = np.asarray(A, dtype=np.float16)
    return oracle.Operator.dense(None, dtype="f16", bits=h.view(np.uint16)), cuda(h), h.astype(np.float64)


def angle_err(X, Y):
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return np.linalg.norm(X - Y * s[None, :], axis=0).max()


@pytest.mark.parametrize("dtype,m,n", [("bf16", 3001, 1496), ("f32", 2999, 1500), ("f16", 2003, 1024),
                                       ("bf16", 20011, 2048), ("bf16", 1203, 40000), ("f32", 1001, 20000),
                                       ("bf16", 9, 8000), ("bf16", 700, 8)])
def test_fused_psvd_matches_fused_oracle(dtype, m, n):
    k = min(8, min(m, n) - 1)
    K = min(max(2 * k, k + 12), min(m, n))
    sig = synth.sigma_power(min(m, n), 1.5)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=m + n, dtype=np.float64)
    op, At, A64 = stored(A, dtype)
    q1 = synth.start_vector(m, m)
    U, S, V, st, info = gk().gk_psvd(At, k, 1e-8, krylov_dim=K, start=cuda(q1), max_restarts=300, fused=True)
    assert st == 0, info
    assert info["reserved"] >= 1  # the fused kernel ran (its cluster size)
    Uo, So, Vo, io = oracle.psvd(op, k, K, q1, tol=1e-12, max_restarts=500, fused=True)
    assert io["converged"]
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    nf = np.linalg.norm(A64)
    floor = 64 * U32 * nf / np.sqrt(n)
    gaps = np.abs(np.diff(sig[: k + 1])).min()  # prescribed gaps (bf16 rounding moves them by < 1e-4)
    np.testing.assert_allclose(S, So, rtol=1e-7, atol=10 * floor)
    assert angle_err(V, Vo) <= max(1e-6, 10 * (1e-8 * So[0] + floor) / gaps)
    r1, r2 = oracle.residuals(op, U, S, V)
    assert max(r1.max(), r2.max()) <= 1e-8 * So[0] + 10 * floor


@pytest.mark.parametrize("dtype,m,n,r,eps", [("f32", 5000, 2000, 120, 1e-5), ("f32", 1999, 4000, 60, 1e-5),
                                             ("bf16", 3000, 1000, 40, 1e-2)])
def test_fused_numrank_matches_fused_oracle(dtype, m, n, r, eps):
    A = synth.gaussian_product(m, n, r, 1e-7, seed=200 + r, dtype=np.float64)
    op, At, _ = stored(A, dtype)
    q1 = synth.start_vector(m, 9)
    rk, sig, st, info = gk().gk_numrank(At, eps, min(m, n, 400), start=cuda(q1), want_sigma=True, fused=True)
    assert st == 0 and info["reserved"] >= 1
    r_or, kp_or, sig_or = oracle.numrank(op, q1, eps=eps, kmax=min(m, n, 400), fused=True)
    assert rk == r_or == r
    np.testing.assert_allclose(sig.cpu().numpy()[:r], sig_or[:r], rtol=2e-6)
    assert abs(info["kprime"] - kp_or) <= 8


def test_fused_and_two_pass_paths_agree():
    """The same operator through the fused sweep (GK_FLAG_FUSED) and through two passes per step:
    the same triplets, the rank and the Algorithm 2 triplets, within the f32 product bounds."""
    M = gk()
    m, n, k, K = 6007, 2048, 10, 36
    sig = synth.sigma_power(n, 1.5)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=5, dtype=np.float64)
    op, At, A64 = stored(A, "bf16")
    q1 = cuda(synth.start_vector(m, 5))
    Uf, Sf, Vf, st1, i1 = M.gk_psvd(At, k, 1e-8, krylov_dim=K, start=q1, fused=True)
    Uu, Su, Vu, st2, i2 = M.gk_psvd(At, k, 1e-8, krylov_dim=K, start=q1)
    assert st1 == st2 == 0 and i1["reserved"] >= 1 and i2["reserved"] == 0
    np.testing.assert_allclose(Sf.cpu().numpy(), Su.cpu().numpy(), rtol=1e-7)
    assert angle_err(Vf.cpu().numpy(), Vu.cpu().numpy()) < 1e-5
    # the fused sweep is as accurate as the two passes: its FP64 true residuals (oracle) stay
    # within twice the two-pass ones (a summation that rounds the row totals to f32 several
    # times would show here as a several-fold larger residual)
    rf = np.maximum(*oracle.residuals(op, Uf.cpu().numpy(), Sf.cpu().numpy(), Vf.cpu().numpy())).max()
    ru = np.maximum(*oracle.residuals(op, Uu.cpu().numpy(), Su.cpu().numpy(), Vu.cpu().numpy())).max()
    assert rf <= 2 * ru + 1e-10 * float(Su[0]), (rf, ru)
    G = synth.gaussian_product(m, n, 70, 1e-7, seed=6, dtype=np.float32)
    Gt = cuda(G)
    r1, _, _, j1 = M.gk_numrank(Gt, 1e-5, 300, start=q1, fused=True)
    r2, _, _, j2 = M.gk_numrank(Gt, 1e-5, 300, start=q1)
    assert r1 == r2 == 70 and j1["reserved"] >= 1 and j2["reserved"] == 0
    U1, S1, V1, s1, f1 = M.gk_fsvd(At, 40, k, start=q1, fused=True)
    U2, S2, V2, s2, f2 = M.gk_fsvd(At, 40, k, start=q1)
    assert s1 == s2 == 0 and f1["reserved"] >= 1 and f2["reserved"] == 0
    np.testing.assert_allclose(S1.cpu().numpy(), S2.cpu().numpy(), rtol=1e-7)


def test_fused_fsvd_matches_fused_oracle():
    m, n, k, r = 4001, 1200, 60, 12
    sig = synth.sigma_geometric(n, 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=71, dtype=np.float64)
    op, At, A64 = stored(A, "f32")
    q1 = synth.start_vector(m, 71)
    U, S, V, st, info = gk().gk_fsvd(At, k, r, route=1, start=cuda(q1), fused=True)
    assert st == 0 and info["reserved"] >= 1
    Uo, So, Vo, kp = oracle.fsvd(op, k, r, q1, route=1, fused=True)
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-7)
    assert angle_err(V.cpu().numpy(), Vo) < 1e-5


def test_fused_rows_not_multiple_of_16_bytes_take_two_passes():
    """n * element size not a multiple of 16 bytes (bf16 n = 1501): the sweep runs two passes."""
    sig = synth.sigma_power(1501, 1.5)
    A, _, _ = synth.prescribed_spectrum(2000, 1501, sig, seed=3, dtype=np.float64)
    op, At, _ = stored(A, "bf16")
    U, S, V, st, info = gk().gk_psvd(At, 6, 1e-8, krylov_dim=24, start=cuda(synth.start_vector(2000, 3)),
                                     fused=True)
    assert st == 0 and info["reserved"] == 0
