"""Full-size checks, in the launch configuration the benchmark uses, on outputs the oracle
can verify one by one (or on properties that hold at any size):

  * dense f32 50000 x 20000 rank-200 product: the rank estimate equals the oracle's,
    computed by the oracle on the same stored bytes.
  * dense bf16 100000 x 40000, sigma_i = i^-1.5, top 100 at tol 1e-8: sampled triplets
    have true residuals (f64, on the stored bf16 operator, computed by the oracle) within
    the tolerance, and every singular value is within the Weyl bound ||E||_F of the
    prescribed one (E = the bf16 rounding of the f32-generated operator).
  * CSR 1e6 x 5e5 with 20 entries per row and a planted rank-50 part, top 50 at tol 1e-8:
    sampled true residuals from the oracle.
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


def _oracle_residual(op, U, S, V, i):
    u = U[:, i].cpu().numpy()
    v = V[:, i].cpu().numpy()
    s = float(S[i])
    r1 = np.linalg.norm(op.matvec(v) - s * u)
    r2 = np.linalg.norm(op.rmatvec(u) - s * v)
    return r1, r2


def test_fullsize_numrank_dense_f32_rank200():
    w = synth.WORKLOADS["dense_f32_50000x20000_rank200"]
    A = synth.torch_gaussian_product(w["m"], w["n"], w["r"], w["noise"], w["seed"])
    q1 = synth.start_vector(w["m"], w["seed"])
    r, sig, st, info = gk().gk_numrank(A, w["eps"], 512, start=torch.from_numpy(q1).cuda(), want_sigma=True)
    assert st == 0 and r == w["r"]
    op = oracle.Operator.dense(A.cpu().numpy())
    oracle.set_threads(0)
    r_or, kp_or, sig_or = oracle.numrank(op, q1, eps=w["eps"], kmax=512)
    assert r == r_or
    np.testing.assert_allclose(sig.cpu().numpy()[: w["r"]], sig_or[: w["r"]], rtol=1e-6)


def test_fullsize_psvd_dense_bf16_top100():
    w = synth.WORKLOADS["dense_bf16_100000x40000_top100"]
    sig = synth.sigma_power(w["n"], w["e"])
    A32, _, _ = synth.torch_prescribed_spectrum(w["m"], w["n"], sig, w["seed"])
    A = A32.to(torch.bfloat16)
    # Weyl: |sigma_i(A_bf16) - sigma_i(A_f32)| <= ||A_bf16 - A_f32||_2 <= ||.||_F
    ef = 0.0
    for i in range(0, w["m"], 8192):
        ef += float(((A[i:i + 8192].float() - A32[i:i + 8192]).double() ** 2).sum())
    ef = ef ** 0.5
    del A32
    torch.cuda.empty_cache()
    U, S, V, st, info = gk().gk_psvd(A, w["k"], w["tol"], krylov_dim=w["K"], seed=w["seed"])
    assert st == 0 and info["resid_est_max"] <= w["tol"]
    s = S.cpu().numpy()
    assert np.all(np.abs(s - sig[: w["k"]]) <= ef + 1e-5 * sig[: w["k"]])
    bits = A.view(torch.int16).cpu().numpy().view(np.uint16)
    op = oracle.Operator.dense(None, dtype="bf16", bits=bits)
    oracle.set_threads(0)
    for i in (0, 49, 99):
        r1, r2 = _oracle_residual(op, U, S, V, i)
        # the f32-accumulated products leave a floor of ~2^-24 ||A||_F / sqrt(n) * c below 1e-9
        assert max(r1, r2) <= 1.2 * w["tol"] * s[0], (i, r1, r2)


def test_fullsize_psvd_csr_top50():
    w = synth.WORKLOADS["csr_f32_1000000x500000_top50"]
    sigp = 100.0 * 0.95 ** np.arange(1, w["k"] + 1)
    d = synth.sparse_planted(w["m"], w["n"], w["per_row"], sigp, w["seed"])
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    M = gk()
    A = M.CSR(w["m"], w["n"], c(d["rowptr"]), c(d["colind"]), c(d["vals"]), c(d["t_rowptr"]), c(d["t_colind"]),
              c(d["t_vals"]))
    U, S, V, st, info = M.gk_psvd(A, w["k"], w["tol"], krylov_dim=w["K"], seed=w["seed"])
    assert st == 0
    op = oracle.Operator.csr(w["m"], w["n"], d["rowptr"], d["colind"], d["vals"], "f32")
    s = S.cpu().numpy()
    for i in (0, 24, 49):
        r1, r2 = _oracle_residual(op, U, S, V, i)
        assert max(r1, r2) <= 1.2 * w["tol"] * s[0], (i, r1, r2)
    # the planted part dominates the top of the spectrum: sigma_1 is close to 100 * 0.95
    assert abs(s[0] - sigp[0]) < 0.05 * sigp[0]
