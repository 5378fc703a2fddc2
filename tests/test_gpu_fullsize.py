"""Full-size checks, in the launch configuration the benchmark uses, on outputs the oracle
can verify one by one (or on properties that hold at any size):

  * dense f32 50000 x 20000 rank-200 product: the rank estimate equals the oracle's,
    computed by the oracle on the same stored bytes.
  * dense bf16 100000 x 40000, sigma_i = i^-1.5, top 100 at tol 1e-8, in the benchmark's
    launch configuration: all 100 triplets against the oracle's complete solve of the same
    stored bytes (values, vectors, FP64 true residuals), and the values within the Weyl bound
    ||E||_F of the prescribed ones (E = the bf16 rounding of the f32-generated operator).
  * CSR 1e6 x 5e5 with 20 entries per row and a planted rank-50 part, top 50 at tol 1e-8:
    all 50 triplets against the oracle's complete solve.
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


def _angles(X, Y):
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return np.linalg.norm(X - Y * s[None, :], axis=0)


def test_fullsize_psvd_dense_bf16_top100_against_complete_oracle_solve():
    """The benchmark's configuration: bf16 100000 x 40000 (sigma_i = i^-1.5), top 100 at tol 1e-8,
    Krylov dimension from the committed network, start vector drawn on the device from the
    workload seed.  The oracle runs its own complete solve (FP64, same K, its own Philox draw of
    the same q1) on the stored bf16 bytes.  Checked for every one of the 100 triplets:
      * sigma_i against the oracle's to 1e-7 relative;
      * the true residual max(||A v - s u||, ||A^T u - s v||), computed by the oracle in FP64 on
        the stored operator, at most tol * sigma_1 (no slack);
      * u_i, v_i against the oracle's within 2 (r_gpu + r_oracle) / gap_i (gap_i from the
        prescribed spectrum, which the bf16 rounding moves by far less than the gaps);
      * sigma_i within the Weyl bound ||E||_F of the prescribed i^-1.5 (E = the bf16 rounding)."""
    from paper_2104_10785_gb300 import predictor

    w = synth.WORKLOADS["dense_bf16_100000x40000_top100"]
    m, n, k, tol = w["m"], w["n"], w["k"], w["tol"]
    sig = synth.sigma_power(n, w["e"])
    A32, _, _ = synth.torch_prescribed_spectrum(m, n, sig, w["seed"])
    A = A32.to(torch.bfloat16)
    ef = 0.0
    for i in range(0, m, 8192):
        ef += float(((A[i:i + 8192].float() - A32[i:i + 8192]).double() ** 2).sum())
    ef = ef ** 0.5
    del A32
    torch.cuda.empty_cache()
    kparams = predictor.load(path=predictor.KRYLOV_PARAMS_FILE)
    assert kparams is not None
    U, S, V, st, info = predictor.learned_psvd(A, kparams, k, tol, seed=w["seed"])
    K = info["krylov_dim"]
    assert st == 0 and info["resid_est_max"] <= tol
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    bits = A.view(torch.int16).cpu().numpy().view(np.uint16)
    del A
    torch.cuda.empty_cache()
    op = oracle.Operator.dense(None, dtype="bf16", bits=bits)
    oracle.set_threads(0)
    q1 = oracle.start_vector(w["seed"], m)
    Uo, So, Vo, io = oracle.psvd(op, k, K, q1, tol=tol, max_restarts=50)
    assert io["converged"]
    np.testing.assert_allclose(S, So, rtol=1e-7)
    r1, r2 = oracle.residuals(op, U, S, V)
    res = np.maximum(r1, r2)
    assert res.max() <= tol * So[0], (res.max() / So[0], int(res.argmax()))
    sp = sig[: k + 1]
    gaps = np.array([min(sp[i - 1] - sp[i] if i > 0 else np.inf, sp[i] - sp[i + 1]) for i in range(k)])
    bound = 2 * (res + tol * So[0]) / gaps
    assert np.all(_angles(V, Vo) <= bound) and np.all(_angles(U, Uo) <= bound)
    assert np.all(np.abs(S - sig[:k]) <= ef + 1e-5 * sig[:k])


def test_fullsize_psvd_csr_top50_against_complete_oracle_solve():
    """CSR 1e6 x 5e5 (20 entries per row and the planted rank-50 part), top 50 at tol 1e-8, K = 100,
    start vector drawn on the device from the workload seed; the oracle's complete solve on the
    same CSR arrays.  All 50 singular values to 1e-8 relative, all 50 true residuals (FP64, oracle)
    at most tol * sigma_1, and the vectors of the triplets whose gap to the neighbouring oracle
    values is at least 1e-3 sigma_1 within 2 (r_gpu + r_oracle) / gap (the top of the spectrum
    meets the random bulk near i = 43, where the gaps close)."""
    w = synth.WORKLOADS["csr_f32_1000000x500000_top50"]
    m, n, k, K, tol = w["m"], w["n"], w["k"], w["K"], w["tol"]
    sigp = 100.0 * 0.95 ** np.arange(1, k + 1)
    d = synth.sparse_planted(m, n, w["per_row"], sigp, w["seed"])
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    M = gk()
    A = M.CSR(m, n, c(d["rowptr"]), c(d["colind"]), c(d["vals"]), c(d["t_rowptr"]), c(d["t_colind"]), c(d["t_vals"]))
    U, S, V, st, info = M.gk_psvd(A, k, tol, krylov_dim=K, seed=w["seed"])
    assert st == 0
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    op = oracle.Operator.csr(m, n, d["rowptr"], d["colind"], d["vals"], "f32")
    oracle.set_threads(0)
    Uo, So, Vo, io = oracle.psvd(op, k, K, oracle.start_vector(w["seed"], m), tol=tol, max_restarts=400)
    assert io["converged"]
    np.testing.assert_allclose(S, So, rtol=1e-8)
    r1, r2 = oracle.residuals(op, U, S, V)
    res = np.maximum(r1, r2)
    assert res.max() <= tol * So[0], (res.max() / So[0], int(res.argmax()))
    gaps = np.array([min(So[i - 1] - So[i] if i > 0 else np.inf, So[i] - So[i + 1] if i + 1 < k else np.inf)
                     for i in range(k)])
    sel = gaps >= 1e-3 * So[0]
    assert sel.sum() >= 30
    bound = 2 * (res + tol * So[0]) / gaps
    assert np.all((_angles(V, Vo) <= bound)[sel]) and np.all((_angles(U, Uo) <= bound)[sel])
    # the planted part dominates the top of the spectrum: sigma_1 is close to 100 * 0.95
    assert abs(S[0] - sigp[0]) < 0.05 * sigp[0]
