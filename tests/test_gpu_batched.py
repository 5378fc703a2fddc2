"""The batched persistent solver against the oracle, problem by problem: a batch of
uneven dense problems (tall, wide, odd sizes, f64/f32/bf16 storage, more problems than
clusters) solved in one launch; every rank equals the oracle's and every partial SVD
matches the oracle's triplets within the tolerances of the single-problem path."""
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


def _problem(i, dtype):
    g = synth.rng(500 + i)
    m = int(g.integers(40, 900))
    n = int(g.integers(20, m + 1)) if i % 5 else int(g.integers(m, 2 * m))  # every fifth one is wide
    r = int(g.integers(3, min(m, n, 30)))
    A = synth.gaussian_product(m, n, r, 1e-7, seed=600 + i, dtype=np.float64)
    return A, r


def _stored(A, dtype):
    if dtype == "f64":
        return oracle.Operator.dense(A), torch.from_numpy(A).cuda(), A
    if dtype == "f32":
        a = A.astype(np.float32)
        return oracle.Operator.dense(a), torch.from_numpy(a).cuda(), a.astype(np.float64)
    bits = synth.to_bf16_bits(A.astype(np.float32))
    t = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    return oracle.Operator.dense(None, dtype="bf16", bits=bits), t, synth.bf16_bits_to_f32(bits).astype(np.float64)


@pytest.mark.parametrize("dtype,eps", [("f64", 1e-6), ("f32", 1e-5), ("bf16", 1e-2)])
def test_batched_numrank_matches_oracle(dtype, eps):
    probs, ops, qs, ranks, kms = [], [], [], [], []
    for i in range(40):
        A, r = _problem(i, dtype)
        op, At, _ = _stored(A, dtype)
        q1 = synth.start_vector(A.shape[0], i)
        km = min(A.shape[0], A.shape[1], 120)
        probs.append(dict(A=At, eps=eps, start=torch.from_numpy(q1).cuda(), kmax=km))
        ops.append(op)
        qs.append(q1)
        ranks.append(r)
        kms.append(km)
    res, st, info = gk().gk_numrank_batched(probs, want_sigma=True)
    assert st == 0
    for i, (rk, sig, r) in enumerate(res):
        r_or, kp_or, sig_or = oracle.numrank(ops[i], qs[i], eps=eps, kmax=kms[i])
        assert rk == r_or, (i, rk, r_or)
        if dtype != "bf16":  # bf16 rounding can push small trailing sigma_r below eps * sigma_1
            assert rk == ranks[i], (i, rk, ranks[i])
        np.testing.assert_allclose(sig.cpu().numpy()[:rk], sig_or[:rk], rtol=2e-6 if dtype != "f64" else 1e-11)


def _angle_err(X, Y):
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return np.linalg.norm(X - Y * s[None, :], axis=0).max()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_batched_psvd_matches_oracle(dtype):
    probs, cases = [], []
    for i in range(24):
        g = synth.rng(900 + i)
        m = int(g.integers(60, 700))
        n = int(g.integers(30, m + 1)) if i % 4 else int(g.integers(m, m + 300))
        sig = 0.9 ** np.arange(1, min(m, n) + 1)
        A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=1000 + i)
        op, At, A64 = _stored(A, dtype)
        k = int(g.integers(1, 9))
        K = min(min(m, n), k + 12)
        q1 = synth.start_vector(m, i)
        probs.append(dict(A=At, k=k, krylov_dim=K, tol=1e-10 if dtype == "f64" else 1e-7,
                          start=torch.from_numpy(q1).cuda()))
        cases.append((op, k, K, q1, A64))
    res, st, info = gk().gk_psvd_batched(probs, max_restarts=300)
    assert st == 0, [r[3] for r in res]
    for i, (U, S, V, rr) in enumerate(res):
        op, k, K, q1, A64 = cases[i]
        Uo, So, Vo, io = oracle.psvd(op, k, K, q1, tol=1e-12, max_restarts=500)
        S = S.cpu().numpy()
        V = V.cpu().numpy()
        U = U.cpu().numpy()
        np.testing.assert_allclose(S, So, rtol=1e-9 if dtype == "f64" else 2e-6)
        assert _angle_err(V, Vo) < (1e-7 if dtype == "f64" else 1e-3), i
        r1, r2 = oracle.residuals(op, U, S, V)
        tol = 1e-10 if dtype == "f64" else 1e-7
        floor = 64 * U32 * np.linalg.norm(A64) / np.sqrt(A64.shape[1]) if dtype != "f64" else 0.0
        assert max(r1.max(), r2.max()) <= (tol + 10 * floor) * So[0] * 1.01, i
        idx = np.argmax(np.abs(V), axis=0)
        assert np.all(V[idx, np.arange(k)] > 0)


def test_batched_psvd_autotune_and_single_problem_agree():
    g = synth.rng(77)
    probs = []
    for i in range(10):
        m, n = int(g.integers(300, 1200)), int(g.integers(100, 300))
        A = synth.gaussian_product(m, n, 12, 1e-6, seed=i, dtype=np.float32)
        probs.append(dict(A=torch.from_numpy(A).cuda(), k=5, krylov_dim=20, tol=1e-8))
    M = gk()
    res1, st1, info1 = M.gk_psvd_batched(probs, autotune=True)
    res2, st2, info2 = M.gk_psvd_batched(probs)
    assert st1 == st2 == 0
    assert info2["reserved"] in (2, 4, 8, 16)
    for (U1, S1, V1, _), (U2, S2, V2, _), pr in zip(res1, res2, probs):
        np.testing.assert_allclose(S1.cpu().numpy(), S2.cpu().numpy(), rtol=1e-12)
        Us, Ss, Vs, st, _ = M.gk_psvd(pr["A"], 5, 1e-8, krylov_dim=20)
        np.testing.assert_allclose(S1.cpu().numpy(), Ss.cpu().numpy(), rtol=1e-6)


def test_batched_recipe_sample_matches_oracle():
    """A sample of the benchmark's own 512-problem recipe (dense f32, m up to 4096, ranks 5..64 plus
    1e-6 noise, rank cut eps = 1e-5, tol 1e-8) in the two configurations the benchmark runs:
      * plain pipeline: k = the true rank, K = max(2r, r + 16) -- the six highest-rank problems,
        whose K > 78 takes the cluster-wide Jacobi branch of the small SVD;
      * learned pipeline: the committed network's (r^, K^) -- the four largest operators (the
        row-ring and panel paths of the products at m, n near 4096).
    Each problem's rank, values and FP64 true residuals (oracle) against the oracle's partial SVD of
    the same stored bytes."""
    from paper_2104_10785_gb300 import predictor

    w = synth.WORKLOADS["batched_f32_512_rank5to64"]
    shapes = synth.batched_shapes(w["count"], w["seed"])
    mats = synth.torch_batched_products(shapes, 1e-6, w["seed"])
    params = predictor.load()
    assert params is not None
    pred = predictor.predict(mats, params)
    high_r = sorted(range(len(mats)), key=lambda i: -shapes[i][2])[:6]
    big = sorted((i for i in range(len(mats)) if i not in high_r), key=lambda i: -shapes[i][0] * shapes[i][1])[:4]
    plain = [dict(A=mats[i], k=shapes[i][2], krylov_dim=min(max(2 * shapes[i][2], shapes[i][2] + 16),
                                                               min(shapes[i][:2])), tol=w["tol"]) for i in high_r]
    assert min(p["krylov_dim"] for p in plain) > 78
    learned = [dict(A=mats[i], k=pred[i][0], krylov_dim=pred[i][1], tol=w["tol"], rank_cut=w["eps"]) for i in big]
    oracle.set_threads(0)
    for probs, idx in ((plain, high_r), (learned, big)):
        res, st, info = gk().gk_psvd_batched(probs)
        assert st == 0, [r[3]["status"] for r in res]
        for (U, S, V, rr), i in zip(res, idx):
            m, n, r = shapes[i]
            assert rr["rank"] == r, (i, rr["rank"], r)
            op = oracle.Operator.dense(np.ascontiguousarray(mats[i].cpu().numpy()))
            K = min(max(2 * r, r + 16), min(m, n))
            Uo, So, Vo, io = oracle.psvd(op, r, K, synth.start_vector(m, i), tol=1e-12, max_restarts=500)
            Sg = S.cpu().numpy()[:r]
            np.testing.assert_allclose(Sg, So, rtol=1e-6)
            r1, r2 = oracle.residuals(op, U.cpu().numpy()[:, :r], Sg, V.cpu().numpy()[:, :r])
            res_rel = max(r1.max(), r2.max()) / So[0]
            # the convergence test bounds the Ritz residual by tol; the f32 products add their floor
            assert res_rel <= 3e-8, (i, shapes[i], res_rel)
