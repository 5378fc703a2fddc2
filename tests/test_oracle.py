"""Pins for the CPU oracle: every check here compares the oracle with something
other than itself -- LAPACK (numpy.linalg), closed forms, exact invariants of the
Golub-Kahan recurrences (Eqs. 2.3-2.4, pq_ortho), published known-answer vectors,
or special cases whose answer the mathematics fixes.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s):
    return np.random.default_rng(1000 + s)


def _angle_ok(U1, U2, tol):
    """Columnwise |cos| between matched singular vectors is 1 within tol."""
    c = np.abs(np.sum(U1 * U2, axis=0)) / (np.linalg.norm(U1, axis=0) * np.linalg.norm(U2, axis=0))
    return np.all(1.0 - c <= tol), (1.0 - c).max()


# ---------------------------------------------------------------------------
# generators and value promotion
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    path = os.path.join(GOLDEN, "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_start_vector_is_normal_2_1():
    # Algorithm 1: q1 ~ N(2, 1)^m.  Moments and a KS test against N(2,1).
    from scipy import stats

    q = oracle.start_vector(2104107, 200000)
    assert abs(q.mean() - 2.0) < 5 / np.sqrt(q.size)
    assert abs(q.var() - 1.0) < 5 * np.sqrt(2.0 / q.size)
    assert stats.kstest(q - 2.0, "norm").pvalue > 1e-4
    # different seeds give different streams; same seed is deterministic
    assert np.array_equal(q[:100], oracle.start_vector(2104107, 100))
    assert not np.allclose(q[:100], oracle.start_vector(2104108, 100))


def test_splitmix64_matches_published_outputs():
    """gko_splitmix64(x) is the generator's output for the state x + gamma, so output i of
    the generator seeded with s is gko_splitmix64(s + i * gamma)."""
    gamma = 0x9E3779B97F4A7C15
    path = os.path.join(GOLDEN, "splitmix64_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for r in rows:
        seed, outs = int(r[0]), [int(x) for x in r[1:]]
        got = [oracle.splitmix64((seed + i * gamma) % 2**64) for i in range(len(outs))]
        assert got == outs


def test_splitmix64_is_a_mixing_bijection_sample():
    xs = [oracle.splitmix64(i) for i in range(4096)]
    assert len(set(xs)) == 4096
    bits = np.array([[(x >> b) & 1 for b in range(64)] for x in xs])
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 0.06)


def test_f16_and_bf16_promotion_match_library_conversions():
    import torch

    allbits = np.arange(65536, dtype=np.uint16)
    # f16: compare with numpy's IEEE half conversion for every bit pattern
    op = oracle.Operator(allbits, 1, 65536, "f16")
    ref = allbits.view(np.float16).astype(np.float64)
    got = np.array([op.value(i) for i in range(65536)])
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    # bf16: compare with torch's bfloat16 -> float64 conversion
    opb = oracle.Operator(allbits, 1, 65536, "bf16")
    refb = torch.from_numpy(allbits.view(np.int16).copy()).view(torch.bfloat16).double().numpy()
    gotb = np.array([opb.value(i) for i in range(65536)])
    finb = np.isfinite(refb)
    assert np.array_equal(gotb[finb], refb[finb])
    # the f16 scale factor multiplies every value
    ops = oracle.Operator(allbits[:100], 1, 100, "f16", scale=0.25)
    assert np.array_equal([ops.value(i) for i in range(100)], ref[:100] * 0.25)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_dense_products_match_numpy(dtype):
    import torch

    rng = _rng(1)
    A = rng.standard_normal((37, 53))
    if dtype == "f64":
        op, Ad = oracle.Operator.dense(A), A
    elif dtype == "f32":
        A32 = A.astype(np.float32)
        op, Ad = oracle.Operator.dense(A32), A32.astype(np.float64)
    else:
        t = torch.from_numpy(A).to(torch.bfloat16)
        bits = t.view(torch.int16).numpy().view(np.uint16)
        op, Ad = oracle.Operator.dense(None, dtype="bf16", bits=bits), t.double().numpy()
    x = rng.standard_normal(53)
    y = rng.standard_normal(37)
    np.testing.assert_allclose(op.matvec(x), Ad @ x, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(op.rmatvec(y), Ad.T @ y, rtol=1e-13, atol=1e-13)


def test_csr_products_match_scipy():
    import scipy.sparse as sp

    rng = _rng(2)
    S = sp.random(300, 170, density=0.05, random_state=3, format="csr", dtype=np.float64)
    S.data = rng.standard_normal(S.nnz)
    S32 = S.astype(np.float32)
    op = oracle.Operator.csr(300, 170, S32.indptr, S32.indices, S32.data, "f32")
    x = rng.standard_normal(170)
    y = rng.standard_normal(300)
    Sd = S32.astype(np.float64)
    np.testing.assert_allclose(op.matvec(x), Sd @ x, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(op.rmatvec(y), Sd.T @ y, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# Jacobi SVD / eigensolver (the small dense kernels of Algorithms 2 and 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (7, 3), (30, 30), (41, 17), (120, 120)])
def test_jacobi_svd_matches_lapack(shape):
    rng = _rng(3)
    M = rng.standard_normal(shape)
    U, s, V, sw = oracle.jacobi_svd(M)
    assert sw >= 0
    s_ref = np.linalg.svd(M, compute_uv=False)
    np.testing.assert_allclose(s, s_ref, rtol=1e-13, atol=1e-14 * s_ref[0])
    np.testing.assert_allclose(U.T @ U, np.eye(shape[1]), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(shape[1]), atol=1e-13)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, M, atol=1e-13 * s_ref[0])


def test_jacobi_svd_closed_forms():
    # 2x2 upper triangular [[a, b], [0, d]]: sigma = (sqrt((a+d)^2+b^2) +- sqrt((a-d)^2+b^2)) / 2
    for a, b, d in [(3.0, 4.0, 1.0), (1.0, 1e-9, 1.0), (2.0, -7.0, 0.5), (5.0, 0.0, -2.0)]:
        M = np.array([[a, b], [0.0, d]])
        _, s, _, _ = oracle.jacobi_svd(M)
        p, q = np.hypot(a + d, b), np.hypot(a - d, b)
        np.testing.assert_allclose(s, [(p + q) / 2, abs(p - q) / 2], rtol=1e-14, atol=1e-15)
    # diagonal: singular values are |d| sorted, singular vectors are +-coordinate axes
    dg = np.array([0.3, -5.0, 2.0, 0.0, 1.0])
    U, s, V, _ = oracle.jacobi_svd(np.diag(dg))
    np.testing.assert_array_equal(s, np.sort(np.abs(dg))[::-1])
    # graded matrix: relative accuracy of tiny singular values (Demmel-Veselic)
    D = np.diag(10.0 ** -np.arange(0, 12, 1.0))
    rng = _rng(4)
    Q1, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    _, s, _, _ = oracle.jacobi_svd(Q1 @ D)  # column scaling only: sigma = 10^-i exactly
    np.testing.assert_allclose(s, np.diag(D), rtol=1e-13)


def test_jacobi_eig_matches_lapack():
    rng = _rng(5)
    M = rng.standard_normal((25, 25))
    S = M + M.T
    th, G, sw = oracle.jacobi_eig(S)
    ref = np.sort(np.linalg.eigvalsh(S))[::-1]
    np.testing.assert_allclose(th, ref, atol=1e-12 * abs(ref).max())
    np.testing.assert_allclose(G.T @ G, np.eye(25), atol=1e-13)
    np.testing.assert_allclose(S @ G, G * th, atol=1e-12 * abs(ref).max())


# ---------------------------------------------------------------------------
# Algorithm 1: recurrences, invariants and special cases
# ---------------------------------------------------------------------------

def _lower_B(d):
    kp = d["kprime"]
    B = np.zeros((kp + 1, kp))
    for j in range(kp):
        B[j, j] = d["alpha"][j]
        B[j + 1, j] = d["beta"][j + 1]
    return B


@pytest.mark.parametrize("shape,passes", [((120, 80), 2), ((80, 120), 2), ((150, 150), 1), ((120, 80), 0),
                                          ((80, 120), 0)])
def test_alg1_bidiagonal_relations(shape, passes):
    """Eq. 2.4: A P_k = Q_{k+1} B_{k+1,k};  A^T Q_{k+1} = P_k B^T + alpha_{k+1} p_{k+1} e_{k+1}^T;
    Eq. pq_ortho: Q^T Q = I, P^T P = I;  alpha_i, beta_i >= 0."""
    rng = _rng(6)
    m, n = shape
    A = rng.standard_normal((m, n)) * np.linspace(1, 0.05, n)[None, :]
    op = oracle.Operator.dense(A)
    k = 40
    d = oracle.gk_lower(op, k, 2 + rng.standard_normal(m), eps=0.0, relative=False, passes=passes)
    assert d["kprime"] == k and d["stop_reason"] == 0
    Q, P, B = d["Q"][:, : k + 1], d["P"], _lower_B(d)
    nA = np.linalg.norm(A, 2)
    assert np.abs(A @ P[:, :k] - Q @ B).max() < 1e-13 * nA
    R = A.T @ Q - P[:, :k] @ B.T
    R[:, k] -= d["alpha"][k] * P[:, k]
    assert np.abs(R).max() < 1e-13 * nA
    tol_o = 1e-10 if passes == 1 else 1e-13
    assert np.abs(Q.T @ Q - np.eye(k + 1)).max() < tol_o
    assert np.abs(P[:, : k + 1].T @ P[:, : k + 1] - np.eye(k + 1)).max() < tol_o
    assert np.all(d["alpha"][: k + 1] >= 0) and np.all(d["beta"][: k + 2] >= 0)
    # Eq. 2.10: A^T A P_k = P_k B^T B + alpha_{k+1} beta_{k+1} p_{k+1} e_k^T
    R2 = A.T @ (A @ P[:, :k]) - P[:, :k] @ (B.T @ B)
    R2[:, k - 1] -= d["alpha"][k] * d["beta"][k] * P[:, k]
    assert np.abs(R2).max() < 1e-12 * nA**2


def test_adaptive_reorthogonalization_repeats_the_pass_under_cancellation():
    """The adaptive rule (passes = 0): a vector almost inside span(Q) (w = Q c + 1e-10 z) loses
    almost all of its norm in the first pass, so the second pass runs and the result is as
    orthogonal as with two passes, where one pass leaves components ~ eps ||c|| / 1e-10; a vector
    with no cancellation gets exactly one pass."""
    rng = _rng(21)
    m, j = 400, 30
    Q, _ = np.linalg.qr(rng.standard_normal((m, j)))
    z = rng.standard_normal(m)
    z -= Q @ (Q.T @ z)
    w = Q @ rng.standard_normal(j) + 1e-10 * z
    res = {}
    for p in (0, 1, 2):
        x = oracle.cgs(w, Q, passes=p)
        res[p] = np.abs(Q.T @ x).max() / np.linalg.norm(x)
    assert res[0] < 1e-14 and res[2] < 1e-14
    assert res[1] > 1e3 * res[0]
    np.testing.assert_array_equal(oracle.cgs(w, Q, passes=0), oracle.cgs(w, Q, passes=2))
    y = rng.standard_normal(m)  # ||y1|| ~ ||y||: no second pass
    np.testing.assert_array_equal(oracle.cgs(y, Q, passes=0), oracle.cgs(y, Q, passes=1))


def test_alg1_orthogonal_invariance():
    """GK on Q1 A Q2^T started at Q1 q1 produces the same alpha, beta."""
    rng = _rng(7)
    m, n = 90, 60
    A = rng.standard_normal((m, n))
    Q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    q1 = 2 + rng.standard_normal(m)
    d0 = oracle.gk_lower(oracle.Operator.dense(A), 30, q1, eps=0.0, relative=False)
    d1 = oracle.gk_lower(oracle.Operator.dense(Q1 @ A @ Q2.T), 30, Q1 @ q1, eps=0.0, relative=False)
    np.testing.assert_allclose(d1["alpha"], d0["alpha"], rtol=1e-11)
    np.testing.assert_allclose(d1["beta"], d0["beta"], rtol=1e-11)


def test_alg1_first_step_closed_form():
    """alpha_1 = ||A^T q1||/||q1||; beta_2 = ||A p1 - alpha_1 q1|| (no earlier q to orthogonalize against
    except q1 itself, which it is orthogonal to in exact arithmetic)."""
    rng = _rng(8)
    A = rng.standard_normal((20, 12))
    q1 = 2 + rng.standard_normal(20)
    d = oracle.gk_lower(oracle.Operator.dense(A), 1, q1, eps=0.0, relative=False)
    qn = q1 / np.linalg.norm(q1)
    a1 = np.linalg.norm(A.T @ qn)
    p1 = A.T @ qn / a1
    w = A @ p1 - a1 * qn
    np.testing.assert_allclose(d["alpha"][0], a1, rtol=1e-14)
    np.testing.assert_allclose(d["beta"][0], np.linalg.norm(q1), rtol=1e-14)
    np.testing.assert_allclose(d["beta"][1], np.linalg.norm(w), rtol=1e-13)


def test_alg1_rank_one_breaks_after_one_step():
    rng = _rng(9)
    x, y = rng.standard_normal(50), rng.standard_normal(30)
    op = oracle.Operator.dense(np.outer(x, y))
    r, kp, sig = oracle.numrank(op, 2 + rng.standard_normal(50), eps=1e-8)
    assert r == 1
    assert kp <= 2
    np.testing.assert_allclose(sig[0], np.linalg.norm(x) * np.linalg.norm(y), rtol=1e-13)


def test_alg1_zero_matrix():
    op = oracle.Operator.dense(np.zeros((10, 7)))
    r, kp, sig = oracle.numrank(op, np.full(10, 2.0), eps=1e-8)
    assert r == 0 and kp == 0


def test_alg3_identity_sees_one_direction():
    """Krylov limitation: K(I, q1) is one-dimensional, so Algorithm 3 reports 1 for A = I."""
    op = oracle.Operator.dense(np.eye(40))
    r, kp, sig = oracle.numrank(op, 2 + _rng(10).standard_normal(40), eps=1e-8)
    assert r == 1 and kp == 1


@pytest.mark.parametrize("m,n,r", [(60, 40, 7), (40, 60, 13), (200, 150, 40), (100, 100, 100)])
def test_alg3_rank_matches_brute_force(m, n, r):
    rng = _rng(11)
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    s = np.linalg.svd(A, compute_uv=False)
    truth = int(np.sum(s > 1e-8 * s[0]))
    assert truth == r
    op = oracle.Operator.dense(A)
    got, kp, sig = oracle.numrank(op, 2 + rng.standard_normal(m), eps=1e-8)
    assert got == truth
    np.testing.assert_allclose(sig[:r], s[:r], rtol=1e-11)


def test_alg3_literal_eigenvalue_count():
    """The printed Algorithm 3 counts eigenvalues of B^T B (= sigma^2) above eps."""
    rng = _rng(12)
    U, _ = np.linalg.qr(rng.standard_normal((50, 20)))
    V, _ = np.linalg.qr(rng.standard_normal((30, 20)))
    s = np.logspace(0, -7, 20)
    A = U @ np.diag(s) @ V.T
    op = oracle.Operator.dense(A)
    q1 = 2 + rng.standard_normal(50)
    lit, _, _ = oracle.numrank(op, q1, eps=1e-6, relative=False, literal=True)
    assert lit == int(np.sum(s**2 > 1e-6))
    rel, _, _ = oracle.numrank(op, q1, eps=1e-6, relative=True)
    assert rel == int(np.sum(s > 1e-6 * s[0]))


def test_alg1_absolute_threshold_reading():
    rng = _rng(13)
    A = 1e-3 * rng.standard_normal((30, 3)) @ rng.standard_normal((3, 20))
    op = oracle.Operator.dense(A)
    r, kp, _ = oracle.numrank(op, 2 + rng.standard_normal(30), eps=1.0, relative=False)
    assert r == 0 or kp <= 1  # everything is below an absolute threshold of 1


# ---------------------------------------------------------------------------
# Algorithm 2 and the restarted partial SVD
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("route", [0, 1])
def test_alg2_fsvd_recovers_low_rank_triplets(route):
    rng = _rng(14)
    m, n, r = 200, 120, 25
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    op = oracle.Operator.dense(A)
    U, S, V, kp = oracle.fsvd(op, r + 5, 10, 2 + rng.standard_normal(m), route=route)
    Ur, Sr, Vtr = np.linalg.svd(A, full_matrices=False)
    np.testing.assert_allclose(S, Sr[:10], rtol=1e-12)
    ok, worst = _angle_ok(U, Ur[:, :10], 1e-12)
    assert ok, worst
    ok, worst = _angle_ok(V, Vtr[:10].T, 1e-12)
    assert ok, worst
    assert oracle.err_rel(op, U, S, V) < 1e-13


def test_alg2_and_first_restart_cycle_share_ritz_values():
    """Lower form (Algorithm 2) and the upper form started at v1 = p1 span the same right Krylov space,
    and P^T A^T A P = B^T B in both, so their Ritz values coincide."""
    rng = _rng(15)
    m, n, K = 150, 110, 25
    A = rng.standard_normal((m, n)) * (0.93 ** np.arange(n))[None, :]
    op = oracle.Operator.dense(A)
    q1 = 2 + rng.standard_normal(m)
    d = oracle.gk_lower(op, K, q1, eps=0.0, relative=False)
    s_lower = np.linalg.svd(_lower_B(d), compute_uv=False)
    al, be, Ub, Vb = oracle.gk_upper(op, K, q1)
    Bu = np.diag(al) + np.diag(be[:-1], 1)
    s_upper = np.linalg.svd(Bu, compute_uv=False)
    np.testing.assert_allclose(s_upper, s_lower, rtol=1e-11)
    # upper-form relations: A V_K = U_K B_K ; A^T U_K = V_K B_K^T + beta_K v_{K+1} e_K^T
    nA = np.linalg.norm(A, 2)
    assert np.abs(A @ Vb[:, :K] - Ub @ Bu).max() < 1e-13 * nA
    R = A.T @ Ub - Vb[:, :K] @ Bu.T
    R[:, K - 1] -= be[K - 1] * Vb[:, K]
    assert np.abs(R).max() < 1e-13 * nA
    np.testing.assert_allclose(Vb.T @ Vb, np.eye(K + 1), atol=1e-13)
    # v1 = A^T q1 / ||A^T q1|| (Algorithm 1)
    v1 = A.T @ q1
    np.testing.assert_allclose(Vb[:, 0], v1 / np.linalg.norm(v1), atol=1e-14)


@pytest.mark.parametrize("m,n,k,K", [(300, 200, 10, 30), (200, 300, 10, 30), (250, 250, 20, 45), (90, 60, 5, 12)])
def test_psvd_matches_lapack(m, n, k, K):
    rng = _rng(16)
    A = rng.standard_normal((m, n)) * (0.95 ** np.arange(n))[None, :]
    op = oracle.Operator.dense(A)
    U, S, V, info = oracle.psvd(op, k, K, 2 + rng.standard_normal(m), tol=1e-12)
    assert info["converged"]
    Ur, Sr, Vtr = np.linalg.svd(A, full_matrices=False)
    np.testing.assert_allclose(S, Sr[:k], rtol=1e-11)
    gaps = np.minimum(np.abs(np.diff(Sr[: k + 1])), np.r_[np.inf, np.abs(np.diff(Sr[:k]))])
    tol_ang = 1e-12 * Sr[0] / gaps.min()
    ok, worst = _angle_ok(V, Vtr[:k].T, max(tol_ang, 1e-11))
    assert ok, worst
    r1, r2 = oracle.residuals(op, U, S, V)
    assert r1.max() < 1e-12 * S[0] and r2.max() < 1e-11 * S[0]
    # sign convention: largest |v_i| entry positive
    for i in range(k):
        assert V[np.argmax(np.abs(V[:, i])), i] > 0


def test_psvd_prescribed_spectrum():
    """A = U diag(0.9^i) V^T with orthonormal U, V: the top singular values are 0.9^i exactly."""
    rng = _rng(17)
    m, n = 400, 200
    U0, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = 0.9 ** np.arange(1, n + 1)
    A = (U0 * s) @ V0.T
    op = oracle.Operator.dense(A)
    U, S, V, info = oracle.psvd(op, 10, 14, 2 + rng.standard_normal(m), tol=1e-13, max_restarts=200)
    assert info["converged"] and info["restarts"] >= 1
    np.testing.assert_allclose(S, s[:10], rtol=1e-12)
    ok, worst = _angle_ok(V, V0[:, :10], 1e-11)
    assert ok, worst
    ok, worst = _angle_ok(U, U0[:, :10], 1e-11)
    assert ok, worst


def test_psvd_residual_estimate_equals_true_residual():
    """||A^T u~_i - sigma_i v~_i|| = |beta_K X_{K,i}|: with a loose tolerance the returned triplets' true
    residual is bounded by the estimate the convergence test used."""
    rng = _rng(18)
    A = rng.standard_normal((160, 120)) * (0.97 ** np.arange(120))[None, :]
    op = oracle.Operator.dense(A)
    U, S, V, info = oracle.psvd(op, 6, 16, 2 + rng.standard_normal(160), tol=1e-4, max_restarts=50)
    r1, r2 = oracle.residuals(op, U, S, V)
    assert r1.max() < 1e-12 * S[0]  # A v~ = sigma u~ holds exactly (to rounding)
    assert r2.max() <= info["resid_est_max"] * S[0] * (1 + 1e-6) + 1e-13 * S[0]
    assert info["resid_est_max"] <= 1e-4


def test_psvd_diagonal_and_rank_deficient():
    rng = _rng(19)
    d = rng.permutation(np.linspace(1.0, 3.0, 50))
    op = oracle.Operator.dense(np.diag(d))
    U, S, V, info = oracle.psvd(op, 5, 20, 2 + rng.standard_normal(50), tol=1e-12, max_restarts=200)
    np.testing.assert_allclose(S, np.sort(d)[::-1][:5], rtol=1e-12)
    # exact rank 3 with k = 5: two zero singular values, no NaN, relations hold
    A = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 30))
    op = oracle.Operator.dense(A)
    U, S, V, info = oracle.psvd(op, 5, 10, 2 + rng.standard_normal(40), tol=1e-12)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(V))
    np.testing.assert_allclose(S[:3], s[:3], rtol=1e-12)
    assert np.all(S[3:] < 1e-12 * s[0])
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-10)
    # zero matrix
    U, S, V, info = oracle.psvd(oracle.Operator.dense(np.zeros((12, 9))), 2, 5, np.full(12, 2.0), tol=1e-12)
    assert np.all(S == 0) and np.all(np.isfinite(V))


def test_psvd_full_dimension_and_tiny_shapes():
    rng = _rng(20)
    for m, n in [(1, 1), (3, 1), (1, 4), (5, 5), (7, 3)]:
        A = rng.standard_normal((m, n))
        mn = min(m, n)
        U, S, V, info = oracle.psvd(oracle.Operator.dense(A), mn, mn, 2 + rng.standard_normal(m), tol=1e-12)
        np.testing.assert_allclose(S, np.linalg.svd(A, compute_uv=False), rtol=1e-12, atol=1e-14)


def test_psvd_transpose_symmetry():
    rng = _rng(21)
    A = rng.standard_normal((70, 50)) * (0.9 ** np.arange(50))[None, :]
    U, S, V, _ = oracle.psvd(oracle.Operator.dense(A), 6, 20, 2 + rng.standard_normal(70), tol=1e-12)
    U2, S2, V2, _ = oracle.psvd(oracle.Operator.dense(A.T.copy()), 6, 20, 2 + rng.standard_normal(50), tol=1e-12)
    np.testing.assert_allclose(S2, S, rtol=1e-12)
    assert _angle_ok(U2, V, 1e-11)[0] and _angle_ok(V2, U, 1e-11)[0]


def test_error_metrics_closed_form():
    """err_res of a rank-k truncation equals the tail norm sqrt(sum_{i>k} sigma_i^2) (Eckart-Young);
    err_rel of exact triplets is ~0 and of a perturbed Sigma equals the perturbation's norm ratio."""
    rng = _rng(22)
    A = rng.standard_normal((40, 30))
    Ur, Sr, Vtr = np.linalg.svd(A, full_matrices=False)
    op = oracle.Operator.dense(A)
    k = 8
    np.testing.assert_allclose(oracle.err_res(op, Ur[:, :k], Sr[:k], Vtr[:k].T), np.sqrt(np.sum(Sr[k:] ** 2)),
                               rtol=1e-12)
    assert oracle.err_rel(op, Ur[:, :k], Sr[:k], Vtr[:k].T) < 1e-14
    Sp = Sr[:k] * 1.01
    # A^T U - V Sp = V (S - Sp)  ->  ||.||_F / ||Sp|| = 0.01 ||S|| / (1.01 ||S||)
    np.testing.assert_allclose(oracle.err_rel(op, Ur[:, :k], Sp, Vtr[:k].T), 0.01 / 1.01, rtol=1e-10)


def test_planted_mistake_is_caught_by_invariants():
    """A dropped recurrence term (alpha_j q_j in Eq. 2.2) breaks Eq. 2.4 by O(||A||); the relation check
    used above therefore detects that class of mistake.  Reproduced here on the host from the oracle's
    own outputs by removing the term."""
    rng = _rng(23)
    A = rng.standard_normal((50, 40))
    op = oracle.Operator.dense(A)
    d = oracle.gk_lower(op, 10, 2 + rng.standard_normal(50), eps=0.0, relative=False)
    B = _lower_B(d)
    Bbad = B.copy()
    Bbad[np.arange(10), np.arange(10)] = 0.0  # as if -alpha_j q_j were dropped
    good = np.abs(A @ d["P"][:, :10] - d["Q"][:, :11] @ B).max()
    bad = np.abs(A @ d["P"][:, :10] - d["Q"][:, :11] @ Bbad).max()
    assert good < 1e-12 and bad > 1e-1


# ---------------------------------------------------------------------------
# the fused sweep (A^T w / beta in place of A^T q): pinned by Eq. 2.4 directly and by
# agreement with the recurrence as printed
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,passes", [((120, 80), 0), ((80, 120), 0), ((150, 150), 2), ((200, 90), 1)])
def test_fused_sweep_keeps_the_bidiagonal_relations(shape, passes):
    """The fused ordering must satisfy Eq. 2.4 and Eq. pq_ortho on its own (these fail if the
    span(P_j) argument were wrong, e.g. a dropped 1/beta or a missing -beta p_j term), and give
    the alpha, beta of the printed recurrence to rounding."""
    rng = _rng(31)
    m, n = shape
    A = rng.standard_normal((m, n)) * np.linspace(1, 0.05, n)[None, :]
    op = oracle.Operator.dense(A)
    k = 40
    q1 = 2 + rng.standard_normal(m)
    d = oracle.gk_lower(op, k, q1, eps=0.0, relative=False, passes=passes, fused=True)
    assert d["kprime"] == k and d["stop_reason"] == 0
    Q, P, B = d["Q"][:, : k + 1], d["P"], _lower_B(d)
    nA = np.linalg.norm(A, 2)
    assert np.abs(A @ P[:, :k] - Q @ B).max() < 1e-13 * nA
    R = A.T @ Q - P[:, :k] @ B.T
    R[:, k] -= d["alpha"][k] * P[:, k]
    assert np.abs(R).max() < 1e-13 * nA
    tol_o = 1e-10 if passes == 1 else 1e-13
    assert np.abs(Q.T @ Q - np.eye(k + 1)).max() < tol_o
    assert np.abs(P[:, : k + 1].T @ P[:, : k + 1] - np.eye(k + 1)).max() < tol_o
    d0 = oracle.gk_lower(op, k, q1, eps=0.0, relative=False, passes=passes)
    sc = max(d0["alpha"].max(), d0["beta"][1:].max())
    assert np.abs(d["alpha"] - d0["alpha"]).max() < 1e-12 * sc
    assert np.abs(d["beta"][1:] - d0["beta"][1:]).max() < 1e-12 * sc


def test_fused_sweep_upper_form_and_restarts_match_lapack():
    """The upper-bidiagonal fused cycle keeps A V_K = U_K B_K, and the restarted partial SVD on it
    (restarts, where the first step after each restart runs unfused) returns LAPACK's triplets."""
    rng = _rng(32)
    m, n, K = 260, 180, 30
    A = rng.standard_normal((m, n)) * (0.93 ** np.arange(n))[None, :]
    op = oracle.Operator.dense(A)
    q1 = 2 + rng.standard_normal(m)
    al, be, Ub, Vb = oracle.gk_upper(op, K, q1, fused=True)
    al0, be0, _, _ = oracle.gk_upper(op, K, q1)
    B = np.diag(al) + np.diag(be[:-1], 1)
    nA = np.linalg.norm(A, 2)
    assert np.abs(A @ Vb[:, :K] - Ub @ B).max() < 1e-13 * nA
    assert np.abs(Ub.T @ Ub - np.eye(K)).max() < 1e-13
    np.testing.assert_allclose(al, al0, rtol=1e-11)
    np.testing.assert_allclose(be, be0, rtol=1e-11)
    U, S, V, info = oracle.psvd(op, 8, 20, q1, tol=1e-12, max_restarts=200, fused=True)
    assert info["converged"] and info["restarts"] >= 1
    Ur, Sr, Vtr = np.linalg.svd(A, full_matrices=False)
    np.testing.assert_allclose(S, Sr[:8], rtol=1e-11)
    ok, worst = _angle_ok(V, Vtr[:8].T, 1e-9)
    assert ok, worst
    r1, r2 = oracle.residuals(op, U, S, V)
    assert max(r1.max(), r2.max()) < 1e-11 * S[0]


@pytest.mark.parametrize("m,n,r", [(300, 200, 17), (150, 260, 40)])
def test_fused_sweep_rank_matches_brute_force(m, n, r):
    rng = _rng(33)
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    op = oracle.Operator.dense(A)
    q1 = 2 + rng.standard_normal(m)
    rank, kp, _ = oracle.numrank(op, q1, eps=1e-9, fused=True)
    assert rank == np.linalg.matrix_rank(A) == r
