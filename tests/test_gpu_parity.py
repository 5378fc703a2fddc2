"""Parity of the CUDA path (through the C ABI) with the CPU oracle on identical seeded
inputs.  Sizes are chosen so that the oracle finishes in seconds while the kernels
still span several tiles, chunks and ragged tails.

Tolerances:
  * f64 operators: the method's own tolerance (tol) bounds the residuals on both
    sides, so singular values agree to ~tol^2/gap and vectors to ~tol*sigma_1/gap.
  * f32/bf16/f16 operators are multiplied in f32 with the vector rounded to f32 and
    runs of at most 64 products summed in f32 (then combined in f64): every entry of
    a product is within 2^-24 (64 + 2) sum_j |a_ij x_j| of the exact product of the
    stored values, and the residual floor of the Krylov relations is of order
    2^-24 ||A||_F / sqrt(n); bounds below are stated from these.
"""
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


def dense_pair(A, dtype):
    """(oracle operator on the stored bytes, device tensor with the same bytes, f64 copy of stored values)."""
    if dtype == "f64":
        A64 = np.asarray(A, dtype=np.float64)
        return oracle.Operator.dense(A64), cuda(A64), A64
    if dtype == "f32":
        A32 = np.asarray(A, dtype=np.float32)
        return oracle.Operator.dense(A32), cuda(A32), A32.astype(np.float64)
    if dtype == "bf16":
        bits = synth.to_bf16_bits(np.asarray(A, dtype=np.float32))
        t = cuda(bits.view(np.int16)).view(torch.bfloat16)
        return oracle.Operator.dense(None, dtype="bf16", bits=bits), t, synth.bf16_bits_to_f32(bits).astype(np.float64)
    if dtype == "f16":
        h = np.asarray(A, dtype=np.float16)
        bits = h.view(np.uint16)
        t = cuda(h)
        return oracle.Operator.dense(None, dtype="f16", bits=bits), t, h.astype(np.float64)
    raise ValueError(dtype)


def angle_err(X, Y):
    """max_i || x_i - sign * y_i || for unit columns (sign-invariant)."""
    X = np.asarray(X)
    Y = np.asarray(Y)
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return np.linalg.norm(X - Y * s[None, :], axis=0).max()


# ---------------------------------------------------------------------------
# the products of Eq. 2.2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("shape", [(1, 1), (7, 3), (33, 65), (1000, 1537), (3001, 2049), (64, 40000)])
def test_dense_products_match_oracle(dtype, shape):
    m, n = shape
    g = synth.rng(11 + m + n)
    A = g.standard_normal((m, n))
    op, At, Ad = dense_pair(A, dtype)
    x = g.standard_normal(n)
    y = g.standard_normal(m)
    M = gk()
    got = M.gk_matvec(At, cuda(x)).cpu().numpy()
    got_t = M.gk_matvec(At, cuda(y), trans=True).cpu().numpy()
    ref = op.matvec(x)
    ref_t = op.rmatvec(y)
    if dtype == "f64":
        # f64 products: within a few ulps of sum_j |a_ij x_j| (different summation order)
        assert np.all(np.abs(got - ref) <= 1e-13 * (np.abs(Ad) @ np.abs(x)) + 1e-300)
        assert np.all(np.abs(got_t - ref_t) <= 1e-13 * (np.abs(Ad).T @ np.abs(y)) + 1e-300)
    else:
        bound = U32 * 66 * (np.abs(Ad) @ np.abs(x)) + 1e-300
        assert np.all(np.abs(got - ref) <= bound)
        bound_t = U32 * 66 * (np.abs(Ad).T @ np.abs(y)) + 1e-300
        assert np.all(np.abs(got_t - ref_t) <= bound_t)


@pytest.mark.parametrize("dtype,m,n", [("bf16", 20000, 8192), ("f32", 50000, 4096)])
def test_dense_products_bulk_path_many_units_per_block(dtype, m, n):
    """16-byte rows take the bulk-copy A x kernel; here the work units (row groups of 128 x
    2048-byte column chunks: 1256 and 3128 of them) outnumber the resident blocks several times,
    so every block runs its ring of stages across several units (the full-size configuration),
    and A^T x runs row blocks of 1024 rows.  Element-wise against the oracle."""
    g = torch.Generator(device="cuda").manual_seed(m + n)
    At = torch.randn(m, n, generator=g, device="cuda", dtype=torch.float32)
    At = At.to(torch.bfloat16) if dtype == "bf16" else At
    x = torch.randn(n, generator=g, device="cuda", dtype=torch.float64)
    y = torch.randn(m, generator=g, device="cuda", dtype=torch.float64)
    M = gk()
    got = M.gk_matvec(At, x).cpu().numpy()
    got_t = M.gk_matvec(At, y, trans=True).cpu().numpy()
    if dtype == "bf16":
        bits = At.view(torch.int16).cpu().numpy().view(np.uint16)
        op = oracle.Operator.dense(None, dtype="bf16", bits=bits)
        Ad = synth.bf16_bits_to_f32(bits).astype(np.float64)
    else:
        A32 = At.cpu().numpy()
        op = oracle.Operator.dense(A32)
        Ad = A32.astype(np.float64)
    oracle.set_threads(0)
    xh, yh = x.cpu().numpy(), y.cpu().numpy()
    ref, ref_t = op.matvec(xh), op.rmatvec(yh)
    assert np.all(np.abs(got - ref) <= U32 * 66 * (np.abs(Ad) @ np.abs(xh)))
    assert np.all(np.abs(got_t - ref_t) <= U32 * 66 * (np.abs(Ad).T @ np.abs(yh)))


def test_dense_products_padded_rows_and_unaligned_ld():
    """ld > n with rows that are not 16-byte aligned takes the scalar path."""
    g = synth.rng(5)
    m, n, ld = 257, 101, 103
    full = g.standard_normal((m, ld)).astype(np.float32)
    At = cuda(full)[:, :n]
    assert At.stride(0) == ld
    op = oracle.Operator(full, m, n, "f32", ld=ld)
    x = g.standard_normal(n)
    y = g.standard_normal(m)
    M = gk()
    A64 = full[:, :n].astype(np.float64)
    assert np.all(np.abs(M.gk_matvec(At, cuda(x)).cpu().numpy() - op.matvec(x)) <= U32 * 66 * (np.abs(A64) @ np.abs(x)))
    assert np.all(np.abs(M.gk_matvec(At, cuda(y), trans=True).cpu().numpy() - op.rmatvec(y))
                  <= U32 * 66 * (np.abs(A64).T @ np.abs(y)))


def _csr_pair(m, n, per_row, sig, seed, dtype=np.float32):
    d = synth.sparse_planted(m, n, per_row, sig, seed, usup=min(200, m // max(1, len(sig))),
                             vsup=min(100, n // max(1, len(sig))), dtype=dtype)
    dt = "f32" if dtype == np.float32 else "f64"
    op = oracle.Operator.csr(m, n, d["rowptr"], d["colind"], d["vals"], dt)
    M = gk()
    A = M.CSR(m, n, cuda(d["rowptr"]), cuda(d["colind"]), cuda(d["vals"]), cuda(d["t_rowptr"]), cuda(d["t_colind"]),
              cuda(d["t_vals"]))
    return op, A, d


def test_csr_products_match_oracle():
    op, A, d = _csr_pair(5003, 2999, 20, 10.0 * 0.9 ** np.arange(1, 6), 3)
    g = synth.rng(9)
    x = g.standard_normal(2999)
    y = g.standard_normal(5003)
    M = gk()
    np.testing.assert_allclose(M.gk_matvec(A, cuda(x)).cpu().numpy(), op.matvec(x), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(M.gk_matvec(A, cuda(y), trans=True).cpu().numpy(), op.rmatvec(y), rtol=1e-12,
                               atol=1e-12)


# ---------------------------------------------------------------------------
# Algorithm 3: numerical rank (exact equality with the oracle)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,r,dtype,eps", [(2000, 1200, 50, "f32", 1e-5), (1200, 2000, 50, "f32", 1e-5),
                                             (5000, 2000, 200, "f32", 1e-5), (777, 555, 31, "f64", 1e-5),
                                             (3000, 1000, 40, "bf16", 1e-2)])
def test_numrank_matches_oracle(m, n, r, dtype, eps):
    # bf16 storage perturbs the product by ~3e-4 sigma_1, so its numerical rank at eps = 1e-5 is full;
    # eps = 1e-2 sits between that floor and sigma_r / sigma_1 ~ 0.5
    A = synth.gaussian_product(m, n, r, 1e-7, seed=100 + m + r, dtype=np.float64)
    op, At, Ad = dense_pair(A, dtype)
    q1 = synth.start_vector(m, 7)
    r_or, kp_or, sig_or = oracle.numrank(op, q1, eps=eps, kmax=min(m, n, 400))
    rk, sig, st, info = gk().gk_numrank(At, eps, min(m, n, 400), start=cuda(q1), want_sigma=True)
    assert st == 0
    assert rk == r_or == r
    sig = sig.cpu().numpy()
    np.testing.assert_allclose(sig[:r], sig_or[:r], rtol=2e-6 if dtype != "f64" else 1e-11)
    assert abs(info["kprime"] - kp_or) <= 8


def test_numrank_seeded_start_matches_oracle_philox():
    """The device draws q1 ~ N(2,1) with Philox4x32-10 + Box-Muller; the oracle draws the same stream."""
    m, n = 900, 700
    A = synth.gaussian_product(m, n, 25, 0.0, seed=3, dtype=np.float64)
    op, At, _ = dense_pair(A, "f64")
    seed = 123456789
    q1 = oracle.start_vector(seed, m)
    r1, s1, _, i1 = gk().gk_numrank(At, 1e-8, 0, seed=seed, want_sigma=True)
    r2, s2, _, i2 = gk().gk_numrank(At, 1e-8, 0, start=cuda(q1), want_sigma=True)
    assert r1 == r2 == 25 and i1["kprime"] == i2["kprime"]
    # the 25 singular values of the rank-25 operator agree; the rest sit at the rounding floor
    np.testing.assert_allclose(s1.cpu().numpy()[:25], s2.cpu().numpy()[:25], rtol=1e-12)


def test_numrank_special_cases():
    M = gk()
    # zero matrix: rank 0
    Z = torch.zeros((50, 30), dtype=torch.float64, device="cuda")
    r, _, st, info = M.gk_numrank(Z, 1e-8)
    assert st == 0 and r == 0 and info["kprime"] == 0
    # rank one
    g = synth.rng(4)
    x, y = g.standard_normal(60), g.standard_normal(45)
    r, sig, st, info = M.gk_numrank(cuda(np.outer(x, y)), 1e-8, want_sigma=True)
    assert r == 1
    np.testing.assert_allclose(sig.cpu().numpy()[0], np.linalg.norm(x) * np.linalg.norm(y), rtol=1e-13)
    # identity: the Krylov space of I is one-dimensional (Algorithm 3 returns 1)
    r, _, _, info = M.gk_numrank(torch.eye(40, dtype=torch.float64, device="cuda"), 1e-8)
    assert r == 1 and info["kprime"] == 1
    # absolute threshold reading
    A = synth.gaussian_product(80, 60, 5, 0.0, seed=8, dtype=np.float64) * 1e-3
    r, _, _, _ = M.gk_numrank(cuda(A), 10.0, eps_absolute=True)
    op = oracle.Operator.dense(A)
    r_or, _, _ = oracle.numrank(op, synth.start_vector(80, 1), eps=10.0, relative=False)
    assert r == r_or


# ---------------------------------------------------------------------------
# restarted partial SVD
# ---------------------------------------------------------------------------

def _compare_psvd(op, At, A64, k, K, tol, q1, s_rtol, v_tol, res_tol, **kw):
    Uo, So, Vo, io = oracle.psvd(op, k, K, q1, tol=min(tol, 1e-12), max_restarts=500)
    assert io["converged"]
    U, S, V, st, info = gk().gk_psvd(At, k, tol, krylov_dim=K, start=cuda(q1), **kw)
    assert st == 0, info
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    np.testing.assert_allclose(S, So, rtol=s_rtol)
    assert angle_err(V, Vo) <= v_tol
    assert angle_err(U, Uo) <= v_tol
    # true residuals of the GPU triplets on the stored operator, in f64 on the CPU
    r1, r2 = oracle.residuals(op, U, S, V)
    assert max(r1.max(), r2.max()) <= res_tol * So[0], (r1.max(), r2.max())
    # sign convention
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(k)] > 0)
    return U, S, V, info


def rank_product(m, n, r, seed):
    g = synth.rng(seed)
    return g.standard_normal((m, r)) @ g.standard_normal((r, n)) + 1e-12 * g.standard_normal((m, n))


def test_psvd_dense_f64_2000x1000_prescribed_spectrum():
    """Dense f64 2000 x 1000, sigma_i = 0.9^i, top 10, Krylov dimension 30, tol 1e-10."""
    w = synth.WORKLOADS["dense_f64_2000x1000_top10"]
    sig = synth.sigma_geometric(w["n"], w["q"])
    A, U0, V0 = synth.prescribed_spectrum(w["m"], w["n"], sig, w["seed"])
    op, At, _ = dense_pair(A, "f64")
    q1 = synth.start_vector(w["m"], w["seed"])
    U, S, V, info = _compare_psvd(op, At, A, w["k"], w["K"], w["tol"], q1, s_rtol=1e-10, v_tol=1e-8, res_tol=1e-10)
    np.testing.assert_allclose(S, sig[: w["k"]], rtol=1e-10)
    assert angle_err(V, V0[:, : w["k"]]) <= 1e-8


@pytest.mark.parametrize("passes", [0, 1, 2])
def test_reorthogonalization_modes_match_oracle(passes):
    """Each Gram-Schmidt rule (0 = second pass only under cancellation, 1 = one pass as printed,
    2 = two passes) on both sides: the partial SVD and the rank agree with the oracle's."""
    sig = synth.sigma_geometric(350, 0.9)
    A, _, _ = synth.prescribed_spectrum(800, 350, sig, seed=31)
    q1 = synth.start_vector(800, 31)
    M = gk()
    At, qt = torch.from_numpy(A).cuda(), torch.from_numpy(q1).cuda()
    U, S, V, st, info = M.gk_psvd(At, 8, 1e-10, krylov_dim=24, reorth_passes=passes, start=qt)
    op = oracle.Operator.dense(A)
    Uo, So, Vo, io = oracle.psvd(op, 8, 24, q1, tol=1e-10, passes=passes, max_restarts=300)
    assert st == 0
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-10)
    assert abs(info["restarts"] - io["restarts"]) <= 1
    G = rank_product(800, 300, 40, 33)
    r, sig_g, st2, _ = M.gk_numrank(torch.from_numpy(G).cuda(), 1e-8, 200, reorth_passes=passes,
                                    start=torch.from_numpy(synth.start_vector(800, 2)).cuda(), want_sigma=True)
    r_o, kp_o, s_o = oracle.numrank(oracle.Operator.dense(G), synth.start_vector(800, 2), eps=1e-8, kmax=200,
                                    passes=passes)
    assert r == r_o == 40


@pytest.mark.parametrize("shape", [(9000, 300), (300, 9000)])
@pytest.mark.parametrize("passes", [0, 1, 2])
def test_reorthogonalization_modes_multiblock(passes, shape):
    """Vectors longer than 8192 entries take the multi-block Gram-Schmidt kernels (shorter ones
    the one-CTA kernel): each rule on a 9000-entry side agrees with the oracle's partial SVD."""
    m, n = shape
    sig = synth.sigma_geometric(min(m, n), 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=41)
    q1 = synth.start_vector(m, 41)
    M = gk()
    At, qt = torch.from_numpy(A).cuda(), torch.from_numpy(q1).cuda()
    U, S, V, st, info = M.gk_psvd(At, 8, 1e-10, krylov_dim=24, reorth_passes=passes, start=qt)
    Uo, So, Vo, io = oracle.psvd(oracle.Operator.dense(A), 8, 24, q1, tol=1e-10, passes=passes, max_restarts=300)
    assert st == 0
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-10)
    assert angle_err(V.cpu().numpy(), Vo) <= 1e-8
    assert abs(info["restarts"] - io["restarts"]) <= 1


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_psvd_reduced_precision_storage(dtype):
    """sigma_i = i^-1.5 spectrum stored in f32 / bf16; parity with the oracle on the stored bytes."""
    m, n, k, K = 3001, 1499, 12, 40
    sig = synth.sigma_power(n, 1.5)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=77, dtype=np.float64)
    op, At, A64 = dense_pair(A, dtype)
    q1 = synth.start_vector(m, 77)
    nf = np.linalg.norm(A64)
    floor = 64 * U32 * nf / np.sqrt(n)  # f32 accumulation floor of the Krylov relations
    gaps = np.abs(np.diff(sig[: k + 1])).min()
    _compare_psvd(op, At, A64, k, K, 1e-8, q1, s_rtol=1e-7, v_tol=max(1e-6, 10 * (1e-8 + floor) / gaps),
                  res_tol=1e-8 + 10 * floor)


def test_psvd_f16_with_scale():
    """f16 storage of A / s with the operator scale s: the same triplets as the oracle on the
    stored bytes times s (entries of A here are ~1e-6, below f16's normal range without it)."""
    m, n, k, K = 1200, 500, 8, 30
    sig = synth.sigma_power(n, 1.5) * 1e-4
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=78, dtype=np.float64)
    s = 2.0 ** -14
    h = np.asarray(A / s, dtype=np.float16)
    op = oracle.Operator.dense(None, dtype="f16", bits=h.view(np.uint16), scale=s)
    q1 = synth.start_vector(m, 78)
    A64 = h.astype(np.float64) * s
    nf = np.linalg.norm(A64)
    floor = 64 * U32 * nf / np.sqrt(n)
    Uo, So, Vo, io = oracle.psvd(op, k, K, q1, tol=1e-12, max_restarts=500)
    U, S, V, st, info = gk().gk_psvd(cuda(h), k, 1e-8, krylov_dim=K, start=cuda(q1), scale=s)
    assert st == 0
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-6)
    r1, r2 = oracle.residuals(op, U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy())
    assert max(r1.max(), r2.max()) <= (1e-8 + 10 * floor / So[0]) * So[0] * 1.01


def test_psvd_csr_planted():
    sigp = 100.0 * 0.95 ** np.arange(1, 11)
    op, A, d = _csr_pair(20011, 9973, 20, sigp, 21)
    q1 = synth.start_vector(20011, 21)
    _compare_psvd(op, A, None, 10, 30, 1e-8, q1, s_rtol=1e-9, v_tol=1e-5, res_tol=2e-8)


def test_psvd_wide_and_tiny_shapes():
    M = gk()
    g = synth.rng(31)
    for m, n, k, K in [(1, 1, 1, 1), (3, 1, 1, 1), (1, 4, 1, 1), (5, 5, 5, 5), (7, 3, 2, 3), (40, 300, 4, 12)]:
        A = g.standard_normal((m, n))
        U, S, V, st, info = M.gk_psvd(cuda(A), k, 1e-12, krylov_dim=K, start=cuda(synth.start_vector(m, 1)))
        assert st in (0, 2)
        np.testing.assert_allclose(S.cpu().numpy(), np.linalg.svd(A, compute_uv=False)[:k], rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("restarts", [0, 3])
def test_ritz_estimates_and_restarts_cycle_by_cycle(restarts):
    """The convergence test's quantity (max_{i<k} |beta_K X_{K,i}| / sigma_1) and the thick restart,
    cycle by cycle: with the same Krylov dimension, keep rule and restart budget, and tol 1e-14 (no
    cycle converges; sigma_i = i^-0.5 and K = 16 leave the estimate at ~8e-2 after one cycle and
    ~2e-4 after four), the GPU and the oracle run the same cycles; the Ritz values and the Ritz
    residual estimate agree after the budget (rounding only: ~1e-13 in the values; the estimate's
    last-row entries carry ~1e-15 absolute, ~1e-11 relative to it)."""
    sig = synth.sigma_power(1000, 0.5)
    A, _, _ = synth.prescribed_spectrum(2000, 1000, sig, seed=17, dtype=np.float64)
    op, At, _ = dense_pair(A, "f64")
    q1 = synth.start_vector(2000, 17)
    Uo, So, Vo, io = oracle.psvd(op, 10, 16, q1, tol=1e-14, max_restarts=restarts)
    U, S, V, st, info = gk().gk_psvd(At, 10, 1e-14, krylov_dim=16, start=cuda(q1), max_restarts=restarts)
    assert not io["converged"] and st == 1  # GK_NOT_CONVERGED: outputs hold the last Ritz triplets
    assert info["cycles"] == io["cycles"] == restarts + 1 and info["restarts"] == restarts
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-10)
    np.testing.assert_allclose(info["resid_est_max"], io["resid_est_max"], rtol=1e-6)
    assert angle_err(V.cpu().numpy()[:, :5], Vo[:, :5]) <= 1e-6


def test_psvd_of_the_transpose_swaps_the_factors():
    """psvd(A^T) = swap(psvd(A)): the same singular values with the left and right vectors
    exchanged (the method is shape-agnostic; here a tall and a wide operator)."""
    sig = synth.sigma_geometric(700, 0.9)
    A, _, _ = synth.prescribed_spectrum(1500, 700, sig, seed=41, dtype=np.float64)
    M = gk()
    U1, S1, V1, st1, _ = M.gk_psvd(cuda(A), 8, 1e-10, krylov_dim=30)
    U2, S2, V2, st2, _ = M.gk_psvd(cuda(A.T), 8, 1e-10, krylov_dim=30)
    assert st1 == st2 == 0
    np.testing.assert_allclose(S1.cpu().numpy(), sig[:8], rtol=1e-10)
    np.testing.assert_allclose(S2.cpu().numpy(), sig[:8], rtol=1e-10)
    # vectors to ~tol sigma_1 / gap (gap >= 0.1 sigma_8 here)
    assert angle_err(U1.cpu().numpy(), V2.cpu().numpy()) < 1e-7
    assert angle_err(V1.cpu().numpy(), U2.cpu().numpy()) < 1e-7


def test_psvd_zero_and_rank_deficient():
    M = gk()
    Z = torch.zeros((30, 20), dtype=torch.float64, device="cuda")
    U, S, V, st, info = M.gk_psvd(Z, 3, 1e-10, krylov_dim=8)
    assert torch.all(S == 0) and torch.isfinite(V).all() and torch.isfinite(U).all()
    g = synth.rng(2)
    A = g.standard_normal((40, 3)) @ g.standard_normal((3, 30))
    U, S, V, st, info = M.gk_psvd(cuda(A), 5, 1e-12, krylov_dim=10)
    s = np.linalg.svd(A, compute_uv=False)
    S = S.cpu().numpy()
    np.testing.assert_allclose(S[:3], s[:3], rtol=1e-12)
    assert np.all(S[3:] < 1e-12 * s[0]) and torch.isfinite(V).all()


def test_psvd_host_buffers_end_to_end():
    """Host (pinned) operator and outputs: the library copies in and out itself."""
    M = gk()
    sig = synth.sigma_geometric(300, 0.9)
    A, _, _ = synth.prescribed_spectrum(1200, 300, sig, seed=5, dtype=np.float32)
    Ah = torch.from_numpy(A).pin_memory()
    U, S, V, st, info = M.gk_psvd(Ah, 6, 1e-8, krylov_dim=20)
    assert st == 0 and U.device.type == "cpu"
    np.testing.assert_allclose(S.numpy(), sig[:6], rtol=1e-6)
    Ud, Sd, Vd, st2, _ = M.gk_psvd(Ah.cuda(), 6, 1e-8, krylov_dim=20)
    np.testing.assert_array_equal(S.numpy(), Sd.cpu().numpy())


def test_library_host_buffers():
    """gk_host_alloc memory: an operator and outputs in it give the device results bit for bit;
    freeing twice (or a foreign address) is rejected."""
    M = gk()
    sig = synth.sigma_geometric(256, 0.85)
    A, _, _ = synth.prescribed_spectrum(900, 256, sig, seed=6, dtype=np.float32)
    Ah = M.host_empty(A.shape, torch.float32)
    assert Ah.is_pinned() and Ah.data_ptr() % 4096 == 0
    Ah.copy_(torch.from_numpy(A))
    outs = (M.host_empty((5, 900), torch.float64), M.host_empty((5,), torch.float64),
            M.host_empty((5, 256), torch.float64))
    U, S, V, st, info = M.gk_psvd(Ah, 5, 1e-8, krylov_dim=18, out=outs)
    Ud, Sd, Vd, st2, _ = M.gk_psvd(Ah.cuda(), 5, 1e-8, krylov_dim=18)
    assert st == st2 == 0
    np.testing.assert_array_equal(S.numpy(), Sd.cpu().numpy())
    np.testing.assert_array_equal(U.numpy(), Ud.cpu().numpy())
    for t in (Ah,) + outs:
        M.host_free(t)
    with pytest.raises(ValueError):
        M.host_free(Ah)
    from paper_2104_10785_gb300 import gk as gkmod

    assert M.lib().gk_host_free(None) == gkmod.GK_INVALID_ARG


def test_invalid_arguments_are_rejected():
    M = gk()
    A = torch.ones((10, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(M.GKError):
        M.gk_psvd(A, 9, 1e-8)  # k > min(m, n)
    with pytest.raises(M.GKError):
        M.gk_psvd(A, 4, 1e-8, krylov_dim=4)  # no room to restart
    with pytest.raises(M.GKError):
        M.gk_psvd(A, 2, -1.0)
    with pytest.raises(M.GKError):
        M.gk_numrank(A, float("nan"))


def test_gpu_residuals_entry_point():
    sig = synth.sigma_geometric(200, 0.8)
    A, U0, V0 = synth.prescribed_spectrum(500, 200, sig, seed=9)
    M = gk()
    r1, r2 = M.gk_residuals(cuda(A), cuda(U0[:, :5]), cuda(sig[:5]), cuda(V0[:, :5]))
    assert r1.max().item() < 1e-13 and r2.max().item() < 1e-13
    Sp = sig[:5] * 1.001
    r1, r2 = M.gk_residuals(cuda(A), cuda(U0[:, :5]), cuda(Sp), cuda(V0[:, :5]))
    np.testing.assert_allclose(r1.cpu().numpy(), 0.001 * sig[:5], rtol=1e-9)


def test_bounded_device_wait_reports_timeout_and_context_survives():
    """A device wait on an mbarrier that nothing arrives at gives up after its limit and the
    host reads GK_TIMEOUT; the context stays usable for the next calls."""
    from paper_2104_10785_gb300 import gk as gkmod

    M = gk()
    assert M.wait_selftest(0) == gkmod.GK_TIMEOUT
    assert M.wait_selftest(200000) == gkmod.GK_TIMEOUT
    assert M.wait_selftest(-1) == gkmod.GK_INVALID_ARG
    A = np.random.default_rng(3).standard_normal((300, 200))
    x = np.random.default_rng(4).standard_normal(200)
    y = M.gk_matvec(cuda(A), cuda(x)).cpu().numpy()
    np.testing.assert_allclose(y, A @ x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_operator_reports_numerical(bad):
    """A NaN or Inf entry: the single-problem calls and the batched item return GK_NUMERICAL
    (no hang, no fault); the other problems of the batch are unaffected."""
    from paper_2104_10785_gb300 import gk as gkmod

    M = gk()
    A = synth.gaussian_product(200, 120, 6, 1e-6, seed=8, dtype=np.float64)
    A[17, 33] = bad
    At = cuda(A)
    st = M.gk_psvd(At, 3, 1e-8, krylov_dim=12, check=False)[3]
    assert st == gkmod.GK_NUMERICAL
    r, _, st2, _ = M.gk_numrank(At, 1e-6, 50, check=False)
    assert st2 == gkmod.GK_NUMERICAL
    good = synth.gaussian_product(220, 100, 6, 1e-9, seed=9, dtype=np.float64)
    out, stb, info = M.gk_psvd_batched([dict(A=At, k=3, krylov_dim=12), dict(A=cuda(good), k=3, krylov_dim=12)],
                                       check=False)
    assert out[0][3]["status"] == gkmod.GK_NUMERICAL and out[1][3]["status"] == 0
    np.testing.assert_allclose(out[1][1].cpu().numpy(), np.linalg.svd(good, compute_uv=False)[:3], rtol=1e-10)
