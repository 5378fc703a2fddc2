"""The opt-in kernels that have not yet run on a GPU, against the default paths they would replace.
Skipped unless GK_EXPERIMENTAL=1: each kernel's host-testable part is covered by the CPU tests
(tests/test_bdsvd_cpu.py, tests/test_ritz_df_cpu.py), and its first GPU run is this file.

  * GK_FLAG_BDSVD (k_bdsvd): the SVD of a restart-free cycle's bidiagonal B by Golub-Kahan SVD
    steps, against the cluster Jacobi: the same triplets (sigma 1e-10 relative to the planted
    values, vectors 1e-8) on f64 operators, one cycle and with restarts;
  * GK_FLAG_RITZ_DF (k_ritz_df): the Ritz vectors from the double-f32 basis copies (exact to
    ~2^-46 of sum |q x|, ~1e-14 here), against the f64 products: sigma 1e-10, vectors 1e-8;
  * GK_FLAG_SKETCH_TC (k_sketch_tc): the sketch on tcgen05 against mma.sync on the same bf16
    operator: both accumulate bf16 products in f32 in the tensor pipe, in different orders, so
    the features (logs of the sketch's singular values) agree to ~1e-5; 1e-4 is the bound;
  * GK_FLAG_BLOCK_F32 (k_acc_gemm_narrow for blocks of up to 16 vectors, its contraction split
    over slices summed by k_acc_reduce; k_acc_gemm's FAST instantiation above): the block rank
    with f32 block products against the oracle: the rank exactly, sigma(B) above the cut within
    1e-5 relative (f32 products carry ~2^-24 (34) sum |a x| per entry);
  * gk_block_fsvd against oracle/block_gk.block_fsvd, and with GK_FLAG_RITZ_DF (U, V from the
    double-f32 basis copies) against itself;
  * GK_FLAG_BLOCK_GS (the block Gram-Schmidt: k_bgs_dots, k_bgs_sub, k_ritz_df): the block rank
    against the oracle (rank-deficient blocks, the largest block, long left vectors, a full
    space, CSR) and gk_block_fsvd against the column-wise flow;
  * GK_FLAG_PROFILE in the block calls: phase times present, results unchanged.
The default block path (k_acc_gemm_narrow in double-f32, the block judge) is in
tests/test_gpu_start_block.py, gated the same way."""
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("GK_EXPERIMENTAL") != "1",
                                 reason="experimental kernels: set GK_EXPERIMENTAL=1 for their first GPU run")]


def gk():
    import paper_2104_10785_gb300 as m

    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def angle_err(X, Y):
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1
    return np.linalg.norm(X - Y * s[None, :], axis=0).max()


@pytest.mark.parametrize("m,n,k,K", [(2000, 1000, 10, 30), (1500, 700, 8, 171), (900, 1200, 5, 64)])
@pytest.mark.parametrize("flag", ["bdsvd", "ritz_df"])
def test_experimental_psvd_matches_the_default(m, n, k, K, flag):
    sig = synth.sigma_geometric(min(m, n), 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=m + K, dtype=np.float64)
    q1 = cuda(synth.start_vector(m, 3))
    At = cuda(A)
    M = gk()
    U1, S1, V1, st1, i1 = M.gk_psvd(At, k, 1e-10, krylov_dim=K, start=q1, **{flag: True})
    U2, S2, V2, st2, i2 = M.gk_psvd(At, k, 1e-10, krylov_dim=K, start=q1)
    assert st1 == st2 == 0
    np.testing.assert_allclose(S1.cpu().numpy(), sig[:k], rtol=1e-10)
    np.testing.assert_allclose(S1.cpu().numpy(), S2.cpu().numpy(), rtol=1e-10)
    assert angle_err(V1.cpu().numpy(), V2.cpu().numpy()) < 1e-8
    assert angle_err(U1.cpu().numpy(), U2.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("m,n", [(1000, 640), (1037, 777), (300, 64), (129, 4000)])
def test_tensor_core_sketch_matches_mma_sync(m, n):
    A = synth.gaussian_product(m, n, 20, 1e-3, seed=m + n, dtype=np.float32)
    At = cuda(synth.to_bf16_bits(A).view(np.int16)).view(torch.bfloat16)
    M = gk()
    f1 = M.gk_sketch_batched([At], seed=5).cpu().numpy()
    f2 = M.gk_sketch_batched([At], seed=5, tcgen05=True).cpu().numpy()
    np.testing.assert_allclose(f2, f1, rtol=0, atol=1e-4)


@pytest.mark.parametrize("m,n,k,r", [(2000, 1000, 60, 10), (700, 1500, 171, 20)])
def test_fsvd_route_1_with_bidiagonal_svd_matches_the_default(m, n, k, r):
    sig = synth.sigma_geometric(min(m, n), 0.9)
    A, _, _ = synth.prescribed_spectrum(m, n, sig, seed=m + k, dtype=np.float64)
    q1 = cuda(synth.start_vector(m, 5))
    M = gk()
    U1, S1, V1, st1, _ = M.gk_fsvd(cuda(A), k, r, route=1, start=q1, bdsvd=True)
    U2, S2, V2, st2, _ = M.gk_fsvd(cuda(A), k, r, route=1, start=q1)
    assert st1 == st2 == 0
    np.testing.assert_allclose(S1.cpu().numpy(), S2.cpu().numpy(), rtol=1e-12)
    assert angle_err(V1.cpu().numpy(), V2.cpu().numpy()) < 1e-9
    assert angle_err(U1.cpu().numpy(), U2.cpu().numpy()) < 1e-9


@pytest.mark.parametrize("dtype,m,n,r,s,eps", [("bf16", 3000, 1000, 40, 5, 1e-2), ("f32", 20000, 1500, 60, 8, 1e-5),
                                                ("f32", 5000, 1300, 50, 12, 1e-5), ("bf16", 2500, 900, 45, 20, 1e-2)])
def test_block_rank_with_f32_products(dtype, m, n, r, s, eps):
    """s <= 8 and s <= 16 take the narrow tiles (k_acc_gemm_narrow, 8 or 16 vectors per CTA), s = 20
    the 32-vector tile of k_acc_gemm's FAST instantiation."""
    from oracle import block_gk as bgk

    A = synth.gaussian_product(m, n, r, 1e-7, seed=m + n + s, dtype=np.float64)
    if dtype == "bf16":
        bits = synth.to_bf16_bits(A.astype(np.float32))
        At, Ad = cuda(bits.view(np.int16)).view(torch.bfloat16), synth.bf16_bits_to_f32(bits).astype(np.float64)
    else:
        A32 = A.astype(np.float32)
        At, Ad = cuda(A32), A32.astype(np.float64)
    Q0 = synth.rng(s + m).standard_normal((m, s))
    rk, sig, steps, st, info = gk().gk_block_numrank(At, s, eps, start=cuda(Q0), want_sigma=True, f32_products=True)
    r_or, sig_or, k_or = bgk.block_numrank(Ad, Q0, eps=eps)
    assert st == 0 and rk == r_or == r
    np.testing.assert_allclose(sig.cpu().numpy()[:r], sig_or[:r], rtol=1e-5)


@pytest.mark.parametrize("m,n,s,steps,r", [(400, 300, 4, 10, 12), (2000, 1200, 8, 12, 40), (300, 200, 1, 30, 5)])
def test_block_fsvd_matches_the_block_oracle(m, n, s, steps, r):
    """gk_block_fsvd against oracle/block_gk.block_fsvd on the same start block: values to 1e-10,
    vectors to 1e-8 (sign-aligned), residuals read from the recurrence to 1e-6 relative (they are
    differences of nearly equal quantities only for converged triplets, ~1e-13 sigma_1 absolute)."""
    from oracle import block_gk as bgk

    A = synth.gaussian_product(m, n, min(m, n), 1e-3, seed=m + s, dtype=np.float64)
    Q0 = synth.rng(m + steps).standard_normal((m, s))
    U, S, V, res, st, info = gk().gk_block_fsvd(cuda(A), s, steps, r, start=cuda(Q0))
    Uo, So, Vo, reso = bgk.block_fsvd(A, Q0, steps, r)
    assert st == 0 and info["steps"] == steps
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=1e-10)
    assert angle_err(V.cpu().numpy(), Vo) < 1e-8 and angle_err(U.cpu().numpy(), Uo) < 1e-8
    np.testing.assert_allclose(res.cpu().numpy(), reso, rtol=1e-6, atol=1e-13 * So[0])


@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_block_fsvd_ritz_vectors_in_double_f32(dtype):
    """gk_block_fsvd with GK_FLAG_RITZ_DF: U = Q X and V = P Y from the bases' double-f32 copies,
    against the f64 products: the values and residuals are the same numbers (they do not depend on
    U, V), the vectors agree to 1e-12 (the copies hold ~2^-48 of each entry, the products ~2^-46
    of sum |q x|)."""
    m, n, s, steps, r = 3000, 1400, 8, 10, 40
    A = synth.gaussian_product(m, n, min(m, n), 1e-3, seed=7, dtype=np.float64)
    if dtype == "bf16":
        At = cuda(synth.to_bf16_bits(A.astype(np.float32)).view(np.int16)).view(torch.bfloat16)
    else:
        At = cuda(A)
    Q0 = cuda(synth.rng(8).standard_normal((m, s)))
    M = gk()
    U1, S1, V1, r1, st1, _ = M.gk_block_fsvd(At, s, steps, r, start=Q0)
    U2, S2, V2, r2, st2, _ = M.gk_block_fsvd(At, s, steps, r, start=Q0, ritz_df=True)
    assert st1 == st2 == 0
    np.testing.assert_array_equal(S1.cpu().numpy(), S2.cpu().numpy())
    np.testing.assert_array_equal(r1.cpu().numpy(), r2.cpu().numpy())
    assert np.abs(U1.cpu().numpy() - U2.cpu().numpy()).max() <= 1e-12
    assert np.abs(V1.cpu().numpy() - V2.cpu().numpy()).max() <= 1e-12


@pytest.mark.parametrize("kind,m,n,r,s,dtype,eps", [
    ("product", 700, 500, 40, 4, "f64", 1e-8),     # rank-deficient blocks: fresh completions in the block QR
    ("product", 2000, 900, 100, 32, "f64", 1e-8),  # the largest block
    ("noisy", 20000, 1500, 60, 8, "f32", 1e-5),    # left vectors past the one-CTA size
    ("full", 60, 40, 40, 8, "f64", 1e-8),          # the blocks fill the space
])
def test_block_rank_with_block_gram_schmidt(kind, m, n, r, s, dtype, eps):
    """GK_FLAG_BLOCK_GS (reorthogonalized block Gram-Schmidt: k_bgs_dots, k_bgs_sub and the
    double-f32 Ritz product project each block against the earlier basis) against the oracle:
    the same steps and rank, sigma(B) within 1e-10 sigma_1 (tests/test_block_reading_cpu.py
    restates the flow)."""
    from oracle import block_gk as bgk

    if kind == "full":
        A = synth.rng(m * n).standard_normal((m, n))
    else:
        A = synth.gaussian_product(m, n, r, 0.0 if kind == "product" else 1e-7, seed=m + n + s, dtype=np.float64)
    if dtype == "f32":
        A32 = A.astype(np.float32)
        At, Ad = cuda(A32), A32.astype(np.float64)
    else:
        At, Ad = cuda(A), A
    Q0 = synth.rng(s + m).standard_normal((m, s))
    rk, sig, steps, st, info = gk().gk_block_numrank(At, s, eps, start=cuda(Q0), want_sigma=True, block_gs=True)
    r_or, sig_or, k_or = bgk.block_numrank(Ad, Q0, eps=eps)
    assert st == 0 and steps == k_or and rk == r_or == r
    np.testing.assert_allclose(sig.cpu().numpy(), sig_or[: steps * s], rtol=0, atol=1e-10 * sig_or[0])


def test_block_rank_csr_with_block_gram_schmidt():
    import scipy.sparse as sp

    from oracle import block_gk as bgk

    m, n, s = 2003, 1499, 4
    d = synth.sparse_planted(m, n, 12, 10.0 * 0.9 ** np.arange(1, 6), 11, usup=200, vsup=100, dtype=np.float64)
    Ad = sp.csr_matrix((d["vals"], d["colind"], d["rowptr"]), shape=(m, n)).toarray()
    M = gk()
    A = M.CSR(m, n, cuda(d["rowptr"]), cuda(d["colind"]), cuda(d["vals"]), cuda(d["t_rowptr"]), cuda(d["t_colind"]),
              cuda(d["t_vals"]))
    Q0 = synth.rng(12).standard_normal((m, s))
    rk, sig, steps, st, info = M.gk_block_numrank(A, s, 1e-8, 8, start=cuda(Q0), want_sigma=True, block_gs=True)
    r_or, sig_or, k_or = bgk.block_numrank(Ad, Q0, eps=1e-8, kmax=8)
    assert st == 0 and steps == k_or == 8 and rk == r_or
    np.testing.assert_allclose(sig.cpu().numpy(), sig_or[: steps * s], rtol=0, atol=1e-10 * sig_or[0])


@pytest.mark.parametrize("m,n,s,steps,r,dtype", [(2000, 1200, 8, 12, 40, "f64"), (3000, 1400, 8, 10, 40, "bf16")])
def test_block_fsvd_with_block_gram_schmidt(m, n, s, steps, r, dtype):
    """gk_block_fsvd with GK_FLAG_BLOCK_GS against the column-wise flow on the same start block:
    values to 1e-10, vectors to 1e-8, residuals to 1e-6 relative (1e-13 sigma_1 absolute)."""
    A = synth.gaussian_product(m, n, min(m, n), 1e-3, seed=m + s, dtype=np.float64)
    if dtype == "bf16":
        At = cuda(synth.to_bf16_bits(A.astype(np.float32)).view(np.int16)).view(torch.bfloat16)
    else:
        At = cuda(A)
    Q0 = cuda(synth.rng(m + steps).standard_normal((m, s)))
    M = gk()
    U1, S1, V1, r1, st1, _ = M.gk_block_fsvd(At, s, steps, r, start=Q0)
    U2, S2, V2, r2, st2, _ = M.gk_block_fsvd(At, s, steps, r, start=Q0, block_gs=True)
    assert st1 == st2 == 0
    S1n = S1.cpu().numpy()
    np.testing.assert_allclose(S2.cpu().numpy(), S1n, rtol=1e-10)
    assert angle_err(U2.cpu().numpy(), U1.cpu().numpy()) < 1e-8 and angle_err(V2.cpu().numpy(), V1.cpu().numpy()) < 1e-8
    np.testing.assert_allclose(r2.cpu().numpy(), r1.cpu().numpy(), rtol=1e-6, atol=1e-13 * S1n[0])


def test_block_calls_report_phase_times():
    """GK_FLAG_PROFILE in the block calls: CUDA-event times of the products (A P, A^T Q), the
    Gram-Schmidt, the small kernels and SVD, and (gk_block_fsvd) the Ritz vectors, all positive,
    and the same results as without it."""
    m, n, s = 3000, 1400, 8
    A = cuda(synth.gaussian_product(m, n, min(m, n), 1e-3, seed=17, dtype=np.float64))
    Q0 = cuda(synth.rng(18).standard_normal((m, s)))
    M = gk()
    r1, s1, k1, st1, i1 = M.gk_block_numrank(A, s, 1e-8, 6, start=Q0, want_sigma=True)
    r2, s2, k2, st2, i2 = M.gk_block_numrank(A, s, 1e-8, 6, start=Q0, want_sigma=True, profile=True)
    assert st1 == st2 == 0 and (r1, k1) == (r2, k2)
    np.testing.assert_array_equal(s1.cpu().numpy(), s2.cpu().numpy())
    assert i1["ms_matvec"] == 0.0
    assert min(i2["ms_matvec"], i2["ms_matvec_t"], i2["ms_orth"], i2["ms_small"]) > 0.0
    *_, st3, i3 = M.gk_block_fsvd(A, s, 6, 20, start=Q0, profile=True)
    assert st3 == 0 and min(i3["ms_matvec"], i3["ms_matvec_t"], i3["ms_orth"], i3["ms_small"], i3["ms_restart"]) > 0.0
