"""Block Golub-Kahan with s start vectors on the GPU (gk_block_numrank: block products, the
blocks' Gram-Schmidt QR, the triangular factors and their 2-norm tests, the SVD of B) against
the oracle (oracle/block_gk.py) on the same operators and start blocks.

The library forms each block's QR column by column (two classical Gram-Schmidt passes against
every earlier column; a column that the passes reduce to rounding is replaced by a fresh
orthonormal direction) and takes the triangular factors as Q_{j+1}^T (A P_j) and
P_{j+1}^T (A^T Q_{j+1}); the oracle reorthogonalizes each block and factors it by Householder
QR.  In exact arithmetic both give the same B (the new columns are orthogonal to the earlier
blocks, and a rank-deficient block's completion lies in the null space the blocks have not
reached); the rounding differences are ~1e-15 sigma_1 (f64 and CSR f64 products in f64, dense
f32/bf16 block products in double-f32, exact to ~2^-47 of sum |a x|).  So block steps and ranks
are equal, and the singular values of B agree to 1e-10 of sigma_1 (margin over the Jacobi
SVD's own ~1e-14).

These tests have not yet run on a GPU: like tests/test_gpu_experimental.py they are skipped unless
GK_EXPERIMENTAL=1, until their first run on a GB300 shows the path green."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import block_gk as bgk

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("GK_EXPERIMENTAL") != "1",
                                 reason="block Golub-Kahan on the GPU: set GK_EXPERIMENTAL=1 for its first GPU run")]


def gk():
    import paper_2104_10785_gb300 as m

    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def stored(A, dtype):
    """(device tensor holding A in `dtype`, f64 copy of the stored values)."""
    if dtype == "f64":
        A64 = np.asarray(A, dtype=np.float64)
        return cuda(A64), A64
    if dtype == "f32":
        A32 = np.asarray(A, dtype=np.float32)
        return cuda(A32), A32.astype(np.float64)
    if dtype == "bf16":
        bits = synth.to_bf16_bits(np.asarray(A, dtype=np.float32))
        return cuda(bits.view(np.int16)).view(torch.bfloat16), synth.bf16_bits_to_f32(bits).astype(np.float64)
    raise ValueError(dtype)


def operator(kind, m, n, r, seed):
    if kind == "repeated":  # sigma = (5, 5, 5, 3, 3, 1, 1, 1): three distinct values, rank 8
        A, _, _ = synth.prescribed_spectrum(m, n, np.array([5.0, 5.0, 5.0, 3.0, 3.0, 1.0, 1.0, 1.0]), seed=seed,
                                            dtype=np.float64)
        return A
    return synth.gaussian_product(m, n, r, 0.0 if kind == "product" else 1e-7, seed=seed, dtype=np.float64)


def check_against_oracle(Ad, Q0, s, eps, kmax, res):
    rk, sig, steps, st, info = res
    r_or, sig_or, steps_or = bgk.block_numrank(Ad, Q0, eps=eps, kmax=kmax)
    assert st == 0
    assert steps == steps_or == info["steps"]
    assert rk == r_or
    sig = sig.cpu().numpy()
    assert sig.shape == (steps * s,) and info["kprime"] == steps * s
    np.testing.assert_allclose(sig, sig_or[: steps * s], rtol=0, atol=1e-10 * sig_or[0])
    np.testing.assert_allclose(sig[:rk], sig_or[:rk], rtol=1e-10)
    assert info["matvecs"] == s * (2 * steps + (1 if info["stop_reason"] == 2 else 0))
    return r_or


@pytest.mark.parametrize("kind,m,n,r,s,dtype,eps,expect,orth_f64", [
    ("repeated", 70, 40, 8, 3, "f64", 1e-8, 8, False),     # a block of 3 counts the multiplicities
    ("repeated", 70, 40, 8, 1, "f64", 1e-8, 3, False),     # one vector: one per distinct value
    ("product", 700, 500, 40, 4, "f64", 1e-8, 40, False),
    ("product", 700, 500, 40, 3, "f64", 1e-8, 40, True),   # the f64 Gram-Schmidt kernels
    ("product", 1500, 1200, 30, 1, "f64", 1e-8, 30, False),
    ("product", 2000, 900, 100, 32, "f64", 1e-8, 100, False),  # the largest block
    ("noisy", 3000, 1000, 40, 5, "bf16", 1e-2, 40, False),  # bf16 storage floor ~3e-4 sigma_1 < eps
    ("noisy", 20000, 1500, 60, 8, "f32", 1e-5, 60, False),  # left vectors past the one-CTA size
])
def test_block_rank_matches_oracle(kind, m, n, r, s, dtype, eps, expect, orth_f64):
    A = operator(kind, m, n, r, seed=m + n + s)
    At, Ad = stored(A, dtype)
    Q0 = synth.rng(s + m).standard_normal((m, s))
    res = gk().gk_block_numrank(At, s, eps, start=cuda(Q0), want_sigma=True, orth_f64=orth_f64)
    assert check_against_oracle(Ad, Q0, s, eps, 0, res) == expect
    assert res[0] == expect


def test_block_rank_csr_matches_oracle():
    """CSR f64 (products one column at a time, in f64), eight block steps of a full-rank operator."""
    import scipy.sparse as sp

    m, n, s = 2003, 1499, 4
    d = synth.sparse_planted(m, n, 12, 10.0 * 0.9 ** np.arange(1, 6), 11, usup=200, vsup=100, dtype=np.float64)
    Ad = sp.csr_matrix((d["vals"], d["colind"], d["rowptr"]), shape=(m, n)).toarray()
    M = gk()
    A = M.CSR(m, n, cuda(d["rowptr"]), cuda(d["colind"]), cuda(d["vals"]), cuda(d["t_rowptr"]), cuda(d["t_colind"]),
              cuda(d["t_vals"]))
    Q0 = synth.rng(12).standard_normal((m, s))
    res = M.gk_block_numrank(A, s, 1e-8, 8, start=cuda(Q0), want_sigma=True)
    assert check_against_oracle(Ad, Q0, s, 1e-8, 8, res) == 32
    assert res[2] == 8 and res[4]["stop_reason"] == 0


@pytest.mark.parametrize("m,n,s", [(30, 20, 4), (50, 20, 20), (20, 30, 4), (21, 20, 4), (24, 24, 8)])
def test_blocks_filling_the_space_give_lapack_singular_values(m, n, s):
    """When the right blocks fill min(m, n) columns, P spans A's row space and sigma(B) = sigma(A);
    a last left block with more columns than R^m has room for (wide, square, m just above n) gets
    zero columns for the excess (the fresh completions find no direction), whose entries of
    S_{k+1} are zero."""
    A = synth.rng(m + s).standard_normal((m, n))
    Q0 = synth.rng(s).standard_normal((m, s))
    rk, sig, steps, st, info = gk().gk_block_numrank(cuda(A), s, 1e-8, start=cuda(Q0), want_sigma=True)
    assert st == 0 and steps * s == min(m, n) and rk == min(m, n)
    np.testing.assert_allclose(sig.cpu().numpy(), np.linalg.svd(A, compute_uv=False), rtol=1e-12)


def test_seeded_start_block_is_algorithm_1s_draw():
    """start = None: column c is Algorithm 1's start vector (Philox4x32-10 + Box-Muller) with seed + c,
    the stream the oracle draws."""
    m, n, s, seed = 900, 700, 3, 987654321
    A = synth.gaussian_product(m, n, 25, 0.0, seed=3, dtype=np.float64)
    Q0 = np.stack([oracle.start_vector(seed + c, m) for c in range(s)], axis=1)
    M = gk()
    r1, s1, k1, st1, _ = M.gk_block_numrank(cuda(A), s, 1e-8, seed=seed, want_sigma=True)
    r2, s2, k2, st2, _ = M.gk_block_numrank(cuda(A), s, 1e-8, start=cuda(Q0), want_sigma=True)
    assert st1 == st2 == 0 and r1 == r2 == 25 and k1 == k2
    np.testing.assert_allclose(s1.cpu().numpy()[:25], s2.cpu().numpy()[:25], rtol=1e-12)
    r_or, sig_or, k_or = bgk.block_numrank(A, Q0, eps=1e-8)
    assert r_or == 25 and k_or == k1


def test_host_operator_start_and_sigma():
    """Host operand, start block and sigma: the library stages the copies; same results as the
    device call."""
    m, n, s = 600, 400, 4
    A = synth.gaussian_product(m, n, 18, 0.0, seed=21, dtype=np.float64)
    Q0 = synth.rng(22).standard_normal((m, s))
    M = gk()
    rh, sh, kh, sth, _ = M.gk_block_numrank(torch.from_numpy(A).pin_memory(), s, 1e-8, start=torch.from_numpy(Q0),
                                            want_sigma=True)
    rd, sd, kd, std, _ = M.gk_block_numrank(cuda(A), s, 1e-8, start=cuda(Q0), want_sigma=True)
    assert sth == std == 0 and rh == rd == 18 and kh == kd
    assert sh.device.type == "cpu"
    np.testing.assert_allclose(sh.numpy(), sd.cpu().numpy(), rtol=0, atol=1e-12 * sd[0].item())


@pytest.mark.parametrize("block_gs", [False, True])
def test_caller_workspace_of_the_queried_size(block_gs):
    """A caller workspace of exactly gk_block_numrank_workspace() bytes gives the same result (with
    the block Gram-Schmidt's buffers when it is asked for)."""
    m, n, s = 800, 500, 4
    A = cuda(synth.gaussian_product(m, n, 22, 0.0, seed=31, dtype=np.float64))
    Q0 = cuda(synth.rng(32).standard_normal((m, s)))
    M = gk()
    nbytes = M.gk_block_numrank_workspace(A, s, block_gs=block_gs)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    r1, s1, k1, st1, _ = M.gk_block_numrank(A, s, 1e-8, start=Q0, want_sigma=True, workspace=ws, block_gs=block_gs)
    r2, s2, k2, st2, _ = M.gk_block_numrank(A, s, 1e-8, start=Q0, want_sigma=True, block_gs=block_gs)
    assert st1 == st2 == 0 and r1 == r2 == 22 and k1 == k2
    np.testing.assert_array_equal(s1.cpu().numpy(), s2.cpu().numpy())
