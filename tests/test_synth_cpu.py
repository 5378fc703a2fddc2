"""The seeded input recipes (synth/) do what the workload table states: shapes and ranges of
the batched family, exact prescribed spectra, the planted sparse structure, bf16 rounding."""
import numpy as np
import scipy.sparse as sp

import synth


def test_batched_shapes_follow_the_recipe():
    w = synth.WORKLOADS["batched_f32_512_rank5to64"]
    shapes = synth.batched_shapes(w["count"], w["seed"])
    assert len(shapes) == 512 and shapes == synth.batched_shapes(512, w["seed"])
    assert shapes[0][:2] == (784, 256) and shapes[1][:2] == (256, 784)
    for m, n, r in shapes[2:]:
        assert 256 <= m <= 4096 and 128 <= n <= m and 5 <= r <= 64
    assert all(5 <= r <= 64 for _, _, r in shapes[:2])


def test_prescribed_spectrum_is_exact():
    sig = synth.sigma_power(40, 1.5)
    A, U, V = synth.prescribed_spectrum(120, 60, sig, seed=3)
    np.testing.assert_allclose(U.T @ U, np.eye(40), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(40), atol=1e-13)
    np.testing.assert_allclose(np.linalg.svd(A, compute_uv=False)[:40], sig, rtol=1e-12)
    assert sig[0] == 1.0 and synth.sigma_geometric(3, 0.9)[0] == 0.9  # 1-based spectra


def test_gaussian_product_has_the_stated_rank():
    A = synth.gaussian_product(90, 70, 12, 0.0, seed=4, dtype=np.float64)
    s = np.linalg.svd(A, compute_uv=False)
    assert s[11] > 1e-6 * s[0] and s[12] < 1e-12 * s[0]


def test_sparse_planted_structure():
    sig = 100.0 * 0.95 ** np.arange(1, 6)
    d = synth.sparse_planted(3000, 1500, 4, sig, seed=5, usup=40, vsup=20, dtype=np.float64)
    m, n = d["shape"]
    A = sp.csr_matrix((d["vals"], d["colind"], d["rowptr"]), shape=(m, n))
    At = sp.csr_matrix((d["t_vals"], d["t_colind"], d["t_rowptr"]), shape=(n, m))
    assert abs(A.T - At).max() == 0  # the stored transpose is the transpose
    assert np.all(np.diff(d["rowptr"]) >= 4)  # 4 distinct background columns per row (plus planted)
    U, V = d["U"], d["V"]
    np.testing.assert_allclose(U.T @ U, np.eye(5), atol=1e-14)  # disjoint unit supports
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-14)
    assert np.all((U != 0).sum(axis=0) == 40) and np.all((V != 0).sum(axis=0) == 20)
    # the planted part is sum_i sigma_i u_i v_i^T on top of the background
    P = (U * sig[None, :]) @ V.T
    rows, cols = np.nonzero(P)
    bg = A.toarray()[rows, cols] - P[rows, cols]
    assert np.all(np.abs(bg) < 10)  # what remains at planted entries is background noise (N(0,1) or 0)


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2.0**-8, 1.0 + 3 * 2.0**-8, 1.0 + 2.0**-7 + 2.0**-9, -2.5, np.nan], np.float32)
    b = synth.to_bf16_bits(x)
    back = synth.bf16_bits_to_f32(b)
    assert back[0] == 1.0
    assert back[1] == 1.0  # a tie rounds to the even neighbour
    assert back[2] == 1.0 + 2.0**-6  # the tie above an odd neighbour rounds up
    assert back[3] == 1.0 + 2.0**-7  # below half an ulp rounds down
    assert back[4] == -2.5 and b[5] == 0x7FC0


def test_rsgd_data_follows_the_recipe():
    """The Algorithm 4 inputs: shapes and dtypes, the same bytes for the same seed, batches drawn
    without replacement inside a batch, labels -sign(x^T W* v) with a rank-r W*, start vectors
    around 2."""
    P, N, d1, d2, r, steps, b = 3, 200, 12, 9, 2, 4, 50
    out = synth.rsgd_data(P, N, d1, d2, r, steps, b, seed=7)
    X, Vd, y, W0, batches, q1, Ws = out
    assert X.shape == (P, N, d1) and Vd.shape == (P, N, d2) and y.shape == (P, N)
    assert W0.shape == (P, d1, d2) and batches.shape == (steps, P, b) and q1.shape == (P, d1)
    assert batches.dtype == np.int32 and X.dtype == np.float64
    again = synth.rsgd_data(P, N, d1, d2, r, steps, b, seed=7)
    for a, c in zip(out, again):
        np.testing.assert_array_equal(a, c)
    assert np.all((batches >= 0) & (batches < N))
    for t in range(steps):
        for p in range(P):
            assert len(set(batches[t, p].tolist())) == b
    for p in range(P):
        assert np.linalg.matrix_rank(Ws[p]) == r
        s = np.array([X[p][i] @ Ws[p] @ Vd[p][i] for i in range(N)])
        np.testing.assert_array_equal(y[p], np.where(s > 0, -1.0, 1.0))
    assert abs(q1.mean() - 2.0) < 0.2
    # zero steps: an empty batch array of the right shape
    assert synth.rsgd_data(P, N, d1, d2, r, 0, b, seed=7)[4].shape == (0, P, b)
