"""Pins of the Algorithm 4 oracle (oracle/rsgd.py) against facts fixed independently of it:
the tangent projection's algebra (idempotent, orthogonal for the trace inner product, the
identity on tangent vectors, zero on the normal part), its closed form when U, V are exact
singular vectors (the rank-r truncation, Eckart-Young), the gradient as the derivative of the
mini-batch objective (central differences are exact for a quadratic), the inner SVD against
LAPACK when the Krylov space is the whole space, and one full step in closed form."""
import numpy as np

import oracle
import synth
from oracle import rsgd


def orth(rows, cols, g):
    return np.linalg.qr(g.standard_normal((rows, cols)))[0]


def trunc(M, r):
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    return (U[:, :r] * S[:r]) @ Vt[:r]


def test_projection_with_exact_singular_vectors_is_the_truncation():
    g = np.random.default_rng(1)
    G = g.standard_normal((30, 20))
    U, S, Vt = np.linalg.svd(G, full_matrices=False)
    for r in (1, 3, 7):
        Z = rsgd.tangent_projection(G, U[:, :r], Vt[:r].T)
        np.testing.assert_allclose(Z, trunc(G, r), atol=1e-12)


def test_projection_algebra():
    g = np.random.default_rng(2)
    d1, d2, r = 30, 20, 4
    U, V = orth(d1, r, g), orth(d2, r, g)
    G = g.standard_normal((d1, d2))
    P = rsgd.tangent_projection(G, U, V)
    np.testing.assert_allclose(rsgd.tangent_projection(P, U, V), P, atol=1e-12)  # idempotent
    Iu, Iv = np.eye(d1) - U @ U.T, np.eye(d2) - V @ V.T
    np.testing.assert_allclose(Iu @ P @ Iv, 0.0, atol=1e-12)  # no normal component
    assert abs(np.sum((G - P) * P)) < 1e-10  # orthogonal for tr(A^T B)
    # tangent vectors U M V^T + U_p V^T + U V_p^T (U_p^T U = 0, V_p^T V = 0) are fixed, one term at a time
    Up = Iu @ g.standard_normal((d1, r))
    Vp = Iv @ g.standard_normal((d2, r))
    M = g.standard_normal((r, r))
    for T in (U @ M @ V.T, Up @ V.T, U @ Vp.T):
        np.testing.assert_allclose(rsgd.tangent_projection(T, U, V), T, atol=1e-12)
    # and the normal part is removed
    N = Iu @ g.standard_normal((d1, d2)) @ Iv
    np.testing.assert_allclose(rsgd.tangent_projection(N, U, V), 0.0, atol=1e-12)


def test_gradient_is_the_derivative_of_the_minibatch_objective():
    X, Vd, y, W0, batches, q1, _ = synth.rsgd_data(1, 300, 12, 9, 2, 1, 40, seed=3)
    X, Vd, y, W, idx = X[0], Vd[0], y[0], W0[0], batches[0, 0]
    lam = 0.3

    def f(W):  # the objective whose gradient the printed steps form: mean(y x^T W v) - lam/2 ||W||^2
        return np.mean([y[i] * X[i] @ W @ Vd[i] for i in idx]) - 0.5 * lam * np.sum(W * W)

    G = rsgd.euclidean_gradient(X, Vd, y, idx, W, lam)
    g = np.random.default_rng(4)
    for _ in range(3):
        E = g.standard_normal(W.shape)
        eps = 1e-3
        fd = (f(W + eps * E) - f(W - eps * E)) / (2 * eps)  # exact for a quadratic
        assert abs(fd - np.sum(G * E)) <= 1e-9 * max(1.0, abs(fd))


def test_inner_svd_with_the_whole_krylov_space_is_exact():
    g = np.random.default_rng(5)
    M = g.standard_normal((40, 24))
    U, S, V = rsgd.inner_svd(M, 5, 24, 2.0 + g.standard_normal(40))
    np.testing.assert_allclose(S, np.linalg.svd(M, compute_uv=False)[:5], rtol=1e-10)
    np.testing.assert_allclose(rsgd.retraction(U, S, V), trunc(M, 5), atol=1e-10)


def test_one_step_in_closed_form():
    """With exact inner SVDs a step is W1 = trunc_r(W0 - eta trunc_r(Gr)) (the projection of Gr
    onto its own top singular vectors is its truncation; the retraction is Eckart-Young)."""
    X, Vd, y, W0, batches, q1, _ = synth.rsgd_data(1, 200, 30, 20, 3, 1, 50, seed=6)
    eta, lam, r = 0.7, 0.1, 3
    W1 = rsgd.rsgd_step(X[0], Vd[0], y[0], batches[0, 0], W0[0], eta, lam, r, 20, q1[0])
    G = rsgd.euclidean_gradient(X[0], Vd[0], y[0], batches[0, 0], W0[0], lam)
    np.testing.assert_allclose(W1, trunc(W0[0] - eta * trunc(G, r), r), atol=1e-9)


def test_rsgd_recovers_the_planted_similarity():
    """Sanity on the synthetic recipe: the sign agreement of x^T W v with x^T W* v rises."""
    X, Vd, y, W0, batches, q1, Ws = synth.rsgd_data(1, 4000, 30, 20, 2, 40, 400, seed=7)

    def agree(W):
        return np.mean(np.sign(np.einsum("ni,ij,nj->n", X[0], W, Vd[0])) ==
                       np.sign(np.einsum("ni,ij,nj->n", X[0], Ws[0], Vd[0])))

    W = rsgd.rsgd(X[0], Vd[0], y[0], W0[0], batches[:, 0], 20.0, 0.0, 2, 20, q1[0])
    assert agree(W) > max(0.85, agree(W0[0]) + 0.2), (agree(W0[0]), agree(W))
