"""Algorithm 4 (fast Riemannian mini-batch gradient descent, Section 4): the oracle.

Test infrastructure: only tests/, the smoke check and bench.py's CPU baseline use this module;
the library never imports it.  Plain numpy in f64, each step in the algorithm's order:

  Gr = (1/b) sum_{i in B} y_i x_i v_i^T          (the mini-batch Euclidean gradient; the
                                                    similarity x^T W v has gradient x v^T)
  Gr = Gr - lam W                                  (printed sign; lam is a parameter)
  U_r S_r V_r^T = rank-r SVD of Gr (Algorithm 2)
  Z = U U^T Gr V V^T + (I - U U^T) Gr V V^T + U U^T Gr (I - V V^T)
                                                   (the projection onto the tangent space,
                                                    the Riemannian gradient equation)
  W = rank-r SVD of (W - eta Z), W = U S V^T       (the SVD retraction)

The inner rank-r SVD ("Algorithm 2") is read as k_inner Golub-Kahan steps from the start
vector q1 without restart, followed by the SVD of the projected bidiagonal matrix and the Ritz
vectors U_K X, V_K Y -- the restart-free cycle of the thick-restart solver (oracle.psvd with
max_restarts = 0), which is what the library's batched solver runs for it."""
import numpy as np

from . import Operator, psvd


def euclidean_gradient(X, Vd, y, idx, W, lam):
    """Gr = (1/b) sum_{i in idx} y_i x_i v_i^T - lam W (Algorithm 4, the gradient steps).
    X: N x d1, Vd: N x d2 (one sample per row), y: N, idx: the batch's b sample indices."""
    d1, d2 = W.shape
    G = np.zeros((d1, d2))
    for i in idx:
        G += y[i] * np.outer(X[i], Vd[i])
    return G / len(idx) - lam * W


def tangent_projection(G, U, V):
    """Z = P_U^H G P_V^H + P_U^V G P_V^H + P_U^H G P_V^V with P_X^H = X X^T and
    P_X^V = I - X X^T (the Riemannian gradient equation; U, V orthonormal columns)."""
    PUh = U @ U.T
    PVh = V @ V.T
    PUv = np.eye(U.shape[0]) - PUh
    PVv = np.eye(V.shape[0]) - PVh
    return PUh @ G @ PVh + PUv @ G @ PVh + PUh @ G @ PVv


def inner_svd(M, r, k_inner, q1):
    """Rank-r SVD of M by k_inner Golub-Kahan steps from q1, no restart (Algorithm 2's fixed
    number of steps, then the small SVD and the Ritz vectors).  Returns U (d1 x r), S, V."""
    U, S, V, _ = psvd(Operator.dense(np.ascontiguousarray(M, dtype=np.float64)), r, k_inner, q1, tol=1e-8,
                      max_restarts=0)
    return U, S, V


def retraction(U, S, V):
    """R_W(xi) = sum_i s_i u_i v_i^T from the first r triplets of W + xi (the SVD retraction)."""
    return (U * S[None, :]) @ V.T


def rsgd_step(X, Vd, y, idx, W, eta, lam, r, k_inner, q1):
    """One pass of Algorithm 4's loop body; returns the new W."""
    G = euclidean_gradient(X, Vd, y, idx, W, lam)
    Ur, _, Vr = inner_svd(G, r, k_inner, q1)
    Z = tangent_projection(G, Ur, Vr)
    U2, S2, V2 = inner_svd(W - eta * Z, r, k_inner, q1)
    return retraction(U2, S2, V2)


def rsgd(X, Vd, y, W0, batches, eta, lam, r, k_inner, q1):
    """Algorithm 4 from W0 over the given batches (steps x b sample indices)."""
    W = np.array(W0, dtype=np.float64)
    for idx in batches:
        W = rsgd_step(X, Vd, y, idx, W, eta, lam, r, k_inner, q1)
    return W
