"""Block Golub-Kahan bidiagonalization with s start vectors, and its rank estimate: the
oracle.  (An extension of Algorithm 1 and Algorithm 3 to blocks; the paper has the
single-vector form only.)

Test infrastructure: only tests/ use this module; the library never imports it.  Plain numpy
in f64, the steps in the order of Algorithm 1 with each vector replaced by an m x s or n x s
block and each normalization by a QR factorization (diag(R) >= 0):

  Q_1 R_0 = Q0                                  (the start block, orthonormalized)
  P_1 R_1 = A^T Q_1
  for j = 1, 2, ...:
      Q_{j+1} S_{j+1} = A P_j - Q_j R_j^T        (reorthogonalized against Q_1..Q_j)
      P_{j+1} R_{j+1} = A^T Q_{j+1} - P_j S_{j+1}^T   (reorthogonalized against P_1..P_j)

so that A [P_1 .. P_k] = [Q_1 .. Q_{k+1}] B with B the block lower bidiagonal matrix whose
diagonal blocks are R_j^T and subdiagonal blocks S_{j+1} ((k+1) s x k s), the block form of
Eq. 2.2.  A Krylov space of one vector holds one direction per distinct singular value, so
Algorithm 1 counts a singular value of multiplicity > 1 once; a block of s >= that
multiplicity holds all of its directions.  The sweep stops (the block form of Algorithm 1's
break test) when ||S_{j+1}||_2 <= eps * sigma~, sigma~ the running estimate of sigma_1 (the
largest block norm so far), or when the right block vanishes, ||R_{j+1}||_2 <= eps * sigma~
(the block form of the alpha break that also ends Algorithm 1), or when the next block would
exceed min(m, n) columns.
The rank (Algorithm 3 on blocks) is the number of singular values of B above eps * sigma_1(B).
block_fsvd is one cycle of the block form of Algorithm 2 (route 1, the SVD of B itself) with each
triplet's right residual from the recurrence (below).
"""
import numpy as np


def _qr_pos(W):
    """W = Q R with diag(R) >= 0 (LAPACK's Householder QR, signs fixed)."""
    Q, R = np.linalg.qr(W)
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn[None, :], R * sgn[:, None]


def _reorth(W, basis, passes):
    """Classical block Gram-Schmidt of W against the columns of `basis`, `passes` times."""
    for _ in range(passes):
        if basis.shape[1]:
            W = W - basis @ (basis.T @ W)
    return W


def block_gk(A, Q0, k, eps=0.0, passes=2):
    """Up to k block steps from the start block Q0 (m x s).  Returns (Q, P, B, steps): Q m x
    (steps+1) s, P n x steps s, B (steps+1) s x steps s with A P = Q B.  eps > 0 enables the
    break test (relative to the running sigma estimate)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    s = Q0.shape[1]
    Q1, _ = _qr_pos(np.asarray(Q0, dtype=np.float64))
    P1, R1 = _qr_pos(A.T @ Q1)
    Qs, Ps, Rs, Ss = [Q1], [P1], [R1], []
    sest = np.linalg.norm(R1, 2)
    steps = 1
    while True:
        Qb = np.hstack(Qs)
        W = _reorth(A @ Ps[-1] - Qs[-1] @ Rs[-1].T, Qb, passes)
        Qn, Sn = _qr_pos(W)
        Qs.append(Qn)
        Ss.append(Sn)
        snorm = np.linalg.norm(Sn, 2)
        sest = max(sest, snorm)
        if (eps > 0 and snorm <= eps * sest) or steps >= k or (steps + 1) * s > min(m, n):
            break
        Pb = np.hstack(Ps)
        Z = _reorth(A.T @ Qn - Ps[-1] @ Sn.T, Pb, passes)
        Pn, Rn = _qr_pos(Z)
        rnorm = np.linalg.norm(Rn, 2)
        if eps > 0 and rnorm <= eps * max(sest, rnorm):
            break  # the right block vanished (the block form of the alpha break)
        Ps.append(Pn)
        Rs.append(Rn)
        sest = max(sest, np.linalg.norm(Rn, 2))
        steps += 1
    B = np.zeros(((steps + 1) * s, steps * s))
    for j in range(steps):
        B[j * s:(j + 1) * s, j * s:(j + 1) * s] = Rs[j].T
        B[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = Ss[j]
    return np.hstack(Qs), np.hstack(Ps), B, steps


def block_numrank(A, Q0, eps=1e-8, kmax=0):
    """Rank estimate: the number of singular values of B above eps * sigma_1(B), with the block
    break test at the same eps.  kmax: block steps (0 = until the blocks fill min(m, n)).
    Returns (rank, singular values of B, steps)."""
    m, n = np.shape(A)
    s = Q0.shape[1]
    k = kmax if kmax > 0 else max(1, min(m, n) // s)
    _, _, B, steps = block_gk(A, Q0, k, eps=eps)
    sig = np.linalg.svd(B, compute_uv=False)
    return int(np.sum(sig > eps * sig[0])), sig, steps


def block_fsvd(A, Q0, steps, r, passes=2):
    """The r largest triplets from `steps` block steps (no break test): B = X diag(sigma) Y^T (the
    SVD of the (k+1)s x ks block lower bidiagonal B), U = Q X_r, V = P Y_r (the block form of
    Algorithm 2, route 1).  A V = U diag(sigma) holds by construction (A P = Q B).  The right
    residual follows from the next right block: A^T Q = P B^T + P_{k+1} R_{k+1} E^T (E picks the
    last block of Q; P_{k+1} R_{k+1} = A^T Q_{k+1} - P_k S_{k+1}^T, reorthogonalized), so
    A^T u_i - sigma_i v_i = P_{k+1} R_{k+1} x_i' with x_i' the last s entries of x_i and
    ||A^T u_i - sigma_i v_i|| = ||R_{k+1} x_i'||.  Returns (U, sigma, V, residuals)."""
    A = np.asarray(A, dtype=np.float64)
    s = Q0.shape[1]
    Q, P, B, st = block_gk(A, Q0, steps, eps=0.0, passes=passes)
    ks = st * s
    X, S, Yt = np.linalg.svd(B, full_matrices=False)
    r = min(r, ks)
    U = Q @ X[:, :r]
    V = P @ Yt[:r].T
    Qn, Sn, Pk = Q[:, ks:], B[ks:, ks - s:ks], P[:, ks - s:]
    Z = _reorth(A.T @ Qn - Pk @ Sn.T, P, passes)
    _, Rn = _qr_pos(Z)
    est = np.linalg.norm(Rn @ X[ks:, :r], axis=0)
    return U, S[:r], V, est
