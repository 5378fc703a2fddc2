"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws matrices and start vectors only; it holds none of the
method's arithmetic.  Both the CUDA path and the CPU oracle read the bytes it
produces.  Recipes (sizes as in the workloads they stand for):

  gaussian_product   A = G1 G2 + noise * N(0,1), G1 m x r, G2 r x n Gaussian,
                     formed in f64 and rounded to the storage type (the paper's
                     synthetic test matrices, Section 5: rank-l products).
  prescribed_spectrum A = U diag(sigma) V^T with U, V from QR of seeded
                     Gaussian matrices (diagonal of R made positive).
  sparse_planted     CSR with `per_row` distinct uniform random columns per row
                     (values N(0,1)) plus planted sigma_i u_i v_i^T with
                     disjoint random supports (u_i: 200 rows, v_i: 100 columns
                     at full size, scaled down for small cases).
  start_vector       q1 ~ N(2,1)^m (Algorithm 1).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2104107


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def start_vector(m: int, seed: int) -> np.ndarray:
    return 2.0 + rng(seed ^ 0x5EED).standard_normal(m)


def orthonormal(rows: int, cols: int, g: np.random.Generator) -> np.ndarray:
    Q, R = np.linalg.qr(g.standard_normal((rows, cols)))
    return Q * np.sign(np.diag(R))[None, :]


def gaussian_product(m: int, n: int, r: int, noise: float, seed: int, dtype=np.float32) -> np.ndarray:
    g = rng(seed)
    A = g.standard_normal((m, r)) @ g.standard_normal((r, n))
    if noise:
        A += noise * g.standard_normal((m, n))
    return A.astype(dtype)


def prescribed_spectrum(m: int, n: int, sigma: np.ndarray, seed: int, dtype=np.float64):
    """A = U diag(sigma) V^T, U m x p, V n x p orthonormal (p = len(sigma) <= min(m, n)).
    Returns (A, U, V) with U, V in f64."""
    g = rng(seed)
    p = len(sigma)
    U = orthonormal(m, p, g)
    V = orthonormal(n, p, g)
    A = (U * sigma[None, :]) @ V.T
    return A.astype(dtype), U, V


def sigma_geometric(p: int, q: float) -> np.ndarray:
    """sigma_i = q^i, i = 1..p (1-based, so sigma_1 = q)."""
    return q ** np.arange(1, p + 1, dtype=np.float64)


def sigma_power(p: int, e: float) -> np.ndarray:
    """sigma_i = i^-e, i = 1..p."""
    return np.arange(1, p + 1, dtype=np.float64) ** (-e)


def to_bf16_bits(A32: np.ndarray) -> np.ndarray:
    """Round f32 to bf16 (round to nearest even) and return the uint16 bit patterns."""
    u = np.ascontiguousarray(A32, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(A32)
    if nan.any():
        r[nan] = 0x7FC0
    return r


def bf16_bits_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def sparse_planted(m: int, n: int, per_row: int, sigma: np.ndarray, seed: int, usup: int = 200, vsup: int = 100,
                   dtype=np.float32):
    """CSR background (per_row distinct random columns per row, N(0,1) values) plus
    sum_i sigma_i u_i v_i^T with disjoint supports; duplicates summed.
    Returns dict(rowptr, colind, vals, t_rowptr, t_colind, t_vals, U, V)."""
    import scipy.sparse as sp

    g = rng(seed)
    cols = np.sort(g.integers(0, n, size=(m, per_row)), axis=1)
    dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1)
    for i in np.nonzero(dup)[0]:
        cols[i] = np.sort(g.choice(n, size=per_row, replace=False))
    rows = np.repeat(np.arange(m), per_row)
    vals = g.standard_normal(m * per_row)
    k = len(sigma)
    rperm = g.permutation(m)[: k * usup].reshape(k, usup)
    cperm = g.permutation(n)[: k * vsup].reshape(k, vsup)
    U = np.zeros((m, k))
    V = np.zeros((n, k))
    pr, pc, pv = [], [], []
    for i in range(k):
        u = g.standard_normal(usup)
        v = g.standard_normal(vsup)
        u /= np.linalg.norm(u)
        v /= np.linalg.norm(v)
        U[rperm[i], i] = u
        V[cperm[i], i] = v
        pr.append(np.repeat(rperm[i], vsup))
        pc.append(np.tile(cperm[i], usup))
        pv.append(sigma[i] * np.outer(u, v).reshape(-1))
    R = np.concatenate([rows] + pr)
    Cc = np.concatenate([cols.reshape(-1)] + pc)
    Vv = np.concatenate([vals] + pv)
    A = sp.coo_matrix((Vv, (R, Cc)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    A = A.astype(dtype)
    At = A.T.tocsr()
    At.sort_indices()
    return dict(rowptr=A.indptr.astype(np.int32), colind=A.indices.astype(np.int32), vals=A.data,
                t_rowptr=At.indptr.astype(np.int32), t_colind=At.indices.astype(np.int32), t_vals=At.data,
                U=U, V=V, shape=(m, n))


# ---------------------------------------------------------------------------
# Workload recipes (full size and reduced size) -- parameters only
# ---------------------------------------------------------------------------
def rsgd_data(P: int, N: int, d1: int, d2: int, r: int, steps: int, b: int, seed: int):
    """Paired data for P independent similarity-learning problems (the shape of the paper's
    Riemannian similarity-learning runs: d1 x d2 parameter matrices of rank r).  Problem p has
    samples x_i ~ N(0, I_d1), v_i ~ N(0, I_d2) (rows of X[p], Vd[p]) and labels
    y_i = -sign(x_i^T W*_p v_i) for a planted rank-r W*_p, so that lowering
    mean(y_i x_i^T W v_i) -- what the printed update W - eta Z does -- moves W towards W*_p.
    Also W0 ~ N(0, 1) (the algorithm's initialization), the mini-batches (steps x P x b sample
    indices, drawn without replacement within a batch), one start vector per problem for the
    inner SVDs (entries N(2, 1), as the library draws them) and W*.  All f64 / int32."""
    g = rng(seed)
    X = g.standard_normal((P, N, d1))
    Vd = g.standard_normal((P, N, d2))
    Wstar = np.stack([g.standard_normal((d1, r)) @ g.standard_normal((r, d2)) for _ in range(P)])
    s = np.stack([np.sum((X[p] @ Wstar[p]) * Vd[p], axis=1) for p in range(P)])  # x_i^T W* v_i
    y = -np.sign(s)
    y[y == 0] = -1.0
    W0 = g.standard_normal((P, d1, d2))
    batches = np.zeros((steps, P, b), dtype=np.int64)
    for t in range(steps):
        for p in range(P):
            batches[t, p] = g.choice(N, size=b, replace=False)
    q1 = 2.0 + g.standard_normal((P, d1))
    return X, Vd, y, W0, batches.astype(np.int32), q1, Wstar


WORKLOADS = {
    # dense f64, prescribed spectrum sigma_i = 0.9^i, top-10, Krylov 30, tol 1e-10
    "dense_f64_2000x1000_top10": dict(kind="spectrum", m=2000, n=1000, q=0.9, k=10, K=30, tol=1e-10,
                                      dtype="f64", seed=BASE_SEED + 1),
    # dense f32 rank-200 product + 1e-7 noise, numerical rank at eps = 1e-5 (relative)
    "dense_f32_50000x20000_rank200": dict(kind="product", m=50000, n=20000, r=200, noise=1e-7, eps=1e-5,
                                          dtype="f32", seed=BASE_SEED + 2),
    # CSR f32 1e6 x 5e5, 20 nnz/row + planted rank 50 (sigma_i = 100 * 0.95^i), top-50, tol 1e-8
    "csr_f32_1000000x500000_top50": dict(kind="sparse", m=1_000_000, n=500_000, per_row=20, k=50, K=100,
                                         tol=1e-8, dtype="f32", seed=BASE_SEED + 3),
    # batched: 512 dense f32 problems, m ~ U[256, 4096], n ~ U[128, m], plus 784 x 256 and 256 x 784,
    # rank r ~ U{5..64} products + 1e-6 noise; rank at eps = 1e-5, then the top-r triplets at tol 1e-8
    "batched_f32_512_rank5to64": dict(kind="batched", count=512, eps=1e-5, tol=1e-8, dtype="f32", seed=BASE_SEED + 5),
    # dense bf16 1e5 x 4e4, sigma_i = i^-1.5, top-100, tol 1e-8
    "dense_bf16_100000x40000_top100": dict(kind="spectrum_pow", m=100000, n=40000, e=1.5, k=100, K=200,
                                           tol=1e-8, dtype="bf16", seed=BASE_SEED + 4),
    # Algorithm 4: 64 similarity-learning problems at the paper's 784 x 256 shape, rank 5, 2048 paired
    # samples each (planted rank-5 similarity), mini-batch 256, eta 50, lam 0, inner Golub-Kahan steps 20
    "rsgd_f64_64x784x256_rank5": dict(kind="rsgd", P=64, N=2048, d1=784, d2=256, r=5, b=256, eta=50.0, lam=0.0,
                                      k_inner=20, dtype="f64", seed=BASE_SEED + 6),
}


# ---------------------------------------------------------------------------
# Full-size generators on the GPU (torch), same recipes; used by the benchmark
# and the full-size tests.  They draw with torch's CUDA generator, so their
# bytes differ from the NumPy recipes above; every consumer reads the bytes.
# ---------------------------------------------------------------------------
def torch_gaussian_product(m: int, n: int, r: int, noise: float, seed: int, device="cuda", block: int = 8192):
    """f32 A = G1 G2 + noise N(0,1), formed in f64 by row blocks and rounded (RNE)."""
    import torch

    g = torch.Generator(device=device).manual_seed(seed)
    G1 = torch.randn(m, r, generator=g, device=device, dtype=torch.float64)
    G2 = torch.randn(r, n, generator=g, device=device, dtype=torch.float64)
    A = torch.empty(m, n, device=device, dtype=torch.float32)
    for i in range(0, m, block):
        blk = G1[i:i + block] @ G2
        if noise:
            blk += noise * torch.randn(blk.shape, generator=g, device=device, dtype=torch.float64)
        A[i:i + block] = blk.to(torch.float32)
    return A


def torch_prescribed_spectrum(m: int, n: int, sigma, seed: int, device="cuda", block: int = 4096, keep_top: int = 0):
    """f32 A = U diag(sigma) V^T with U (m x n), V (n x n) from f32 QR of seeded Gaussians
    (diag R > 0), formed by row blocks without TF32.  Returns (A, U[:, :keep_top], V[:, :keep_top])."""
    import torch

    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        g = torch.Generator(device=device).manual_seed(seed)
        p = len(sigma)
        U, R = torch.linalg.qr(torch.randn(m, p, generator=g, device=device, dtype=torch.float32))
        U *= torch.sign(torch.diagonal(R))[None, :]
        del R
        V, R = torch.linalg.qr(torch.randn(n, p, generator=g, device=device, dtype=torch.float32))
        V *= torch.sign(torch.diagonal(R))[None, :]
        del R
        s = torch.as_tensor(np.asarray(sigma), device=device, dtype=torch.float32)
        A = torch.empty(m, n, device=device, dtype=torch.float32)
        Vt = V.T.contiguous()
        for i in range(0, m, block):
            A[i:i + block] = (U[i:i + block] * s[None, :]) @ Vt
        top = (U[:, :keep_top].double().clone(), V[:, :keep_top].double().clone()) if keep_top else (None, None)
        del U, V, Vt
        return A, top[0], top[1]
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32


def batched_shapes(count: int, seed: int):
    """(m, n, r) of a batch: m ~ U[256, 4096], n ~ U[128, m], r ~ U{5..64}; the first two problems
    are the 784 x 256 and 256 x 784 shapes of the similarity-learning setting."""
    g = rng(seed)
    out = [(784, 256, int(g.integers(5, 65))), (256, 784, int(g.integers(5, 65)))]
    while len(out) < count:
        m = int(g.integers(256, 4097))
        n = int(g.integers(128, m + 1))
        out.append((m, n, int(g.integers(5, 65))))
    return out[:count]


def torch_batched_products(shapes, noise: float, seed: int, device="cuda", fast: bool = False):
    """Dense f32 operators G1 G2 + noise N(0,1) (formed in f64, or in f32 with fast=True) for each
    (m, n, r); each stored with its row stride rounded up to a multiple of 4 elements (16-byte
    rows); returns views m x n."""
    import torch

    g = torch.Generator(device=device).manual_seed(seed)
    dt = torch.float32 if fast else torch.float64
    mats = []
    for (m, n, r) in shapes:
        G1 = torch.randn(m, r, generator=g, device=device, dtype=dt)
        G2 = torch.randn(r, n, generator=g, device=device, dtype=dt)
        A = G1 @ G2
        if noise:
            A += noise * torch.randn(m, n, generator=g, device=device, dtype=dt)
        ld = (n + 3) // 4 * 4
        buf = torch.zeros(m, ld, device=device, dtype=torch.float32)
        buf[:, :n] = A.to(torch.float32)
        mats.append(buf[:, :n])
    return mats
