"""FP64 CPU oracle of the learned predictor: sketch features and the 35-256-256-2 MLP.

TEST INFRASTRUCTURE ONLY (like the rest of this package).  Plain NumPy, written from
the definitions the CUDA path documents:

  sketch_features: Y = A Omega, Omega (n x 32) with entry (j, c) = draw 32 j + c of the
      N(0,1) stream of the start-vector construction (Philox4x32-10 + Box-Muller, here the
      oracle's own implementation minus its +2 shift); the singular values of Y (LAPACK SVD
      as a step); features log(sigma_i / (sqrt(32) ||A||_F)), log ||A||_F, log m, log n.
  forward / loss / grad: standardize the inputs, two GELU layers (exact, erf), a linear
      output layer; loss 0.5 * mean over rows of the squared error of the standardized
      targets; gradients by the chain rule written out layer by layer.
  adam_step: one update of the Adam method (Kingma and Ba, ICLR 2015, Algorithm 1) with
      its bias-corrected moment estimates.
"""
from __future__ import annotations

import math

import numpy as np

from . import start_vector

S = 32
F = 35
H = 256
N_TRAINABLE = H * F + H + H * H + H + 2 * H + 2
N_PARAMS = N_TRAINABLE + F + F + 2 + 2


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + 2 * H].reshape(2, H); o += 2 * H
    b3 = p[o:o + 2]; o += 2
    xmu = p[o:o + F]; o += F
    xsd = p[o:o + F]; o += F
    ymu = p[o:o + 2]; o += 2
    ysd = p[o:o + 2]; o += 2
    return W1, b1, W2, b2, W3, b3, xmu, xsd, ymu, ysd


_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X, destandardize=True):
    W1, b1, W2, b2, W3, b3, xmu, xsd, ymu, ysd = unpack(params)
    Xs = (np.asarray(X, dtype=np.float64) - xmu) / xsd
    Z1 = Xs @ W1.T + b1
    A1 = gelu(Z1)
    Z2 = A1 @ W2.T + b2
    A2 = gelu(Z2)
    O = A2 @ W3.T + b3
    cache = (Xs, Z1, A1, Z2, A2, O)
    return (O * ysd + ymu if destandardize else O), cache


def loss_and_grad(params, X, Y):
    """0.5 * mean_b sum_o (O - Y~)^2 and its gradient w.r.t. the trainable parameters."""
    W1, b1, W2, b2, W3, b3, xmu, xsd, ymu, ysd = unpack(params)
    _, (Xs, Z1, A1, Z2, A2, O) = forward(params, X, destandardize=False)
    B = O.shape[0]
    Yt = (np.asarray(Y, dtype=np.float64) - ymu) / ysd
    D = O - Yt
    loss = 0.5 * np.sum(D * D) / B
    dO = D / B
    gW3 = dO.T @ A2
    gb3 = dO.sum(axis=0)
    dZ2 = (dO @ W3) * gelu_grad(Z2)
    gW2 = dZ2.T @ A1
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    gW1 = dZ1.T @ Xs
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def omega(seed: int, n: int):
    """Omega (n x 32): entry (j, c) is draw 32 j + c of the N(0,1) stream."""
    return (start_vector(seed, n * S) - 2.0).reshape(n, S)


def round_bf16(x):
    """x rounded to bf16 (round to nearest, ties to even), returned as f64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def sketch_features(A, seed: int, omega_bf16: bool = False):
    """The 35 features of A's sketch Y = A Omega.  omega_bf16: Omega rounded to bf16 first (the
    library's definition for bf16-stored operators, whose product runs on the tensor pipe)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    Om = omega(seed, n)
    Y = A @ (round_bf16(Om) if omega_bf16 else Om)
    s = np.linalg.svd(Y, compute_uv=False)
    s = np.concatenate([s, np.zeros(S - len(s))]) if len(s) < S else s
    nf = math.sqrt(float(np.sum(A * A)))
    ref = math.sqrt(S) * nf
    f = np.log(np.maximum(s, 1e-30 * ref) / ref)
    return np.concatenate([f, [math.log(nf), math.log(m), math.log(n)]])


def adam_step(p, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based), Kingma and Ba (ICLR 2015), Algorithm 1:
    m <- beta1 m + (1 - beta1) g;  v <- beta2 v + (1 - beta2) g^2;
    m^ = m / (1 - beta1^t);  v^ = v / (1 - beta2^t);  p <- p - lr m^ / (sqrt(v^) + eps).
    Returns (p, m, v) after the update, in f64."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m1 = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v1 = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m1 / (1.0 - beta1 ** t)
    vhat = v1 / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m1, v1
