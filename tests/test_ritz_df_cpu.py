"""The double-f32 Ritz-vector product (paper_2104_10785_gb300/csrc/gk_ritz_df.cuh), compiled for the
host (g++, no FMA contraction) and run row by row and column group by column group as the GPU grid
runs it, against the f64 product of the same (split) values.  Bound: each output within
2^-45 sum_k |q_ik x_kj| of the exact product (the double-f32 accumulation, renormalized every
four terms, keeps ~2^-46 of it; measured 2^-46.3 at K = 171 and 2^-47 at K = 500 in a NumPy
restatement of the same operations)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ritz(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("ritz") / "ritz_df_host.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", out,
                    os.path.join(HERE, "native", "ritz_df_host.cpp")], check=True)
    L = C.CDLL(out)
    P = C.POINTER(C.c_double)
    L.ritz_df_host.argtypes = [P, C.c_longlong, C.c_longlong, C.c_int, P, C.c_longlong, C.c_int, P, C.c_longlong]
    L.ritz_df_host.restype = None

    def run(Q, ldq, X, ncol):
        len_, K = Q.shape
        Qc = np.zeros((K, ldq))
        Qc[:, :len_] = Q.T
        Xc = np.ascontiguousarray(X.T)  # ncol x K: column c of X contiguous
        Cm = np.full((ncol, len_), np.nan)
        L.ritz_df_host(Qc.ctypes.data_as(P), ldq, len_, K, Xc.ctypes.data_as(P), K, ncol, Cm.ctypes.data_as(P), len_)
        return Cm.T

    return run


def split_exact(a):
    """The f64 value of the (hi, lo) f32 pair the copy holds for each entry."""
    hi = a.astype(np.float32)
    lo = (a - hi.astype(np.float64)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


@pytest.mark.parametrize("len_,K,ncol", [(1, 1, 1), (37, 5, 3), (1000, 30, 10), (777, 171, 100), (300, 500, 17)])
def test_double_f32_product_matches_f64(ritz, len_, K, ncol):
    g = np.random.default_rng(len_ + K)
    Q, _ = np.linalg.qr(g.standard_normal((len_, K))) if len_ >= K else (g.standard_normal((len_, K)), None)
    X = g.standard_normal((K, ncol))
    got = ritz(Q, len_ + (len_ % 3), X, ncol)
    Qe, Xe = split_exact(Q), split_exact(X)
    want = Qe @ Xe
    bound = 2.0**-45 * (np.abs(Qe) @ np.abs(Xe))
    assert np.all(np.abs(got - want) <= bound + 1e-300), np.max(np.abs(got - want) / (bound + 1e-300))
    # and the copy's own rounding (~2^-48 per entry) keeps it within 1e-13 of the f64 product
    assert np.max(np.abs(got - Q @ X)) <= 1e-13 * max(1.0, np.abs(Q @ X).max())


def test_cancellation_and_scales(ritz):
    """Outputs that cancel to ~1e-8 of their terms, and entries spanning 1e-12..1e12 (products well
    inside f32's range): the error stays relative to the sum of |terms|, not to the small result."""
    g = np.random.default_rng(9)
    K = 64
    Q = g.standard_normal((200, K))
    X = np.zeros((K, 2))
    X[:, 0] = g.standard_normal(K)
    X[:, 1] = -X[:, 0] * (1 + 1e-8 * g.standard_normal(K))
    got = ritz(Q, 200, X, 2)
    Qe, Xe = split_exact(Q), split_exact(X)
    bound = 2.0**-45 * (np.abs(Qe) @ np.abs(Xe))
    assert np.all(np.abs(got - Qe @ Xe) <= bound)
    Q2 = Q * 10.0 ** g.integers(-12, 12, size=(1, K))
    X2 = g.standard_normal((K, 3)) * 10.0 ** g.integers(-12, 12, size=(K, 1))
    got2 = ritz(Q2, 200, X2, 3)
    Qe2, Xe2 = split_exact(Q2), split_exact(X2)
    assert np.all(np.abs(got2 - Qe2 @ Xe2) <= 2.0**-45 * (np.abs(Qe2) @ np.abs(Xe2)))
