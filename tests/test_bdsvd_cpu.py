"""The bidiagonal SVD's step and row functions (paper_2104_10785_gb300/csrc/gk_bdsvd.cuh: the
Golub-Kahan SVD step with a Wilkinson shift and the zero-diagonal chases), compiled for the host
by g++ and driven as the GPU kernel drives them (tests/native/bdsvd_host.cpp), against LAPACK's
singular values and the definition of an SVD: B = X diag(sigma) Y^T with X, Y orthogonal and
sigma descending.  Bounds: backward-stable rotations give |sigma_i - sigma_i(B)| <= c n eps ||B||
and orthogonality to c n eps; the tests allow 1e-13 ||B|| (values) and 2e-13 (reconstruction and
orthogonality) at n <= 300."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bdsvd(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("bdsvd") / "bdsvd_host.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                    os.path.join(HERE, "native", "bdsvd_host.cpp")], check=True)
    L = C.CDLL(out)
    P = C.POINTER(C.c_double)
    L.bd_svd_host.argtypes = [P, P, C.c_int, P, P, P, C.POINTER(C.c_int), C.POINTER(C.c_int * 2)]
    L.bd_svd_host.restype = C.c_int

    def run(d, e):
        n = len(d)
        d = np.ascontiguousarray(d, dtype=np.float64)
        e = np.ascontiguousarray(e if n > 1 else [0.0], dtype=np.float64)
        s, X, Y = np.zeros(n), np.zeros(n * n), np.zeros(n * n)
        steps = C.c_int(0)
        chases = (C.c_int * 2)()
        rc = L.bd_svd_host(d.ctypes.data_as(P), e.ctypes.data_as(P), n, s.ctypes.data_as(P), X.ctypes.data_as(P),
                           Y.ctypes.data_as(P), C.byref(steps), C.byref(chases))
        run.chases = (chases[0], chases[1])
        return rc, s, X.reshape(n, n).T, Y.reshape(n, n).T, steps.value

    return run


def check(run, d, e):
    n = len(d)
    B = np.diag(d) + (np.diag(e, 1) if n > 1 else 0.0)
    rc, s, X, Y, steps = run(d, e)
    assert rc == 0
    nb = max(np.abs(B).max(), 1e-300)
    assert np.all(s >= 0) and np.all(np.diff(s) <= 0)
    assert np.abs(s - np.linalg.svd(B, compute_uv=False)).max() <= 1e-13 * nb
    assert np.linalg.norm(B - X @ np.diag(s) @ Y.T) <= 2e-13 * nb * max(1.0, np.sqrt(n) / 4)
    assert np.linalg.norm(X.T @ X - np.eye(n)) <= 2e-13 * max(1.0, np.sqrt(n) / 4)
    assert np.linalg.norm(Y.T @ Y - np.eye(n)) <= 2e-13 * max(1.0, np.sqrt(n) / 4)
    return steps


@pytest.mark.parametrize("n", [1, 2, 3, 10, 50, 171, 300])
def test_random_bidiagonal(bdsvd, n):
    g = np.random.default_rng(n)
    steps = check(bdsvd, g.standard_normal(n), g.standard_normal(max(n - 1, 0)))
    assert steps <= 4 * n + 10  # about two steps per singular value


def test_graded_clustered_and_toeplitz(bdsvd):
    n = 120
    check(bdsvd, 10.0 ** (-np.arange(n) / 10), 10.0 ** (-np.arange(n - 1) / 10))
    check(bdsvd, np.ones(80), 1e-9 * np.ones(79))   # a tight cluster at 1
    check(bdsvd, np.ones(80), np.ones(79))          # values 2 cos(k pi / 161): a smooth spectrum


def test_zero_entries(bdsvd):
    """Zero diagonal entries (first, inside, last: the chases), zero off-diagonal entries (a split
    from the start), an all-zero diagonal, and the zero matrix."""
    g = np.random.default_rng(7)
    d = g.standard_normal(60)
    d[[0, 17, 59]] = 0.0
    check(bdsvd, d, g.standard_normal(59))
    assert bdsvd.chases[1] > 0  # the zero-diagonal chases ran (the general rotation form)
    e = g.standard_normal(59)
    e[[5, 30]] = 0.0
    check(bdsvd, g.standard_normal(60), e)
    check(bdsvd, np.zeros(20), np.ones(19))
    check(bdsvd, np.zeros(6), np.zeros(5))


def test_golub_kahan_bidiagonal_of_a_power_law_operator(bdsvd):
    """The projected matrix of an actual Golub-Kahan run (upper form, f64, full reorthogonalization)
    on A = U diag(i^-1.5) V^T: its singular values approximate A's leading ones."""
    g = np.random.default_rng(3)
    m, n, K = 400, 300, 60
    U, _ = np.linalg.qr(g.standard_normal((m, n)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    A = (U * np.arange(1, n + 1) ** -1.5) @ V.T
    P = np.zeros((n, K))
    Q = np.zeros((m, K))
    d, e = np.zeros(K), np.zeros(K - 1)
    p = A.T @ np.full(m, 2.0)
    P[:, 0] = p / np.linalg.norm(p)
    for j in range(K):
        q = A @ P[:, j] - (e[j - 1] * Q[:, j - 1] if j else 0.0)
        q -= Q[:, :j] @ (Q[:, :j].T @ q)
        d[j] = np.linalg.norm(q)
        Q[:, j] = q / d[j]
        if j + 1 < K:
            p = A.T @ Q[:, j] - d[j] * P[:, j]
            p -= P[:, :j + 1] @ (P[:, :j + 1].T @ p)
            e[j] = np.linalg.norm(p)
            P[:, j + 1] = p / e[j]
    check(bdsvd, d, e)
    rc, s, X, Y, _ = bdsvd(d, e)
    np.testing.assert_allclose(s[:5], np.arange(1, 6) ** -1.5, rtol=1e-8)


def test_lower_bidiagonal_through_its_transpose(bdsvd):
    """gk_fsvd's route 1 reading: B_{k'+1,k'} (alpha on the diagonal, beta below it) padded with a
    zero column has an upper-bidiagonal transpose (alpha then 0 on the diagonal, beta above it);
    B^T = X' S Y'^T gives B = Y' S X'^T, so X' holds B's right vectors and Y' its left ones, with a
    zero last entry in every right vector of a nonzero value (the padding column is never used)."""
    g = np.random.default_rng(11)
    kp = 40
    alpha, beta = np.abs(g.standard_normal(kp)) + 0.1, np.abs(g.standard_normal(kp)) + 0.1
    K = kp + 1
    Bpad = np.zeros((K, K))
    Bpad[np.arange(kp), np.arange(kp)] = alpha
    Bpad[np.arange(1, K), np.arange(kp)] = beta
    rc, s, Xp, Yp, _ = bdsvd(np.append(alpha, 0.0), beta)
    assert rc == 0
    np.testing.assert_allclose(s, np.linalg.svd(Bpad, compute_uv=False), rtol=0, atol=1e-13 * s[0])
    assert np.linalg.norm(Bpad - Yp @ np.diag(s) @ Xp.T) <= 1e-13 * s[0] * K
    assert np.all(np.abs(Xp[K - 1, :kp]) <= 1e-13)


def test_no_access_outside_the_kernels_buffers_under_sanitizers(tmp_path):
    """The step and row functions, built with AddressSanitizer and UndefinedBehaviorSanitizer and
    driven over orders 1..64 (random, zero diagonal entries, splits, graded, clustered;
    tests/native/bdsvd_fuzz.cpp): no access outside d, e (n entries) and the n rotations a side
    that the GPU kernel gives each step, no undefined behaviour, every call finished."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "bdsvd_fuzz")
    build = subprocess.run([cxx, "-O1", "-g", "-std=c++17", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                            "-o", exe, os.path.join(HERE, "native", "bdsvd_fuzz.cpp"),
                            os.path.join(HERE, "native", "bdsvd_host.cpp")], capture_output=True, text=True)
    if build.returncode != 0:
        pytest.skip("the compiler has no sanitizer runtime: " + build.stderr.strip().splitlines()[-1][:200])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0")
    out = subprocess.run([exe, "64"], capture_output=True, text=True, env=env)
    assert out.returncode == 0, out.stdout + out.stderr
    assert int(out.stdout.split()[-1]) == 64 * 5
