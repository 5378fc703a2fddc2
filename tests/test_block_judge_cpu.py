"""The block judge of block Golub-Kahan (paper_2104_10785_gb300/csrc/gk_block_judge.cuh, run on one
warp by k_block_judge), compiled for the host by g++ and run lane after lane as the warp runs it,
against LAPACK's 2-norm of the triangular factor and the break tests of Algorithm 1 with block
norms; the placement of T (left blocks) and T^T (right blocks) into B.  Bound: the norm within
4e-15 relative of numpy's (Jacobi on the scaled Gram matrix: eigenvalue error ~s eps lambda_max,
halved by the square root)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def judge(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("judge") / "block_judge_host.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                    os.path.join(HERE, "native", "block_judge_host.cpp")], check=True)
    L = C.CDLL(out)
    P = C.POINTER(C.c_double)
    L.block_judge_host.argtypes = [P, C.c_int, C.c_int, C.c_double, P, P, C.POINTER(C.c_int), P, C.c_longlong,
                                   C.c_int, C.c_int]
    L.block_judge_host.restype = C.c_int

    def run(raw, side=2, eps=0.0, sest=0.0, B=None, row0=0, col0=0):
        s = raw.shape[0]
        r = np.asfortranarray(raw, dtype=np.float64)
        se, nr, sw = C.c_double(sest), C.c_double(0.0), C.c_int(0)
        Bp, ldb = (None, 0) if B is None else (B.ctypes.data_as(P), B.shape[0])
        brk = L.block_judge_host(r.ctypes.data_as(P), s, side, eps, C.byref(se), C.byref(nr), C.byref(sw), Bp, ldb,
                                 row0, col0)
        return brk, se.value, nr.value, sw.value

    return run


@pytest.mark.parametrize("s", [1, 2, 3, 5, 8, 17, 32])
def test_norm_of_the_triangle_matches_lapack(judge, s):
    g = np.random.default_rng(s)
    for trial in range(5):
        raw = g.standard_normal((s, s))  # the strictly lower part must be ignored
        if trial == 1:
            raw[:, ::2] *= 1e-6           # graded columns
        if trial == 2 and s > 1:
            raw[:, 1] = 0.0               # a rank-deficient block (a completed column)
        if trial == 3:
            raw = raw * 1e-3 + np.triu(np.ones((s, s)))  # nearly rank one
        brk, sest, nrm, sweeps = judge(raw)
        want = np.linalg.norm(np.triu(raw), 2)
        assert brk == 0 and abs(nrm - want) <= 4e-15 * want, (trial, nrm, want)
        assert sest == nrm and 0 <= sweeps < 60


def test_scales_past_the_gram_range_and_special_blocks(judge):
    """Entries at 1e200 and 1e-200 (an unscaled T^T T would overflow or underflow), the zero block,
    and blocks holding inf or NaN (status 2)."""
    g = np.random.default_rng(1)
    raw = np.triu(g.standard_normal((6, 6)))
    want = np.linalg.norm(raw, 2)
    for sc in (1e200, 1e-200, 1e-300):
        brk, _, nrm, _ = judge(raw * sc)
        assert brk == 0 and abs(nrm / sc - want) <= 4e-15 * want, sc
    brk, sest, nrm, sweeps = judge(np.zeros((4, 4)), side=2, sest=3.0)
    assert brk == 0 and nrm == 0.0 and sest == 3.0 and sweeps == 0
    for bad in (np.inf, np.nan):
        r = raw.copy()
        r[1, 3] = bad
        brk, _, nrm, _ = judge(r, side=1, eps=1e-8, sest=1.0)
        assert brk == 2 and not np.isfinite(nrm), bad
    r = raw.copy()
    r[4, 0] = np.nan  # below the diagonal: not part of T
    assert judge(r)[0] == 0


def test_break_tests_of_the_three_sides(judge):
    """side 0 (left block S): sest grows first, break when ||S|| <= eps sest; side 1 (right block R):
    break when ||R|| <= eps max(sest, ||R||), sest grows only otherwise; side 2 (R_1): no test."""
    raw = np.diag([2.0, 1.0])  # ||T|| = 2
    assert judge(raw, side=0, eps=1e-8, sest=1.0)[:2] == (0, 2.0)
    assert judge(raw, side=0, eps=0.1, sest=30.0)[:2] == (1, 30.0)    # 2 <= 0.1 * 30
    assert judge(raw, side=0, eps=0.0, sest=1e300)[:2] == (0, 1e300)  # eps = 0: never breaks
    assert judge(raw, side=1, eps=0.1, sest=30.0)[:2] == (1, 30.0)
    assert judge(raw, side=1, eps=0.1, sest=19.0)[:2] == (0, 19.0)    # 2 > 0.1 * 19
    assert judge(raw, side=1, eps=1e-8, sest=1.0)[:2] == (0, 2.0)
    assert judge(raw * 1e-20, side=1, eps=1e-8, sest=0.0)[0] == 0     # ||R|| <= eps ||R|| is false
    assert judge(raw, side=2, eps=0.9, sest=100.0)[:2] == (0, 100.0)
    assert judge(np.zeros((2, 2)), side=0, eps=1e-8, sest=1.0)[0] == 1   # an exact zero block
    assert judge(np.zeros((2, 2)), side=1, eps=1e-8, sest=1.0)[0] == 1


def test_placement_of_left_and_right_blocks(judge):
    """A left block's T goes to B[row0 + a, col0 + c]; a right block's T^T to B[row0 + c, col0 + a];
    a right block that breaks is not placed, a left one that breaks is (B's last row block)."""
    g = np.random.default_rng(4)
    raw = g.standard_normal((3, 3))
    T = np.triu(raw)
    for side in (0, 1, 2):
        B = np.zeros((9, 9), order="F")
        judge(raw, side=side, B=B, row0=3, col0=2)
        want = np.zeros((9, 9))
        want[3:6, 2:5] = T if side == 0 else T.T
        np.testing.assert_array_equal(B, want)
    B = np.zeros((9, 9), order="F")
    assert judge(raw * 1e-12, side=1, eps=1e-8, sest=1.0, B=B, row0=3, col0=3)[0] == 1
    assert not B.any()
    assert judge(raw * 1e-12, side=0, eps=1e-8, sest=1.0, B=B, row0=3, col0=0)[0] == 1
    np.testing.assert_array_equal(B[3:6, 0:3], T * 1e-12)
