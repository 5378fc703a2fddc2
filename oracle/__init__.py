"""Plain FP64 CPU oracle for the Golub-Kahan partial SVD / numerical rank method
of "Accurate and fast matrix factorization for low-rank learning" (arXiv 2104.10785).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with the
CUDA library in ``paper_2104_10785_gb300``; it is compiled from ``gk_oracle.c`` with
the host C compiler and called through ctypes on NumPy arrays.

Functions follow the paper:
  gk_lower  -- Algorithm 1 (GK bidiagonalization, reorthogonalization, break test)
  numrank   -- Algorithm 3 (rank determination)
  fsvd      -- Algorithm 2 (F-SVD), literal eig(B^T B) route or SVD-of-B route
  psvd      -- thick-restarted partial SVD built on the upper-bidiagonal form
  gk_upper  -- one restart-free cycle of the upper-bidiagonal process
  jacobi_svd / jacobi_eig -- textbook one-sided / cyclic Jacobi
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgk_oracle.so")
_lock = threading.Lock()
_lib = None

F64, F32, BF16, F16 = 0, 1, 2, 3
DENSE, CSR = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libgk_oracle.so (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gk_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Op(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("dtype", C.c_int), ("m", C.c_int64), ("n", C.c_int64),
        ("ld", C.c_int64), ("scale", C.c_double), ("vals", C.c_void_p),
        ("rowptr", C.c_void_p), ("colind", C.c_void_p),
    ]


class _GkInfo(C.Structure):
    _fields_ = [("kprime", C.c_int), ("stop_reason", C.c_int), ("sigma_est", C.c_double)]


class _PsvdInfo(C.Structure):
    _fields_ = [
        ("cycles", C.c_int), ("restarts", C.c_int), ("matvecs", C.c_int64),
        ("converged", C.c_int), ("kdim_used", C.c_int), ("resid_est_max", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.POINTER
            d, i64, i32, u64 = C.c_double, C.c_int64, C.c_int, C.c_uint64
            vp = C.c_void_p
            L.gko_apply.argtypes = [P(_Op), vp, vp]
            L.gko_apply_t.argtypes = [P(_Op), vp, vp]
            L.gko_elem_value.argtypes = [P(_Op), i64]
            L.gko_elem_value.restype = d
            L.gko_philox4x32_10.argtypes = [vp, vp, vp]
            L.gko_start_vector.argtypes = [u64, i64, vp]
            L.gko_splitmix64.argtypes = [u64]
            L.gko_splitmix64.restype = u64
            L.gko_set_threads.argtypes = [i32]
            L.gko_jacobi_svd.argtypes = [i64, i64, vp, vp, vp, vp]
            L.gko_jacobi_eig.argtypes = [i64, vp, vp, vp]
            L.gko_gk_lower.argtypes = [P(_Op), i32, d, i32, i32, vp, vp, vp, vp, vp, P(_GkInfo), i32]
            L.gko_cgs.argtypes = [i32, vp, vp, i64, i64, i32]
            L.gko_cgs.restype = None
            L.gko_numrank.argtypes = [P(_Op), i32, d, i32, i32, i32, vp, P(i32), P(_GkInfo), vp, i32]
            L.gko_fsvd.argtypes = [P(_Op), i32, i32, i32, i32, vp, vp, vp, vp, P(_GkInfo), i32]
            L.gko_psvd.argtypes = [P(_Op), i32, i32, i32, d, i32, i32, vp, u64, vp, vp, vp, P(_PsvdInfo), i32]
            L.gko_gk_upper.argtypes = [P(_Op), i32, i32, vp, u64, vp, vp, vp, vp, i32]
            L.gko_residuals.argtypes = [P(_Op), i32, vp, vp, vp, vp, vp]
            L.gko_err_rel.argtypes = [P(_Op), i32, vp, vp, vp]
            L.gko_err_rel.restype = d
            L.gko_err_res.argtypes = [P(_Op), i32, vp, vp, vp]
            L.gko_err_res.restype = d
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().gko_set_threads(int(n))


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n
    return a


class Operator:
    """A stored matrix the oracle reads: dense row-major or CSR.

    ``vals`` keeps the stored bytes: float64, float32, or uint16 bit patterns
    for bf16/f16 (``dtype`` = 'bf16' or 'f16'); ``scale`` multiplies every value.
    """

    def __init__(self, vals, m, n, dtype, kind=DENSE, ld=None, rowptr=None, colind=None, scale=1.0):
        self.m, self.n = int(m), int(n)
        code = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}[dtype]
        want = {F64: np.float64, F32: np.float32, BF16: np.uint16, F16: np.uint16}[code]
        self.vals = np.ascontiguousarray(vals, dtype=want).reshape(-1)
        self.kind = kind
        self.rowptr = None if rowptr is None else np.ascontiguousarray(rowptr, dtype=np.int32)
        self.colind = None if colind is None else np.ascontiguousarray(colind, dtype=np.int32)
        self.ld = int(ld if ld is not None else n)
        self._s = _Op(kind, code, self.m, self.n, self.ld, float(scale), self.vals.ctypes.data,
                      None if self.rowptr is None else self.rowptr.ctypes.data,
                      None if self.colind is None else self.colind.ctypes.data)

    @classmethod
    def dense(cls, a, dtype=None, bits=None, scale=1.0):
        """Dense row-major operator from an ndarray (or bf16/f16 bit patterns + shape)."""
        if bits is not None:
            m, n = bits.shape
            return cls(bits, m, n, dtype, scale=scale)
        a = np.asarray(a)
        m, n = a.shape
        dt = dtype or {np.dtype(np.float64): "f64", np.dtype(np.float32): "f32"}[a.dtype]
        return cls(a, m, n, dt, scale=scale)

    @classmethod
    def csr(cls, m, n, rowptr, colind, vals, dtype="f32"):
        return cls(vals, m, n, dtype, kind=CSR, rowptr=rowptr, colind=colind)

    @property
    def ref(self):
        return C.byref(self._s)

    def matvec(self, x):
        x = _f64(x, self.n)
        y = np.empty(self.m)
        lib().gko_apply(self.ref, _p(x), _p(y))
        return y

    def rmatvec(self, x):
        x = _f64(x, self.m)
        y = np.empty(self.n)
        lib().gko_apply_t(self.ref, _p(x), _p(y))
        return y

    def value(self, idx: int) -> float:
        return lib().gko_elem_value(self.ref, int(idx))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().gko_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def start_vector(seed: int, m: int):
    q = np.empty(m)
    lib().gko_start_vector(C.c_uint64(seed & (2**64 - 1)), m, _p(q))
    return q


def splitmix64(x: int) -> int:
    return int(lib().gko_splitmix64(C.c_uint64(x & (2**64 - 1))))


def jacobi_svd(M):
    """One-sided Jacobi SVD of a rows x cols (rows >= cols) matrix: (U, s, V, sweeps)."""
    M = np.asarray(M, dtype=np.float64)
    rows, cols = M.shape
    Mc = np.asfortranarray(M)
    s = np.empty(cols)
    U = np.empty((rows, cols), order="F")
    V = np.empty((cols, cols), order="F")
    sw = lib().gko_jacobi_svd(rows, cols, Mc.ctypes.data_as(C.c_void_p), _p(s),
                              U.ctypes.data_as(C.c_void_p), V.ctypes.data_as(C.c_void_p))
    return U, s, V, sw


def jacobi_eig(S):
    S = np.asfortranarray(np.asarray(S, dtype=np.float64))
    n = S.shape[0]
    th = np.empty(n)
    G = np.empty((n, n), order="F")
    sw = lib().gko_jacobi_eig(n, S.ctypes.data_as(C.c_void_p), _p(th), G.ctypes.data_as(C.c_void_p))
    return th, G, sw


def cgs(w, Q, passes=0):
    """Gram-Schmidt of w against the columns of Q (the oracle's step, as Algorithm 1 applies it)."""
    Q = np.asarray(Q, dtype=np.float64)
    len_, j = Q.shape
    Qc = np.ascontiguousarray(Q.T)  # row c = column c
    out = np.array(w, dtype=np.float64, copy=True)
    lib().gko_cgs(int(passes), _p(out), _p(Qc), C.c_int64(len_), C.c_int64(len_), int(j))
    return out


def gk_lower(op: Operator, k: int, q1, eps=0.0, relative=True, passes=0, fused=False):
    """Algorithm 1 (fused=True: the fused-sweep ordering, A^T w / beta for A^T q).  Returns
    dict(alpha, beta, Q, P, kprime, stop_reason, sigma_est)."""
    m, n = op.m, op.n
    q1 = _f64(q1, m)
    alpha = np.zeros(k + 1)
    beta = np.zeros(k + 2)
    Q = np.zeros((k + 1, m))  # row c is column c of Q (column-major storage)
    P = np.zeros((k + 1, n))
    info = _GkInfo()
    rc = lib().gko_gk_lower(op.ref, k, eps, int(relative), passes, _p(q1), _p(alpha), _p(beta),
                            _p(Q), _p(P), C.byref(info), int(bool(fused)))
    if rc != 0:
        raise ValueError(f"gko_gk_lower rc={rc}")
    return dict(alpha=alpha, beta=beta, Q=Q.T.copy(), P=P.T.copy(), kprime=info.kprime,
                stop_reason=info.stop_reason, sigma_est=info.sigma_est)


def numrank(op: Operator, q1, eps=1e-8, relative=True, literal=False, kmax=0, passes=0, fused=False):
    """Algorithm 3.  Returns (rank, kprime, sigma(B) descending)."""
    q1 = _f64(q1, op.m)
    mn = min(op.m, op.n)
    km = mn if kmax <= 0 or kmax > mn else kmax
    sig = np.zeros(km + 1)
    r = C.c_int(0)
    info = _GkInfo()
    rc = lib().gko_numrank(op.ref, km, eps, int(relative), int(literal), passes, _p(q1), C.byref(r),
                           C.byref(info), _p(sig), int(bool(fused)))
    if rc != 0:
        raise ValueError(f"gko_numrank rc={rc}")
    return r.value, info.kprime, sig[: info.kprime].copy()


def fsvd(op: Operator, k: int, r: int, q1, route=1, passes=0, fused=False):
    """Algorithm 2 (F-SVD).  route 0 = eig(B^T B) + A v / sigma; route 1 = SVD of B."""
    q1 = _f64(q1, op.m)
    U = np.zeros((r, op.m))
    V = np.zeros((r, op.n))
    S = np.zeros(r)
    info = _GkInfo()
    rc = lib().gko_fsvd(op.ref, k, r, route, passes, _p(q1), _p(U), _p(S), _p(V), C.byref(info), int(bool(fused)))
    if rc != 0:
        raise ValueError(f"gko_fsvd rc={rc}")
    return U.T.copy(), S, V.T.copy(), info.kprime


def psvd(op: Operator, k: int, K: int, q1, tol=1e-10, keep=0, max_restarts=100, passes=0, seed=0, fused=False):
    """Thick-restarted partial SVD.  Returns (U m x k, S k, V n x k, info dict)."""
    q1 = _f64(q1, op.m)
    U = np.zeros((k, op.m))
    V = np.zeros((k, op.n))
    S = np.zeros(k)
    info = _PsvdInfo()
    rc = lib().gko_psvd(op.ref, k, K, keep, tol, max_restarts, passes, _p(q1), C.c_uint64(seed), _p(U),
                        _p(S), _p(V), C.byref(info), int(bool(fused)))
    if rc < 0:
        raise ValueError(f"gko_psvd rc={rc}")
    d = dict(cycles=info.cycles, restarts=info.restarts, matvecs=info.matvecs,
             converged=bool(info.converged), kdim_used=info.kdim_used,
             resid_est_max=info.resid_est_max, rc=rc)
    return U.T.copy(), S, V.T.copy(), d


def gk_upper(op: Operator, K: int, q1, passes=0, seed=0, fused=False):
    """One restart-free upper-bidiagonal cycle: (alpha[K], beta[K], U m x K, V n x (K+1))."""
    q1 = _f64(q1, op.m)
    alpha = np.zeros(K)
    beta = np.zeros(K)
    Ub = np.zeros((K, op.m))
    Vb = np.zeros((K + 1, op.n))
    rc = lib().gko_gk_upper(op.ref, K, passes, _p(q1), C.c_uint64(seed), _p(alpha), _p(beta), _p(Ub), _p(Vb),
                            int(bool(fused)))
    if rc != 0:
        raise ValueError(f"gko_gk_upper rc={rc}")
    return alpha, beta, Ub.T.copy(), Vb.T.copy()


def residuals(op: Operator, U, S, V):
    """Per-triplet (||A v_i - s_i u_i||, ||A^T u_i - s_i v_i||)."""
    k = len(S)
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.float64).T)
    Vc = np.ascontiguousarray(np.asarray(V, dtype=np.float64).T)
    S = _f64(S)
    r1 = np.empty(k)
    r2 = np.empty(k)
    lib().gko_residuals(op.ref, k, _p(Uc), _p(S), _p(Vc), _p(r1), _p(r2))
    return r1, r2


def err_rel(op: Operator, U, S, V) -> float:
    """The paper's relative error ||A^T U - V Sigma||_F / ||Sigma||_F."""
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.float64).T)
    Vc = np.ascontiguousarray(np.asarray(V, dtype=np.float64).T)
    S = _f64(S)
    return lib().gko_err_rel(op.ref, len(S), _p(Uc), _p(S), _p(Vc))


def err_res(op: Operator, U, S, V) -> float:
    """The paper's residual error ||A - U Sigma V^T||_F (dense operators)."""
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.float64).T)
    Vc = np.ascontiguousarray(np.asarray(V, dtype=np.float64).T)
    S = _f64(S)
    return lib().gko_err_res(op.ref, len(S), _p(Uc), _p(S), _p(Vc))
