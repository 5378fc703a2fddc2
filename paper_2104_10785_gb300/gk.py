"""ctypes binding of libgk.so (include/gk.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch provides device memory and the current stream.  There is no
host fallback: if the library or a CUDA device is missing, calls raise.

Names follow the C ABI: gk_psvd, gk_numrank, gk_psvd_workspace, ...
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import torch

from . import build as _build

GK_OK, GK_NOT_CONVERGED, GK_RANK_DEFICIENT = 0, 1, 2
GK_INVALID_ARG, GK_CUDA_ERROR, GK_NUMERICAL, GK_TIMEOUT = -1, -2, -3, -4
GK_OUT_OF_MEMORY, GK_NOT_IMPLEMENTED, GK_NO_DEVICE = -5, -6, -7
GK_F64, GK_F32, GK_BF16, GK_F16 = 0, 1, 2, 3
GK_DENSE, GK_CSR = 0, 1
GK_FLAG_PROFILE = 1
GK_FLAG_AUTOTUNE = 2
GK_FLAG_FUSED = 4
GK_FLAG_REFINE = 8
GK_FLAG_ORTH_F64 = 16
GK_FLAG_PERSISTENT = 32
GK_FLAG_SKETCH_TC = 64
GK_FLAG_BDSVD = 128
GK_FLAG_RITZ_DF = 256
GK_FLAG_BLOCK_F32 = 512
GK_FLAG_BLOCK_GS = 1024

_DTYPE = {torch.float64: GK_F64, torch.float32: GK_F32, torch.bfloat16: GK_BF16, torch.float16: GK_F16}


class gk_matrix(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("dtype", C.c_int32), ("m", C.c_int64), ("n", C.c_int64), ("ld", C.c_int64),
        ("scale", C.c_double), ("vals", C.c_void_p), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
        ("t_vals", C.c_void_p), ("t_rowptr", C.c_void_p), ("t_colind", C.c_void_p),
    ]


class gk_opts(C.Structure):
    _fields_ = [
        ("krylov_dim", C.c_int32), ("keep", C.c_int32), ("max_restarts", C.c_int32),
        ("reorth_passes", C.c_int32), ("eps_absolute", C.c_int32), ("flags", C.c_int32),
        ("seed", C.c_uint64), ("start", C.c_void_p), ("stream", C.c_void_p),
        ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t), ("predictor", C.c_void_p),
    ]


class gk_info(C.Structure):
    _fields_ = [
        ("steps", C.c_int32), ("restarts", C.c_int32), ("cycles", C.c_int32), ("kprime", C.c_int32),
        ("stop_reason", C.c_int32), ("breakdowns", C.c_int32), ("svd_sweeps", C.c_int32), ("reserved", C.c_int32),
        ("matvecs", C.c_int64),
        ("resid_est_max", C.c_double), ("sigma_est", C.c_double), ("seconds", C.c_double),
        ("ms_matvec", C.c_double), ("ms_matvec_t", C.c_double), ("ms_orth", C.c_double), ("ms_small", C.c_double),
        ("ms_restart", C.c_double), ("n_matvec", C.c_int64), ("n_matvec_t", C.c_int64), ("launches", C.c_int64),
        ("ms_copy", C.c_double), ("resid_true_max", C.c_double), ("ms_refine", C.c_double),
        ("refine_checks", C.c_int32), ("fallbacks", C.c_int32), ("err_rel", C.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gk_batch_item(C.Structure):
    _fields_ = [
        ("A", gk_matrix), ("k", C.c_int32), ("krylov_dim", C.c_int32), ("tol", C.c_double),
        ("U", C.c_void_p), ("S", C.c_void_p), ("V", C.c_void_p), ("start", C.c_void_p),
        ("rank_cut", C.c_double), ("status", C.c_int32), ("rank", C.c_int32), ("steps", C.c_int32), ("restarts", C.c_int32),
        ("cycles", C.c_int32), ("breakdowns", C.c_int32), ("matvecs", C.c_int64),
        ("resid_est_max", C.c_double), ("sigma_est", C.c_double), ("sigma_next", C.c_double),
    ]


class gk_rsgd_args(C.Structure):
    _fields_ = [
        ("P", C.c_int32), ("N", C.c_int32), ("d1", C.c_int32), ("d2", C.c_int32), ("r", C.c_int32),
        ("k_inner", C.c_int32), ("steps", C.c_int32), ("b", C.c_int32), ("eta", C.c_double), ("lam", C.c_double),
        ("X", C.c_void_p), ("Vd", C.c_void_p), ("y", C.c_void_p), ("batches", C.c_void_p), ("q1", C.c_void_p),
        ("W", C.c_void_p),
    ]


class GKError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} {last_cuda_error()}".strip())


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libgk.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build_library()
            if not os.path.exists(path):
                raise RuntimeError(f"libgk.so missing at {path}")
            L = C.CDLL(path)
            P = C.POINTER
            L.gk_default_opts.argtypes = [P(gk_opts)]
            L.gk_default_opts.restype = None
            L.gk_psvd_workspace.argtypes = [P(gk_matrix), C.c_int, P(gk_opts)]
            L.gk_psvd_workspace.restype = C.c_size_t
            L.gk_psvd.argtypes = [P(gk_matrix), C.c_int, C.c_double, P(gk_opts), C.c_void_p, C.c_void_p, C.c_void_p,
                                  P(gk_info)]
            L.gk_psvd.restype = C.c_int
            L.gk_numrank_workspace.argtypes = [P(gk_matrix), C.c_int, P(gk_opts)]
            L.gk_numrank_workspace.restype = C.c_size_t
            L.gk_numrank.argtypes = [P(gk_matrix), C.c_double, C.c_int, P(gk_opts), P(C.c_int), C.c_void_p,
                                     P(gk_info)]
            L.gk_numrank.restype = C.c_int
            L.gk_fsvd.argtypes = [P(gk_matrix), C.c_int, C.c_int, C.c_int, P(gk_opts), C.c_void_p, C.c_void_p,
                                  C.c_void_p, P(gk_info)]
            L.gk_fsvd.restype = C.c_int
            L.gk_block_numrank.argtypes = [P(gk_matrix), C.c_int, C.c_void_p, C.c_double, C.c_int, P(gk_opts),
                                           P(C.c_int), C.c_void_p, P(C.c_int), P(gk_info)]
            L.gk_block_numrank.restype = C.c_int
            L.gk_block_fsvd.argtypes = [P(gk_matrix), C.c_int, C.c_void_p, C.c_int, C.c_int, P(gk_opts), C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, P(gk_info)]
            L.gk_block_fsvd.restype = C.c_int
            L.gk_block_numrank_workspace.argtypes = [P(gk_matrix), C.c_int, C.c_int, P(gk_opts)]
            L.gk_block_numrank_workspace.restype = C.c_size_t
            L.gk_matvec.argtypes = [P(gk_matrix), C.c_int, C.c_void_p, C.c_void_p, P(gk_opts)]
            L.gk_matvec.restype = C.c_int
            L.gk_residuals.argtypes = [P(gk_matrix), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, P(gk_opts)]
            L.gk_residuals.restype = C.c_int
            L.gk_matvec_static.argtypes = [P(gk_matrix), C.c_int, C.c_void_p, C.c_void_p, P(gk_opts)]
            L.gk_matvec_static.restype = C.c_int
            L.gk_psvd_batched.argtypes = [P(gk_batch_item), C.c_int, P(gk_opts), P(gk_info)]
            L.gk_psvd_batched.restype = C.c_int
            L.gk_numrank_batched.argtypes = [P(gk_batch_item), C.c_int, P(gk_opts), P(gk_info)]
            L.gk_numrank_batched.restype = C.c_int
            L.gk_rsgd_batched.argtypes = [P(gk_rsgd_args), P(gk_opts), P(gk_info)]
            L.gk_rsgd_batched.restype = C.c_int
            L.gk_sketch_batched.argtypes = [P(gk_matrix), C.c_int, C.c_uint64, C.c_void_p, P(gk_opts)]
            L.gk_sketch_batched.restype = C.c_int
            L.gk_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, P(gk_opts)]
            L.gk_mlp_forward.restype = C.c_int
            L.gk_mlp_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, P(gk_opts)]
            L.gk_mlp_grad.restype = C.c_int
            L.gk_mlp_train.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                       C.c_int, C.c_int, C.c_float, C.c_uint64, C.c_void_p, P(gk_opts)]
            L.gk_mlp_train.restype = C.c_int
            L.gk_status_string.argtypes = [C.c_int]
            L.gk_status_string.restype = C.c_char_p
            L.gk_last_cuda_error.argtypes = []
            L.gk_last_cuda_error.restype = C.c_char_p
            L.gk_version.argtypes = []
            L.gk_version.restype = C.c_char_p
            L.gk_launch_count.argtypes = []
            L.gk_launch_count.restype = C.c_int64
            L.gk_wait_selftest.argtypes = [C.c_longlong]
            L.gk_wait_selftest.restype = C.c_int
            L.gk_predictor_load.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]
            L.gk_predictor_load.restype = C.c_int
            L.gk_predictor_free.argtypes = [C.c_void_p]
            L.gk_predictor_free.restype = C.c_int
            L.gk_predictor_predict.argtypes = [C.c_void_p, P(gk_matrix), C.c_int, C.c_void_p, P(gk_opts)]
            L.gk_predictor_predict.restype = C.c_int
            L.gk_predictor_margins.argtypes = [C.c_double, C.c_double, C.c_int64, C.c_int, C.POINTER(C.c_int),
                                               C.POINTER(C.c_int)]
            L.gk_predictor_margins.restype = C.c_int
            L.gk_host_alloc.argtypes = [C.c_size_t, C.POINTER(C.c_void_p)]
            L.gk_host_alloc.restype = C.c_int
            L.gk_host_free.argtypes = [C.c_void_p]
            L.gk_host_free.restype = C.c_int
            _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().gk_status_string(int(s)).decode()


def last_cuda_error() -> str:
    return lib().gk_last_cuda_error().decode()


def version() -> str:
    return lib().gk_version().decode()


_host_bufs = {}


def host_empty(shape, dtype=torch.float32):
    """A host tensor in huge-page-backed pinned memory from gk_host_alloc (release with host_free).
    The mapping is rounded up to the huge-page size (512 MB with 64 KB pages): carve small operands
    from one buffer instead of allocating each."""
    import numpy as np

    shape = tuple(int(x) for x in shape)
    esz = torch.empty((), dtype=dtype).element_size()
    nbytes = esz
    for d in shape:
        nbytes *= d
    p = C.c_void_p()
    st = lib().gk_host_alloc(max(nbytes, 1), C.byref(p))
    if st < 0:
        raise GKError(st, "gk_host_alloc")
    raw = (C.c_uint8 * max(nbytes, 1)).from_address(p.value)
    t = torch.from_numpy(np.frombuffer(raw, dtype=np.uint8, count=nbytes)).view(dtype).view(shape)
    _host_bufs[t.data_ptr()] = (p.value, raw)
    return t


def host_free(t) -> None:
    ent = _host_bufs.pop(t.data_ptr(), None)
    if ent is None:
        raise ValueError("not a tensor from host_empty")
    st = lib().gk_host_free(C.c_void_p(ent[0]))
    if st < 0:
        raise GKError(st, "gk_host_free")


def wait_selftest(cycles: int) -> int:
    """Status of a device wait on a flag that nothing sets, bounded to `cycles` SM cycles."""
    return int(lib().gk_wait_selftest(int(cycles)))


def launch_count() -> int:
    """Kernels this host thread has launched through the library so far."""
    return int(lib().gk_launch_count())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Predictor:
    """A learned predictor loaded into the library (gk_predictor_load): pass it as predictor= to
    gk_psvd (the Krylov dimension) or gk_psvd_batched (the learned pipeline)."""

    def __init__(self, params):
        w = params.detach().to(torch.float32).contiguous()
        h = C.c_void_p()
        st = lib().gk_predictor_load(C.c_void_p(w.data_ptr()), w.numel() * 4, C.byref(h))
        if st < 0:
            raise GKError(st, "gk_predictor_load")
        self.handle = h.value
        self._lib = lib()

    def predict(self, mats, stream=None):
        """(count x 2) float32 host array of (log r, log K) for dense device operators."""
        import numpy as np

        n = len(mats)
        arr = (gk_matrix * n)()
        for i, A in enumerate(mats):
            arr[i], _ = make_matrix(A)
        out = np.zeros((n, 2), dtype=np.float32)
        o = default_opts()
        s = stream if stream is not None else torch.cuda.current_stream(mats[0].device)
        o.stream = s.cuda_stream
        st = lib().gk_predictor_predict(C.c_void_p(self.handle), arr, n, C.c_void_p(out.ctypes.data), C.byref(o))
        if st < 0:
            raise GKError(st, "gk_predictor_predict")
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self._lib.gk_predictor_free(C.c_void_p(h))
            self.handle = None


@dataclass
class CSR:
    """A CSR operator and the CSR of its transpose (both required by the library)."""
    m: int
    n: int
    rowptr: torch.Tensor
    colind: torch.Tensor
    vals: torch.Tensor
    t_rowptr: torch.Tensor
    t_colind: torch.Tensor
    t_vals: torch.Tensor

    @property
    def device(self):
        return self.vals.device


def make_matrix(A, scale: float = 1.0) -> tuple[gk_matrix, tuple]:
    """gk_matrix describing a dense row-major tensor (m x n, unit column stride) or a CSR."""
    if isinstance(A, CSR):
        for t in (A.rowptr, A.colind, A.t_rowptr, A.t_colind):
            if t.dtype != torch.int32 or not t.is_contiguous():
                raise ValueError("CSR index arrays must be contiguous int32")
        if A.vals.dtype not in _DTYPE or A.t_vals.dtype != A.vals.dtype:
            raise ValueError("unsupported CSR value dtype")
        M = gk_matrix(GK_CSR, _DTYPE[A.vals.dtype], A.m, A.n, 0, float(scale), A.vals.data_ptr(),
                      A.rowptr.data_ptr(), A.colind.data_ptr(), A.t_vals.data_ptr(), A.t_rowptr.data_ptr(),
                      A.t_colind.data_ptr())
        return M, (A,)
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("dense operator must be a 2-D row-major tensor with unit column stride")
    if A.dtype not in _DTYPE:
        raise ValueError(f"unsupported dtype {A.dtype}")
    M = gk_matrix(GK_DENSE, _DTYPE[A.dtype], A.shape[0], A.shape[1], A.stride(0), float(scale), A.data_ptr(),
                  None, None, None, None, None)
    return M, (A,)


def default_opts() -> gk_opts:
    o = gk_opts()
    lib().gk_default_opts(C.byref(o))
    return o


def _check_start(start, m):
    """The library reads m values from a start vector: refuse any other length here."""
    if start is not None and start.numel() != m:
        raise ValueError(f"start vector must have m = {m} entries, got {start.numel()}")


def _opts(device, krylov_dim=0, keep=0, max_restarts=None, reorth_passes=None, eps_absolute=False, seed=None,
          start=None, stream=None, workspace=None, profile=False, fused=False, refine=False, orth_f64=False,
          persistent=False, bdsvd=False):
    o = default_opts()
    o.flags = ((GK_FLAG_PROFILE if profile else 0) | (GK_FLAG_FUSED if fused else 0) | (GK_FLAG_REFINE if refine else 0)
               | (GK_FLAG_ORTH_F64 if orth_f64 else 0) | (GK_FLAG_PERSISTENT if persistent else 0)
               | (GK_FLAG_BDSVD if bdsvd else 0))
    o.krylov_dim = int(krylov_dim)
    o.keep = int(keep)
    if max_restarts is not None:
        o.max_restarts = int(max_restarts)
    if reorth_passes is not None:
        o.reorth_passes = int(reorth_passes)
    o.eps_absolute = int(bool(eps_absolute))
    if seed is not None:
        o.seed = int(seed) & (2**64 - 1)
    keep_alive = []
    if start is not None:
        st = start.to(torch.float64).contiguous()
        keep_alive.append(st)
        o.start = st.data_ptr()
    if device.type == "cuda":
        s = stream if stream is not None else torch.cuda.current_stream(device)
        o.stream = s.cuda_stream
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o, keep_alive


def gk_psvd(A, k: int, tol: float = 1e-8, *, krylov_dim: int = 0, keep: int = 0, max_restarts: int | None = None,
            reorth_passes: int | None = None, seed: int | None = None, start=None, stream=None, workspace=None,
            scale: float = 1.0, out=None, check: bool = True, profile: bool = False, fused: bool = False,
            refine: bool = False, predictor: "Predictor | None" = None, orth_f64: bool = False,
            persistent: bool = False, bdsvd: bool = False, sketch_tc: bool = False, ritz_df: bool = False):
    """k largest singular triplets of A.  Returns (U m x k, S k, V n x k, status, info dict).

    Outputs live where A lives (device tensors for a CUDA operator, host tensors
    for a host operator: the library copies host data itself).  fused=True runs the fused
    sweep, one pass over A per step (GK_FLAG_FUSED); info["reserved"] is the fused kernel's
    cluster size (0 when the steps ran as two passes).  refine=True checks the returned
    triplets' true residuals with FP64-grade products and keeps restarting while one exceeds
    tol (GK_FLAG_REFINE; info["resid_true_max"], info["ms_refine"]).  predictor (a Predictor)
    chooses the Krylov dimension from A's sketch when krylov_dim is 0 (info["kprime"] = K used).
    bdsvd=True takes the SVD of a cycle's bidiagonal projected matrix by Golub-Kahan SVD steps
    (GK_FLAG_BDSVD, experimental); sketch_tc=True runs the predictor's sketch of a bf16 operator
    on the tcgen05 tensor cores (GK_FLAG_SKETCH_TC, experimental); ritz_df=True forms the Ritz
    vectors from the bases' double-f32 copies on the FP32 pipes (GK_FLAG_RITZ_DF, experimental).
    """
    M, keep_a = make_matrix(A, scale)
    _check_start(start, M.m)
    dev = A.device
    if dev.type != "cuda" and not torch.cuda.is_available():
        raise RuntimeError("gk_psvd needs a CUDA device (no host fallback)")
    m, n = M.m, M.n
    if out is None:
        pin = dev.type == "cpu"
        U = torch.empty((k, m), dtype=torch.float64, device=dev, pin_memory=pin)
        V = torch.empty((k, n), dtype=torch.float64, device=dev, pin_memory=pin)
        S = torch.empty(k, dtype=torch.float64, device=dev, pin_memory=pin)
    else:
        U, S, V = out
    o, ka = _opts(dev if dev.type == "cuda" else torch.device("cuda"), krylov_dim, keep, max_restarts,
                  reorth_passes, False, seed, start, stream, workspace, profile, fused, refine, orth_f64, persistent,
                  bdsvd)
    if sketch_tc:
        o.flags |= GK_FLAG_SKETCH_TC
    if ritz_df:
        o.flags |= GK_FLAG_RITZ_DF
    if predictor is not None:
        o.predictor = predictor.handle
    info = gk_info()
    st = lib().gk_psvd(C.byref(M), int(k), float(tol), C.byref(o), _ptr(U), _ptr(S), _ptr(V), C.byref(info))
    if check and st < 0:
        raise GKError(st, "gk_psvd")
    return U.T, S, V.T, st, info.as_dict()


def gk_fsvd(A, k: int, r: int, *, route: int = 1, reorth_passes: int | None = None, seed: int | None = None,
            start=None, stream=None, workspace=None, scale: float = 1.0, check: bool = True, profile: bool = False,
            fused: bool = False, orth_f64: bool = False, bdsvd: bool = False):
    """Algorithm 2 as printed: k steps of Algorithm 1, the SVD of B, the r largest triplets
    (route 1: U = Q X; route 0: u_i = A v_i / sigma_i).  Returns (U m x r, S r, V n x r, status,
    info dict); outputs live where A lives."""
    M, keep_a = make_matrix(A, scale)
    _check_start(start, M.m)
    dev = A.device
    if dev.type != "cuda" and not torch.cuda.is_available():
        raise RuntimeError("gk_fsvd needs a CUDA device (no host fallback)")
    pin = dev.type == "cpu"
    U = torch.empty((r, M.m), dtype=torch.float64, device=dev, pin_memory=pin)
    V = torch.empty((r, M.n), dtype=torch.float64, device=dev, pin_memory=pin)
    S = torch.empty(r, dtype=torch.float64, device=dev, pin_memory=pin)
    o, ka = _opts(dev if dev.type == "cuda" else torch.device("cuda"), 0, 0, None, reorth_passes, False, seed, start,
                  stream, workspace, profile, fused, orth_f64=orth_f64)
    if bdsvd:
        o.flags |= GK_FLAG_BDSVD
    info = gk_info()
    st = lib().gk_fsvd(C.byref(M), int(k), int(r), int(route), C.byref(o), _ptr(U), _ptr(S), _ptr(V), C.byref(info))
    if check and st < 0:
        raise GKError(st, "gk_fsvd")
    return U.T, S, V.T, st, info.as_dict()


def gk_numrank(A, eps: float = 1e-8, kmax: int = 0, *, eps_absolute: bool = False, reorth_passes: int | None = None,
               seed: int | None = None, start=None, stream=None, workspace=None, scale: float = 1.0,
               want_sigma: bool = False, check: bool = True, profile: bool = False, fused: bool = False,
               orth_f64: bool = False):
    """Numerical rank by Algorithm 3.  Returns (rank, sigma(B) or None, status, info dict)."""
    M, keep_a = make_matrix(A, scale)
    _check_start(start, M.m)
    dev = A.device
    if dev.type != "cuda" and not torch.cuda.is_available():
        raise RuntimeError("gk_numrank needs a CUDA device (no host fallback)")
    mn = min(M.m, M.n)
    km = mn if kmax <= 0 or kmax > mn else kmax
    sig = torch.zeros(km + 1, dtype=torch.float64, device=dev) if want_sigma else None
    o, ka = _opts(dev if dev.type == "cuda" else torch.device("cuda"), 0, 0, None, reorth_passes, eps_absolute,
                  seed, start, stream, workspace, profile, fused, orth_f64=orth_f64)
    info = gk_info()
    r = C.c_int(-1)
    st = lib().gk_numrank(C.byref(M), float(eps), int(kmax), C.byref(o), C.byref(r), _ptr(sig), C.byref(info))
    if check and st < 0:
        raise GKError(st, "gk_numrank")
    d = info.as_dict()
    return r.value, (sig[: d["kprime"]] if sig is not None else None), st, d


def gk_block_numrank(A, s: int, eps: float = 1e-8, kmax: int = 0, *, start=None, seed: int | None = None,
                     stream=None, workspace=None, scale: float = 1.0, want_sigma: bool = False, check: bool = True,
                     orth_f64: bool = False, f32_products: bool = False, block_gs: bool = False,
                     profile: bool = False):
    """Numerical rank from a block of s start vectors (block Algorithm 1 + Algorithm 3).
    start: optional m x s start block.  f32_products: the block products of a reduced-precision
    dense operator in f32 (GK_FLAG_BLOCK_F32, experimental); block_gs: the block Gram-Schmidt
    (GK_FLAG_BLOCK_GS, experimental); profile: the info dict's ms_* phase times (GK_FLAG_PROFILE).
    Returns (rank, sigma(B) or None, block steps, status, info dict)."""
    M, keep_a = make_matrix(A, scale)
    if start is not None and tuple(start.shape) != (M.m, int(s)):
        raise ValueError(f"start block must be m x s = {M.m} x {int(s)}, got {tuple(start.shape)}")
    dev = A.device
    if dev.type != "cuda" and not torch.cuda.is_available():
        raise RuntimeError("gk_block_numrank needs a CUDA device (no host fallback)")
    mn = min(M.m, M.n)
    s = int(s)
    cap_steps = int(kmax) if kmax > 0 else max(1, min(mn // max(s, 1), 1024 // max(s, 1) - 1))
    sig = torch.zeros(max(cap_steps * s, 1), dtype=torch.float64, device=dev) if want_sigma else None
    q0 = None
    if start is not None:
        # start is m x s; the library reads it column-major (column c contiguous)
        q0 = start.to(torch.float64).t().contiguous()
    o, ka = _opts(dev if dev.type == "cuda" else torch.device("cuda"), seed=seed, stream=stream, workspace=workspace,
                  orth_f64=orth_f64, profile=profile)
    if f32_products:
        o.flags |= GK_FLAG_BLOCK_F32
    if block_gs:
        o.flags |= GK_FLAG_BLOCK_GS
    info = gk_info()
    r = C.c_int(-1)
    steps = C.c_int(0)
    st = lib().gk_block_numrank(C.byref(M), s, _ptr(q0), float(eps), int(kmax), C.byref(o), C.byref(r), _ptr(sig),
                                C.byref(steps), C.byref(info))
    if check and st < 0:
        raise GKError(st, "gk_block_numrank")
    d = info.as_dict()
    return r.value, (sig[: d["kprime"]] if sig is not None else None), steps.value, st, d


def gk_block_fsvd(A, s: int, steps: int, r: int, *, start=None, seed: int | None = None, stream=None,
                  workspace=None, scale: float = 1.0, check: bool = True, orth_f64: bool = False,
                  f32_products: bool = False, ritz_df: bool = False, block_gs: bool = False,
                  profile: bool = False):
    """One cycle of the block form of Algorithm 2 on a CUDA operator (gk_block_fsvd, experimental).
    f32_products: GK_FLAG_BLOCK_F32; ritz_df: the Ritz vectors from the bases' double-f32 copies
    (GK_FLAG_RITZ_DF); block_gs: the block Gram-Schmidt (GK_FLAG_BLOCK_GS); profile: the info dict's
    ms_* phase times (GK_FLAG_PROFILE).  Returns (U m x r, S r, V n x r, residuals r, status, info dict), all on
    A's device."""
    M, keep_a = make_matrix(A, scale)
    if start is not None and tuple(start.shape) != (M.m, int(s)):
        raise ValueError(f"start block must be m x s = {M.m} x {int(s)}, got {tuple(start.shape)}")
    dev = A.device
    if dev.type != "cuda":
        raise ValueError("gk_block_fsvd takes a CUDA operator (its outputs are device tensors)")
    U = torch.empty((r, M.m), dtype=torch.float64, device=dev)
    V = torch.empty((r, M.n), dtype=torch.float64, device=dev)
    S = torch.empty(r, dtype=torch.float64, device=dev)
    res = torch.empty(r, dtype=torch.float64, device=dev)
    q0 = start.to(torch.float64).t().contiguous() if start is not None else None
    o, ka = _opts(dev, seed=seed, stream=stream, workspace=workspace, orth_f64=orth_f64, profile=profile)
    if f32_products:
        o.flags |= GK_FLAG_BLOCK_F32
    if ritz_df:
        o.flags |= GK_FLAG_RITZ_DF
    if block_gs:
        o.flags |= GK_FLAG_BLOCK_GS
    info = gk_info()
    st = lib().gk_block_fsvd(C.byref(M), int(s), _ptr(q0), int(steps), int(r), C.byref(o), _ptr(U), _ptr(S), _ptr(V),
                             _ptr(res), C.byref(info))
    if check and st < 0:
        raise GKError(st, "gk_block_fsvd")
    return U.T, S, V.T, res, st, info.as_dict()


def gk_block_numrank_workspace(A, s: int, kmax: int = 0, *, orth_f64: bool = False, block_gs: bool = False) -> int:
    M, _ = make_matrix(A)
    o = default_opts()
    o.flags = (GK_FLAG_ORTH_F64 if orth_f64 else 0) | (GK_FLAG_BLOCK_GS if block_gs else 0)
    return int(lib().gk_block_numrank_workspace(C.byref(M), int(s), int(kmax), C.byref(o)))


def gk_matvec(A, x, trans: bool = False, *, stream=None, scale: float = 1.0):
    """y = A x (or A^T x) through the library's product kernels; x, y f64."""
    M, keep_a = make_matrix(A, scale)
    if x.numel() != (M.m if trans else M.n):
        raise ValueError(f"x must have {M.m if trans else M.n} entries, got {x.numel()}")
    dev = A.device
    xx = x.to(torch.float64).contiguous()
    y = torch.empty(M.n if trans else M.m, dtype=torch.float64, device=xx.device)
    o, ka = _opts(dev if dev.type == "cuda" else torch.device("cuda"), stream=stream)
    st = lib().gk_matvec(C.byref(M), int(bool(trans)), _ptr(xx), _ptr(y), C.byref(o))
    if st < 0:
        raise GKError(st, "gk_matvec")
    return y


def gk_matvec_static(A, x, out, trans: bool = False, *, stream=None, scale: float = 1.0) -> int:
    """y = A x (or A^T x) into the caller's device tensor `out`, with the library's
    static scratch instead of any device allocation (see gk_matvec_static in gk.h).
    Returns the status code."""
    M, keep_a = make_matrix(A, scale)
    if x.dtype != torch.float64 or not x.is_contiguous() or out.dtype != torch.float64 or not out.is_contiguous():
        raise ValueError("x and out must be contiguous float64 device tensors")
    if x.numel() != (M.m if trans else M.n) or out.numel() != (M.n if trans else M.m):
        raise ValueError("x and out must have the lengths of the product's input and output")
    o = gk_opts()
    lib().gk_default_opts(C.byref(o))
    s = stream if stream is not None else torch.cuda.current_stream(out.device)
    o.stream = s.cuda_stream
    return int(lib().gk_matvec_static(C.byref(M), int(bool(trans)), _ptr(x), _ptr(out), C.byref(o)))


def gk_residuals(A, U, S, V, *, stream=None, scale: float = 1.0):
    """(||A v_i - s_i u_i||, ||A^T u_i - s_i v_i||) for the columns of U, V."""
    M, keep_a = make_matrix(A, scale)
    dev = A.device
    k = S.numel()
    if tuple(U.shape) != (M.m, k) or tuple(V.shape) != (M.n, k):
        raise ValueError(f"U must be {M.m} x {k} and V {M.n} x {k}, got {tuple(U.shape)} and {tuple(V.shape)}")
    Uc = U.T.contiguous().to(torch.float64)
    Vc = V.T.contiguous().to(torch.float64)
    Sc = S.to(torch.float64).contiguous()
    r1 = torch.empty(k, dtype=torch.float64, device=Sc.device)
    r2 = torch.empty(k, dtype=torch.float64, device=Sc.device)
    o, ka = _opts(dev if dev.type == "cuda" else torch.device("cuda"), stream=stream)
    st = lib().gk_residuals(C.byref(M), int(k), _ptr(Uc), _ptr(Sc), _ptr(Vc), _ptr(r1), _ptr(r2), C.byref(o))
    if st < 0:
        raise GKError(st, "gk_residuals")
    return r1, r2


def gk_psvd_workspace(A, k: int, krylov_dim: int = 0) -> int:
    M, _ = make_matrix(A)
    o = default_opts()
    o.krylov_dim = int(krylov_dim)
    return int(lib().gk_psvd_workspace(C.byref(M), int(k), C.byref(o)))


def gk_numrank_workspace(A, kmax: int = 0) -> int:
    M, _ = make_matrix(A)
    return int(lib().gk_numrank_workspace(C.byref(M), int(kmax), None))


def _batch_opts(device, seed=None, max_restarts=None, reorth_passes=None, eps_absolute=False, autotune=False,
                stream=None, profile=False):
    o, _ = _opts(device, 0, 0, max_restarts, reorth_passes, eps_absolute, seed, None, stream)
    o.flags = (GK_FLAG_AUTOTUNE if autotune else 0) | (GK_FLAG_PROFILE if profile else 0)
    return o


def _item_result(it):
    return dict(status=it.status, rank=it.rank, steps=it.steps, restarts=it.restarts, cycles=it.cycles,
                breakdowns=it.breakdowns, matvecs=it.matvecs, resid_est_max=it.resid_est_max, sigma_est=it.sigma_est,
                sigma_next=it.sigma_next)


def gk_psvd_batched(problems, *, seed=None, max_restarts=None, reorth_passes=None, autotune=False, stream=None,
                    check=True, profile=False, predictor=None):
    """Partial SVDs of many dense device operators in one persistent launch.

    problems: sequence of dicts with keys A (2-D CUDA tensor, n <= 4096), k, and optionally
    krylov_dim, tol (default 1e-8), start, rank_cut (relative eps; triplets below it are not converged).
    With predictor (a Predictor) the library runs the learned pipeline: k is each problem's output
    capacity and rank_cut its eps (see gk_psvd_batched in gk.h).  Returns (list of (U, S, V, result
    dict), status, info)."""
    n = len(problems)
    items = (gk_batch_item * n)()
    keep = []
    outs = []
    dev = problems[0]["A"].device
    # one output buffer per kind for the whole batch (views per problem)
    ks = [int(pr["k"]) for pr in problems]
    shapes = [pr["A"].shape for pr in problems]
    uoff, soff, voff = [0], [0], [0]
    for kk, (mm, nn) in zip(ks, shapes):
        uoff.append(uoff[-1] + kk * mm)
        soff.append(soff[-1] + kk)
        voff.append(voff[-1] + kk * nn)
    Ubig = torch.empty(max(uoff[-1], 1), dtype=torch.float64, device=dev)
    Sbig = torch.empty(max(soff[-1], 1), dtype=torch.float64, device=dev)
    Vbig = torch.empty(max(voff[-1], 1), dtype=torch.float64, device=dev)
    for i, pr in enumerate(problems):
        A = pr["A"]
        M, _ = make_matrix(A)
        k = ks[i]
        U = Ubig[uoff[i]:uoff[i + 1]].view(k, A.shape[0])
        S = Sbig[soff[i]:soff[i + 1]]
        V = Vbig[voff[i]:voff[i + 1]].view(k, A.shape[1])
        st = None
        if pr.get("start") is not None:
            _check_start(pr["start"], A.shape[0])
            st = pr["start"].to(torch.float64).contiguous()
            keep.append(st)
        items[i].A = M
        items[i].k = k
        items[i].krylov_dim = int(pr.get("krylov_dim", 0))
        items[i].tol = float(pr.get("tol", 1e-8))
        items[i].rank_cut = float(pr.get("rank_cut", 0.0))
        items[i].U, items[i].S, items[i].V = U.data_ptr(), S.data_ptr(), V.data_ptr()
        items[i].start = st.data_ptr() if st is not None else None
        outs.append((U, S, V))
        keep.append(A)
    o = _batch_opts(dev, seed, max_restarts, reorth_passes, False, autotune, stream, profile)
    if predictor is not None:
        o.predictor = predictor.handle
    info = gk_info()
    status = lib().gk_psvd_batched(items, n, C.byref(o), C.byref(info))
    if check and status < 0:
        raise GKError(status, "gk_psvd_batched")
    d = info.as_dict()
    d["sigma_1"] = Sbig[torch.tensor(soff[:-1], device=dev)]  # each problem's largest value (device)
    # the three device buffers behind the views: problem i's k x m block of U^T, its k values and
    # its k x n block of V^T, back to back in problem order
    d["outputs"] = (Ubig[:uoff[-1]], Sbig[:soff[-1]], Vbig[:voff[-1]])
    return [(U.T, S, V.T, _item_result(items[i])) for i, (U, S, V) in enumerate(outs)], status, d


def gk_numrank_batched(problems, *, seed=None, reorth_passes=None, eps_absolute=False, autotune=False, stream=None,
                       want_sigma=False, check=True, profile=False):
    """Rank estimates (Algorithm 3) of many dense device operators in one persistent launch.

    problems: sequence of dicts with keys A, and optionally kmax (0 = min(m, n, 256)), eps (default 1e-8),
    start.  Returns (list of (rank, sigma or None, result dict), status, info)."""
    n = len(problems)
    items = (gk_batch_item * n)()
    keep = []
    sigs = []
    dev = problems[0]["A"].device
    for i, pr in enumerate(problems):
        A = pr["A"]
        M, _ = make_matrix(A)
        km = int(pr.get("kmax", 0))
        mn = min(A.shape)
        cap = min(mn, 256) if km <= 0 or km > mn else km
        sg = torch.zeros(cap + 2, dtype=torch.float64, device=A.device) if want_sigma else None
        st = None
        if pr.get("start") is not None:
            _check_start(pr["start"], A.shape[0])
            st = pr["start"].to(torch.float64).contiguous()
            keep.append(st)
        items[i].A = M
        items[i].k = km
        items[i].tol = float(pr.get("eps", 1e-8))
        items[i].S = sg.data_ptr() if sg is not None else None
        items[i].start = st.data_ptr() if st is not None else None
        sigs.append(sg)
        keep.append(A)
    o = _batch_opts(dev, seed, None, reorth_passes, eps_absolute, autotune, stream, profile)
    info = gk_info()
    status = lib().gk_numrank_batched(items, n, C.byref(o), C.byref(info))
    if check and status < 0:
        raise GKError(status, "gk_numrank_batched")
    res = []
    for i in range(n):
        r = _item_result(items[i])
        sg = sigs[i][: r["steps"]] if sigs[i] is not None else None
        res.append((items[i].rank, sg, r))
    return res, status, info.as_dict()


# ---------------------------------------------------------------------------
# learned predictor (sketch features and the MLP)
# ---------------------------------------------------------------------------
GK_FEATURES = 35
GK_MLP_TRAINABLE = 75522
GK_MLP_PARAMS = 75596


def _stream_opts(device, stream=None):
    o = default_opts()
    s = stream if stream is not None else torch.cuda.current_stream(device)
    o.stream = s.cuda_stream
    return o


def gk_sketch_batched(mats, seed: int = 2104107, stream=None, tcgen05: bool = False):
    """35 sketch features per dense device operator (count x 35 float32, device).
    tcgen05: the tensor-core form for one bf16 operator (GK_FLAG_SKETCH_TC)."""
    n = len(mats)
    arr = (gk_matrix * n)()
    for i, A in enumerate(mats):
        arr[i], _ = make_matrix(A)
    feats = torch.empty((n, GK_FEATURES), dtype=torch.float32, device=mats[0].device)
    o = _stream_opts(mats[0].device, stream)
    if tcgen05:
        o.flags |= GK_FLAG_SKETCH_TC
    st = lib().gk_sketch_batched(arr, n, C.c_uint64(seed & (2**64 - 1)), _ptr(feats), C.byref(o))
    if st < 0:
        raise GKError(st, "gk_sketch_batched")
    return feats


def gk_mlp_forward(params, x, bf16_weights: bool = False, stream=None):
    x = x.to(torch.float32).contiguous()
    out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
    st = lib().gk_mlp_forward(_ptr(params), _ptr(x), x.shape[0], _ptr(out), int(bf16_weights),
                              C.byref(_stream_opts(x.device, stream)))
    if st < 0:
        raise GKError(st, "gk_mlp_forward")
    return out


def gk_mlp_grad(params, x, y, stream=None):
    x = x.to(torch.float32).contiguous()
    y = y.to(torch.float32).contiguous()
    g = torch.empty(GK_MLP_TRAINABLE, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    st = lib().gk_mlp_grad(_ptr(params), _ptr(x), _ptr(y), x.shape[0], _ptr(g), _ptr(loss),
                           C.byref(_stream_opts(x.device, stream)))
    if st < 0:
        raise GKError(st, "gk_mlp_grad")
    return g, float(loss)


def gk_mlp_train(params, adam_m, adam_v, t0, x, y, batch=256, epochs=1, lr=1e-3, seed=0, stream=None):
    x = x.to(torch.float32).contiguous()
    y = y.to(torch.float32).contiguous()
    losses = torch.zeros(epochs, dtype=torch.float32, device=x.device)
    st = lib().gk_mlp_train(_ptr(params), _ptr(adam_m), _ptr(adam_v), int(t0), _ptr(x), _ptr(y), x.shape[0],
                            int(batch), int(epochs), float(lr), C.c_uint64(seed), _ptr(losses),
                            C.byref(_stream_opts(x.device, stream)))
    if st < 0:
        raise GKError(st, "gk_mlp_train")
    return losses


def gk_rsgd_batched(X, Vd, y, W, batches, q1, eta: float, lam: float, r: int, k_inner: int, *,
                    reorth_passes: int | None = None, autotune: bool = False, stream=None):
    """Algorithm 4 for P problems of one shape (see gk_rsgd_batched in gk.h): X (P, N, d1),
    Vd (P, N, d2), y (P, N), W (P, d1, d2; W0 in, the iterate out, updated in place),
    batches (steps, P, b) int32, q1 (P, d1): contiguous CUDA tensors (f64 but batches).
    Returns (status, info dict)."""
    for t in (X, Vd, y, W, q1):
        if t.dtype != torch.float64 or not t.is_contiguous() or t.device.type != "cuda":
            raise ValueError("X, Vd, y, W, q1 must be contiguous float64 CUDA tensors")
    if batches.dtype != torch.int32 or not batches.is_contiguous() or batches.device.type != "cuda":
        raise ValueError("batches must be a contiguous int32 CUDA tensor")
    if X.dim() != 3 or Vd.dim() != 3 or batches.dim() != 3:
        raise ValueError("X, Vd and batches must be 3-D")
    P, N, d1 = X.shape
    d2 = Vd.shape[2]
    steps, _, b = batches.shape
    if (tuple(Vd.shape) != (P, N, d2) or tuple(y.shape) != (P, N) or tuple(W.shape) != (P, d1, d2)
            or tuple(q1.shape) != (P, d1) or batches.shape[1] != P):
        raise ValueError("shapes: X (P, N, d1), Vd (P, N, d2), y (P, N), W (P, d1, d2), q1 (P, d1), "
                         "batches (steps, P, b)")
    if batches.numel() and (int(batches.min()) < 0 or int(batches.max()) >= N):
        raise ValueError("batch indices must lie in [0, N)")
    a = gk_rsgd_args(P=P, N=N, d1=d1, d2=d2, r=int(r), k_inner=int(k_inner), steps=steps, b=b, eta=float(eta),
                     lam=float(lam), X=X.data_ptr(), Vd=Vd.data_ptr(), y=y.data_ptr(), batches=batches.data_ptr(),
                     q1=q1.data_ptr(), W=W.data_ptr())
    o, ka = _opts(W.device, reorth_passes=reorth_passes, stream=stream)
    if autotune:
        o.flags |= GK_FLAG_AUTOTUNE
    info = gk_info()
    st = lib().gk_rsgd_batched(C.byref(a), C.byref(o), C.byref(info))
    if st < 0:
        raise GKError(st, "gk_rsgd_batched")
    return st, info.as_dict()
