"""gk_matvec_static: the operator product for callers that cannot call cudaMalloc
(their device memory is owned by another allocator, or an allocation would stall a
latency-critical loop).  Its scratch is a static device array inside the library.

Checked through the C ABI against gk_matvec, the allocating entry point that runs the
same kernels, on two calls in a row (the second call finds the first call's leftovers
in the shared array): dense f64/f32/bf16, f16 with a power-of-two scale, CSR (f32 and
bf16, both directions), the size limit on both sides of it, and the arguments it
refuses.  This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

U32 = 2.0**-24


def _raw():
    from paper_2104_10785_gb300 import gk as raw

    return raw


def _static_call(raw, A, x, trans, scale=1.0, y=None):
    M, _ = raw.make_matrix(A, scale)
    if y is None:
        y = torch.full((M.n if trans else M.m,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = raw.lib().gk_matvec_static(C.byref(M), int(trans), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), None)
    return st, y


def _check_twice(raw, A, x, trans, ref, tol, scale=1.0):
    import paper_2104_10785_gb300 as gk

    for call in range(2):
        st, y = _static_call(raw, A, x, trans, scale)
        assert st == raw.GK_OK, gk.status_string(st)
        y = y.cpu().numpy()
        assert np.all(np.isfinite(y))
        assert np.all(np.abs(y - ref) <= tol), (call, np.abs(y - ref).max())


@pytest.mark.parametrize("dtype,shape,scale", [(torch.float32, (3001, 2049), 1.0), (torch.bfloat16, (1000, 1537), 1.0),
                                               (torch.float64, (777, 555), 1.0), (torch.float32, (64, 40000), 1.0),
                                               (torch.float16, (1203, 517), 0.25)])
def test_static_scratch_product_matches_gk_matvec(dtype, shape, scale):
    import paper_2104_10785_gb300 as gk

    raw = _raw()
    g = np.random.default_rng(shape[0] * 7 + shape[1])
    A = torch.from_numpy(g.standard_normal(shape)).to(dtype).cuda()
    Ad = A.double().cpu().numpy() * scale
    for trans in (0, 1):
        x = torch.from_numpy(g.standard_normal(shape[0] if trans else shape[1])).cuda()
        ref = gk.gk_matvec(A, x, trans=bool(trans), scale=scale).cpu().numpy()
        mag = (np.abs(Ad).T if trans else np.abs(Ad)) @ np.abs(x.cpu().numpy())
        tol = (1e-13 if dtype == torch.float64 else U32 * 66) * mag + 1e-300
        _check_twice(raw, A, x, trans, ref, tol, scale)


@pytest.mark.parametrize("dtype", [np.float32, "bf16"])
def test_static_scratch_csr_matches_gk_matvec(dtype):
    """CSR operators: the static call takes the default lanes per row (it reads no device
    value on the host), gk_matvec sizes them from nnz; both multiply in f64."""
    import paper_2104_10785_gb300 as gk

    raw = _raw()
    m, n = 4007, 2503
    d = synth.sparse_planted(m, n, 20, 10.0 * 0.9 ** np.arange(1, 6), 17, usup=200, vsup=100, dtype=np.float32)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    if dtype == "bf16":
        vals = dev(synth.to_bf16_bits(d["vals"]).view(np.int16)).view(torch.bfloat16)
        tvals = dev(synth.to_bf16_bits(d["t_vals"]).view(np.int16)).view(torch.bfloat16)
    else:
        vals, tvals = dev(d["vals"]), dev(d["t_vals"])
    A = gk.CSR(m, n, dev(d["rowptr"]), dev(d["colind"]), vals, dev(d["t_rowptr"]), dev(d["t_colind"]), tvals)
    g = np.random.default_rng(5)
    for trans in (0, 1):
        x = torch.from_numpy(g.standard_normal(m if trans else n)).cuda()
        ref = gk.gk_matvec(A, x, trans=bool(trans)).cpu().numpy()
        tol = 1e-13 * (np.abs(ref) + np.abs(ref).max()) + 1e-300
        _check_twice(raw, A, x, trans, ref, tol)


def test_static_scratch_limit_both_sides():
    """Dense A^T x needs 8 n (row blocks) bytes of partial sums, row blocks of 1024 rows at this
    size: n = 32000 fits the 32 MiB array with m = 131072 (128 row blocks), n = 33000 does not."""
    import paper_2104_10785_gb300 as gk

    raw = _raw()
    m = 131072
    A = torch.empty((m, 33000), dtype=torch.float32, device="cuda")
    x = torch.zeros(m, dtype=torch.float64, device="cuda")
    st, y = _static_call(raw, A, x, 1)
    assert st == raw.GK_OUT_OF_MEMORY
    assert torch.isnan(y).all()  # nothing was written
    del A, y
    torch.cuda.empty_cache()
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn((m, 32000), dtype=torch.float32, device="cuda", generator=g)
    x = torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
    ref = gk.gk_matvec(A, x, trans=True)
    mag = (A.abs().T @ x.abs().float()).double()
    for _ in range(2):
        st, y = _static_call(raw, A, x, 1)
        assert st == raw.GK_OK, gk.status_string(st)
        assert bool(((y - ref).abs() <= U32 * 66 * mag * 1.01 + 1e-300).all())
    del A, x, y, ref, mag
    torch.cuda.empty_cache()


def test_static_scratch_refused_arguments():
    raw = _raw()
    # host operands would need a staging allocation: refused
    Ah = torch.ones((8, 4), dtype=torch.float32)
    M, _ = raw.make_matrix(Ah)
    xh = torch.ones(4, dtype=torch.float64)
    yd = torch.empty(8, dtype=torch.float64, device="cuda")
    st = raw.lib().gk_matvec_static(C.byref(M), 0, C.c_void_p(xh.data_ptr()), C.c_void_p(yd.data_ptr()), None)
    assert st == raw.GK_INVALID_ARG
    # x and y sharing memory (a square operator in place): refused
    A = torch.randn((64, 64), dtype=torch.float64, device="cuda")
    buf = torch.randn(96, dtype=torch.float64, device="cuda")
    for trans in (0, 1):
        st, _ = _static_call(raw, A, buf[:64], trans, y=buf[:64])
        assert st == raw.GK_INVALID_ARG
        st, _ = _static_call(raw, A, buf[:64], trans, y=buf[32:96])
        assert st == raw.GK_INVALID_ARG
    # memory of another GPU: refused before any launch
    if torch.cuda.device_count() > 1:
        A1 = torch.randn((64, 64), dtype=torch.float64, device="cuda:1")
        x0 = torch.randn(64, dtype=torch.float64, device="cuda:0")
        with torch.cuda.device(0):
            st, _ = _static_call(raw, A1, x0, 0)
        assert st == raw.GK_INVALID_ARG
