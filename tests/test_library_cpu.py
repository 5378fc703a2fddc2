"""Host-side checks of the CUDA library that need no GPU: it builds for sm_103a, loads,
exports every entry point declared in include/gk.h, and refuses to compute without a
device (no host fallback)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|size_t|char)\s*\*?\s*(gk_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["gk_psvd", "gk_numrank", "gk_psvd_workspace", "gk_numrank_workspace", "gk_matvec",
                 "gk_residuals", "gk_status_string", "gk_default_opts"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_2104_10785_gb300 as gk

    path = gk.library_path()
    gk.lib()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(gk_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    """Every translation unit is compiled for sm_103a alone (one -gencode, no PTX for other targets)."""
    import paper_2104_10785_gb300 as gk
    from paper_2104_10785_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    gk.lib()
    assert gk.library_path().endswith("libgk.so")


def test_status_strings_and_defaults():
    import paper_2104_10785_gb300 as gk
    from paper_2104_10785_gb300 import gk as raw

    assert gk.status_string(0) == "GK_OK"
    assert gk.status_string(-7) == "GK_NO_DEVICE"
    o = raw.default_opts()
    assert o.reorth_passes == 0 and o.max_restarts == 200 and o.krylov_dim == 0
    assert "sm_103a" in gk.version()


def test_no_device_means_no_compute():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C

    import numpy as np
    from paper_2104_10785_gb300 import gk as raw

    A = np.ones((4, 3))
    M = raw.gk_matrix(raw.GK_DENSE, raw.GK_F64, 4, 3, 3, 1.0, A.ctypes.data, None, None, None, None, None)
    r = C.c_int(-1)
    st = raw.lib().gk_numrank(C.byref(M), 1e-8, 0, None, C.byref(r), None, None)
    assert st == raw.GK_NO_DEVICE and r.value == -1
    U = np.zeros((3, 4)); S = np.zeros(3); V = np.zeros((3, 3))
    st = raw.lib().gk_psvd(C.byref(M), 1, 1e-8, None, U.ctypes.data, S.ctypes.data, V.ctypes.data, None)
    assert st == raw.GK_NO_DEVICE
    st = raw.lib().gk_fsvd(C.byref(M), 2, 1, 1, None, U.ctypes.data, S.ctypes.data, V.ctypes.data, None)
    assert st == raw.GK_NO_DEVICE


def test_operator_descriptors_from_tensors():
    """The binding describes what it is given (row stride, storage type, CSR arrays) and
    refuses layouts the library cannot read, before any call."""
    import torch

    from paper_2104_10785_gb300 import gk as raw

    buf = torch.zeros(6, 12, dtype=torch.bfloat16)
    M, keep = raw.make_matrix(buf[:, :10])
    assert (M.kind, M.dtype, M.m, M.n, M.ld) == (raw.GK_DENSE, raw.GK_BF16, 6, 10, 12)
    assert M.vals == buf.data_ptr() and keep[0].data_ptr() == buf.data_ptr()
    for dt, code in ((torch.float64, raw.GK_F64), (torch.float32, raw.GK_F32), (torch.float16, raw.GK_F16)):
        assert raw.make_matrix(torch.zeros(3, 2, dtype=dt), scale=2.0)[0].dtype == code
    with pytest.raises(ValueError):
        raw.make_matrix(torch.zeros(4, 5).T)  # column stride 4
    with pytest.raises(ValueError):
        raw.make_matrix(torch.zeros(4, 5, dtype=torch.int32))
    with pytest.raises(ValueError):
        raw.make_matrix(torch.zeros(4))
    i32 = lambda *v: torch.tensor(v, dtype=torch.int32)
    C = raw.CSR(2, 3, i32(0, 1, 2), i32(0, 2), torch.ones(2), i32(0, 1, 1, 2), i32(0, 1), torch.ones(2))
    M, _ = raw.make_matrix(C)
    assert (M.kind, M.dtype, M.m, M.n) == (raw.GK_CSR, raw.GK_F32, 2, 3)
    with pytest.raises(ValueError):
        raw.make_matrix(raw.CSR(2, 3, C.rowptr.long(), C.colind, C.vals, C.t_rowptr, C.t_colind, C.t_vals))


def test_rsgd_entry_checks_arguments_before_the_device():
    """gk_rsgd_batched refuses sizes outside its limits with GK_INVALID_ARG, and a valid request
    without a device with GK_NO_DEVICE (no host fallback)."""
    import ctypes as C

    import torch
    from paper_2104_10785_gb300 import gk as raw

    def args(**kw):
        base = dict(P=2, N=100, d1=30, d2=20, r=3, k_inner=12, steps=2, b=10, eta=0.5, lam=0.0, X=1, Vd=1, y=1,
                    batches=1, q1=1, W=1)
        base.update(kw)
        return raw.gk_rsgd_args(**base)

    L = raw.lib()
    for bad in (dict(P=0), dict(b=0), dict(N=5), dict(r=0), dict(r=17), dict(k_inner=4), dict(k_inner=21),
                dict(d2=5000), dict(d1=1), dict(steps=-1), dict(eta=float("nan"))):
        assert L.gk_rsgd_batched(C.byref(args(**bad)), None, None) == raw.GK_INVALID_ARG, bad
    if not torch.cuda.is_available():
        assert L.gk_rsgd_batched(C.byref(args()), None, None) == raw.GK_NO_DEVICE


def test_block_numrank_checks_arguments_before_the_device():
    """gk_block_numrank refuses a block size outside 1..min(32, m, n), a negative or non-finite
    eps, the absolute threshold and a block count past the small SVD's order with
    GK_INVALID_ARG; a valid request without a device gets GK_NO_DEVICE (no host fallback)."""
    import ctypes as C

    import numpy as np
    import torch
    from paper_2104_10785_gb300 import gk as raw

    A = np.ones((40, 30))
    M = raw.gk_matrix(raw.GK_DENSE, raw.GK_F64, 40, 30, 30, 1.0, A.ctypes.data, None, None, None, None, None)
    L = raw.lib()

    def call(s=4, eps=1e-8, kmax=0, absolute=0):
        o = raw.default_opts()
        o.eps_absolute = absolute
        r = C.c_int(-1)
        return L.gk_block_numrank(C.byref(M), s, None, eps, kmax, C.byref(o), C.byref(r), None, None, None)

    for bad in (dict(s=0), dict(s=33), dict(s=31), dict(eps=-1.0), dict(eps=float("nan")), dict(eps=float("inf")),
                dict(absolute=1), dict(s=4, kmax=256), dict(s=1, kmax=1024)):
        assert call(**bad) == raw.GK_INVALID_ARG, bad
    for s_bad in (0, 33, 31):
        assert L.gk_block_numrank_workspace(C.byref(M), s_bad, 0, None) == 0
    assert L.gk_block_numrank_workspace(C.byref(M), 4, 256, None) == 0
    if not torch.cuda.is_available():
        assert call() == raw.GK_NO_DEVICE
        assert call(s=4, kmax=255) == raw.GK_NO_DEVICE  # (255 + 1) * 4 = 1024
        assert L.gk_block_numrank_workspace(C.byref(M), 4, 0, None) == 0


def test_block_numrank_binding_checks_the_start_block_shape():
    """The binding refuses a start block that is not m x s before anything reaches the library
    (the library reads m * s values from it)."""
    import torch

    import paper_2104_10785_gb300 as gk

    A = torch.zeros(10, 6, dtype=torch.float64)
    for bad in (torch.zeros(10, 3), torch.zeros(9, 2), torch.zeros(20)):
        with pytest.raises(ValueError):
            gk.gk_block_numrank(A, 2, start=bad)


def test_bindings_check_the_start_vector_length():
    """gk_psvd, gk_fsvd and gk_numrank refuse a start vector whose length is not m before the
    library would read m values from it."""
    import torch

    import paper_2104_10785_gb300 as gk

    A = torch.zeros(10, 6, dtype=torch.float64)
    bad = torch.zeros(9, dtype=torch.float64)
    with pytest.raises(ValueError):
        gk.gk_psvd(A, 2, start=bad)
    with pytest.raises(ValueError):
        gk.gk_fsvd(A, 3, 2, start=bad)
    with pytest.raises(ValueError):
        gk.gk_numrank(A, 1e-8, start=bad)


def test_bindings_check_vector_and_factor_shapes():
    """gk_matvec and gk_residuals refuse vectors and factors whose sizes do not match the
    operator before the library would read past them."""
    import torch

    import paper_2104_10785_gb300 as gk

    A = torch.zeros(10, 6, dtype=torch.float64)
    with pytest.raises(ValueError):
        gk.gk_matvec(A, torch.zeros(10, dtype=torch.float64))
    with pytest.raises(ValueError):
        gk.gk_matvec(A, torch.zeros(6, dtype=torch.float64), trans=True)
    with pytest.raises(ValueError):
        gk.gk_residuals(A, torch.zeros(10, 2), torch.zeros(2), torch.zeros(5, 2))
    with pytest.raises(ValueError):
        gk.gk_residuals(A, torch.zeros(10, 3), torch.zeros(2), torch.zeros(6, 2))


def test_plain_c_client_compiles_links_and_gets_no_device(tmp_path):
    """tests/native/abi_client.c references every entry point of include/gk.h from C11 (pedantic,
    warnings as errors) and links against libgk.so; without a device its calls return
    GK_NO_DEVICE, and a refused argument GK_INVALID_ARG, before any pointer is touched."""
    import shutil

    import torch

    import paper_2104_10785_gb300 as gk

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = gk.library_path()
    gk.lib()
    exe = str(tmp_path / "abi_client")
    subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-o", exe,
                    os.path.join(ROOT, "tests", "native", "abi_client.c"), "-L" + os.path.dirname(lib), "-lgk",
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    if torch.cuda.is_available():
        return  # the expected statuses below are those of a machine without a GPU
    env = dict(os.environ)
    dirs = ["/usr/local/cuda/lib64", os.path.join(os.path.dirname(torch.__file__), "lib")]
    env["LD_LIBRARY_PATH"] = ":".join(dirs + [env.get("LD_LIBRARY_PATH", "")])
    out = subprocess.run([exe], capture_output=True, text=True, env=env, check=True).stdout.split()
    no_dev, inval = str(-7), str(-1)
    assert out[:6] == [no_dev, no_dev, no_dev, no_dev, inval, no_dev], out
    assert out[6] == "GK_NO_DEVICE"


def test_block_fsvd_checks_arguments_before_the_device():
    """gk_block_fsvd refuses a block size outside 1..min(32, m, n), no steps, (steps + 1) s past
    1024, and r outside 1..steps s with GK_INVALID_ARG before it looks for a device."""
    import ctypes as C

    import numpy as np
    import torch
    from paper_2104_10785_gb300 import gk as raw

    A = np.ones((40, 30))
    M = raw.gk_matrix(raw.GK_DENSE, raw.GK_F64, 40, 30, 30, 1.0, A.ctypes.data, None, None, None, None, None)
    L = raw.lib()
    buf = np.zeros(40 * 30)
    p = buf.ctypes.data

    def call(s=4, steps=3, r=5):
        return L.gk_block_fsvd(C.byref(M), s, None, steps, r, None, p, p, p, p, None)

    for bad in (dict(s=0), dict(s=33), dict(steps=0), dict(s=4, steps=256), dict(r=0), dict(s=4, steps=3, r=13)):
        assert call(**bad) == raw.GK_INVALID_ARG, bad
    if not torch.cuda.is_available():
        assert call() == raw.GK_NO_DEVICE


def test_binding_structs_match_the_c_layout(tmp_path):
    """Every struct the binding mirrors (gk_matrix, gk_opts, gk_info, gk_batch_item, gk_rsgd_args)
    has, under the C compiler and include/gk.h, the same size and the same offset for each field
    as its ctypes class: a field added on one side only would shift every field after it."""
    import ctypes
    import shutil

    from paper_2104_10785_gb300 import gk as binding

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [binding.gk_matrix, binding.gk_opts, binding.gk_info, binding.gk_batch_item, binding.gk_rsgd_args]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gk.h"', "int main(void) {"]
    want = []
    for cls in structs:
        name = cls.__name__
        lines.append('  printf("%%zu\\n", sizeof(%s));' % name)
        want.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (name, f))
            want.append(getattr(cls, f).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"), "-o", exe, str(src)],
                   check=True)
    got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want
