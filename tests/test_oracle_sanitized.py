"""The oracle's C part (oracle/gk_oracle.c) built with AddressSanitizer and
UndefinedBehaviorSanitizer, and the oracle's pin tests run against that build in a child process:
an access outside a buffer or undefined behaviour in the oracle would fail them here, where in the
ordinary build it could go unnoticed and corrupt an expected value."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import oracle
oracle._LIB_PATH = {lib!r}
oracle.build = lambda force=False: oracle._LIB_PATH
assert oracle.lib()._name == {lib!r}
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + {files!r}))
"""


def runtime(name):
    cc = shutil.which("gcc")
    p = subprocess.run([cc, "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_oracle_pins_pass_under_sanitizers(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    asan, ubsan = runtime("libasan.so"), runtime("libubsan.so")
    if asan is None or ubsan is None:
        pytest.skip("no sanitizer runtime")
    lib = str(tmp_path / "libgk_oracle_asan.so")
    subprocess.run([cc, "-O1", "-g", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fsanitize=address,undefined",
                    "-fno-sanitize-recover=all", "-o", lib, os.path.join(ROOT, "oracle", "gk_oracle.c"), "-lm"],
                   check=True)
    files = [os.path.join(ROOT, "tests", f) for f in
             ("test_oracle.py", "test_oracle_block_gk.py", "test_oracle_rsgd.py", "test_oracle_mlp.py")]
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib, files=files))
    env = dict(os.environ, LD_PRELOAD=asan + ":" + ubsan, ASAN_OPTIONS="detect_leaks=0", OMP_NUM_THREADS="2")
    out = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, env=env, cwd=str(tmp_path),
                         timeout=900)
    assert out.returncode == 0, (out.stdout[-3000:] + out.stderr[-3000:])
