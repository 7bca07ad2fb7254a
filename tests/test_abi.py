"""The C-ABI library builds, loads and exports every function that
include/xengine.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xengine.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(corr_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1904_07778_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("corr_create", "corr_push", "corr_dump", "corr_normalise", "corr_sync",
              "corr_destroy", "corr_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for name in _declared():
        assert name in exported, name


def test_pure_host_calls(lib_path):
    """Calls that touch no device: status strings, baseline counts, argument checks."""
    from paper_1904_07778_gb300 import xengine as xe
    assert xe.corr_strerror(0) == "ok"
    assert xe.corr_strerror(xe.CORR_ESEQ) == "block sequence gap or duplicate"
    assert xe.corr_n_baselines(32) == 528
    assert xe.corr_n_baselines(192) == 18528
    assert xe.corr_n_baselines(512) == 131328
    assert xe.corr_n_baselines(0) == 0
    lib = ctypes.CDLL(lib_path)
    lib.corr_create.argtypes = [ctypes.c_int] * 5 + [ctypes.c_uint, ctypes.c_void_p, ctypes.c_void_p]
    ctx = ctypes.c_void_p()
    # invalid shapes are rejected before any device work
    assert lib.corr_create(0, 1, 1, 4, 0, 0, None, ctypes.byref(ctx)) == xe.CORR_EINVAL
    assert lib.corr_create(4, 1, 1, 5, 0, 0, None, ctypes.byref(ctx)) == xe.CORR_EINVAL
    assert lib.corr_create(4, 1, 1, 4, 7, 0, None, ctypes.byref(ctx)) == xe.CORR_EINVAL
    assert lib.corr_create(4, 1, 1, 4, 0, 0, None, None) == xe.CORR_EINVAL
    lib.corr_destroy.argtypes = [ctypes.c_void_p]
    assert lib.corr_destroy(None) == 0


def test_binding_has_no_cpu_fallback():
    """The product path imports nothing from the oracle."""
    pkg = os.path.join(ROOT, "paper_1904_07778_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f
