"""The C-ABI library builds, loads and exports every function that
include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:corr|fe|pk)_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_1904_07778_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("corr_create", "corr_push", "corr_dump", "corr_normalise", "corr_sync",
              "corr_destroy", "corr_strerror", "fe_create", "fe_channelise", "fe_gains_from_power",
              "pk_create", "pk_push", "pk_next", "pk_release", "pk_crc32"):
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
    # corr_push_many checks its context and block list before any device work
    lib.corr_push_many.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t,
                                   ctypes.c_uint64]
    blocks = (ctypes.c_void_p * 2)(None, None)
    assert lib.corr_push_many(None, blocks, 2, 64, xe.CORR_SEQ_ANY) == xe.CORR_EINVAL
    assert lib.corr_push_many(None, None, 2, 64, xe.CORR_SEQ_ANY) == xe.CORR_EINVAL


def test_binding_has_no_cpu_fallback():
    """The product path imports nothing from the oracle."""
    pkg = os.path.join(ROOT, "paper_1904_07778_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f


def test_fengine_host_calls(lib_path):
    """fe_create rejects bad shapes before any device work; the Eq. 3 gain
    rule (pure host code) equals the oracle's bit for bit."""
    import numpy as np
    from oracle import fengine as ofe
    from paper_1904_07778_gb300 import fengine as fe
    from paper_1904_07778_gb300 import xengine as xe
    lib = ctypes.CDLL(lib_path)
    lib.fe_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_uint, ctypes.c_void_p, ctypes.c_void_p]
    f = ctypes.c_void_p()
    for args in ((0, 64, 4, 0), (4, 100, 4, 0), (4, 8, 4, 0), (4, 4096, 4, 0), (4, 64, 0, 0),
                 (4, 64, 17, 0), (4, 64, 4, 25), (4, 64, 4, -1)):
        assert lib.fe_create(*args, 0, None, ctypes.byref(f)) == xe.CORR_EINVAL, args
    assert lib.fe_create(4, 64, 4, 0, 2, None, ctypes.byref(f)) == xe.CORR_EINVAL
    rng = np.random.default_rng(8)
    P = rng.integers(0, 1 << 40, (64, 12))
    P[3, 4] = 0
    P[5, 6] = 1
    for n, target in ((1000, 2.5), (7, 2.0), (123456, 3.0)):
        got = fe.fe_gains_from_power(P, n, target)
        assert np.array_equal(got.astype(np.int64), ofe.gains_from_power(P, n, target))
