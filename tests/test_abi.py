"""The C ABI library builds, loads and exports every declared entry point.

No compute calls here: this runs without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2007_16076_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gapsp_[a-z_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib_path():
    try:
        return _build.build()
    except (FileNotFoundError, RuntimeError) as e:  # no nvcc
        pytest.skip(f"cannot build: {e}")


def test_header_declares_the_boundary():
    assert {"gapsp_create", "gapsp_all_pairs", "gapsp_rows", "gapsp_destroy",
            "gapsp_strerror"} <= _declared()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gapsp_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing


def test_library_loads(lib_path):
    try:
        lib = ctypes.CDLL(lib_path)
    except OSError as e:  # libcudart missing on a machine without CUDA
        pytest.skip(str(e))
    for name in _declared():
        assert hasattr(lib, name)
    lib.gapsp_strerror.restype = ctypes.c_char_p
    assert lib.gapsp_strerror(3) == b"memory budget exceeded"


def test_default_opts(lib_path):
    from paper_2007_16076_gb300 import Opts
    try:
        lib = ctypes.CDLL(lib_path)
    except OSError as e:
        pytest.skip(str(e))
    o = Opts()
    lib.gapsp_default_opts(ctypes.byref(o))
    assert (o.conn, o.kind, o.B, o.seed, o.mem_budget) == (8, 0, 32, 0, 0)


def test_invalid_arguments_rejected_without_gpu(lib_path):
    """Argument checks come before any CUDA call."""
    from paper_2007_16076_gb300 import Opts
    try:
        lib = ctypes.CDLL(lib_path)
    except OSError as e:
        pytest.skip(str(e))
    P = ctypes.c_void_p
    lib.gapsp_create.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(Opts),
                                 ctypes.POINTER(P)]
    h = P()
    img = (ctypes.c_uint8 * 4)()
    o = Opts()
    lib.gapsp_default_opts(ctypes.byref(o))
    assert lib.gapsp_create(img, 0, 4, None, ctypes.byref(o), ctypes.byref(h)) == 1
    assert lib.gapsp_create(img, 300, 4, None, ctypes.byref(o), ctypes.byref(h)) == 1
    o.conn = 6
    assert lib.gapsp_create(img, 2, 2, None, ctypes.byref(o), ctypes.byref(h)) == 1
    o.conn = 8
    o.kind = 1  # mask kind without a mask
    assert lib.gapsp_create(img, 2, 2, None, ctypes.byref(o), ctypes.byref(h)) == 1
    o.kind = 0
    o.warm_start = 1  # 0 (on) or -1 (off) only
    assert lib.gapsp_create(img, 2, 2, None, ctypes.byref(o), ctypes.byref(h)) == 1
    o.warm_start = 0
    for fr in (-4, 33):  # fill variants -3..32 only
        o.fill_rows = fr
        assert lib.gapsp_create(img, 2, 2, None, ctypes.byref(o), ctypes.byref(h)) == 1
    assert not h
    lib.gapsp_destroy(None)  # NULL-safe
