"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/mix.h declares (CPU only: no device calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:int|const char\s*\*|void)\s+(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libmix():
    from paper_2502_19081_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(libmix):
    names = _declared()
    assert "mix_init" in names and "mix_step" in names and len(names) >= 19
    missing = [n for n in names if not hasattr(libmix, n)]
    assert not missing, missing


def test_binding_lists_the_header(libmix):
    from paper_2502_19081_gb300 import mix
    assert sorted(mix.EXPORTS) == sorted(n for n in _declared() if n in mix.EXPORTS)
    assert set(mix.EXPORTS) <= set(_declared())


def test_strerror_is_host_only(libmix):
    libmix.mix_strerror.restype = ctypes.c_char_p
    assert libmix.mix_strerror(0) == b"ok"
    assert libmix.mix_strerror(-4) == b"capacity overflow"
    assert libmix.mix_strerror(12345) == b"unknown status"


def test_null_arguments_rejected_without_device(libmix):
    out = ctypes.c_void_p()
    assert libmix.mix_init(None, None, None, None, None, ctypes.byref(out)) == -1
    assert libmix.mix_destroy(None) == 0


def test_product_code_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_2502_19081_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f
