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


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding passes through the ABI has the size and field
    offsets the C header gives it (a host C program compiled against
    include/mix.h prints them; no device involved)."""
    import shutil
    import subprocess

    from paper_2502_19081_gb300 import mix
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [getattr(mix, n) for n in dir(mix)
               if n.startswith("mix_") and isinstance(getattr(mix, n), type)
               and issubclass(getattr(mix, n), ctypes.Structure)]
    assert len(structs) >= 10
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mix.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'    printf("%s sizeof %zu\\n", "{s.__name__}", sizeof({s.__name__}));')
        for f, _ in s._fields_:
            lines.append(f'    printf("%s %s %zu\\n", "{s.__name__}", "{f}", offsetof({s.__name__}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        name, field, val = line.split()
        s = getattr(mix, name)
        want = ctypes.sizeof(s) if field == "sizeof" else getattr(s, field).offset
        assert int(val) == want, (name, field, int(val), want)
        seen += 1
    assert seen == sum(len(s._fields_) + 1 for s in structs)
