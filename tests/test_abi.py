"""The C ABI boundary without a GPU: the in-tree library builds, loads, and
exports exactly the entry points that include/sptrsv.h declares; the Python
binding declares the same names.  No compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sptrsv.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sptrsv_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2609_40159_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if ln.split()[-1].startswith("sptrsv_")})
    assert exported == _declared()


def test_binding_declares_same_names(lib_path):
    from paper_2609_40159_gb300 import _lib
    assert _lib.DECLARED == _declared()
    lib = _lib.load(lib_path)
    for name in _declared():
        assert hasattr(lib, name)
    assert lib.sptrsv_status_string(7) == b"a bounded device wait gave up"
    assert lib.sptrsv_status_string(0) == b"ok"


def test_checked_variant_exports_the_same_abi(lib_path):
    """The bounds-checked debug variant (SPTRSV_CHECKED) is built beside the
    product library, exports the same entry points and says which it is."""
    from paper_2609_40159_gb300 import _lib
    assert os.path.exists(_lib.LIB_CHECKED_PATH)
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_CHECKED_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if ln.split()[-1].startswith("sptrsv_")})
    assert exported == _declared()
    assert _lib.load(_lib.LIB_CHECKED_PATH).sptrsv_checked_build() == 1
    assert _lib.load(lib_path).sptrsv_checked_build() == 0


def test_missing_library_fails_loudly(tmp_path):
    from paper_2609_40159_gb300 import _lib
    with pytest.raises(OSError, match="no CPU fallback"):
        _lib.load(str(tmp_path / "missing.so"))


def test_header_compiles_as_plain_c(tmp_path):
    c = tmp_path / "use.c"
    c.write_text('#include "sptrsv.h"\nint main(void){ sptrsv_plan_opts o = {0}; return (int)o.mode; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-c", str(c), "-o", str(tmp_path / "use.o")], check=True)


def test_status_codes_match_header():
    from paper_2609_40159_gb300 import _lib
    src = open(HEADER).read()
    for name, val in re.findall(r"(SPTRSV_E[A-Z]+|SPTRSV_OK)\s*=\s*(\d+)", src):
        assert getattr(_lib, name) == int(val)


def test_every_entry_point_rejects_null_arguments():
    """With NULL handles, plans and descriptors (and zero sizes) every entry
    point returns SPTRSV_EINVAL before it touches a device (this runs on a
    machine without a GPU)."""
    import ctypes as C
    from paper_2609_40159_gb300 import _lib as L
    lib = L.lib()
    for name, sig in L._SIGS.items():
        if name == "sptrsv_status_string":
            continue
        args = [t(0) if t in (C.c_int32, C.c_int64, C.c_double) else None for t in sig]
        assert getattr(lib, name)(*args) == L.SPTRSV_EINVAL, name
