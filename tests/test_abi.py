"""The C-ABI library loads and exports every entry point include/ls.h declares (CPU only)."""
import os
import re

from paper_1602_07652_gb300 import binding, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    lib = binding.load_library()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(binding.EXPORTED)


def test_status_strings_and_defaults():
    lib = binding.load_library()
    assert lib.ls_strerror(0) == b"ok"
    assert b"NaN" in lib.ls_strerror(-6)
    o = binding.default_opts()
    assert o.inner_tol == 1e-3 and o.shift == 10.0 and o.inner_restart == 30
