"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/emucov.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "emucov.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emu_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_04440_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("emu_cov_build", "emu_potrf_mp", "emu_solve_refine", "emu_sample"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    import paper_2408_04440_gb300 as E

    assert sorted(E.EXPORTED) == _declared()


def test_status_strings(lib):
    lib.emu_status_str.restype = ctypes.c_char_p
    assert lib.emu_status_str(0) == b"ok"
    assert b"positive definite" in lib.emu_status_str(3)


def test_library_is_built_for_sm103a_only():
    from paper_2408_04440_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2408_04440_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "emu_oracle" not in text, f
