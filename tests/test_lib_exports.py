"""The C-ABI library builds, loads and exports every entry point of include/dcf.h
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "dcf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9\s\*]*?\b(dcf_[A-Za-z_0-9]+)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2207_11669_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["dcf_create", "dcf_load_blocks", "dcf_step", "dcf_solve", "dcf_get_LS",
                     "dcf_destroy", "dcf_load_init", "dcf_get_factors", "dcf_get_stats"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2207_11669_gb300 import dcf
    assert set(header_functions()) <= set(dcf.exported_symbols())


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2207_11669_gb300 import dcf
    monkeypatch.setattr(dcf, "_LIB", None)
    monkeypatch.setattr(dcf, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(dcf.DcfError):
        dcf.lib()
