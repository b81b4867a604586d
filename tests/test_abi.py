"""The C-ABI library loads and exports every symbol include/hom.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hom_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_00733_gb300 import build, hom
    build.build()
    return hom.load_library()


def test_header_declares_the_north_star_calls():
    syms = declared_symbols()
    for s in ["hom_create", "hom_solve", "hom_effective_stiffness", "hom_fields", "hom_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2110_00733_gb300 import hom
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert sorted(hom.EXPORTED) == declared_symbols()


def test_struct_layouts_match_header():
    import ctypes
    from paper_2110_00733_gb300 import hom
    # hom_options: 3 ints, (pad), pointer, 5 ints, (pad)
    assert ctypes.sizeof(hom.hom_options) == 48
    # hom_solve_info: 4 ints + 2 doubles + 6 doubles + 1 double
    assert ctypes.sizeof(hom.hom_solve_info) == 16 + 8 * 9


def test_missing_library_fails_loudly(tmp_path):
    from paper_2110_00733_gb300 import hom
    saved = hom._lib
    hom._lib = None
    try:
        with pytest.raises(ImportError):
            hom.load_library(str(tmp_path / "nope.so"))
    finally:
        hom._lib = saved
