"""The C-ABI library loads and exports every symbol include/hom.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header="hom.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hom_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_00733_gb300 import build, hom
    build.build()
    return hom.load_library()


def test_header_declares_the_solver_calls():
    syms = declared_symbols()
    for s in ["hom_create", "hom_solve", "hom_effective_stiffness", "hom_fields", "hom_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2110_00733_gb300 import hom
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert sorted(hom.EXPORTED) == declared_symbols()


def test_library_exports_every_network_symbol(lib):
    from paper_2110_00733_gb300 import net
    for s in declared_symbols("hom_net.h"):
        assert hasattr(lib, s), s
    assert sorted(net.EXPORTED) == declared_symbols("hom_net.h")
    assert sum(27 * ci * co + co for _, ci, co in net.LAYERS) > 500000


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the header's structs have the C compiler's sizes and
    field offsets."""
    import ctypes
    import subprocess
    from paper_2110_00733_gb300 import hom
    src = tmp_path / "layout.c"
    fields_o = [f for f, _ in hom.hom_options._fields_]
    fields_i = [f for f, _ in hom.hom_solve_info._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hom.h"', "int main(void) {",
             'printf("%zu %zu\\n", sizeof(hom_options), sizeof(hom_solve_info));']
    lines += [f'printf("%zu\\n", offsetof(hom_options, {f}));' for f in fields_o]
    lines += [f'printf("%zu\\n", offsetof(hom_solve_info, {f}));' for f in fields_i]
    lines += ["return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    so, si = int(out[0]), int(out[1])
    assert ctypes.sizeof(hom.hom_options) == so
    assert ctypes.sizeof(hom.hom_solve_info) == si
    offs = [int(v) for v in out[2:]]
    py = [getattr(hom.hom_options, f).offset for f in fields_o] + \
         [getattr(hom.hom_solve_info, f).offset for f in fields_i]
    assert offs == py


def test_missing_library_fails_loudly(tmp_path):
    from paper_2110_00733_gb300 import hom
    saved = hom._lib
    hom._lib = None
    try:
        with pytest.raises(ImportError):
            hom.load_library(str(tmp_path / "nope.so"))
    finally:
        hom._lib = saved


@pytest.mark.parametrize("kw, msg", [
    (dict(E=0.0), "E > 0"),
    (dict(nu=0.5), "nu < 0.5"),
    (dict(input_kind=7), "input_kind"),
    (dict(smoothing=3), "smoothing"),
    (dict(derivative=5), "derivative"),
    (dict(solver=9), "solver"),
    (dict(precision=4), "precision"),
    (dict(shape=(65, 0, 0)), "launch-shape"),
    (dict(sweep_floor=1.0), "sweep_floor"),
])
def test_create_rejects_bad_arguments_before_device_work(lib, kw, msg):
    """hom_create checks its arguments before it touches a device: each bad
    one returns HOM_EINVAL with its message (this runs without a GPU)"""
    import numpy as np
    from paper_2110_00733_gb300 import hom
    phi = np.zeros((8, 8, 8), np.float32)
    with pytest.raises(hom.HomError) as e:
        hom.hom_create((8, 8, 8), phi, **kw)
    assert e.value.code == hom.HOM_EINVAL
    assert msg in str(e.value)


@pytest.mark.parametrize("grid, kw, code", [
    ((65, 8, 8), {}, "HOM_EUNSUPPORTED_GRID"),
    ((7, 8, 8), {}, "HOM_EUNSUPPORTED_GRID"),
    ((64, 32, 20), {}, "HOM_EUNSUPPORTED_GRID"),
    ((8, 8, 8), dict(E=-1.0), "HOM_EINVAL"),
    ((8, 8, 8), dict(derivative=3), "HOM_EINVAL"),
])
def test_noalloc_rejects_bad_arguments_before_device_work(lib, grid, kw, code):
    """the allocation-free A(eps) checks grid sizes (each in [2, 64] of the
    form 2^a 3^b 5^c, at most 32768 voxels), E, nu and the derivative before
    it touches a device"""
    import numpy as np
    from paper_2110_00733_gb300 import hom
    phi = np.zeros(grid, np.float32)
    eps = np.zeros((6,) + grid, np.float32)
    with pytest.raises(hom.HomError) as e:
        hom.hom_apply_noalloc(grid, phi, eps, np.zeros_like(eps), **kw)
    assert e.value.code == getattr(hom, code)
