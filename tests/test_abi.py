"""CPU checks of the C ABI: the library loads, exports every symbol include/pfc.h
declares, the Python struct mirrors the C struct, and the host-only helpers
work.  No CUDA computation is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pfc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2103_04856_gb300 import build, pfc
    if not os.path.exists(pfc.LIB_PATH):
        build.build()
    return pfc.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pfc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_what_binding_exports():
    from paper_2103_04856_gb300 import pfc
    assert declared_functions() == sorted(pfc.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof as the C compiler lays out `struct` of pfc.h."""
    import subprocess
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pfc.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


def test_problem_struct_layout_matches_header(tmp_path):
    from paper_2103_04856_gb300 import pfc
    fields = [name for name, _ in pfc._CProblem._fields_]
    got = _c_layout(tmp_path, "pfc_problem", fields)
    assert ctypes.sizeof(pfc._CProblem) == got[0]
    for name, off in zip(fields, got[1:]):
        assert getattr(pfc._CProblem, name).offset == off, name


def test_hflow_params_layout_matches_header(tmp_path):
    from paper_2103_04856_gb300 import pfc
    fields = [name for name, _ in pfc._CHFlow._fields_]
    got = _c_layout(tmp_path, "pfc_hflow_params", fields)
    assert ctypes.sizeof(pfc._CHFlow) == got[0]
    for name, off in zip(fields, got[1:]):
        assert getattr(pfc._CHFlow, name).offset == off, name


def test_status_strings_and_b_to_a(lib):
    from paper_2103_04856_gb300 import pfc
    assert lib.pfc_status_string(0) == b"ok"
    assert lib.pfc_status_string(pfc.PFC_ENONFINITE) == b"non-finite result"
    # sponges row of the paper's Table four_shapes, host-only helper
    np.testing.assert_allclose(pfc.pfc_b_to_a([1, 5, 0.8, 0, 0, 1, 0]), [1, 2.8, 2, -10, -10, 25])


def test_create_rejects_bad_problems_without_touching_the_gpu(lib):
    from paper_2103_04856_gb300 import pfc
    h = ctypes.c_void_p()
    bad = [dict(eps=0.0), dict(nx=0), dict(xi=-1.0), dict(tile_y=12), dict(h=float("nan")),
           dict(mu=float("inf")), dict(theta=(0.0, float("nan"), 1.0)), dict(flags=2)]
    for kw in bad:
        base = dict(nx=8, ny=8, nz=8, eps=1.5, a=(1, 0, 1, 0, 0, 0))
        base.update(kw)
        p = pfc.Problem(**base)
        rc = lib.pfc_create(ctypes.byref(p._c()), ctypes.byref(h))
        assert rc == pfc.PFC_EINVAL, kw
        assert lib.pfc_last_error()
    p = pfc.Problem(nx=8, ny=8, nz=8, eps=1.5, a=(1, 0, 1, 0, 0, 0))
    c = p._c()
    c.well = 7
    assert lib.pfc_create(ctypes.byref(c), ctypes.byref(h)) == pfc.PFC_EINVAL
    assert lib.pfc_energy(None, None, None, None) == pfc.PFC_EINVAL
    # the orientation term is a fused-path feature
    p = pfc.Problem(nx=8, ny=8, nz=8, eps=1.5, a=(1, 0, 1, 0, 0, 0), impl="plain", mu=1.0, theta=(0, 0, 1))
    assert lib.pfc_create(ctypes.byref(p._c()), ctypes.byref(h)) == pfc.PFC_EUNSUPPORTED


def test_noalloc_rejects_host_memory_without_launching(lib):
    """The no-allocation entry point checks its fields before it touches the
    GPU: host memory (or, on a machine without a GPU, any pointer) is refused
    with a message, and nothing is launched."""
    from paper_2103_04856_gb300 import pfc
    p = pfc.Problem(nx=8, ny=8, nz=8, eps=1.5, a=(1, 0, 1, 0, 0, 0))
    u = np.zeros(512, dtype=np.float32)
    g = np.zeros(512, dtype=np.float32)
    rc = lib.pfc_energy_and_grad_noalloc(ctypes.byref(p._c()), ctypes.c_void_p(u.ctypes.data),
                                         ctypes.c_void_p(g.ctypes.data), None, None)
    assert rc == pfc.PFC_EINVAL
    assert b"device memory" in lib.pfc_last_error()
    c = p._c()
    c.flags = 4
    assert lib.pfc_energy_and_grad_noalloc(ctypes.byref(c), None, None, None, None) == pfc.PFC_EINVAL


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2103_04856_gb300 import pfc
    monkeypatch.setattr(pfc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pfc, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        pfc.load_library()


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2103_04856_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "pf_oracle" not in src, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2103_04856_gb300" not in src and "pfc.h" not in src, f
