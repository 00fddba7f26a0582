"""The C-ABI library builds, loads and exports every entry point that
include/cbs.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2507_16087_gb300 import build_lib, cbs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "cbs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(?:cbs_status|void|const char\*)\s+(\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return ctypes.CDLL(build_lib.LIB)


def test_header_declares_expected_entry_points():
    names = _declared()
    for n in ("solver_create", "solve_forward", "solve_adjoint", "residual_norm", "solver_destroy",
              "cbs_last_error"):
        assert n in names
    assert set(names) == set(cbs.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", build_lib.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(_declared()) <= exported


def test_binding_loads_and_reports_create_errors_without_gpu(lib):
    L = cbs.load()
    # a NULL grid is rejected on the host before any device call
    h = ctypes.c_void_p()
    st = L.solver_create(None, 1.0, 1.0, None, None, None, None, None, ctypes.byref(h))
    assert st == cbs.CBS_EINVAL
    assert b"NULL" in L.cbs_last_error(None)
    g = cbs.cbs_grid()
    g.ndim = 2
    g.n[0], g.n[1] = 100, 64  # 100 is not a supported extent
    st = L.solver_create(ctypes.byref(g), 1e-3, 1e6, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8),
                         None, None, ctypes.byref(h))
    assert st == cbs.CBS_EINVAL
    assert b"unsupported extent" in L.cbs_last_error(None)


def test_oracle_shares_nothing_with_the_cuda_path():
    """The oracle and the CUDA path never include, import or link each other."""
    pkg = os.path.join(ROOT, "paper_2507_16087_gb300")
    for d in (pkg, os.path.join(pkg, "csrc")):
        for f in os.listdir(d):
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(d, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), f
                assert "cbs_oracle" not in src and "orc_" not in src, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "csrc" not in src and "import cbs" not in src and "libcbs_gb300" not in src, f
            assert "paper_2507_16087_gb300" not in src, f


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the header's size and field offsets (compiled with gcc)."""
    structs = {"cbs_grid": cbs.cbs_grid, "cbs_boundary": cbs.cbs_boundary, "cbs_options": cbs.cbs_options,
               "cbs_info": cbs.cbs_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cbs.h"', "int main(void) {"]
    for name, ct in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in ct._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(ln.rsplit(" ", 1) for ln in out.splitlines())
    for name, ct in structs.items():
        assert int(got[name]) == ctypes.sizeof(ct), name
        for fname, _ in ct._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(ct, fname).offset, (name, fname)


def test_allocator_callbacks_must_come_in_pairs():
    """solver_create rejects a dev_alloc without dev_free before touching the device (CPU-only check)."""
    lib = cbs.load()
    g = cbs.cbs_grid()
    g.ndim = 2
    g.n[0], g.n[1] = 16, 16
    o = cbs.cbs_options()
    o.dev_alloc = cbs.DEV_ALLOC_FN(lambda nbytes, stream, ctx: None)
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the options are checked first
    st = lib.solver_create(ctypes.byref(g), 1e-3, 1e6, dummy, dummy, dummy, None, ctypes.byref(o), ctypes.byref(h))
    assert st == cbs.CBS_EINVAL
    assert b"dev_alloc and dev_free" in lib.cbs_last_error(None)
    assert not h.value
