"""The C ABI library loads and exports every symbol the public headers declare
(no GPU needed; no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2506_01120_gb300 import binding
from paper_2506_01120_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def built_lib():
    if not os.path.exists(binding.LIB_PATH):
        build()
    return binding.lib()


def declared_symbols():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        names += re.findall(r"LC_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)
    return names


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for required in ("lie_closure", "lie_closure_dev", "lie_closure_batched"):
        assert required in names
    assert sorted(names) == sorted(binding.EXPORTED)


def test_every_declared_symbol_is_exported(built_lib):
    for name in declared_symbols():
        assert hasattr(built_lib, name), name
        assert ctypes.cast(getattr(built_lib, name), ctypes.c_void_p).value


def test_host_only_calls(built_lib):
    o = binding.make_options("fp64")
    assert o.precision == binding.LC_PREC_FP64
    assert o.eta_abs == 1e-12 and o.tau_screen == 0.0 and o.saturation_exit == 0
    assert o.screen_kappa == 10.0 and o.tol_mode == binding.LC_TOL_RELATIVE
    assert o.autotune == 0 and o.ortho_check == 0
    assert binding.status_string(binding.LC_ERR_CAPACITY).startswith("basis capacity")
    assert binding.status_string(12345) == "unknown status"
    assert "sm_103a" in binding.version()


def test_struct_layouts_match_compiled_header(tmp_path):
    """Every field offset of the ctypes mirrors equals offsetof() in C."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lieclosure.h"', 'int main(void) {']
    for cname, py in (("lc_options", binding.Options), ("lc_report", binding.Report)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in (("lc_options", binding.Options), ("lc_report", binding.Report)):
        assert got[(cname, "size")] == ctypes.sizeof(py)
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_struct_layouts_match_header():
    """ctypes mirrors of lc_options / lc_report have the C sizes."""
    assert ctypes.sizeof(binding.Options) == 4 + 4 + 8 + 8 + 4 + 4 + 4 + 4 + 8 + 8 + 4 + 4 + 4 + 4 + 4 + 4 + 8 + 4 + 4 + 4 + 4
    assert ctypes.sizeof(binding.Report) == 8 * 8 + 8 * 5 + 8 + 8 + 8 + 8 + 8 * 6 + 4 * 2 + 8 * 5 + 4 * 6 + 8 + 8 + 8


def test_argument_errors_need_no_gpu(built_lib):
    """Invalid arguments are rejected on the host before any CUDA call."""
    import numpy as np
    g = np.zeros((1, 4, 4), dtype=np.complex128)
    dim = ctypes.c_longlong(7)
    L = built_lib
    assert L.lie_closure(None, 1, 4, 1e-8, None, ctypes.byref(dim), 16, None, None) == binding.LC_ERR_ARG
    assert dim.value == 0
    assert L.lie_closure(g.ctypes.data, 0, 4, 1e-8, None, ctypes.byref(dim), 16, None, None) == binding.LC_ERR_ARG
    assert L.lie_closure(g.ctypes.data, 1, 4, -1.0, None, ctypes.byref(dim), 16, None, None) == binding.LC_ERR_ARG
    assert L.lie_closure(g.ctypes.data, 1, 4, 1e-8, None, ctypes.byref(dim), 0, None, None) == binding.LC_ERR_ARG
    o = binding.make_options("fp64")
    o.precision = 7
    assert L.lie_closure(g.ctypes.data, 1, 4, 1e-8, None, ctypes.byref(dim), 16, ctypes.byref(o), None) \
        == binding.LC_ERR_ARG


def test_pauli_entry_rejects_bad_arguments_before_any_device_call(built_lib):
    """Argument errors of lie_closure_pauli are found on the host (no GPU needed)."""
    import numpy as np
    L = built_lib
    s = np.array([1, 2], dtype=np.uint64)
    c = np.array([1.0, 1.0])
    good = np.array([0, 1, 2], dtype=np.int64)
    out_s = np.zeros(8, dtype=np.uint64)
    out_c = np.zeros(8)
    out_o = np.zeros(9, dtype=np.int64)
    dim = ctypes.c_longlong(7)

    def call(off, nq=2, tol=1e-8, k=2, tcap=8, max_dim=8):
        return L.lie_closure_pauli(s.ctypes.data, c.ctypes.data, off.ctypes.data, k, nq, tol, out_s.ctypes.data,
                                   out_c.ctypes.data, out_o.ctypes.data, tcap, ctypes.byref(dim), max_dim, None, None)

    assert call(good, nq=0) == binding.LC_ERR_ARG
    assert call(good, nq=32) == binding.LC_ERR_ARG
    assert call(good, tol=0.0) == binding.LC_ERR_ARG
    assert call(good, k=0) == binding.LC_ERR_ARG
    assert call(good, tcap=0) == binding.LC_ERR_ARG
    assert call(good, max_dim=0) == binding.LC_ERR_ARG
    assert call(np.array([1, 1, 2], dtype=np.int64)) == binding.LC_ERR_ARG      # offsets[0] != 0
    assert call(np.array([0, 2, 1], dtype=np.int64)) == binding.LC_ERR_ARG      # decreasing
    assert dim.value == 0
