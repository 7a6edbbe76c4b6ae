"""CPU checks of the C ABI: the library builds, loads, and exports every function
that include/komega_gb300.h declares; argument validation that needs no GPU."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_2001_08707_gb300 import build as kwbuild
from paper_2001_08707_gb300 import komega as kw

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "komega_gb300.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kw_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(kw.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        kwbuild.build()
    return kw.load_library()


def test_header_declares_expected_entry_points():
    names = _declared_functions()
    for n in ("kw_create", "kw_destroy", "kw_set_csr", "kw_solve", "kw_solve_host", "kw_get_shift_status",
              "kw_get_residual_history", "kw_spmv_dot", "kw_status_string", "kw_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_strings(lib):
    assert lib.kw_abi_version() == kw.ABI_VERSION == 2
    assert lib.kw_status_string(0) == b"KW_OK"
    assert lib.kw_status_string(4) == b"KW_ERR_BREAKDOWN"
    assert lib.kw_status_string(8) == b"KW_NOT_CONVERGED"
    assert lib.kw_status_string(99) == b"KW_UNKNOWN"


def test_default_options(lib):
    o = kw.kw_options()
    lib.kw_default_options(C.byref(o))
    assert o.prec == kw.KW_F64 and o.tol == 1e-10 and o.maxiter == 100000 and o.seed_switch == 1
    assert o.use_graph == 1


def test_create_rejects_bad_options_without_touching_the_gpu(lib):
    ctx = C.c_void_p()
    bad = [kw.kw_options(7, 1e-10, 100, 1, 0, 0),      # precision
           kw.kw_options(0, -1.0, 100, 1, 0, 0),       # tol
           kw.kw_options(0, 1e-10, 0, 1, 0, 0),        # maxiter
           kw.kw_options(0, float("nan"), 10, 1, 0, 0),
           kw.kw_options(0, 1e-10, 10, 1, -1, 0)]      # hist_stride
    for o in bad:
        assert lib.kw_create(C.byref(ctx), C.byref(o), None) == kw.KW_ERR_ARG
        assert not ctx.value
    assert lib.kw_create(None, None, None) == kw.KW_ERR_ARG


def test_null_context_is_rejected(lib):
    info = kw.kw_solve_info()
    assert lib.kw_solve(None, None, 1, None, 0, None, None, None, C.byref(info)) == kw.KW_ERR_ARG
    assert lib.kw_set_csr(None, 1, 1, None, None, None) == kw.KW_ERR_ARG
    lib.kw_destroy(None)


_MIRRORS = {"kw_options": kw.kw_options, "kw_c128": kw.kw_c128, "kw_solve_info": kw.kw_solve_info,
            "kw_instance": kw.kw_instance, "kw_rci_io": kw.kw_rci_io, "kw_stats": kw.kw_stats,
            "kw_csr_term": kw.kw_csr_term}


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors have the size and field offsets that a C compiler gives
    the header's structures (fields matched by name)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "komega_gb300.h"', "int main(void) {"]
    for name, mirror in _MIRRORS.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in mirror._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name, mirror in _MIRRORS.items():
        assert got[(name, "size")] == C.sizeof(mirror), name
        for field, _ in mirror._fields_:
            assert got[(name, field)] == getattr(mirror, field).offset, (name, field)
