"""The C ABI without a GPU: the library builds, loads, exports every function that
include/pf_gb300.h declares, and the ctypes structures match the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pf_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:pf_status|void|size_t|const\s+char\s*\*)\s*\**\s*(pf_\w+)\s*\(", text,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_04060_gb300 import build, _binding
    build.build()
    return _binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pf_create_grid", "pf_set_coeffs", "pf_linear_solve", "pf_nonlinear_solve", "pf_submit", "pf_poll",
              "pf_destroy_grid", "pf_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1711_04060_gb300 import _binding
    for n in declared_functions():
        assert hasattr(lib, n), f"{n} not exported"
        assert n in _binding.SIGNATURES, f"{n} has no ctypes signature"
    assert set(_binding.SIGNATURES) == set(declared_functions())


def test_struct_layouts_match_c(tmp_path):
    from paper_1711_04060_gb300 import _binding as B
    structs = {"pf_species": B.pf_species, "pf_coeffs": B.pf_coeffs, "pf_solve_opts": B.pf_solve_opts,
               "pf_report": B.pf_report, "pf_nl_opts": B.pf_nl_opts, "pf_result": B.pf_result,
               "pf_request": B.pf_request, "pf_profile": B.pf_profile, "pf_batch_tune": B.pf_batch_tune,
               "pf_sites": B.pf_sites, "pf_batch_stats": B.pf_batch_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_errors_without_device_are_reported(lib):
    """Argument errors are caught before any device work and leave a message."""
    h = ctypes.c_void_p()
    org = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    assert lib.pf_create_grid(1, 4, 4, 1.0, org, None, ctypes.byref(h)) == 1  # PF_E_INVAL
    assert b"nz" in lib.pf_last_error() or b"nx" in lib.pf_last_error()
    assert lib.pf_destroy_grid(None) == 0
    b = ctypes.c_void_p()
    assert lib.pf_batch_create(None, 0, None, ctypes.byref(b)) == 1
    assert b"grid" in lib.pf_last_error()
    assert lib.pf_batch_destroy(None) == 0
    assert lib.pf_set_filter(None, None, None, 0) == 1
    for fn in (lib.pf_linear_solve, lib.pf_linear_solve_cg):
        assert fn(None, 0, None, None, 0, None, None) == 1
        assert b"required" in lib.pf_last_error()


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1711_04060_gb300 import _binding, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_binding, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _binding.load()


def test_size_limit_is_refused_before_allocation(lib):
    h = ctypes.c_void_p()
    org = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    assert lib.pf_create_grid(2000, 2000, 1000, 1.0, org, None, ctypes.byref(h)) == 1  # PF_E_INVAL
    assert b"too large" in lib.pf_last_error()


def test_grid_bytes_without_device(lib):
    """The device footprint the server budgets by: about 393 bytes per padded node plus fixed buffers, four FP64
    history vectors of the predicted starting vectors, and two FP64 vectors per Anderson history column plus three."""
    from paper_1711_04060_gb300 import api
    n = 257
    np_ = (n + 7) // 8 * 8 * n * n
    b0 = api.pf_grid_bytes(n, n, n)
    assert (393 + 32) * np_ < b0 < (393 + 32) * np_ + (1 << 20)
    assert api.pf_grid_bytes(n, n, n, 5) - b0 == (2 * 5 + 3) * 8 * np_
    assert api.pf_grid_bytes(0, 4, 4) == 0
