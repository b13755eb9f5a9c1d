"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every function include/bdss.h declares, the binding's signature table matches
the header, and host-side argument checks reject bad input before anything
touches the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bdss.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2509_03015_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bdss_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bdss_create", "bdss_factor", "bdss_solve", "bdss_destroy", "bdss_factor_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in bdss.h but not exported"


def test_binding_covers_the_header():
    from paper_2509_03015_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_no_cuda_symbols_leak_into_abi(lib):
    # the exported C ABI carries no torch or C++ types
    src = open(HEADER).read()
    assert "torch" not in src and "std::" not in src and "at::" not in src


def test_status_strings(lib):
    for code in range(0, 10):
        s = lib.bdss_status_string(code)
        assert s and isinstance(s, bytes)
    assert lib.bdss_status_string(0) == b"ok"
    assert b"guard" in lib.bdss_status_string(9)


def test_host_argument_checks(lib):
    from paper_2509_03015_gb300 import _lib
    h = ctypes.c_void_p()
    # invalid sizes are rejected before any CUDA call
    assert lib.bdss_create(ctypes.byref(h), 0, 8, 1, 0, None) == 1
    assert lib.bdss_create(ctypes.byref(h), 10, 0, 1, 0, None) == 1
    assert lib.bdss_create(ctypes.byref(h), 10, 8, 0, 0, None) == 1
    assert lib.bdss_create(ctypes.byref(h), 10, 8, 65, 0, None) == 1
    assert lib.bdss_create(ctypes.byref(h), 10, 8, 1, 7, None) == 1
    assert lib.bdss_create(None, 10, 8, 1, 0, None) == 1
    assert lib.bdss_create(ctypes.byref(h), 10, 257, 1, 0, None) == 8  # n > 256 not supported
    assert h.value is None
    # NULL handles
    assert lib.bdss_destroy(None) == 0
    assert lib.bdss_set_option(None, 0, 1) == 1
    info = _lib.bdss_info()
    assert lib.bdss_factor(None, None, None, ctypes.byref(info)) == 1
    assert lib.bdss_solve(None, None, None, 1, ctypes.byref(info)) == 1
    out = ctypes.c_double()
    assert lib.bdss_logdet(None, ctypes.byref(out)) == 1
    assert lib.bdss_debug_fail_alloc(-1) == 1
    assert lib.bdss_debug_fail_alloc(0) == 0
    # Kalman assembly: sizes first, then NULL inputs, all before any CUDA call
    nul = [None] * 10
    assert lib.bdss_kalman_assemble(0, 8, 4, 0, *nul) == 1
    assert lib.bdss_kalman_assemble(4, 0, 4, 0, *nul) == 1
    assert lib.bdss_kalman_assemble(4, 8, 0, 0, *nul) == 1
    assert lib.bdss_kalman_assemble(4, 8, 4, 2, *nul) == 1
    assert lib.bdss_kalman_assemble(4, 257, 4, 0, *nul) == 8
    assert lib.bdss_kalman_assemble(4, 8, 4097, 1, *nul) == 8
    assert lib.bdss_kalman_assemble(1 << 31, 64, 64, 0, *nul) == 8
    assert lib.bdss_kalman_assemble(4, 8, 4, 1, *nul) == 1


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2509_03015_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()


def test_binding_rejects_pageable_host_tensors():
    # inputs may be CUDA or pinned host tensors (read in place by the
    # kernels); a pageable CPU tensor or a CPU output is refused up front
    import torch
    from paper_2509_03015_gb300.solver import _check_tensor
    t = torch.zeros(2, 3, 3, dtype=torch.float64)
    with pytest.raises(ValueError, match="pinned host"):
        _check_tensor(t, "A_diag", (2, 3, 3), host_ok=True)
    with pytest.raises(ValueError, match="CUDA tensor"):
        _check_tensor(t, "X", (2, 3, 3))
    with pytest.raises(ValueError):
        _check_tensor(t.float(), "A_diag", (2, 3, 3), host_ok=True)


def _enum_values(name):
    """Members and values of the C enum `name` in include/bdss.h."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef enum \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    return {k: int(v) for k, v in re.findall(r"\b([A-Z][A-Z0-9_]+)\s*=\s*(\d+)", body)}


def test_binding_option_table_matches_the_header():
    """Every bdss_option the header declares has the same number in the
    binding's option table, and the table names no other number."""
    from paper_2509_03015_gb300 import _lib
    opts = _enum_values("bdss_option")
    assert opts["BDSS_OPT_SMALL_CLUSTER"] == 14
    assert sorted(_lib.OPTIONS.values()) == sorted(opts.values())
    for key, value in _lib.OPTIONS.items():
        assert opts["BDSS_OPT_" + key.upper()] == value, key
