"""Host-side checks of the phase trace: the argument rules of
bdss_last_trace and the split of barrier stamps into per-level steps."""
import ctypes
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_03015_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_trace_argument_checks(lib):
    cnt = ctypes.c_int32()
    buf = (ctypes.c_int64 * 4)()
    assert lib.bdss_last_trace(None, buf, 4, ctypes.byref(cnt)) == 1
    assert lib.bdss_get_launch_config(None, None, None, None) == 1


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_phase_split_layout():
    # L = 3: barrier 0, (A, B) x 3, top, then downward levels 2 and 1
    stamps = [0, 10_000, 30_000, 40_000, 55_000, 60_000, 62_000, 70_000, 73_000, 75_000]
    ph = _bench().phase_split(stamps, 3, launch_ms=0.080)
    assert ph["A"] == [10.0, 10.0, 5.0]
    assert ph["B"] == [20.0, 15.0, 2.0]
    assert ph["top"] == 8.0
    assert ph["C"] == [3.0, 2.0]
    assert ph["edges"] == pytest.approx(80.0 - 75.0)


def test_phase_split_factor_only_and_short():
    ph = _bench().phase_split([0, 5_000, 9_000], 1, launch_ms=0.012)
    assert ph["A"] == [5.0] and ph["B"] == [4.0] and "top" not in ph
    assert _bench().phase_split([0, 1], 2, launch_ms=1.0) is None
