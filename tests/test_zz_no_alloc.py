"""The no-allocation entry point (bdss_factor_solve_noalloc), called through
the C ABI, must give the same solution as the allocating entry point
(bdss_create + bdss_factor_solve) within the parity tolerance used elsewhere,
and meet the oracle's forward- and backward-error bars, on calls in a row
with different systems (so that what one call leaves in the shared scratch
cannot leak into the next).  One system has n >= 32, so the tail levels split
blocks over CTAs as the allocating entry point does.  It serves callers that
may not allocate device memory while they run, such as a real-time control
loop or a plugin whose host owns all device memory.

Kept in a file of its own, collected last."""
import ctypes

import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_TOL = 1e-10


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _noalloc(lib, s):
    from paper_2509_03015_gb300 import _lib
    N, n, _ = s["A_diag"].shape
    d = s["B"].shape[-1]
    Ad, As, B = _dev(s["A_diag"]), _dev(s["A_sub"] if N > 1 else np.zeros((1, n, n))), _dev(s["B"])
    X = torch.full_like(B, float("nan"))
    info = _lib.bdss_info()
    stream = torch.cuda.current_stream()
    st = lib.bdss_factor_solve_noalloc(N, n, d, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(As.data_ptr()),
                                       ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream), ctypes.byref(info))
    return st, X.cpu().numpy()


def _allocating(s):
    from paper_2509_03015_gb300 import Solver
    N, n, _ = s["A_diag"].shape
    d = s["B"].shape[-1]
    solver = Solver(N, n, d_max=d)
    X = solver.factor_solve(_dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"]))
    out = X.cpu().numpy()
    solver.close()
    return out


def _rel(X, Y):
    return np.abs(X - Y).sum(axis=-1).max() / np.abs(Y).sum(axis=-1).max()


def test_noalloc_matches_allocating_entry_point_twice(oracle_mod):
    from paper_2509_03015_gb300 import _lib
    lib = _lib.load()
    systems = [inputs.random_btd(300, 16, 2, seed=21), inputs.workload("kalman-N64-n8-d1"),
               inputs.random_btd(300, 48, 2, seed=22)]
    for s in systems:
        st, X = _noalloc(lib, s)
        assert st == 0, _lib.STATUS_NAMES.get(st)
        Xr = _allocating(s)
        assert np.all(np.isfinite(X))
        assert _rel(X, Xr) <= FWD_TOL
        Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
        assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
        assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14


def test_noalloc_rejects_systems_beyond_its_scratch():
    from paper_2509_03015_gb300 import _lib
    lib = _lib.load()
    info = _lib.bdss_info()
    # 4096 blocks of 64 x 64 need ~400 MB of workspace, far beyond the array
    st = lib.bdss_factor_solve_noalloc(4096, 64, 1, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                       ctypes.c_void_p(16), ctypes.c_void_p(16), None, ctypes.byref(info))
    assert st == 8  # BDSS_ERR_UNSUPPORTED, returned before any launch
    # blocks beyond n = 64 (the tiled path) are not offered without allocation
    st = lib.bdss_factor_solve_noalloc(4, 96, 1, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                       ctypes.c_void_p(16), ctypes.c_void_p(16), None, ctypes.byref(info))
    assert st == 8
