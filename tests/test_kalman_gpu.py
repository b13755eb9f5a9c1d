"""Device assembly of the Kalman-smoother normal equations (Sec. 4.2) against
the oracle's assembly, element by element, and the assembled system solved
end to end on the device."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP64 sums of at most n + m <= 400 products of O(1) terms: rounding-order
# differences stay below 400 eps of the largest magnitude; 1e-12 leaves room.
RTOL = 1e-12


def _dev(model):
    return {k: torch.from_numpy(v).cuda() for k, v in model.items()}


def _close(got, want):
    want = np.asarray(want)
    scale = max(1.0, float(np.abs(want).max())) if want.size else 1.0
    np.testing.assert_allclose(got.cpu().numpy(), want, rtol=0, atol=RTOL * scale)


@pytest.mark.parametrize("N,n,m", [(1, 3, 2), (2, 8, 5), (5, 70, 20), (7, 130, 65), (33, 64, 32), (3, 256, 96),
                                   (4, 17, 200)])
def test_assembly_matches_oracle(N, n, m):
    from paper_2509_03015_gb300 import kalman_assemble
    mod = inputs.kalman_model(N, n, m, seed=N + n + m)
    d = _dev(mod)
    A_diag, A_sub, B = kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"], d["zeta"])
    torch.cuda.synchronize()
    rd, rs, rb = oracle.kalman_assemble(mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["z"], mod["zeta"])
    _close(A_diag, rd)
    _close(A_sub, rs)
    _close(B, rb)


def test_matrix_only_and_zero_offsets():
    from paper_2509_03015_gb300 import kalman_assemble
    mod = inputs.kalman_model(6, 40, 12, seed=3)
    d = _dev(mod)
    A_diag, A_sub, B = kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"])
    assert B is None
    rd, rs, _ = oracle.kalman_assemble(mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["z"])
    _close(A_diag, rd)
    _close(A_sub, rs)
    _, _, B = kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"])
    _, _, rb = oracle.kalman_assemble(mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["z"], None)
    _close(B, rb)


def test_assembled_system_solves_end_to_end():
    from paper_2509_03015_gb300 import Solver, kalman_assemble
    N, n, m = 257, 24, 10
    mod = inputs.kalman_model(N, n, m, seed=11)
    d = _dev(mod)
    A_diag, A_sub, B = kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"], d["zeta"])
    sol = Solver(N, n, d_max=1)
    X = sol.factor_solve(A_diag, A_sub, B)
    sol.close()
    rd, rs, rb = oracle.kalman_assemble(mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["z"], mod["zeta"])
    Xr = oracle.solve_system(rd, rs, rb)
    np.testing.assert_allclose(X.cpu().numpy(), Xr, rtol=0, atol=1e-9 * max(1.0, np.abs(Xr).max()))


def test_rejects_bad_arguments_and_reports_alloc_failure():
    from paper_2509_03015_gb300 import _lib, kalman_assemble
    mod = inputs.kalman_model(3, 8, 4, seed=0)
    d = _dev(mod)
    with pytest.raises(ValueError):
        kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"].cpu())
    lib = _lib.load()
    # the library itself rejects a page-locked host input and a size past its limits
    zh = d["z"].cpu().pin_memory()
    out = torch.empty((3, 8, 8), dtype=torch.float64, device="cuda")
    sub = torch.empty((2, 8, 8), dtype=torch.float64, device="cuda")
    rhs = torch.empty((3, 8, 1), dtype=torch.float64, device="cuda")
    p = [ctypes.c_void_p(t.data_ptr()) for t in (d["G"], d["H"], d["Qinv"], d["Rinv"])]
    tail = [ctypes.c_void_p(d["zeta"].data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(sub.data_ptr()), ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(None)]
    assert lib.bdss_kalman_assemble(3, 8, 4, 0, *p, ctypes.c_void_p(zh.data_ptr()), *tail) == 1
    assert lib.bdss_kalman_assemble(3, 8, 4, 0, *p, ctypes.c_void_p(d["z"].data_ptr()), *tail) == 0
    assert lib.bdss_kalman_assemble(3, 8, 4097, 0, *p, ctypes.c_void_p(d["z"].data_ptr()), *tail) == 8
    assert lib.bdss_debug_fail_alloc(1) == 0
    try:
        with pytest.raises(_lib.BDSSError) as e:
            kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"])
        assert e.value.status == 4
    finally:
        lib.bdss_debug_fail_alloc(0)
    A_diag, _, _ = kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"])
    rd, _, _ = oracle.kalman_assemble(mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["z"])
    _close(A_diag, rd)


@pytest.mark.parametrize("N,n,m", [(3, 16, 64), (4, 70, 130)])
def test_assembly_with_diagonal_R_matches_oracle(N, n, m):
    from paper_2509_03015_gb300 import kalman_assemble
    mod = inputs.kalman_model(N, n, m, seed=5 * N + m)
    mod["Rinv"] = np.ascontiguousarray(np.stack([np.diag(R) for R in mod["Rinv"]]))
    d = _dev(mod)
    A_diag, A_sub, B = kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"], d["zeta"])
    rd, rs, rb = oracle.kalman_assemble(mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["z"], mod["zeta"])
    _close(A_diag, rd)
    _close(A_sub, rs)
    _close(B, rb)


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_neuro_shaped_instance_solves(precision):
    from paper_2509_03015_gb300 import Solver, kalman_assemble
    N, n, m = 20, 32, 128
    mod = inputs.kalman_neuro_model(N, n, m, seed=2)
    d = _dev(mod)
    A_diag, A_sub, B = kalman_assemble(d["G"], d["H"], d["Qinv"], d["Rinv"], d["z"], d["zeta"])
    rd, rs, rb = oracle.kalman_assemble(mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["z"], mod["zeta"])
    _close(A_diag, rd)
    _close(B, rb)
    sol = Solver(N, n, d_max=1, precision=precision)
    X = sol.factor_solve(A_diag, A_sub, B)
    sol.close()
    Xr = oracle.solve_system(rd, rs, rb)
    np.testing.assert_allclose(X.cpu().numpy(), Xr, rtol=0, atol=1e-9 * max(1.0, np.abs(Xr).max()))
