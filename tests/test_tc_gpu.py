"""Tensor-core path (BDSS_TF32_IR, n > 64): the TMA + tcgen05 3xTF32 Schur
tile against an FP64 product, then the solver in TF32 mode refined to the
FP64 backward-error bar against the oracle."""
import ctypes

import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs
from tests._helpers import assert_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_tc_tile_selftest():
    from paper_2509_03015_gb300 import _lib
    lib = _lib.load()
    err = ctypes.c_double(-1.0)
    st = lib.bdss_tc_selftest(ctypes.byref(err))
    assert st == 0, _lib.STATUS_NAMES.get(st)
    # 3xTF32 keeps ~2^-21 of every product: far below plain TF32 (2^-11)
    assert 0.0 <= err.value <= 2e-6, err.value


@pytest.mark.parametrize("N,n,d", [(2, 128, 1), (5, 128, 4), (9, 200, 2), (33, 256, 2), (64, 96, 3)])
def test_tf32_ir_parity(oracle_mod, N, n, d):
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(N, n, d, seed=300 + N + n)
    solver = Solver(N, n, d_max=d, precision="tf32_ir")
    X = solver.factor_solve(_dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"])).cpu().numpy()
    info = solver.last_info
    solver.close()
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert info.backward_err <= 1e-14
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14
    assert oracle_mod.forward_error(X, Xo) <= 1e-10
    assert_elementwise(X, Xo, rtol=1e-9, atol_frac=1e-11)


def test_tf32_ir_kalman_N4096_n256(oracle_mod, mixed_workload_oracle):
    """The mixed-precision workload at full size in TF32 mode: backward error
    <= 1e-14 after refinement and the error against the FP64 oracle, bounded
    by about kappa u_64 (kappa ~ 1e5) with room for the refinement's stop."""
    from paper_2509_03015_gb300 import Solver
    s, Xo = mixed_workload_oracle
    solver = Solver(4096, 256, d_max=16, precision="tf32_ir")
    X = solver.factor_solve(_dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"])).cpu().numpy()
    info = solver.last_info
    solver.close()
    assert info.backward_err <= 1e-14
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14
    fe = oracle_mod.forward_error(X, Xo)
    print(f"tf32_ir N4096 n256: iters {info.iters}, backward {info.backward_err:.2e}, forward vs oracle {fe:.2e}")
    assert fe <= 1e-9
    assert_elementwise(X, Xo, rtol=1e-7, atol_frac=1e-9)
