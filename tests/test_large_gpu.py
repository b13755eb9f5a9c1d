"""GPU parity of the large-block path (64 < n <= 256, tiled through shared
memory) against the CPU oracle, FP64 and FP32 + FP64 refinement, including
the full N = 4096, n = 256, d = 16 Kalman workload with rho = 0.99."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs
from tests._helpers import assert_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_TOL = 1e-10
BWD_TOL = 1e-14


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _solve(s, precision="fp64", persistent=True, fused=True):
    from paper_2509_03015_gb300 import Solver
    N, n, _ = s["A_diag"].shape
    d = s["B"].shape[-1]
    Ad, As, B = _dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"])
    solver = Solver(N, n, d_max=d, precision=precision, persistent=persistent)
    try:
        if fused:
            X = solver.factor_solve(Ad, As, B)
        else:
            solver.factor(Ad, As)
            X = solver.solve(B)
        ld = solver.logdet()
        return X.cpu().numpy(), ld, solver.last_info
    finally:
        solver.close()


SWEEP = [(1, 65, 1), (1, 256, 3), (2, 96, 2), (3, 65, 1), (5, 128, 4), (8, 100, 2), (9, 200, 1),
         (17, 128, 16), (33, 256, 2), (64, 130, 5), (100, 192, 3)]


@pytest.mark.parametrize("N,n,d", SWEEP)
def test_large_fp64_parity(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=50 + N + n)
    X, ld, _ = _solve(s)
    L, C = oracle_mod.factor(s["A_diag"], s["A_sub"])
    Xo = oracle_mod.solve(L, C, s["B"])
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert_elementwise(X, Xo, rtol=1e-10, atol_frac=1e-12)
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    ldo = oracle_mod.logdet(L)
    assert abs(ld - ldo) <= 1e-12 * max(1.0, abs(ldo))


@pytest.mark.parametrize("N,n,d", [(2, 96, 2), (9, 200, 1), (33, 256, 2)])
def test_large_fp64_separate_factor_solve(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=7 + N)
    X, _, _ = _solve(s, fused=False)
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL


@pytest.mark.parametrize("N,n,d", [(5, 128, 4), (33, 256, 2)])
def test_large_per_level_matches_persistent(N, n, d):
    s = inputs.random_btd(N, n, d, seed=3)
    X1, ld1, _ = _solve(s, persistent=True)
    X2, ld2, _ = _solve(s, persistent=False)
    assert np.array_equal(X1, X2) and ld1 == ld2


@pytest.mark.parametrize("N,n,d", [(1, 65, 1), (5, 128, 4), (17, 128, 16), (33, 256, 2), (100, 192, 3)])
def test_large_fp32_ir(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=90 + N)
    X, _, info = _solve(s, precision="fp32_ir")
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert info.backward_err <= BWD_TOL


def test_large_not_spd():
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(9, 128, 1, seed=2)
    s["A_diag"][6] -= 1e4 * np.eye(128)
    solver = Solver(9, 128, d_max=1)
    with pytest.raises(BDSSError) as e:
        solver.factor_solve(_dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"]))
    assert e.value.status == 2 and e.value.info.block == 6 and e.value.info.level == 1
    solver.close()


def test_kalman_N4096_n256_fp32_ir_full(oracle_mod, mixed_workload_oracle):
    """The mixed-precision workload at full size: FP32 factors, FP64
    residual refinement to backward error <= 1e-14; forward error against
    the FP64 oracle (kappa ~ 1e5 bounds it by ~kappa * u)."""
    s, Xo = mixed_workload_oracle
    X, _, info = _solve(s, precision="fp32_ir")
    assert info.backward_err <= BWD_TOL
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    fe = oracle_mod.forward_error(X, Xo)
    print(f"N4096 n256: refine iters {info.iters}, backward {info.backward_err:.2e}, forward vs oracle {fe:.2e}")
    assert fe <= 1e-9
    assert_elementwise(X, Xo, rtol=1e-7, atol_frac=1e-9)


def test_kalman_N4096_n256_fp64_full(oracle_mod, mixed_workload_oracle):
    """The same workload on the plain FP64 tiled path, against the oracle."""
    s, Xo = mixed_workload_oracle
    X, _, _ = _solve(s, precision="fp64")
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    assert_elementwise(X, Xo, rtol=1e-7, atol_frac=1e-10)
