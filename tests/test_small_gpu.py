"""GPU: the one-cluster path for short systems of small blocks (one launch
of a single thread-block cluster, cluster barriers between the phases).

Against the oracle element by element with the log-determinant, over every
N parity class through several levels, n up to 32 and d up to 16; bitwise
against the persistent grid kernel and the per-level launches (the same
operations in the same order); mixed with them through the stored factors;
and the failure report of a non-SPD block."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs
from tests._helpers import assert_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_TOL = 1e-10
BWD_TOL = 1e-14


def _dev(s):
    d = torch.device("cuda:0")
    N, n, _ = s["A_diag"].shape
    As = s["A_sub"] if N > 1 else np.zeros((1, n, n))
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in (s["A_diag"], As, s["B"]))


def _solve(s, small, persistent=True, fused=True):
    from paper_2509_03015_gb300 import Solver
    N, n, _ = s["A_diag"].shape
    d = s["B"].shape[-1]
    Ad, As, B = _dev(s)
    sol = Solver(N, n, d_max=d, persistent=persistent)
    try:
        sol.set_option("small_cluster", small)
        if fused:
            X = sol.factor_solve(Ad, As, B)
        else:
            sol.factor(Ad, As)
            X = sol.solve(B)
        stats = sol.launch_stats()
        return X.cpu().numpy(), sol.logdet(), stats
    finally:
        sol.close()


SWEEP = [(1, 1, 1), (1, 8, 3), (2, 8, 2), (3, 3, 1), (4, 5, 2), (5, 16, 3), (7, 12, 1), (8, 8, 8),
         (9, 24, 2), (15, 31, 1), (16, 32, 4), (17, 2, 16), (33, 7, 5), (63, 16, 1), (64, 8, 1),
         (65, 1, 1), (100, 3, 16), (128, 16, 2), (129, 8, 1), (300, 12, 3), (1000, 4, 1)]


@pytest.mark.parametrize("N,n,d", SWEEP)
def test_small_path_parity(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=900 + 3 * N + n)
    X, ld, stats = _solve(s, 1)
    assert stats == (1, 0)  # one launch, no grid barrier: the one-cluster path ran
    L, C = oracle_mod.factor(s["A_diag"], s["A_sub"])
    Xo = oracle_mod.solve(L, C, s["B"])
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert_elementwise(X, Xo, rtol=1e-10, atol_frac=1e-12)
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    ldo = oracle_mod.logdet(L)
    assert abs(ld - ldo) <= 1e-12 * max(1.0, abs(ldo))


@pytest.mark.parametrize("N,n,d", [(1, 5, 2), (3, 4, 1), (64, 8, 1), (65, 16, 4), (100, 3, 5), (127, 32, 2)])
def test_small_path_bitwise_equals_grid_and_per_level(N, n, d):
    s = inputs.random_btd(N, n, d, seed=77 + N)
    X1, ld1, st1 = _solve(s, 1)
    X2, ld2, st2 = _solve(s, 0)
    X3, ld3, _ = _solve(s, 0, persistent=False)
    assert st1 == (1, 0) and st2[1] > 0
    assert np.array_equal(X1, X2) and np.array_equal(X1, X3)
    assert ld1 == ld2 == ld3


def test_small_factors_serve_the_other_paths(oracle_mod):
    """Factor on one path, solve on the other: the stored factors have one
    layout; separate factor and solve give the fused call's bits."""
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(90, 12, 3, seed=5)
    Ad, As, B = _dev(s)
    sol = Solver(90, 12, d_max=3)
    try:
        sol.set_option("small_cluster", 1)
        Xf = sol.factor_solve(Ad, As, B).cpu().numpy()
        sol.factor(Ad, As)
        X1 = sol.solve(B).cpu().numpy()
        sol.set_option("small_cluster", 0)
        X2 = sol.solve(B).cpu().numpy()        # grid kernel on the cluster's factors
        sol.factor(Ad, As)
        sol.set_option("small_cluster", 1)
        X3 = sol.solve(B).cpu().numpy()        # cluster on the grid kernel's factors
        assert np.array_equal(Xf, X1) and np.array_equal(X1, X2) and np.array_equal(X2, X3)
    finally:
        sol.close()
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(Xf, Xo) <= FWD_TOL


@pytest.mark.parametrize("N,n,blk", [(1, 6, 0), (2, 4, 1), (9, 8, 4), (64, 8, 48), (100, 12, 57)])
def test_small_not_spd_reports_level_and_block(N, n, blk):
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(N, n, 1, seed=2)
    s["A_diag"][blk] -= 1000.0 * np.eye(n)
    Ad, As, B = _dev(s)
    sol = Solver(N, n, d_max=1)
    try:
        sol.set_option("small_cluster", 1)
        with pytest.raises(BDSSError) as e:
            sol.factor_solve(Ad, As, B)
        assert e.value.status == 2
        if blk == 0:
            assert e.value.info.block == 0
        else:
            assert e.value.info.level == (blk & -blk).bit_length() - 1 and e.value.info.block == blk
        s2 = inputs.random_btd(N, n, 1, seed=3)
        Ad2, As2, B2 = _dev(s2)
        sol.factor_solve(Ad2, As2, B2)  # the handle stays usable
    finally:
        sol.close()


def test_small_path_default_rule():
    """By size: taken for the short Kalman system (N = 64, n = 8), not for a
    long one, and never with per-level launches."""
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.workload("kalman-N64-n8-d1")
    Ad, As, B = _dev(s)
    sol = Solver(64, 8, d_max=1)
    sol.factor_solve(Ad, As, B)
    assert sol.launch_stats() == (1, 0)
    sol.set_option("persistent", 0)
    sol.factor_solve(Ad, As, B)
    assert sol.launch_stats()[0] > 1
    sol.close()
    sol = Solver(5000, 8, d_max=1)
    s = inputs.random_btd(5000, 8, 1, seed=1)
    Ad, As, B = _dev(s)
    sol.factor_solve(Ad, As, B)
    assert sol.launch_stats()[1] > 0
    sol.close()
    sol = Solver(64, 8, d_max=1, precision="fp32_ir")
    with pytest.raises(BDSSError) as e:
        sol.set_option("small_cluster", 1)
    assert e.value.status == 8
    sol.close()


def test_small_trace_stamps():
    """The one-cluster launch stamps every cluster barrier: start-up, phases A
    and B of each level, then (with right-hand sides) the top block and each
    downward level, and the end."""
    from paper_2509_03015_gb300 import Solver
    s = inputs.workload("kalman-N64-n8-d1")
    Ad, As, B = _dev(s)
    sol = Solver(64, 8, d_max=1)
    try:
        sol.set_option("small_cluster", 1)
        L = sol.plan_levels
        sol.factor_solve(Ad, As, B)
        st = sol.trace()
        assert len(st) == 3 * L + 2 and all(b >= a for a, b in zip(st, st[1:]))
        sol.factor(Ad, As)
        assert len(sol.trace()) == 2 * L + 2
    finally:
        sol.close()
