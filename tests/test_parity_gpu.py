"""GPU parity: the CUDA cyclic-reduction path (called through the C ABI)
against the CPU FP64 oracle, element by element, on the same seeded inputs.

Bars (FP64 path, kappa(A) <= 1e6): relative forward error <= 1e-10 against
the oracle and backward error ||B - A X||_inf / (||A||_inf ||X||_inf) <= 1e-14
with the residual taken in compensated FP64 by the oracle.  log det from the
GPU factors must equal the oracle's.  Mixed precision: the same backward-error
bar after refinement."""
import math

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
    return (torch.from_numpy(np.ascontiguousarray(s["A_diag"])).to(d),
            torch.from_numpy(np.ascontiguousarray(s["A_sub"])).to(d),
            torch.from_numpy(np.ascontiguousarray(s["B"])).to(d))


def _gpu_solve(s, precision="fp64", persistent=True, fused=True):
    from paper_2509_03015_gb300 import Solver
    N, n, _ = s["A_diag"].shape
    d = s["B"].shape[-1]
    Ad, As, B = _dev(s)
    solver = Solver(N, n, d_max=d, precision=precision, persistent=persistent)
    try:
        if fused:
            X = solver.factor_solve(Ad, As, B)
        else:
            solver.factor(Ad, As)
            X = solver.solve(B)
        ld = solver.logdet()
        info = solver.last_info
        torch.cuda.synchronize()
        return X.cpu().numpy(), ld, info
    finally:
        solver.close()


SWEEP = [
    # (N, n, d): every N parity class through several levels, n across the
    # warp / tile boundaries, d from 1 to 16
    (1, 1, 1), (1, 7, 3), (1, 64, 2), (2, 1, 1), (2, 8, 2), (3, 3, 1), (3, 64, 4),
    (4, 5, 2), (5, 2, 3), (5, 33, 1), (7, 12, 1), (8, 8, 8), (9, 24, 2), (15, 31, 1),
    (16, 32, 4), (17, 48, 1), (33, 7, 5), (33, 64, 2), (63, 16, 1), (64, 8, 1),
    (65, 1, 1), (100, 3, 16), (127, 12, 2), (128, 24, 1), (255, 48, 3), (257, 64, 1),
    (1000, 8, 4), (1025, 2, 1), (2047, 32, 2), (4099, 12, 1),
]


@pytest.mark.parametrize("N,n,d", SWEEP)
def test_fp64_parity_random(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=1000 + 7 * N + n)
    X, ld, _ = _gpu_solve(s)
    L, C = oracle_mod.factor(s["A_diag"], s["A_sub"])
    Xo = oracle_mod.solve(L, C, s["B"])
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert_elementwise(X, Xo, rtol=1e-10, atol_frac=1e-12)
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    ldo = oracle_mod.logdet(L)
    assert abs(ld - ldo) <= 1e-12 * max(1.0, abs(ldo))


@pytest.mark.parametrize("N,n,d", [(1, 5, 2), (2, 8, 1), (9, 24, 2), (100, 3, 4), (257, 64, 1), (1000, 8, 4)])
def test_fp64_separate_factor_then_solve(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=N + n)
    X, ld, _ = _gpu_solve(s, fused=False)
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL


@pytest.mark.parametrize("N,n,d", [(3, 4, 1), (64, 8, 1), (1000, 16, 2), (4099, 12, 1),
                                   (1, 5, 3), (2, 16, 8), (100, 3, 5), (255, 16, 8), (256, 1, 1)])
def test_per_level_launches_match_persistent(N, n, d):
    """The per-level launch structure (Algorithms 4, 7) and the persistent
    kernel run the same arithmetic in the same order: bitwise equal."""
    s = inputs.random_btd(N, n, d, seed=5 + N)
    X1, ld1, _ = _gpu_solve(s, persistent=True)
    X2, ld2, _ = _gpu_solve(s, persistent=False)
    assert np.array_equal(X1, X2)
    assert ld1 == ld2


def test_repeat_runs_bitwise_identical():
    s = inputs.random_btd(1000, 24, 2, seed=3)
    X1, _, _ = _gpu_solve(s)
    X2, _, _ = _gpu_solve(s)
    assert np.array_equal(X1, X2)


@pytest.mark.parametrize("name", ["kalman-N64-n8-d1", "kalman-N2048-n32-d8-grad"])
def test_kalman_workloads_full(oracle_mod, name):
    s = inputs.workload(name)
    X, ld, _ = _gpu_solve(s)
    L, C = oracle_mod.factor(s["A_diag"], s["A_sub"])
    Xo = oracle_mod.solve(L, C, s["B"])
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert_elementwise(X, Xo, rtol=1e-9, atol_frac=1e-11)
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    assert abs(ld - oracle_mod.logdet(L)) <= 1e-12 * abs(oracle_mod.logdet(L))


def test_kalman_N16384_n64_full(oracle_mod):
    """The benchmark workload at full size, in the launch configuration the
    benchmark times (persistent, fused factor + solve), against the oracle
    on every element."""
    s = inputs.workload("kalman-N16384-n64-d4")
    X, ld, _ = _gpu_solve(s)
    L, C = oracle_mod.factor(s["A_diag"], s["A_sub"])
    Xo = oracle_mod.solve(L, C, s["B"])
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert_elementwise(X, Xo, rtol=1e-9, atol_frac=1e-11)
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    assert abs(ld - oracle_mod.logdet(L)) <= 1e-12 * abs(oracle_mod.logdet(L))


@pytest.mark.parametrize("N", [1, 2, 3, 10, 1000, 100000])
def test_tridiag_closed_form_gpu(N):
    s = inputs.tridiag_121(N)
    X, ld, _ = _gpu_solve(s)
    i = np.arange(1, N + 1, dtype=np.float64)
    exact = i * (N + 1 - i) / 2.0
    kappa = 4.0 * (N + 1) ** 2 / math.pi ** 2
    assert np.max(np.abs(X.reshape(-1) - exact)) / np.max(exact) <= max(1e-14, 8 * kappa * 2.2e-16)
    # First-order perturbation: |d logdet| = |tr(A^-1 dA)| <= u |A| tr(A^-1)
    # per rounding of the Schur updates, tr(A^-1) = N (N+2) / 6 here; cyclic
    # reduction rounds every (identical) block alike, so the terms add up.
    tol = 8 * 2.0 ** -53 * 2.0 * N * (N + 2) / 6.0 + 1e-13
    assert abs(ld - math.log(N + 1)) <= tol


def test_single_block_is_plain_cholesky():
    s = inputs.random_btd(1, 40, 3, seed=9)
    X, ld, _ = _gpu_solve(s)
    A = 0.5 * (s["A_diag"][0] + s["A_diag"][0].T)
    np.testing.assert_allclose(X[0], np.linalg.solve(A, s["B"][0]), rtol=1e-12, atol=1e-13)
    assert abs(ld - np.linalg.slogdet(A)[1]) < 1e-11


def test_block_diagonal_independent():
    s = inputs.random_btd(37, 16, 2, seed=4)
    s["A_sub"][:] = 0.0
    X, _, _ = _gpu_solve(s)
    for i in range(37):
        A = 0.5 * (s["A_diag"][i] + s["A_diag"][i].T)
        np.testing.assert_allclose(X[i], np.linalg.solve(A, s["B"][i]), rtol=1e-12, atol=1e-13)


def test_in_place_solve(oracle_mod):
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(300, 16, 2, seed=8)
    Ad, As, B = _dev(s)
    solver = Solver(300, 16, d_max=2)
    solver.factor_solve(Ad, As, B, X=B)
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(B.cpu().numpy(), Xo) <= FWD_TOL
    solver.close()


@pytest.mark.parametrize("N,n,blk", [(1, 6, 0), (2, 4, 1), (9, 8, 4), (9, 8, 0), (100, 12, 57), (1000, 8, 999)])
def test_not_spd_reports_level_and_block(N, n, blk):
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(N, n, 1, seed=2)
    s["A_diag"][blk] -= 1000.0 * np.eye(n)
    Ad, As, B = _dev(s)
    solver = Solver(N, n, d_max=1)
    with pytest.raises(BDSSError) as e:
        solver.factor_solve(Ad, As, B)
    assert e.value.status == 2
    # the pivot fails where the block is eliminated: level = trailing zeros
    if blk == 0:
        assert e.value.info.block == 0
    else:
        lvl = (blk & -blk).bit_length() - 1
        assert e.value.info.level == lvl and e.value.info.block == blk
    # the device stays usable: a good system factors on the same handle
    s2 = inputs.random_btd(N, n, 1, seed=3)
    Ad2, As2, B2 = _dev(s2)
    solver.factor_solve(Ad2, As2, B2)
    solver.close()


def test_nan_input_is_an_error():
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(50, 8, 1, seed=2)
    s["A_diag"][21][3, 3] = np.nan
    Ad, As, B = _dev(s)
    solver = Solver(50, 8, d_max=1)
    with pytest.raises(BDSSError) as e:
        solver.factor_solve(Ad, As, B)
    assert e.value.status == 2
    solver.close()


def test_barrier_timeout_is_reported_and_device_stays_usable(oracle_mod):
    """A wait that nothing releases (CTA 0 skips its arrival at the third grid
    barrier) ends after the configured limit with BDSS_ERR_TIMEOUT; the handle
    and the context remain usable."""
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(5000, 8, 1, seed=2)
    Ad, As, B = _dev(s)
    solver = Solver(5000, 8, d_max=1, timeout_ms=300)
    solver.set_option("debug_skip_arrive", 3)
    with pytest.raises(BDSSError) as e:
        solver.factor_solve(Ad, As, B)
    assert e.value.status == 6
    solver.set_option("debug_skip_arrive", 0)
    X = solver.factor_solve(Ad, As, B)
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(X.cpu().numpy(), Xo) <= FWD_TOL
    solver.close()


def test_invalid_arguments_rejected():
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(10, 4, 2, seed=1)
    Ad, As, B = _dev(s)
    solver = Solver(10, 4, d_max=1)
    with pytest.raises(BDSSError) as e:
        solver.factor_solve(Ad, As, B)  # d = 2 > d_max
    assert e.value.status == 1
    with pytest.raises(BDSSError) as e:
        solver.solve(B[:, :, :1].contiguous())  # before factor
    assert e.value.status == 3
    solver.close()


# ---- mixed precision: FP32 factor + FP64 refinement --------------------------

@pytest.mark.parametrize("N,n,d", [(1, 8, 1), (2, 3, 2), (9, 24, 2), (257, 64, 1), (1000, 8, 4), (2047, 32, 2)])
def test_fp32_ir_reaches_fp64_backward_error(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=77 + N)
    X, ld, info = _gpu_solve(s, precision="fp32_ir")
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL
    assert 0 <= info.iters <= 10 and info.backward_err <= BWD_TOL


def test_fp32_ir_kalman_N16384_n64(oracle_mod):
    s = inputs.workload("kalman-N16384-n64-d4")
    X, ld, info = _gpu_solve(s, precision="fp32_ir")
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= BWD_TOL
    assert oracle_mod.forward_error(X, Xo) <= FWD_TOL


@pytest.mark.parametrize("N,n,d", [(300, 64, 2), (65, 160, 3)])
def test_reported_backward_error_matches_oracle(oracle_mod, N, n, d):
    # max_refine = 0: the library stops after its first residual and reports
    # ||B - A X||_inf / (||A||_inf ||X||_inf) of the FP32 solution (~1e-7),
    # with ||A||_inf estimated from FP64 bit fields; at that size the plain
    # FP64 residual is exact to many digits, so the report must agree with
    # the oracle's compensated value to well within the 2^-20 norm estimate
    from paper_2509_03015_gb300 import Solver
    from paper_2509_03015_gb300._lib import BDSSError
    s = inputs.random_btd(N, n, d, seed=5 + N)
    Ad, As, B = _dev(s)
    solver = Solver(N, n, d_max=d, precision="fp32_ir")
    try:
        solver.set_option("max_refine", 0)
        with pytest.raises(BDSSError) as e:
            X = torch.empty_like(B)
            solver.factor_solve(Ad, As, B, X)
        assert e.value.status == 7  # NO_CONVERGENCE after zero corrections
        reported = e.value.info.backward_err
        ref = oracle_mod.backward_error(s["A_diag"], s["A_sub"], X.cpu().numpy(), s["B"])
        assert 1e-12 < ref < 1e-3
        assert abs(reported - ref) <= 1e-5 * ref
    finally:
        solver.close()


@pytest.mark.parametrize("N,n,blk", [(64, 8, 0), (64, 8, 12), (200, 16, 96), (7, 4, 6)])
def test_small_systems_report_not_spd(N, n, blk):
    # a failing pivot in a small system (few CTAs, tail levels only)
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(N, n, 1, seed=4)
    s["A_diag"][blk] -= 1000.0 * np.eye(n)
    Ad, As, B = _dev(s)
    solver = Solver(N, n, d_max=1)
    try:
        with pytest.raises(BDSSError) as e:
            solver.factor_solve(Ad, As, B)
        assert e.value.status == 2
        if blk == 0:
            assert e.value.info.block == 0
        else:
            assert e.value.info.level == (blk & -blk).bit_length() - 1 and e.value.info.block == blk
    finally:
        solver.close()
