"""The FP64-accurate residual on the tensor cores (BF16 digit slices, exact
FP32 accumulation) against the oracle's compensated residual, element by
element, and against the FP64-ALU residual of the same handle; its use
inside the mixed-precision refinement is covered by the large-block parity
tests, which run with it on by default."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _norm_inf_A(Ad, As):
    N, n, _ = Ad.shape
    best = 0.0
    for i in range(N):
        s = np.abs(0.5 * (Ad[i] + Ad[i].T)).sum(axis=1)
        if i > 0:
            s = s + np.abs(As[i - 1]).sum(axis=1)
        if i + 1 < N:
            s = s + np.abs(As[i]).sum(axis=0)
        best = max(best, float(s.max()))
    return best


def _residuals(s, X, emu):
    from paper_2509_03015_gb300 import Solver
    N, n, _ = s["A_diag"].shape
    d = s["B"].shape[-1]
    solver = Solver(N, n, d_max=d, precision="fp32_ir")
    try:
        solver.set_option("residual_emu", 1 if emu else 0)
        Ad, As, B = _dev(s["A_diag"]), _dev(s["A_sub"] if N > 1 else np.zeros((1, n, n))), _dev(s["B"])
        solver.factor(Ad, As)
        return solver.residual(B, _dev(X)).cpu().numpy()
    finally:
        solver.close()


CASES = [(1, 96, 1), (2, 128, 5), (3, 200, 16), (5, 65, 2), (9, 130, 16), (17, 256, 4), (33, 192, 3)]


@pytest.mark.parametrize("N,n,d", CASES)
def test_tensor_core_residual_matches_oracle(oracle_mod, N, n, d):
    """|R - R_exact| <= 1e-15 (max|B| + ||A||_inf max|X|) for every entry: the
    59-bit digits and the FP64 combination keep the residual at FP64 accuracy;
    an inexact (rounded) FP32 accumulation would be off by ~1e-7."""
    s = inputs.random_btd(N, n, d, seed=40 + N + n)
    rng = np.random.default_rng(N * n)
    # columns of very different magnitudes, and one block far smaller than the rest
    X = rng.standard_normal((N, n, d)) * np.logspace(-3, 3, d)
    X[N // 2] *= 1e-5
    R = _residuals(s, X, emu=True)
    Ro = oracle_mod.residual(s["A_diag"], s["A_sub"], X, s["B"])
    scale = np.abs(s["B"]).max() + _norm_inf_A(s["A_diag"], s["A_sub"]) * np.abs(X).max()
    err = np.abs(R - Ro)
    assert err.max() <= 1e-15 * scale, err.max() / scale
    # the FP64-ALU residual of the same handle meets the same bound
    R64 = _residuals(s, X, emu=False)
    assert np.abs(R64 - Ro).max() <= 1e-15 * scale


def test_tensor_core_residual_wide_exponents(oracle_mod):
    """Operator rows and X columns spread over many binades: each row and
    column is cut below its own maximum."""
    N, n, d = 4, 128, 8
    s = inputs.random_btd(N, n, d, seed=9)
    rowscale = np.logspace(-4, 4, n)
    s["A_diag"] = s["A_diag"] * rowscale[None, :, None] * rowscale[None, None, :]
    s["A_sub"] = s["A_sub"] * rowscale[None, :, None] * rowscale[None, None, :]
    X = np.random.default_rng(3).standard_normal((N, n, d)) / rowscale[None, :, None]
    R = _residuals(s, X, emu=True)
    Ro = oracle_mod.residual(s["A_diag"], s["A_sub"], X, s["B"])
    scale = np.abs(s["B"]).max() + _norm_inf_A(s["A_diag"], s["A_sub"]) * np.abs(X).max()
    assert np.abs(R - Ro).max() <= 1e-15 * scale


def test_tensor_core_residual_propagates_nan():
    N, n, d = 3, 128, 2
    s = inputs.random_btd(N, n, d, seed=4)
    X = np.ones((N, n, d))
    X[1, 5, 1] = np.nan
    R = _residuals(s, X, emu=True)
    assert np.isnan(R[..., 1]).any() and np.isfinite(R[..., 0]).all()


def test_residual_option_is_refused_without_tensor_core_buffers():
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = Solver(8, 32, d_max=2, precision="fp32_ir")  # n <= 64: FP64-ALU residual only
    with pytest.raises(BDSSError) as e:
        s.set_option("residual_emu", 1)
    assert e.value.status == 8
    s.close()


# ---------------------------------------------------------------------------
# The Schur products of the tiled FP64 factorisation on the tensor cores
# (separator update of Algorithm 3).  The FP64 large-block parity tests run
# with them by default; these compare the two product engines directly.
# ---------------------------------------------------------------------------
def _fp64_solve(s, schur_emu, persistent=True):
    from paper_2509_03015_gb300 import Solver
    N, n, _ = s["A_diag"].shape
    d = s["B"].shape[-1]
    solver = Solver(N, n, d_max=d, precision="fp64", persistent=persistent)
    try:
        solver.set_option("schur_emu", 1 if schur_emu else 0)
        As = s["A_sub"] if N > 1 else np.zeros((1, n, n))
        X = solver.factor_solve(_dev(s["A_diag"]), _dev(As), _dev(s["B"]))
        return X.cpu().numpy(), solver.logdet()
    finally:
        solver.close()


def _integer_couplings(n, d, seed):
    """N = 3 with A_11 = I, integer couplings in [-2, 2] and diagonals chosen
    so that every Schur complement is an integer matrix (D_2 = I at level 0,
    the top block 4 I): every product of the factorisation is an exact
    integer sum, so both engines must give the same bits, and the solution of
    an integer B is exact (denominators are powers of two)."""
    rng = np.random.default_rng(seed)
    A10 = rng.integers(-2, 3, (n, n)).astype(float)
    A21 = rng.integers(-2, 3, (n, n)).astype(float)
    I = np.eye(n)
    E = A21 @ A10
    A_diag = np.stack([A10.T @ A10 + E.T @ E + 4.0 * I, I, I + A21 @ A21.T])
    A_sub = np.stack([A10, A21])
    B = rng.integers(-8, 9, (3, n, d)).astype(float)
    return {"A_diag": A_diag, "A_sub": A_sub, "B": B}


def _exact_residual_is_zero(s, X, scale_bits=8):
    """A X == B in integer arithmetic: X scaled by 2^scale_bits must be
    integral, and the products are formed with Python integers."""
    Xs = X * 2.0 ** scale_bits
    if not np.array_equal(Xs, np.round(Xs)):
        return False
    Xi = Xs.astype(np.int64).astype(object)
    Ad = s["A_diag"].astype(np.int64).astype(object)
    As = s["A_sub"].astype(np.int64).astype(object)
    Bi = (s["B"] * 2.0 ** scale_bits).astype(np.int64).astype(object)
    N = Ad.shape[0]
    for i in range(N):
        r = Ad[i].dot(Xi[i])
        if i > 0:
            r = r + As[i - 1].dot(Xi[i - 1])
        if i + 1 < N:
            r = r + As[i].T.dot(Xi[i + 1])
        if not np.array_equal(r, Bi[i]):
            return False
    return True


@pytest.mark.parametrize("n,d", [(32, 2), (48, 1), (64, 4), (96, 1), (200, 3), (256, 2)])
def test_schur_emu_exact_on_integer_couplings(n, d):
    """Both engines give the same bits, and that is the exact solution (the
    FP64 oracle, which eliminates in another order, is not exact here: the
    system's condition number is ~1e8)."""
    s = _integer_couplings(n, d, seed=n)
    Xe, lde = _fp64_solve(s, schur_emu=True)
    Xa, lda = _fp64_solve(s, schur_emu=False)
    assert np.array_equal(Xe, Xa) and lde == lda
    assert _exact_residual_is_zero(s, Xe)


SCHUR_CASES = [(2, 96, 2), (3, 65, 1), (5, 128, 4), (9, 200, 3), (17, 256, 16), (33, 130, 2), (64, 192, 5)]


@pytest.mark.parametrize("N,n,d", SCHUR_CASES)
def test_schur_emu_matches_oracle_and_alu(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=60 + N + n)
    Xe, lde = _fp64_solve(s, schur_emu=True)
    Xa, _ = _fp64_solve(s, schur_emu=False)
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(Xe, Xo) <= 1e-10
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], Xe, s["B"]) <= 1e-14
    # the two engines differ by rounding only
    assert oracle_mod.forward_error(Xe, Xa) <= 1e-12
    L, _ = oracle_mod.factor(s["A_diag"], s["A_sub"])
    ldo = oracle_mod.logdet(L)
    assert abs(lde - ldo) <= 1e-12 * max(1.0, abs(ldo))


def test_schur_emu_wide_row_scales(oracle_mod):
    """Rows and columns of the system spread over sixteen binades, so that
    the rows of every coupling block are cut below very different maxima."""
    N, n, d = 9, 160, 3
    s = inputs.random_btd(N, n, d, seed=11)
    sc = np.logspace(-8, 8, n)
    s["A_diag"] = s["A_diag"] * sc[None, :, None] * sc[None, None, :]
    s["A_sub"] = s["A_sub"] * sc[None, :, None] * sc[None, None, :]
    s["B"] = s["B"] * sc[None, :, None]
    Xe, _ = _fp64_solve(s, schur_emu=True)
    Xa, _ = _fp64_solve(s, schur_emu=False)
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], Xe, s["B"]) <= 1e-14
    # both engines reach the same backward error class; the forward
    # difference is bounded through the scaled condition number
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], Xa, s["B"]) <= 1e-14


def test_schur_emu_per_level_matches_persistent():
    s = inputs.random_btd(17, 128, 2, seed=5)
    X1, ld1 = _fp64_solve(s, schur_emu=True, persistent=True)
    X2, ld2 = _fp64_solve(s, schur_emu=True, persistent=False)
    assert np.array_equal(X1, X2) and ld1 == ld2


def test_schur_emu_not_spd_reports_block():
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(9, 128, 1, seed=2)
    s["A_diag"][6] -= 1e4 * np.eye(128)
    solver = Solver(9, 128, d_max=1)
    solver.set_option("schur_emu", 1)
    with pytest.raises(BDSSError) as e:
        solver.factor_solve(_dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"]))
    assert e.value.status == 2 and e.value.info.block == 6 and e.value.info.level == 1
    solver.close()


@pytest.mark.parametrize("n,prec", [(16, "fp64"), (128, "fp32_ir")])
def test_schur_emu_option_is_refused_elsewhere(n, prec):
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = Solver(8, n, d_max=2, precision=prec)
    with pytest.raises(BDSSError) as e:
        s.set_option("schur_emu", 1)
    assert e.value.status == 8
    s.set_option("schur_emu", 0)
    s.close()


# n <= 64: the per-level FP64 factorisation with the Schur products on the
# tensor cores (default for n = 64 and N >= 1024; forced on for the others).
@pytest.mark.parametrize("N,n,d", [(1024, 64, 4), (2000, 64, 1), (37, 64, 3), (100, 32, 2), (513, 48, 2),
                                   (2, 64, 2)])
def test_schur_emu_small_blocks_match_oracle(oracle_mod, N, n, d):
    s = inputs.random_btd(N, n, d, seed=70 + N + n)
    Xe, lde = _fp64_solve(s, schur_emu=True)
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(Xe, Xo) <= 1e-10
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], Xe, s["B"]) <= 1e-14
    Xa, _ = _fp64_solve(s, schur_emu=False)
    assert oracle_mod.forward_error(Xe, Xa) <= 1e-12
    L, _ = oracle_mod.factor(s["A_diag"], s["A_sub"])
    ldo = oracle_mod.logdet(L)
    assert abs(lde - ldo) <= 1e-12 * max(1.0, abs(ldo))


def test_schur_emu_small_opt_in_and_separate_solve(oracle_mod):
    """At the headline's block size the engine is opt-in; a factor followed
    by a separate solve gives the fused call's result."""
    from paper_2509_03015_gb300 import Solver
    N, n, d = 1500, 64, 4
    s = inputs.kalman_btd(N, n, 32, d, 0.95, 1)
    Ad, As, B = _dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"])
    sol = Solver(N, n, d_max=d)
    assert sol.factor_solve(Ad, As, B) is not None and sol.launch_stats()[0] == 1  # persistent FP64 ALU
    sol.set_option("schur_emu", 1)
    X1 = sol.factor_solve(Ad, As, B).cpu().numpy()
    assert sol.launch_stats()[0] > 1  # per-level launches, not the single persistent one
    sol.factor(Ad, As)
    X2 = sol.solve(B).cpu().numpy()
    sol.close()
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(X1, Xo) <= 1e-10
    assert oracle_mod.forward_error(X2, X1) <= 1e-13
