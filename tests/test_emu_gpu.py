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
