"""Mixed precision beyond plain refinement: FP64 conjugate gradients
preconditioned by the FP32 (or TF32) factors, on systems whose condition
number stalls X += M^-1 r.  The solution is checked against the oracle's FP64
solve (forward error within the kappa-scaled bound) and its backward error
recomputed by the oracle."""
import numpy as np
import pytest

import oracle
from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TARGET = 1e-14  # the library's default target backward error


def _dev(s):
    return (torch.from_numpy(np.ascontiguousarray(s[k])).cuda() for k in ("A_diag", "A_sub", "B"))


def _solve(N, n, d, precision, A_diag, A_sub, B, krylov, **opts):
    from paper_2509_03015_gb300 import Solver, _lib
    sol = Solver(N, n, d_max=d, precision=precision)
    try:
        sol.set_option("refine_krylov", krylov)
        for k, v in opts.items():
            sol.set_option(k, v)
        try:
            X = sol.factor_solve(A_diag, A_sub, B)
            status, info = 0, sol.last_info
        except _lib.BDSSError as e:
            X, status, info = None, e.status, e.info
        return X, status, sol.refine_stats(), info
    finally:
        sol.close()


def _check(s, X, kappa):
    Xh = X.cpu().numpy()
    berr = oracle.backward_error(s["A_diag"], s["A_sub"], Xh, s["B"])
    assert berr <= TARGET, berr
    Xr = oracle.solve_system(s["A_diag"], s["A_sub"], s["B"])
    # a backward error e bounds the forward error by about kappa e; the
    # oracle's FP64 solve is backward stable too (e ~ u_64 << TARGET)
    assert oracle.forward_error(Xh, Xr) <= 10 * kappa * TARGET


def test_cg_refinement_converges_where_plain_refinement_stalls():
    # kappa ~ 0.7 N^2 = 7.5e8, kappa u_32 ~ 45: plain refinement does not reach
    # the target within its 10 steps
    N, n, d = 32768, 4, 2
    s = inputs.laplace_btd(N, n, d, seed=1)
    kappa = 0.7 * N * N
    Ad, As, B = _dev(s)
    X0, st0, (plain0, cg0), _ = _solve(N, n, d, "fp32_ir", Ad, As, B, krylov=0)
    assert cg0 == 0
    X1, st1, (plain1, cg1), info = _solve(N, n, d, "fp32_ir", Ad, As, B, krylov=1)
    assert st1 == 0
    assert info.iters == plain1 + cg1
    assert info.backward_err <= TARGET
    _check(s, X1, kappa)
    if st0 == 7:  # plain refinement stalled or ran out of steps: CG did the work
        assert cg1 > 0
    else:
        pytest.skip(f"plain refinement converged (status {st0}) at kappa ~ {kappa:.1e}")


@pytest.mark.parametrize("precision,N,n,d", [("fp32_ir", 300, 16, 3), ("fp32_ir", 97, 80, 2), ("tf32_ir", 256, 80, 1)])
def test_cg_from_the_start(precision, N, n, d):
    s = inputs.laplace_btd(N, n, d, seed=N + n)
    Ad, As, B = _dev(s)
    X, st, (plain, cg), info = _solve(N, n, d, precision, Ad, As, B, krylov=2)
    assert st == 0
    assert plain == 0 and cg > 0
    assert info.backward_err <= TARGET
    _check(s, X, 0.7 * N * N)


def test_well_conditioned_systems_never_reach_cg():
    N, n, d = 1000, 32, 2
    s = inputs.random_btd(N, n, d, seed=3)
    Ad, As, B = _dev(s)
    X, st, (plain, cg), _ = _solve(N, n, d, "fp32_ir", Ad, As, B, krylov=1)
    assert st == 0 and cg == 0 and plain >= 1


def test_zero_corrections_and_cg_allocation_failure():
    from paper_2509_03015_gb300 import _lib
    N, n, d = 2048, 8, 1
    s = inputs.laplace_btd(N, n, d, seed=4)
    Ad, As, B = _dev(s)
    # max_refine = 0 stops before any correction, CG included
    _, st, (plain, cg), _ = _solve(N, n, d, "fp32_ir", Ad, As, B, krylov=2, max_refine=0)
    assert st == 7 and plain == 0 and cg == 0
    # the CG buffers are allocated on first use; a failed allocation is reported
    from paper_2509_03015_gb300 import Solver
    lib = _lib.load()
    sol = Solver(N, n, d_max=d, precision="fp32_ir")
    try:
        sol.set_option("refine_krylov", 2)
        assert lib.bdss_debug_fail_alloc(2) == 0
        try:
            with pytest.raises(_lib.BDSSError) as e:
                sol.factor_solve(Ad, As, B)
            assert e.value.status == 4
        finally:
            lib.bdss_debug_fail_alloc(0)
        X = sol.factor_solve(Ad, As, B)  # the remaining buffers are allocated now
        _check(s, X, 0.7 * N * N)
    finally:
        sol.close()


@pytest.mark.parametrize("N,n,d,prec", [(64, 8, 2, "fp32_ir"), (33, 24, 1, "fp32_ir"), (9, 96, 2, "tf32_ir")])
def test_shifted_factorisation_beyond_fp32(oracle_mod, N, n, d, prec):
    """kappa ~ 1e9: the FP32 Cholesky fails (a pivot goes non-positive in
    FP32), the default mode factors A + sigma diag(A) and the FP64 CG
    refinement on the unshifted A reaches the backward-error bar; with the
    shift switched off the call reports BDSS_ERR_NOT_SPD."""
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.illcond_btd(N, n, d, seed=N + n, kappa=1e9)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
    Ad, As, B = dev(s["A_diag"]), dev(s["A_sub"]), dev(s["B"])
    off = Solver(N, n, d_max=d, precision=prec)
    off.set_option("shift", 0)
    with pytest.raises(BDSSError) as e:
        off.factor_solve(Ad, As, B)
    assert e.value.status == 2
    off.close()
    sol = Solver(N, n, d_max=d, precision=prec)
    X = sol.factor_solve(Ad, As, B).cpu().numpy()
    sigma = sol.factor_shift()
    plain, cg = sol.refine_stats()
    sol.close()
    assert sigma > 0 and cg > 0
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    # forward error bounded by about kappa u_64 (both solutions are backward stable)
    assert oracle_mod.forward_error(X, Xo) <= 1e9 * 2.2e-16 * 50
