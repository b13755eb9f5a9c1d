"""The crossover N_* (Sec. 3.3): the reduction stops at the first level with
at most N_* blocks and one CTA factors and solves them by the serial
block-Cholesky sweep (Algorithms 1 and 2 with K = 1).  Against the oracle,
element by element, with the log-determinant, for N_* below, at and above
the level sizes (N <= N_* is a serial solve of the whole system)."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs
from tests._helpers import assert_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.mark.parametrize("N,n,d,nstar", [(1, 5, 1, 4), (3, 8, 2, 4), (9, 8, 1, 2), (17, 1, 1, 16), (64, 8, 1, 64),
                                         (100, 32, 3, 7), (257, 64, 2, 8), (1000, 12, 4, 33), (4099, 24, 1, 3)])
def test_serial_top_sweep_parity(oracle_mod, N, n, d, nstar):
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(N, n, d, seed=500 + N + nstar)
    sol = Solver(N, n, d_max=d)
    sol.set_option("nstar", nstar)
    Ad, As, B = _dev(s["A_diag"]), _dev(s["A_sub"] if N > 1 else np.zeros((1, n, n))), _dev(s["B"])
    X = sol.factor_solve(Ad, As, B).cpu().numpy()
    ld = sol.logdet()
    X2 = sol.solve(B).cpu().numpy()           # the stored sweep factors again
    sol.set_option("persistent", 0)
    sol.factor(Ad, As)
    X3 = sol.solve(B).cpu().numpy()           # one launch per level and the top
    sol.close()
    L, C = oracle_mod.factor(s["A_diag"], s["A_sub"])
    Xo = oracle_mod.solve(L, C, s["B"])
    assert oracle_mod.forward_error(X, Xo) <= 1e-10
    assert_elementwise(X, Xo, rtol=1e-10, atol_frac=1e-12)
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14
    ldo = oracle_mod.logdet(L)
    assert abs(ld - ldo) <= 1e-12 * max(1.0, abs(ldo))
    assert np.array_equal(X, X2) and np.array_equal(X2, X3)


def test_nstar_limits():
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = Solver(16, 8, d_max=1, precision="fp32_ir")
    with pytest.raises(BDSSError) as e:
        s.set_option("nstar", 4)
    assert e.value.status == 8
    s.close()
    s = Solver(16, 96, d_max=1)
    with pytest.raises(BDSSError) as e:
        s.set_option("nstar", 4)
    assert e.value.status == 8
    with pytest.raises(BDSSError) as e:
        s.set_option("nstar", 0)
    assert e.value.status == 1
    s.close()


def test_tune_nstar_keeps_a_candidate(oracle_mod):
    from paper_2509_03015_gb300 import Solver
    s = inputs.workload("kalman-N64-n8-d1")
    sol = Solver(64, 8, d_max=1)
    Ad, As, B = _dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"])
    best, times = sol.tune_nstar(Ad, As, B, candidates=(1, 2, 4, 8, 64), reps=3)
    assert best in times and times[best] == min(times.values())
    X = sol.factor_solve(Ad, As, B).cpu().numpy()
    sol.close()
    assert oracle_mod.forward_error(X, oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])) <= 1e-10
