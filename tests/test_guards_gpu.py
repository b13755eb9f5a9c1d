"""GPU: workspace guard bands and injected allocation failures.

Every workspace buffer carries a 256-byte guard band of a fixed pattern; with
the debug option on, each call checks them.  The faults here are planted from
the host (a byte of a guard overwritten by cudaMemset, an allocation made to
fail): nothing faults on the device."""
import ctypes

import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(s):
    return tuple(torch.from_numpy(np.ascontiguousarray(s[k])).cuda() for k in ("A_diag", "A_sub", "B"))


@pytest.mark.parametrize("N,n,d,precision,persistent", [
    (1000, 24, 2, "fp64", True), (777, 64, 4, "fp64", False), (300, 32, 3, "fp32_ir", True),
    (65, 96, 4, "fp64", True), (65, 96, 4, "tf32_ir", True)])
def test_guard_bands_hold(N, n, d, precision, persistent):
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(N, n, d, seed=N)
    Ad, As, B = _dev(s)
    sol = Solver(N, n, d_max=d, precision=precision, persistent=persistent)
    try:
        sol.set_option("debug_guards", 1)
        X = sol.factor_solve(Ad, As, B)
        sol.solve(B, torch.empty_like(X))
        sol.logdet()
    finally:
        sol.close()


def test_overwritten_guard_is_reported():
    from paper_2509_03015_gb300 import BDSSError, Solver
    s = inputs.random_btd(200, 16, 1, seed=1)
    Ad, As, B = _dev(s)
    sol = Solver(200, 16, d_max=1)
    try:
        sol.set_option("debug_guards", 1)
        sol.factor_solve(Ad, As, B)
        sol.set_option("debug_corrupt_guard", 2)  # the coupling buffer's band
        with pytest.raises(BDSSError) as e:
            sol.factor_solve(Ad, As, B)
        assert e.value.status == 9
        with pytest.raises(BDSSError):
            sol.set_option("debug_corrupt_guard", 99)  # no such buffer
    finally:
        sol.close()


@pytest.mark.parametrize("precision,n", [("fp64", 32), ("fp32_ir", 32), ("tf32_ir", 128)])
def test_injected_allocation_failure_frees_everything(precision, n):
    from paper_2509_03015_gb300 import BDSSError, Solver, _lib
    lib = _lib.load()
    Solver(500, n, d_max=2, precision=precision).close()  # warm the context
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failures = 0
    try:
        for k in range(1, 40):
            assert lib.bdss_debug_fail_alloc(k) == 0
            try:
                sol = Solver(500, n, d_max=2, precision=precision)
            except BDSSError as e:
                assert e.status == 4
                failures += 1
                continue
            sol.close()  # k beyond the number of allocations: creation succeeds
            break
    finally:
        lib.bdss_debug_fail_alloc(0)
    assert failures >= 6
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < (4 << 20)  # nothing left allocated
    sol = Solver(500, n, d_max=2, precision=precision)
    sol.close()
