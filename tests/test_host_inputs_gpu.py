"""GPU: inputs in page-locked host memory are read in place by the kernels
(the level-0 steps stage them through L2), giving the same bits as device
inputs; outputs must be device memory."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("N,n,d", [(1, 8, 1), (2, 5, 2), (257, 64, 4), (1000, 12, 3)])
def test_pinned_host_inputs_match_device_inputs(N, n, d, persistent):
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(N, n, d, seed=11 + N)
    h = {k: torch.from_numpy(np.ascontiguousarray(s[k])).pin_memory() for k in ("A_diag", "A_sub", "B")}
    dv = {k: v.cuda() for k, v in h.items()}
    sol = Solver(N, n, d_max=d, persistent=persistent)
    try:
        X_dev = sol.factor_solve(dv["A_diag"], dv["A_sub"], dv["B"])
        X_host = sol.factor_solve(h["A_diag"], h["A_sub"], h["B"])
        assert X_host.is_cuda
        assert torch.equal(X_dev, X_host)
        sol.factor(h["A_diag"], h["A_sub"])
        X2 = sol.solve(h["B"])
        X3 = sol.solve(dv["B"])
        assert torch.equal(X2, X3)
    finally:
        sol.close()


def test_pinned_host_inputs_mixed_precision(oracle_mod):
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(300, 32, 2, seed=3)
    h = {k: torch.from_numpy(np.ascontiguousarray(s[k])).pin_memory() for k in ("A_diag", "A_sub", "B")}
    sol = Solver(300, 32, d_max=2, precision="fp32_ir")
    try:
        X = sol.factor_solve(h["A_diag"], h["A_sub"], h["B"]).cpu().numpy()
        assert sol.last_info.backward_err <= 1e-14
        assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14
    finally:
        sol.close()


def test_host_output_is_rejected():
    import ctypes
    from paper_2509_03015_gb300 import Solver, _lib
    s = inputs.random_btd(10, 4, 1, seed=1)
    dv = {k: torch.from_numpy(np.ascontiguousarray(s[k])).cuda() for k in ("A_diag", "A_sub", "B")}
    Xh = torch.empty(dv["B"].shape, dtype=torch.float64).pin_memory()
    sol = Solver(10, 4, d_max=1)
    try:
        info = _lib.bdss_info()
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        st = sol.lib.bdss_factor_solve(sol.h, p(dv["A_diag"]), p(dv["A_sub"]), p(dv["B"]), p(Xh), 1,
                                       ctypes.byref(info))
        assert st == 1  # X must be device memory
    finally:
        sol.close()
