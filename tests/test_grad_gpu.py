"""Differentiation: the hand-written adjoint backward of BlockTriSolve
against (a) the oracle's adjoint gradients at the full N = 2048, n = 32, d = 8
workload, (b) central finite differences (step 1e-6) through the GPU solve on
random entries and on random directions supported on 1% of the entries, and
(c) a dense torch.linalg gradient at N = 16.  Loss L = sum(W * X)."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _grads(s, W):
    from paper_2509_03015_gb300 import block_tri_solve
    Ad = _dev(s["A_diag"]).requires_grad_(True)
    As = _dev(s["A_sub"]).requires_grad_(True)
    B = _dev(s["B"]).requires_grad_(True)
    X = block_tri_solve(Ad, As, B)
    loss = (X * _dev(W)).sum()
    loss.backward()
    return (X.detach().cpu().numpy(), Ad.grad.cpu().numpy(), As.grad.cpu().numpy(), B.grad.cpu().numpy())


def _loss(solver, Ad, As, B, W):
    X = solver.factor_solve(Ad, As, B)
    return float((X * W).sum().item())


def test_grads_vs_oracle_full_size(oracle_mod):
    s = inputs.workload("kalman-N2048-n32-d8-grad", with_W=True)
    X, gD, gS, gB = _grads(s, s["W"])
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    Lo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["W"])
    oD, oS = oracle_mod.adjoint_grads(Lo, Xo)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(X, Xo) <= 1e-10
    assert rel(gB, Lo) <= 1e-10
    assert rel(gD, oD) <= 1e-10
    assert rel(gS, oS) <= 1e-10


def test_grads_vs_central_differences():
    from paper_2509_03015_gb300 import Solver
    s = inputs.workload("kalman-N2048-n32-d8-grad", with_W=True)
    N, n, _ = s["A_diag"].shape
    _, gD, gS, gB = _grads(s, s["W"])
    Ad, As, B, W = _dev(s["A_diag"]), _dev(s["A_sub"]), _dev(s["B"]), _dev(s["W"])
    solver = Solver(N, n, d_max=8)
    h = 1e-6
    rng = np.random.default_rng(0)

    def fd(which, idx=None, V=None):
        base = {"D": Ad, "S": As, "B": B}[which]
        P, M = base.clone(), base.clone()
        if V is None:
            P[idx] += h
            M[idx] -= h
        else:
            P += h * V
            M -= h * V
        args_p = {"D": (P, As, B), "S": (Ad, P, B), "B": (Ad, As, P)}[which]
        args_m = {"D": (M, As, B), "S": (Ad, M, B), "B": (Ad, As, M)}[which]
        return (_loss(solver, *args_p, W) - _loss(solver, *args_m, W)) / (2 * h)
    # single entries
    for _ in range(16):
        i, r, c = int(rng.integers(0, N)), int(rng.integers(0, n)), int(rng.integers(0, n))
        g = fd("D", (i, r, c))
        assert abs(g - gD[i, r, c]) <= 1e-6 * max(1.0, abs(g))
        i = int(rng.integers(0, N - 1))
        g = fd("S", (i, r, c))
        assert abs(g - gS[i, r, c]) <= 1e-6 * max(1.0, abs(g))
    # random directions supported on a random 1% of the entries
    for which, grad in (("D", gD), ("S", gS), ("B", gB)):
        for _ in range(4):
            shape = grad.shape
            mask = rng.random(shape) < 0.01
            V = np.where(mask, rng.standard_normal(shape), 0.0)
            g = fd(which, V=_dev(V))
            ref = float((grad * V).sum())
            assert abs(g - ref) <= 1e-6 * max(1.0, abs(ref)), (which, g, ref)
    solver.close()


def test_grads_vs_dense_torch_N16():
    s = inputs.kalman_btd(16, 32, 16, 8, 0.95, 0, with_W=True)
    N, n, d = 16, 32, 8
    _, gD, gS, gB = _grads(s, s["W"])
    Ad = torch.tensor(s["A_diag"], requires_grad=True)
    As = torch.tensor(s["A_sub"], requires_grad=True)
    Bt = torch.tensor(s["B"], requires_grad=True)
    rows = []
    for i in range(N):
        row = []
        for j in range(N):
            if i == j:
                row.append(0.5 * (Ad[i] + Ad[i].T))
            elif i == j + 1:
                row.append(As[j])
            elif j == i + 1:
                row.append(As[i].T)
            else:
                row.append(torch.zeros(n, n, dtype=torch.float64))
        rows.append(torch.cat(row, 1))
    A = torch.cat(rows, 0)
    X = torch.linalg.solve(A, Bt.reshape(N * n, d))
    (X * torch.tensor(s["W"].reshape(N * n, d))).sum().backward()
    np.testing.assert_allclose(gD, Ad.grad.numpy(), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(gS, As.grad.numpy(), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(gB, Bt.grad.numpy(), rtol=1e-9, atol=1e-11)
