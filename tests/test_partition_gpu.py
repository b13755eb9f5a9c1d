"""The partitioned solve's library side on one GPU: bdss_chunk_reduce
against the chunk contribution computed by the oracle from its definition,
and the whole partitioned solve with G ranks played in turn by one process
(phase 1 for every rank, the exchange as a list, then phase 2), against the
oracle's solution of the full system.  No rank waits on another's kernels."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs, partition
from tests.test_partition_cpu import _cpu_ops

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Ni,n,d,sides", [(1, 4, 1, "both"), (5, 8, 2, "left"), (6, 16, 3, "right"),
                                          (9, 32, 2, "both"), (17, 96, 4, "both"), (4, 130, 1, "both")])
def test_chunk_reduce_matches_definition(oracle_mod, Ni, n, d, sides):
    from paper_2509_03015_gb300 import Solver
    s = inputs.random_btd(Ni + 2, n, d, seed=Ni * n)
    Ad, As, B = s["A_diag"][1:-1], s["A_sub"][1:-1], s["B"][1:-1]
    A_left = s["A_sub"][0] if sides in ("both", "left") else None
    A_right = s["A_sub"][-1] if sides in ("both", "right") else None
    elim, back, _ = _cpu_ops(oracle_mod)
    S_ref, bh_ref = elim(Ad, As, A_left, A_right, B)
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    sol = Solver(Ni, n, d_max=max(d, min(n, 64)))
    S, bh = sol.chunk_reduce(dev(Ad), dev(As if Ni > 1 else np.zeros((1, n, n))), dev(A_left), dev(A_right), dev(B))
    scale = max(1.0, np.abs(S_ref).max())
    np.testing.assert_allclose(S.cpu().numpy(), S_ref, rtol=1e-10, atol=1e-12 * scale)
    np.testing.assert_allclose(bh.cpu().numpy(), bh_ref, rtol=1e-10, atol=1e-12 * max(1.0, np.abs(bh_ref).max()))
    xl = np.random.default_rng(1).standard_normal((n, d))
    xr = np.random.default_rng(2).standard_normal((n, d))
    X = sol.chunk_backsolve(dev(B), dev(A_left), dev(A_right), dev(xl if A_left is not None else None),
                            dev(xr if A_right is not None else None)).cpu().numpy()
    Xo = back(B, A_left, A_right, xl if A_left is not None else None, xr if A_right is not None else None)
    assert oracle_mod.forward_error(X, Xo) <= 1e-10
    sol.close()


@pytest.mark.parametrize("N,G,n,d", [(37, 2, 5, 2), (64, 4, 16, 1), (257, 8, 24, 3), (99, 3, 80, 2)])
def test_partitioned_solve_ranks_in_turn(oracle_mod, N, G, n, d):
    s = inputs.random_btd(N, n, d, seed=N + G)
    ops = [partition.gpu_chunk_ops(n, d) for _ in range(G)]
    msgs = [partition.chunk_message(s["A_diag"], s["A_sub"], s["B"], G, g, ops[g][0]) for g in range(G)]
    X = np.empty_like(s["B"])
    for g in range(G):
        (a, b), Xg = partition.chunk_finish(s["A_sub"], s["B"], G, g, msgs, ops[g][1], ops[g][2])
        X[a:b] = Xg
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(X, Xo) <= 1e-10
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14
