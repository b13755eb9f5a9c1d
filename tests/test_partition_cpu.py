"""The partitioned solve's host logic on CPU: chunking, the exchange, the
reduced system of the separators and the back-solve.  The chunk elimination
is done here by the oracle (standing in for the GPU's bdss_chunk_reduce),
written from its definition in partition.py: S_LL = A_left^T (A_I^-1)_ff
A_left and so on.  The reduced system is pinned to the oracle's dense Eq. 5
(schur_partition), and the whole solve, over gloo ranks (world size 2 and 4),
to the oracle's solution of the full system."""
import os

import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs, partition


def _cpu_ops(oracle):
    def eliminate(Ad, As, A_left, A_right, B_I):
        Ni, n, _ = Ad.shape
        d = B_I.shape[-1]
        y = oracle.solve_system(Ad, As, B_I)
        S = np.zeros((3, n, n))
        bh = np.zeros((2, n, d))
        if A_left is not None:
            R = np.zeros((Ni, n, n))
            R[0] = A_left
            ZL = oracle.solve_system(Ad, As, R)
            S[0] = A_left.T @ ZL[0]
            bh[0] = A_left.T @ y[0]
            if A_right is not None:
                S[2] = A_right @ ZL[-1]
        if A_right is not None:
            R = np.zeros((Ni, n, n))
            R[-1] = A_right.T
            ZR = oracle.solve_system(Ad, As, R)
            S[1] = A_right @ ZR[-1]
            bh[1] = A_right @ y[-1]
        return S, bh

    def backsolve(B_I, A_left, A_right, x_left, x_right):
        Bp = np.array(B_I, dtype=np.float64)
        if A_left is not None:
            Bp[0] -= A_left @ x_left
        if A_right is not None:
            Bp[-1] -= A_right.T @ x_right
        Ni = Bp.shape[0]
        return None if Ni == 0 else oracle.solve_system(_keep["Ad"], _keep["As"], Bp)

    _keep = {}

    def eliminate_keep(Ad, As, A_left, A_right, B_I):
        _keep["Ad"], _keep["As"] = Ad, As
        return eliminate(Ad, As, A_left, A_right, B_I)

    def reduced_solve(D, E, b):
        return oracle.solve_system(D, E, b)
    return eliminate_keep, backsolve, reduced_solve


@pytest.mark.parametrize("N,G", [(1, 1), (5, 1), (3, 2), (4, 2), (9, 3), (10, 4), (37, 4), (64, 8)])
def test_chunks_cover_and_leave_interiors(N, G):
    b = partition.chunk_bounds(N, G)
    assert b[0][0] == 0 and b[-1][1] == N and all(b[g][1] == b[g + 1][0] for g in range(G - 1))
    for g in range(G):
        (i0, i1), left, right = partition.chunk_layout(N, G, g)
        assert i1 > i0  # every chunk has a nonempty interior
        assert (left is None) == (g == 0) and (right is None) == (g == G - 1)
    with pytest.raises(ValueError):
        partition.chunk_bounds(4, 3)


@pytest.mark.parametrize("N,G,n,d", [(9, 3, 2, 1), (12, 4, 3, 2), (7, 2, 4, 3)])
def test_reduced_system_is_the_dense_schur_complement(oracle_mod, N, G, n, d):
    """The assembled separator system equals Eq. 5 with A_uu = all interiors,
    computed densely by the oracle."""
    s = inputs.random_btd(N, n, d, seed=N * 10 + G)
    elim, _, _ = _cpu_ops(oracle_mod)
    msgs = [partition.chunk_message(s["A_diag"], s["A_sub"], s["B"], G, g, elim) for g in range(G)]
    D, E, b = partition.reduced_system(msgs, n, d)
    seps = [partition.chunk_layout(N, G, g)[2] for g in range(G - 1)]
    S, b_hat, _, _, _ = oracle_mod.schur_partition(s["A_diag"], s["A_sub"], s["B"], seps)
    Gm = G - 1
    dense = np.zeros((Gm * n, Gm * n))
    for g in range(Gm):
        dense[g * n:(g + 1) * n, g * n:(g + 1) * n] = 0.5 * (D[g] + D[g].T)
        if g + 1 < Gm:
            dense[(g + 1) * n:(g + 2) * n, g * n:(g + 1) * n] = E[g]
            dense[g * n:(g + 1) * n, (g + 1) * n:(g + 2) * n] = E[g].T
    np.testing.assert_allclose(dense, S, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b.reshape(-1, d), b_hat, rtol=1e-12, atol=1e-12)


def _worker(rank, world, port, N, n, d, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    s = inputs.random_btd(N, n, d, seed=77)
    elim, back, red = _cpu_ops(oracle)
    (a, b), X = partition.partitioned_solve(s["A_diag"], s["A_sub"], s["B"], world, rank, elim, back, red,
                                            partition.torch_allgather())
    np.save(os.path.join(out, f"x{rank}.npy"), X)
    np.save(os.path.join(out, f"r{rank}.npy"), np.array([a, b]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_partitioned_solve_over_gloo_ranks(oracle_mod, tmp_path, world):
    torch = pytest.importorskip("torch")
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    N, n, d = 37, 5, 2
    mp.start_processes(_worker, args=(world, port, N, n, d, str(tmp_path)), nprocs=world, start_method="spawn")
    s = inputs.random_btd(N, n, d, seed=77)
    X = np.empty_like(s["B"])
    covered = np.zeros(N, dtype=bool)
    for r in range(world):
        a, b = np.load(tmp_path / f"r{r}.npy")
        X[a:b] = np.load(tmp_path / f"x{r}.npy")
        assert not covered[a:b].any()
        covered[a:b] = True
    assert covered.all()
    Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
    assert oracle_mod.forward_error(X, Xo) <= 1e-12
    assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X, s["B"]) <= 1e-14
    del torch
