"""Batched solves in one launch (device work queue): every instance against
the oracle, including the 512-instance uneven MPC batch; CUDA-graph replay is
bitwise equal to a plain launch; the autotuner picks a valid configuration;
a non-SPD instance fails alone."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _to_dev(systems):
    out = []
    for s in systems:
        N, n, _ = s["A_diag"].shape
        As = s["A_sub"] if N > 1 else np.zeros((1, n, n))
        out.append((_dev(s["A_diag"]), _dev(As), _dev(s["B"])))
    return out


def _mixed_batch(K=48, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(K):
        N = int(rng.choice([1, 2, 3, 5, 8, 17, 33, 64, 100, 257, 300]))
        n = int(rng.choice([1, 3, 8, 12, 24, 31, 48, 64]))
        out.append(inputs.random_btd(N, n, 2, seed=seed * 1000 + k))
    return out


def test_batched_mixed_parity(oracle_mod):
    from paper_2509_03015_gb300 import BatchSolver
    systems = _mixed_batch()
    bs = BatchSolver(_to_dev(systems))
    X = bs.run()
    for s, Xk in zip(systems, X):
        Xk = Xk.cpu().numpy()
        Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
        assert oracle_mod.forward_error(Xk, Xo) <= 1e-10
        assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], Xk, s["B"]) <= 1e-14
    bs.close()


def test_mpc_batch_512_full(oracle_mod):
    from paper_2509_03015_gb300 import BatchSolver
    systems = inputs.mpc_batch(**{k: v for k, v in inputs.MPC_BATCH.items() if k in ("K", "d", "rho", "seed")})
    assert len(systems) == 512
    bs = BatchSolver(_to_dev(systems))
    X = bs.run(graph=True)
    status, lat = bs.wait()
    assert all(s == 0 for s in status) and all(t > 0 for t in lat)
    Xo, _ = oracle_mod.factor_solve_batched(systems)
    for s, Xk, xo in zip(systems, X, Xo):
        Xk = Xk.cpu().numpy()
        assert oracle_mod.forward_error(Xk, xo) <= 1e-10
    # backward error on a sample of instances (compensated residual is costly)
    for k in range(0, 512, 37):
        s = systems[k]
        assert oracle_mod.backward_error(s["A_diag"], s["A_sub"], X[k].cpu().numpy(), s["B"]) <= 1e-14
    bs.close()


def test_graph_replay_bitwise_equal():
    from paper_2509_03015_gb300 import BatchSolver
    systems = _mixed_batch(K=32, seed=3)
    dev = _to_dev(systems)
    bs = BatchSolver(dev)
    X0 = [x.clone() for x in bs.run(graph=False)]
    for _ in range(2):
        for x in bs.X:
            x.zero_()
        X1 = bs.run(graph=True)
        for a, b in zip(X0, X1):
            assert torch.equal(a, b)
    bs.close()


def test_autotune_and_reuse(oracle_mod):
    from paper_2509_03015_gb300 import BatchSolver
    systems = _mixed_batch(K=24, seed=5)
    bs = BatchSolver(_to_dev(systems), autotune=2)
    t, i = bs.config
    assert t in (32, 64, 128, 256) and t >= max(s["A_diag"].shape[1] for s in systems) and i in (1, 2, 4)
    X = bs.run()
    for s, Xk in zip(systems, X):
        Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
        assert oracle_mod.forward_error(Xk.cpu().numpy(), Xo) <= 1e-10
    bs.close()


def test_non_spd_instance_fails_alone(oracle_mod):
    from paper_2509_03015_gb300 import BatchSolver
    systems = _mixed_batch(K=16, seed=7)
    bad = 5
    N, n, _ = systems[bad]["A_diag"].shape
    systems[bad]["A_diag"][N - 1] -= 1e4 * np.eye(n)
    bs = BatchSolver(_to_dev(systems))
    bs.launch()
    status, _ = bs.wait(raise_on_error=False)
    assert status[bad] == 2
    for k, s in enumerate(systems):
        if k == bad:
            continue
        assert status[k] == 0
        Xo = oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
        assert oracle_mod.forward_error(bs.X[k].cpu().numpy(), Xo) <= 1e-10
    bs.close()
