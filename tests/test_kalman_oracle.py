"""Pins of the oracle's Kalman-smoother assembly (Sec. 4.2) against things
other than its own block formulas: the dense normal equations built from the
stacked state and observation operators, and the time-invariant generator the
workloads use."""
import numpy as np
import pytest

import oracle
from paper_2509_03015_gb300 import inputs


def _spd(rng, n, scale=1.0):
    M = rng.standard_normal((n, n))
    return scale * (M @ M.T / n + np.eye(n))


def _dense(A_diag, A_sub):
    N = A_diag.shape[0]
    blk = oracle.dense_blocks(A_diag, A_sub)
    return np.block([[blk(r, c) for c in range(N)] for r in range(N)])


def _model(N, n, m, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((N, n, n)) / np.sqrt(n)
    H = rng.standard_normal((N, m, n)) / np.sqrt(n)
    Qinv = np.stack([_spd(rng, n, 3.0) for _ in range(N)])
    Rinv = np.stack([_spd(rng, m, 0.5) for _ in range(N)])
    z = rng.standard_normal((N, m))
    zeta = rng.standard_normal((N, n))
    return G, H, Qinv, Rinv, z, zeta


@pytest.mark.parametrize("diag_r", [False, True])
@pytest.mark.parametrize("N,n,m", [(1, 3, 2), (2, 2, 3), (5, 4, 3), (6, 3, 5)])
def test_assembly_equals_dense_normal_equations(N, n, m, diag_r):
    # minimise 1/2 |Hx - z|^2_{R^-1} + 1/2 |Gx - zeta|^2_{Q^-1}: the stacked state
    # operator has I on its block diagonal and -G_k below it; the normal
    # equations are (H^T R^-1 H + G^T Q^-1 G) x = H^T R^-1 z + G^T Q^-1 zeta
    G, H, Qinv, Rinv, z, zeta = _model(N, n, m, seed=N * 10 + n)
    r_in = Rinv
    if diag_r:
        r_in = np.stack([np.diag(R) for R in Rinv])  # keep only the diagonals
        Rinv = np.stack([np.diag(r) for r in r_in])
    Gbig = np.eye(N * n)
    for k in range(1, N):
        Gbig[k * n:(k + 1) * n, (k - 1) * n:k * n] = -G[k]
    Hbig = np.zeros((N * m, N * n))
    Qbig = np.zeros((N * n, N * n))
    Rbig = np.zeros((N * m, N * m))
    for k in range(N):
        Hbig[k * m:(k + 1) * m, k * n:(k + 1) * n] = H[k]
        Qbig[k * n:(k + 1) * n, k * n:(k + 1) * n] = Qinv[k]
        Rbig[k * m:(k + 1) * m, k * m:(k + 1) * m] = Rinv[k]
    A = Hbig.T @ Rbig @ Hbig + Gbig.T @ Qbig @ Gbig
    b = Hbig.T @ Rbig @ z.reshape(-1) + Gbig.T @ Qbig @ zeta.reshape(-1)
    A_diag, A_sub, B = oracle.kalman_assemble(G, H, Qinv, r_in, z, zeta)
    Ad = _dense(A_diag, A_sub)
    np.testing.assert_allclose(Ad, A, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(B.reshape(-1), b, rtol=1e-12, atol=1e-12)


def test_assembly_reproduces_the_time_invariant_generator():
    # the workloads' generator: F = rho * Haar, H, Q = 0.1 I, R = 0.5 I, P0 = I,
    # A_11 = P0^-1 + ...: the assembly with Qinv[0] = P0^-1 gives the same blocks
    N, n, m, rho, seed = 7, 5, 3, 0.95, 4
    s = inputs.kalman_btd(N, n, m, 1, rho, seed)
    rng = np.random.default_rng(seed)
    F = rho * inputs.haar_orthogonal(rng, n)
    Hm = rng.standard_normal((m, n)) / np.sqrt(n)
    G = np.stack([np.eye(n)] + [F] * (N - 1))
    H = np.stack([Hm] * N)
    Qinv = np.stack([np.eye(n)] + [10.0 * np.eye(n)] * (N - 1))
    Rinv = np.stack([2.0 * np.eye(m)] * N)
    A_diag, A_sub, _ = oracle.kalman_assemble(G, H, Qinv, Rinv, np.zeros((N, m)))
    np.testing.assert_allclose(A_diag, s["A_diag"], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(A_sub, s["A_sub"], rtol=1e-13, atol=1e-13)


def test_assembled_system_is_spd_and_solves():
    G, H, Qinv, Rinv, z, zeta = _model(9, 6, 4, seed=2)
    A_diag, A_sub, B = oracle.kalman_assemble(G, H, Qinv, Rinv, z, zeta)
    A = _dense(A_diag, A_sub)
    np.linalg.cholesky(A)  # SPD
    X = oracle.solve_system(A_diag, A_sub, B)
    np.testing.assert_allclose(A @ X.reshape(-1), B.reshape(-1), rtol=1e-10, atol=1e-10)


def test_neuro_shaped_model_follows_its_recipe():
    # damped 2-D rotations (|eigenvalues| = rho in [0.95, 0.999]), G_0 = I,
    # dense SPD Q^-1, tall well-conditioned H, diagonal R^-1 = 1, zeta only at 0
    N, n, m = 5, 16, 64
    mod = inputs.kalman_neuro_model(N, n, m, seed=7)
    G, H, Qinv, Rinv, zeta = mod["G"], mod["H"], mod["Qinv"], mod["Rinv"], mod["zeta"]
    np.testing.assert_array_equal(G[0], np.eye(n))
    ev = np.abs(np.linalg.eigvals(G[1]))
    assert ev.min() >= 0.95 - 1e-12 and ev.max() <= 0.999 + 1e-12
    GtG = G[1].T @ G[1]
    np.testing.assert_allclose(GtG, np.diag(np.diag(GtG)), atol=1e-14)  # scaled orthogonal blocks
    assert np.linalg.eigvalsh(Qinv[0]).min() > 0 and np.count_nonzero(Qinv[0]) == n * n
    sv = np.linalg.svd(H[0], compute_uv=False)
    assert sv.max() / sv.min() < 10
    assert Rinv.shape == (N, m) and np.all(Rinv == 1.0)
    assert np.any(zeta[0] != 0) and not np.any(zeta[1:])
    A_diag, A_sub, _ = oracle.kalman_assemble(G, H, Qinv, Rinv, mod["z"], zeta)
    np.linalg.cholesky(_dense(A_diag, A_sub))
