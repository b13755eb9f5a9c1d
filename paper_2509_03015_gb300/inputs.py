"""Seeded synthetic inputs for the block-tridiagonal SPD solver.

This module only *draws* problems; it holds none of the solver's arithmetic
(no factorisation, no solve, no Schur complement).  Both the CUDA path's tests
and benchmark and the CPU oracle's tests take their inputs from here.

Layout of every problem (the operator of Eq. 1, Sec. 1):
  A_diag : (N, n, n) float64, A_diag[i] = A_{i+1,i+1} in the paper's 1-based
           numbering (row-major; the solver uses sym(A_diag[i])).
  A_sub  : (N-1, n, n) float64, A_sub[i] = A_{i+2,i+1}, the block *below* the
           diagonal; the block above it is its transpose.
  B      : (N, n, d) float64, i.e. the (N*n) x d right-hand side, row-major.

Generators:
  kalman_btd     -- the Kalman-smoother normal equations of Sec. 4.2 (Eq. 6 and
                    the block formulas after it), time-invariant F, H, Q, R.
  mpc_batch_shapes -- (N_k, n_k) of the 512-instance uneven batch.
  random_btd     -- per-block random SPD systems (every block distinct), used by
                    the parity tests so that an indexing mistake cannot hide
                    behind repeated blocks.
  tridiag_121    -- n = 1, A = tridiag(-1, 2, -1), B = 1.
  laplace_btd    -- block 1-D Laplacian with PSD block perturbations sharing a
                    null vector: kappa(A) ~ N^2, beyond plain FP32 refinement.
  kalman_model   -- a time-varying state-space model (G_k, H_k, Q_k^-1, R_k^-1,
                    z_k, zeta_k), the input of the on-device assembly of the
                    Kalman-smoother normal equations.
  kalman_neuro_model -- the same inputs shaped like the neuroscience instance of
                    Sec. 4.2 (damped-rotation G, tall H, dense Q, diagonal R).
"""
from __future__ import annotations

import math

import numpy as np

# Named workloads.  Sizes follow the Kalman-smoother recipe: F = rho * Haar
# orthogonal, H Gaussian / sqrt(n), Q = 0.1 I, R = 0.5 I, P0 = I.
WORKLOADS = {
    # small plain FP64 solve
    "kalman-N64-n8-d1": dict(N=64, n=8, m=4, d=1, rho=0.95, seed=0),
    # the fused persistent FP64 path (roofline and level-fusion benchmark)
    "kalman-N16384-n64-d4": dict(N=16384, n=64, m=32, d=4, rho=0.95, seed=0),
    # mixed precision with refinement, kappa(A) pushed towards 1e5
    "kalman-N4096-n256-d16-rho0.99": dict(N=4096, n=256, m=128, d=16, rho=0.99, seed=0),
    # differentiation (forward + adjoint backward); W drawn after B
    "kalman-N2048-n32-d8-grad": dict(N=2048, n=32, m=16, d=8, rho=0.95, seed=0),
}

# The uneven batch: 512 condensed-MPC-like systems.
MPC_BATCH = dict(K=512, N_lo=32, N_hi=2048, n_choices=(12, 24, 48), d=1, rho=0.95, seed=0)


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a standard Gaussian with the
    sign of diag(R) folded into Q (Mezzadri 2007)."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def kalman_blocks(n: int, m: int, rho: float, rng: np.random.Generator):
    """The distinct blocks of the time-invariant Kalman-smoother Hessian.

    Sec. 4.2: A_kk = Q^-1 + G_{k+1}^T Q^-1 G_{k+1} + H^T R^-1 H,
    A_{k+1,k} = -Q^-1 G_{k+1}, G_{N+1} = 0; the first block carries the prior
    P0^-1 in place of Q^-1.  Returns (first, middle, last, only, sub) where
    `only` is the single block of an N = 1 system.
    """
    F = rho * haar_orthogonal(rng, n)
    H = rng.standard_normal((m, n)) / math.sqrt(n)
    Qinv = 10.0 * np.eye(n)          # Q = 0.1 I
    Rinv = 2.0 * np.eye(m)           # R = 0.5 I (m x m)
    P0inv = np.eye(n)                # P0 = I
    HtRH = H.T @ Rinv @ H
    FtQF = F.T @ Qinv @ F
    first = P0inv + HtRH + FtQF
    middle = Qinv + HtRH + FtQF
    last = Qinv + HtRH
    only = P0inv + HtRH
    sub = -(Qinv @ F)
    return first, middle, last, only, sub


def kalman_btd(N: int, n: int, m: int, d: int, rho: float, seed: int, with_W: bool = False):
    """One Kalman-smoother system.  Draw order: the Haar Gaussian, then H,
    then B, then (optionally) W, all from numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    first, middle, last, only, sub = kalman_blocks(n, m, rho, rng)
    A_diag = np.empty((N, n, n), dtype=np.float64)
    if N == 1:
        A_diag[0] = only
    else:
        A_diag[:] = middle
        A_diag[0] = first
        A_diag[N - 1] = last
    A_sub = np.empty((max(N - 1, 0), n, n), dtype=np.float64)
    A_sub[:] = sub
    B = rng.standard_normal((N * n, d)).reshape(N, n, d)
    out = dict(A_diag=A_diag, A_sub=A_sub, B=np.ascontiguousarray(B))
    if with_W:
        out["W"] = rng.standard_normal((N * n, d)).reshape(N, n, d)
    return out


def kalman_model(N: int, n: int, m: int, seed: int, g_scale: float = 0.5):
    """Per-step model with every block distinct, drawn from
    numpy.random.default_rng(seed) in the order G, H, M_Q, M_R, z, zeta:
    G_k = g_scale * Gaussian / sqrt(n), H_k = Gaussian / sqrt(n),
    Qinv_k = M_Q M_Q^T / n + I, Rinv_k = M_R M_R^T / m + I, z_k and zeta_k
    standard Gaussian.  Returns a dict of C-contiguous float64 arrays with the
    shapes G, Qinv (N, n, n), H (N, m, n), Rinv (N, m, m), z (N, m),
    zeta (N, n)."""
    rng = np.random.default_rng(seed)
    G = g_scale * rng.standard_normal((N, n, n)) / math.sqrt(n)
    H = rng.standard_normal((N, m, n)) / math.sqrt(n)
    Mq = rng.standard_normal((N, n, n))
    Mr = rng.standard_normal((N, m, m))
    z = rng.standard_normal((N, m))
    zeta = rng.standard_normal((N, n))
    Qinv = np.matmul(Mq, Mq.transpose(0, 2, 1)) / n + np.eye(n)
    Rinv = np.matmul(Mr, Mr.transpose(0, 2, 1)) / m + np.eye(m)
    return dict(G=G, H=H, Qinv=np.ascontiguousarray(Qinv), Rinv=np.ascontiguousarray(Rinv), z=z, zeta=zeta)


def kalman_neuro_model(N: int = 100, n: int = 256, m: int = 1024, seed: int = 0):
    """Synthetic stand-in for the neuroscience instance of Sec. 4.2, whose
    data, damping and covariances are not given.  Drawn from
    numpy.random.default_rng(seed) in the order rho, theta, H, M, x0, z:
      G_k = G for k >= 1: block diagonal of n/2 damped 2-D rotations
            rho_i [[cos t_i, -sin t_i], [sin t_i, cos t_i]],
            rho_i ~ U(0.95, 0.999), t_i ~ U(0, pi/4); G_0 = I;
      H_k = H: Gaussian / sqrt(m), m x n with m >= n (well conditioned);
      Q = 0.05 (M M^T / n + I), dense SPD, Qinv = Q^-1 for every step;
      R = I (diagonal, larger than Q): Rinv given as its diagonal, (N, m);
      zeta_0 = G_0 x0 = x0 (the known initial state), zeta_k = 0 after it;
      z_k standard Gaussian.
    Returns the arrays of kalman_model, Rinv of shape (N, m)."""
    if n % 2:
        raise ValueError("n must be even (2-D rotations)")
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.95, 0.999, n // 2)
    theta = rng.uniform(0.0, math.pi / 4, n // 2)
    Hm = rng.standard_normal((m, n)) / math.sqrt(m)
    M = rng.standard_normal((n, n))
    x0 = rng.standard_normal(n)
    z = rng.standard_normal((N, m))
    Gm = np.zeros((n, n))
    for i in range(n // 2):
        c, s_ = math.cos(theta[i]), math.sin(theta[i])
        Gm[2 * i:2 * i + 2, 2 * i:2 * i + 2] = rho[i] * np.array([[c, -s_], [s_, c]])
    Qinv1 = np.linalg.inv(0.05 * (M @ M.T / n + np.eye(n)))
    Qinv1 = 0.5 * (Qinv1 + Qinv1.T)
    G = np.empty((N, n, n))
    G[:] = Gm
    G[0] = np.eye(n)
    H = np.ascontiguousarray(np.broadcast_to(Hm, (N, m, n)))
    Qinv = np.ascontiguousarray(np.broadcast_to(Qinv1, (N, n, n)))
    Rinv = np.ones((N, m))
    zeta = np.zeros((N, n))
    zeta[0] = x0
    return dict(G=G, H=H, Qinv=Qinv, Rinv=Rinv, z=z, zeta=zeta)


def workload(name: str, with_W: bool = False):
    cfg = WORKLOADS[name]
    return kalman_btd(cfg["N"], cfg["n"], cfg["m"], cfg["d"], cfg["rho"], cfg["seed"], with_W=with_W)


def mpc_batch_shapes(K: int = 512, N_lo: int = 32, N_hi: int = 2048, n_choices=(12, 24, 48), seed: int = 0):
    """(N_k, n_k) for the uneven batch: a master default_rng(seed) draws
    N_k = floor(exp(U(ln N_lo, ln N_hi))) and n_k uniformly from n_choices,
    for k = 0..K-1 (N first, then n, per instance)."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(K):
        Nk = int(math.floor(math.exp(rng.uniform(math.log(N_lo), math.log(N_hi)))))
        nk = int(n_choices[int(rng.integers(0, len(n_choices)))])
        shapes.append((max(Nk, 1), nk))
    return shapes


def mpc_batch(K: int = 512, d: int = 1, rho: float = 0.95, seed: int = 0, **kw):
    """The batch: instance k is a Kalman system with seed k, m = n_k / 2."""
    shapes = mpc_batch_shapes(K=K, seed=seed, **kw)
    return [kalman_btd(Nk, nk, max(nk // 2, 1), d, rho, k) for k, (Nk, nk) in enumerate(shapes)]


def random_btd(N: int, n: int, d: int, seed: int, coupling: float = 1.0):
    """Per-block random SPD block-tridiagonal system.

    A_sub[i] ~ coupling * Gaussian / sqrt(n); A_diag[i] = M M^T / n + s_i I with
    s_i = ||A_{i,i-1}||_2 + ||A_{i,i+1}||_2 + 1, which makes A block diagonally
    dominant in the 2-norm and hence SPD.  A_diag is returned slightly
    non-symmetric on purpose (a skew part of size 1e-3) so that the sym(.)
    reading of the diagonal blocks is exercised.
    """
    rng = np.random.default_rng(seed)
    A_sub = coupling * rng.standard_normal((max(N - 1, 0), n, n)) / math.sqrt(n)
    norms = np.array([np.linalg.norm(A_sub[i], 2) for i in range(N - 1)]) if N > 1 else np.zeros(0)
    A_diag = np.empty((N, n, n))
    for i in range(N):
        M = rng.standard_normal((n, n))
        s = 1.0 + (norms[i - 1] if i > 0 else 0.0) + (norms[i] if i < N - 1 else 0.0)
        skew = rng.standard_normal((n, n)) * 1e-3
        A_diag[i] = M @ M.T / n + s * np.eye(n) + (skew - skew.T)
    B = rng.standard_normal((N, n, d))
    return dict(A_diag=A_diag, A_sub=A_sub, B=B)


def laplace_btd(N: int, n: int, d: int, seed: int):
    """Ill-conditioned SPD system: a 1-D Laplacian coupling of blocks,
    A_{i+1,i} = -I, A_ii = 2 I + S_i with S_i = P M_i M_i^T P / (2n) and
    P = I - v v^T for one random unit vector v, so every S_i is PSD with v in
    its null space.  On span{v} (x) R^N the matrix is tridiag(-1, 2, -1)
    exactly, with smallest eigenvalue 4 sin^2(pi / (2 (N + 1))), and
    kappa(A) ~ 0.6 N^2 (about 6e8 at N = 32768).  Drawn from
    numpy.random.default_rng(seed) in the order v, M (N, n, n), B (N n, d)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    Pv = np.eye(n) - np.outer(v, v)
    M = rng.standard_normal((N, n, n))
    PM = np.matmul(Pv, M)
    A_diag = 2.0 * np.eye(n) + np.matmul(PM, PM.transpose(0, 2, 1)) / (2 * n)
    A_sub = np.empty((max(N - 1, 0), n, n))
    A_sub[:] = -np.eye(n)
    B = rng.standard_normal((N * n, d)).reshape(N, n, d)
    return dict(A_diag=A_diag, A_sub=A_sub, B=np.ascontiguousarray(B))


def illcond_btd(N: int, n: int, d: int, seed: int, kappa: float = 1e9):
    """SPD system with condition number about kappa whose FP32 Cholesky
    fails: every diagonal block is Q diag(lambda) Q^T with lambda spaced
    log-uniformly from 1 down to 1/kappa (Q Haar), and A_{i+1,i} has 2-norm
    1/(4 kappa), so the couplings move no eigenvalue by more than half of the
    smallest.  Drawn from numpy.random.default_rng(seed) in the order Q (per
    block), the couplings, B."""
    rng = np.random.default_rng(seed)
    lam = np.logspace(0.0, -math.log10(kappa), n)
    A_diag = np.empty((N, n, n))
    for i in range(N):
        Q = haar_orthogonal(rng, n)
        A_diag[i] = (Q * lam) @ Q.T
        A_diag[i] = 0.5 * (A_diag[i] + A_diag[i].T)
    A_sub = np.empty((max(N - 1, 0), n, n))
    for i in range(N - 1):
        G = rng.standard_normal((n, n))
        A_sub[i] = G * (0.25 / kappa / np.linalg.norm(G, 2))
    B = rng.standard_normal((N, n, d))
    return dict(A_diag=A_diag, A_sub=A_sub, B=B)


def tridiag_121(N: int, d: int = 1):
    """n = 1: A = tridiag(-1, 2, -1), B = all ones."""
    return dict(A_diag=np.full((N, 1, 1), 2.0), A_sub=np.full((max(N - 1, 0), 1, 1), -1.0),
                B=np.ones((N, 1, d)))
