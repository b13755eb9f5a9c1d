"""CPU FP64 oracle for SPD block-tridiagonal solves -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg may import this package.  The CUDA path never
imports it and shares no code with it.

What it computes (all FP64, on the host):
  factor / solve   block-Thomas = Algorithm 1 + Algorithm 2 with one segment
                   (K = 1, J = N), the serial base case of Algorithms 4 and 7.
  logdet           2 * sum log diag(L_j).
  residual         R = B - A X with compensated (Dot2) accumulation.
  backward_error   ||B - A X||_inf / (||A||_inf ||X||_inf).
  adjoint_grads    dL/dA_ii = -sym(Lam_i X_i^T),
                   dL/dA_{i+1,i} = -(Lam_{i+1} X_i^T + X_{i+1} Lam_i^T).
  schur_partition  the separator/interior permutation of Sec. 3.1 (Eq. 2-4)
                   and the reduced system of Eq. 5, densely (numpy).
  tally            flop counts of the block-Thomas sweep.
  kalman_assemble  the Kalman-smoother Hessian blocks and right-hand side of
                   Sec. 4.2 from (G_k, H_k, Q_k^{-1}, R_k^{-1}, z_k, zeta_k).

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself: dense LAPACK Cholesky on tiny inputs, the closed form of
tridiag(-1,2,-1), N = 1 plain Cholesky, block-diagonal A, exact rational
arithmetic, manufactured solutions, finite differences, and the printed
structure of the N = 9 example of Eq. 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdss_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP for the batched CPU baseline)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32 = ctypes.c_int64, ctypes.c_int
        lib.oracle_factor.argtypes = [i64, i32, _dp, _dp, _dp, _dp]
        lib.oracle_factor.restype = i32
        lib.oracle_solve.argtypes = [i64, i32, i32, _dp, _dp, _dp, _dp]
        lib.oracle_solve.restype = None
        lib.oracle_logdet.argtypes = [i64, i32, _dp]
        lib.oracle_logdet.restype = ctypes.c_double
        lib.oracle_residual.argtypes = [i64, i32, i32, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_residual.restype = None
        lib.oracle_norm_inf_A.argtypes = [i64, i32, _dp, _dp]
        lib.oracle_norm_inf_A.restype = ctypes.c_double
        lib.oracle_adjoint_grads.argtypes = [i64, i32, i32, _dp, _dp, _dp, _dp]
        lib.oracle_adjoint_grads.restype = None
        lib.oracle_tally.argtypes = [i64, i32, i32, _dp]
        lib.oracle_tally.restype = None
        pp = ctypes.POINTER(_dp)
        lib.oracle_factor_solve_batched.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(i32), i32,
                                                    pp, pp, pp, pp, ctypes.POINTER(i32)]
        lib.oracle_factor_solve_batched.restype = None
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = i32
        _lib = lib
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _sub_ptr(A_sub, n):
    # a valid pointer even when N == 1 (no sub-diagonal blocks)
    if A_sub.size == 0:
        A_sub = np.zeros((1, n, n))
    return _c(A_sub)


class NotSPDError(RuntimeError):
    def __init__(self, block):
        super().__init__(f"block {block}: Cholesky pivot not positive/finite")
        self.block = block


def factor(A_diag, A_sub):
    """Block-Thomas factor (Algorithm 1, K = 1).  Returns (L, C): L (N,n,n)
    lower-triangular diagonal factors, C (N-1,n,n) sub-diagonal factors."""
    lib = _load()
    A_diag, pd = _c(A_diag)
    N, n, _ = A_diag.shape
    A_sub, ps = _sub_ptr(np.asarray(A_sub), n)
    L = np.zeros((N, n, n))
    C = np.zeros((max(N - 1, 1), n, n))
    rc = lib.oracle_factor(N, n, pd, ps, L.ctypes.data_as(_dp), C.ctypes.data_as(_dp))
    if rc != 0:
        raise NotSPDError(rc - 1)
    return L, C[: N - 1]


def solve(L, C, B):
    """Block forward/backward substitution (Algorithm 2, K = 1)."""
    lib = _load()
    L, pl = _c(L)
    N, n, _ = L.shape
    C, pc = _sub_ptr(np.asarray(C), n)
    B, pb = _c(B)
    d = B.shape[-1]
    X = np.empty_like(B)
    lib.oracle_solve(N, n, d, pl, pc, pb, X.ctypes.data_as(_dp))
    return X


def solve_system(A_diag, A_sub, B):
    L, C = factor(A_diag, A_sub)
    return solve(L, C, B)


def logdet(L):
    lib = _load()
    L, pl = _c(L)
    return lib.oracle_logdet(L.shape[0], L.shape[1], pl)


def residual(A_diag, A_sub, X, B):
    """R = B - A X, compensated (Dot2) accumulation."""
    lib = _load()
    A_diag, pd = _c(A_diag)
    N, n, _ = A_diag.shape
    A_sub, ps = _sub_ptr(np.asarray(A_sub), n)
    X, px = _c(X)
    B, pb = _c(B)
    R = np.empty_like(B)
    lib.oracle_residual(N, n, B.shape[-1], pd, ps, px, pb, R.ctypes.data_as(_dp))
    return R


def norm_inf_A(A_diag, A_sub):
    lib = _load()
    A_diag, pd = _c(A_diag)
    N, n, _ = A_diag.shape
    A_sub, ps = _sub_ptr(np.asarray(A_sub), n)
    return lib.oracle_norm_inf_A(N, n, pd, ps)


def norm_inf(X):
    """Max absolute row sum of the (N*n) x d matrix X."""
    X = np.asarray(X)
    return float(np.abs(X.reshape(-1, X.shape[-1])).sum(axis=1).max()) if X.size else 0.0


def backward_error(A_diag, A_sub, X, B):
    """||B - A X||_inf / (||A||_inf ||X||_inf), residual in compensated FP64."""
    R = residual(A_diag, A_sub, X, B)
    den = norm_inf_A(A_diag, A_sub) * norm_inf(X)
    return norm_inf(R) / den if den > 0 else norm_inf(R)


def forward_error(X, X_ref):
    """||X - X_ref||_inf / ||X_ref||_inf."""
    return norm_inf(np.asarray(X) - np.asarray(X_ref)) / max(norm_inf(X_ref), 1e-300)


def adjoint_grads(Lam, X):
    lib = _load()
    Lam, pl = _c(Lam)
    X, px = _c(X)
    N, n, d = X.shape
    dA_diag = np.empty((N, n, n))
    dA_sub = np.zeros((max(N - 1, 1), n, n))
    lib.oracle_adjoint_grads(N, n, d, pl, px, dA_diag.ctypes.data_as(_dp), dA_sub.ctypes.data_as(_dp))
    return dA_diag, dA_sub[: N - 1]


def tally(N, n, d):
    """Block-Thomas flop tally: dict(factor=..., solve=...)."""
    lib = _load()
    out = np.zeros(2)
    lib.oracle_tally(N, n, d, out.ctypes.data_as(_dp))
    return dict(factor=float(out[0]), solve=float(out[1]))


def factor_solve_batched(systems):
    """CPU baseline over independent systems, one per OpenMP thread.  Returns
    (list of X, number of threads)."""
    lib = _load()
    K = len(systems)
    keep = []
    Xs = []
    Nk = (ctypes.c_int64 * K)()
    nk = (ctypes.c_int * K)()
    pd, ps, pb, px = ((_dp * K)() for _ in range(4))
    for k, s in enumerate(systems):
        A_diag, p1 = _c(s["A_diag"])
        N, n, _ = A_diag.shape
        A_sub, p2 = _sub_ptr(np.asarray(s["A_sub"]), n)
        B, p3 = _c(s["B"])
        X = np.empty_like(B)
        keep += [A_diag, A_sub, B]
        Xs.append(X)
        Nk[k], nk[k] = N, n
        pd[k], ps[k], pb[k], px[k] = p1, p2, p3, X.ctypes.data_as(_dp)
    info = (ctypes.c_int * K)()
    d = systems[0]["B"].shape[-1]
    lib.oracle_factor_solve_batched(K, Nk, nk, d, pd, ps, pb, px, info)
    for k in range(K):
        if info[k] != 0:
            raise NotSPDError((k, info[k] - 1))
    return Xs, int(lib.oracle_num_threads())


# ---------------------------------------------------------------------------
# Sec. 3.1: separator / interior partition and the reduced system (Eq. 2-5),
# written densely with numpy.  Block indices here are 0-based.
# ---------------------------------------------------------------------------

def partition(N, separators):
    """Order of Eq. 2-3: interiors (ascending) first, then separators
    (ascending).  Returns (interiors, separators)."""
    seps = sorted(set(int(s) for s in separators))
    ints = [i for i in range(N) if i not in seps]
    return ints, seps


def dense_blocks(A_diag, A_sub):
    """Block (r, c) of A for the block-tridiagonal operator: sym(A_ii) on the
    diagonal, A_sub below, A_sub^T above, zero elsewhere (Eq. 1)."""
    N, n, _ = A_diag.shape

    def blk(r, c):
        if r == c:
            return 0.5 * (A_diag[r] + A_diag[r].T)
        if r == c + 1:
            return A_sub[c]
        if c == r + 1:
            return A_sub[r].T
        return np.zeros((n, n))
    return blk


def permuted_structure(N, separators):
    """Which original block (r, c) sits at each block position of the
    permuted matrix of Eq. 2, or None where the permuted matrix is zero."""
    ints, seps = partition(N, separators)
    order = ints + seps
    out = []
    for r in order:
        row = []
        for c in order:
            row.append((r, c) if abs(r - c) <= 1 else None)
        out.append(row)
    return out


def schur_partition(A_diag, A_sub, B, separators):
    """Eq. 5: S = A_ll - A_lu^T A_uu^{-1} A_lu and
    b_hat = B_l - A_lu^T A_uu^{-1} B_u, densely.  Returns (S, b_hat, A_uu,
    A_lu, A_ll) as dense numpy arrays in the order of `partition`."""
    N, n, _ = A_diag.shape
    ints, seps = partition(N, separators)
    blk = dense_blocks(A_diag, A_sub)

    def assemble(rows, cols):
        M = np.zeros((len(rows) * n, len(cols) * n))
        for a, r in enumerate(rows):
            for b, c in enumerate(cols):
                M[a * n:(a + 1) * n, b * n:(b + 1) * n] = blk(r, c)
        return M
    A_uu = assemble(ints, ints)
    A_lu = assemble(ints, seps)   # rows: interiors, cols: separators (Eq. 2)
    A_ll = assemble(seps, seps)
    Bf = np.asarray(B)
    B_u = np.concatenate([Bf[i] for i in ints]) if ints else np.zeros((0, Bf.shape[-1]))
    B_l = np.concatenate([Bf[i] for i in seps])
    if ints:
        F = np.linalg.solve(A_uu, A_lu)
        G = np.linalg.solve(A_uu, B_u)
        S = A_ll - A_lu.T @ F
        b_hat = B_l - A_lu.T @ G
    else:
        S, b_hat = A_ll, B_l
    return S, b_hat, A_uu, A_lu, A_ll


def kalman_assemble(G, H, Qinv, Rinv, z, zeta=None):
    """Normal equations of the MAP Kalman smoother (Sec. 4.2, "Kalman Smoothing
    Experiment"), blocks 0-based: step k has transition G[k] (G[0] enters only
    through zeta[0] = G_1 x_0), observation H[k], precisions Qinv[k], Rinv[k],
    measurement z[k].  With G_{N+1} = 0:
      A_kk      = Qinv[k] + G[k+1]^T Qinv[k+1] G[k+1] + H[k]^T Rinv[k] H[k]
      A_{k+1,k} = -Qinv[k+1] G[k+1]
      b_k       = H[k]^T Rinv[k] z[k] + Qinv[k] zeta[k] - G[k+1]^T Qinv[k+1] zeta[k+1]
    (the right-hand side read from G^T Q^{-1} zeta with G the block-bidiagonal
    state operator).  Rinv of shape (N, m) holds diagonal precisions (the
    neuroscience instance of Sec. 4.2 has a diagonal R).  Returns
    (A_diag, A_sub, B) with B of shape (N, n, 1)."""
    G, H, Qinv, Rinv, z = (np.asarray(a, dtype=np.float64) for a in (G, H, Qinv, Rinv, z))
    if Rinv.ndim == 2:
        Rinv = np.stack([np.diag(r) for r in Rinv])
    N, n = G.shape[0], G.shape[1]
    zeta = np.zeros((N, n)) if zeta is None else np.asarray(zeta, dtype=np.float64)
    A_diag = np.empty((N, n, n))
    A_sub = np.empty((max(N - 1, 0), n, n))
    B = np.empty((N, n, 1))
    for k in range(N):
        Akk = Qinv[k] + H[k].T @ Rinv[k] @ H[k]
        b = H[k].T @ (Rinv[k] @ z[k]) + Qinv[k] @ zeta[k]
        if k + 1 < N:
            Akk = Akk + G[k + 1].T @ Qinv[k + 1] @ G[k + 1]
            A_sub[k] = -(Qinv[k + 1] @ G[k + 1])
            b = b - G[k + 1].T @ (Qinv[k + 1] @ zeta[k + 1])
        A_diag[k] = Akk
        B[k, :, 0] = b
    return A_diag, A_sub, B
