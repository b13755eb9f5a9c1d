"""Test-side helpers written independently of both the oracle and the CUDA
path: dense assembly of the block-tridiagonal operator (Eq. 1) and exact
rational arithmetic for brute-force checks."""
from fractions import Fraction

import numpy as np


def dense_A(A_diag, A_sub):
    """Dense Nn x Nn operator of Eq. 1: sym(A_ii) on the diagonal, A_{i+1,i}
    below it and A_{i+1,i}^T above it."""
    A_diag = np.asarray(A_diag)
    N, n, _ = A_diag.shape
    A = np.zeros((N * n, N * n))
    for i in range(N):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = 0.5 * (A_diag[i] + A_diag[i].T)
    for i in range(N - 1):
        A[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = A_sub[i]
        A[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = np.asarray(A_sub[i]).T
    return A


def dense_B(B):
    B = np.asarray(B)
    return B.reshape(-1, B.shape[-1])


def to_frac(M):
    return [[Fraction(float(x)) for x in row] for row in np.asarray(M)]


def frac_solve(A, B):
    """Exact Gauss-Jordan elimination over the rationals: A X = B."""
    n = len(A)
    m = len(B[0])
    M = [list(A[i]) + list(B[i]) for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [x / piv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [row[n:] for row in M]


def frac_matmul(A, X):
    return [[sum(a * x for a, x in zip(row, col)) for col in zip(*X)] for row in A]


def assert_elementwise(X, X_ref, rtol, atol_frac):
    """Element by element: |X - X_ref| <= rtol |X_ref| + atol_frac max|X_ref|
    for every entry, so that no single entry can be far off while a norm of
    the difference stays small."""
    X = np.asarray(X)
    X_ref = np.asarray(X_ref)
    assert X.shape == X_ref.shape
    scale = float(np.abs(X_ref).max()) if X_ref.size else 0.0
    err = np.abs(X - X_ref)
    bound = rtol * np.abs(X_ref) + atol_frac * scale
    bad = err > bound
    if bad.any():
        i = np.unravel_index(int(np.argmax(err - bound)), err.shape)
        raise AssertionError(f"{int(bad.sum())} entries beyond tolerance; worst at {i}: got {X[i]!r}, "
                             f"expected {X_ref[i]!r} (|diff| {err[i]:.3e} > {bound[i]:.3e})")
