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
