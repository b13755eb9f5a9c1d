"""Host-side accounting of the cyclic-reduction schedule: level sizes and the
flops the kernels execute (counting a fused multiply-add as two flops), for
roofline reporting.  Pure integer/float bookkeeping; no solver arithmetic."""
from __future__ import annotations


def levels(N: int):
    """N_l for l = 0..L (N_0 = N, N_{l+1} = ceil(N_l / 2), N_L = 1)."""
    out = [int(N)]
    while out[-1] > 1:
        out.append((out[-1] + 1) // 2)
    return out


def chol_flops(n: int) -> float:
    return n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0


def cr_flops(N: int, n: int, d: int):
    """Flops executed by odd-even cyclic reduction: dict(factor=..., solve=...).

    Per eliminated block: Cholesky, one forward substitution per coupling
    (n^3 each).  Per separator: one symmetric update per eliminated neighbour
    (n^2 (n+1)) and the new coupling (2 n^3) when it exists.  RHS: forward
    substitution (n^2 d), W^T y per neighbour (2 n^2 d), the top solve
    (2 n^2 d), back-substitution n^2 d + 2 n^2 d per coupling."""
    fac = 0.0
    sol = 0.0
    Ns = levels(N)
    for Nl in Ns[:-1]:
        for j in range(1, Nl, 2):
            ncoup = 1 + (1 if j + 1 < Nl else 0)
            fac += chol_flops(n) + ncoup * n ** 3
            sol += n * n * d + ncoup * 2 * n * n * d       # up: y_j; down: couplings
            sol += n * n * d                                # down: L^-T
        for s in range(0, Nl, 2):
            nb = (1 if s >= 2 else 0) + (1 if s + 1 < Nl else 0)
            fac += nb * n * n * (n + 1)
            if s + 2 < Nl:
                fac += 2 * n ** 3
            sol += nb * 2 * n * n * d
    fac += chol_flops(n)
    sol += 2 * n * n * d
    return dict(factor=fac, solve=sol)


def thomas_flops(N: int, n: int, d: int):
    """Block-Thomas flop tally (the oracle's): per block Cholesky, per coupling
    trsm n^3 and symmetric update n^2 (n+1); solve 2 n^2 d per block and
    4 n^2 d per coupling."""
    fac = N * chol_flops(n) + (N - 1) * (n ** 3 + n * n * (n + 1))
    sol = N * 2.0 * n * n * d + (N - 1) * 4.0 * n * n * d
    return dict(factor=fac, solve=sol)


def tc_tile_flops(N: int, n: int) -> float:
    """Flops of the Schur-update products (Algorithm 3, Eq. 5) that the TF32
    mode of the tiled path runs on the tensor cores, summed over the levels:
    per separator one symmetric product n^2 (n+1) per eliminated neighbour and
    the new coupling 2 n^3 when it exists (the separator part of cr_flops)."""
    fl = 0.0
    for Nl in levels(N)[:-1]:
        for s in range(0, Nl, 2):
            nb = (1 if s >= 2 else 0) + (1 if s + 1 < Nl else 0)
            fl += nb * n * n * (n + 1) + (2 * n ** 3 if s + 2 < Nl else 0)
    return fl
