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


def emu_schur_mma_flops(N: int, n: int) -> float:
    """BF16 tensor-core flops the FP64 tiled factorisation executes for its
    Schur products with the digit-slice engine: per separator, 128 x 16
    output tiles of D's lower part (one accumulation round per eliminated
    neighbour) and of the new coupling E (one round); a round is ten
    128 x 160 x np products (np = n rounded up to 64), one per A slice."""
    MT, CT, np_ = -(-n // 128), -(-n // 16), -(-n // 64) * 64
    d_tiles = sum(min(CT, (mt + 1) * 8) for mt in range(MT))
    per_round = 2.0 * 10 * 128 * 160 * np_
    rounds = 0
    for Nl in levels(N)[:-1]:
        for s in range(0, Nl, 2):
            rounds += d_tiles * ((1 if s >= 2 else 0) + (1 if s + 1 < Nl else 0))
            rounds += MT * CT * (1 if s + 2 < Nl else 0)
    return rounds * per_round


def emu_wslice_bytes(N: int, n: int) -> float:
    """HBM bytes of the coupling-block slicing over the levels: each stored
    n x n FP64 block read once, its ten BF16 digit planes (n x np) written."""
    np_ = -(-n // 64) * 64
    blocks = sum(Nl - 1 for Nl in levels(N)[:-1])
    return blocks * (8.0 * n * n + 20.0 * n * np_)


def segment_levels(N: int, J: int, n_star: int = 1):
    """Level sizes of the recursion with interior segments of J blocks
    (Sec. 3.1, Eq. 2-4): at a level of N_l blocks the separators sit at
    positions 0, J+1, 2(J+1), ..., so N_{l+1} = ceil(N_l / (J+1)); the
    recursion stops once N_l <= n_star (Sec. 3.3's crossover N_*), where the
    remaining system is factored by the serial sweep."""
    out = [int(N)]
    while out[-1] > max(1, int(n_star)):
        out.append(-(-out[-1] // (J + 1)))
    return out


def segment_flops(N: int, n: int, d: int, J: int, n_star: int = 1):
    """Flops of the recursive Schur-complement method with segments of J
    interior blocks (Algorithms 1-3 for the factor, 5-7 for the solve), with
    the same per-routine counts as cr_flops: Cholesky chol_flops(n), a
    triangular solve with n columns n^3, a symmetric update n^2 (n+1), a
    product of n x n blocks 2 n^3, and 2 n^2 (triangular: n^2) per n x d
    block product.  Per segment of J' interior blocks between a left
    separator and, unless it is the trailing segment, a right separator:
      interior sweep   J' chol + (J'-1) (trsm + syrk)            (Alg. 1, K = 1)
      left coupling    F_L = L^{-1} [A_{first,sL}; 0; ...]: it fills every
                       interior block: trsm, then (J'-1) (gemm + trsm)
      right coupling   F_R touches the last interior block only: trsm
      Schur updates    S_LL -= F_L^T F_L (J' syrk), S_RR -= F_R^T F_R (syrk),
                       new coupling S_RL = -F_R^T F_L,last (gemm)  (Alg. 3, Eq. 5)
    The level whose size is <= n_star is factored by the serial sweep
    (block-Thomas, thomas_flops).  With J = 1 this is odd-even cyclic
    reduction and equals cr_flops; with n_star >= N it is block-Thomas."""
    c, t3, sy, g3 = chol_flops(n), float(n) ** 3, float(n * n * (n + 1)), 2.0 * n ** 3
    v1, v2 = float(n * n * d), 2.0 * n * n * d
    fac = sol = 0.0
    sizes = segment_levels(N, J, n_star)
    for Nl in sizes[:-1]:
        seps = list(range(0, Nl, J + 1))
        for k, s in enumerate(seps):
            last = seps[k + 1] if k + 1 < len(seps) else Nl
            Jp = last - s - 1                    # interior blocks after separator s
            if Jp <= 0:
                continue
            has_r = k + 1 < len(seps)
            fac += Jp * c + (Jp - 1) * (t3 + sy)            # interior sweep
            fac += t3 + (Jp - 1) * (g3 + t3)                # F_L with fill
            fac += Jp * sy                                  # S_LL update
            if has_r:
                fac += t3 + sy + g3                         # F_R, S_RR, S_RL
            # solve: forward sweep of the interior RHS, separator updates,
            # then z = y - F_L x_L - F_R x_R and the backward sweep
            sol += Jp * v1 + (Jp - 1) * v2
            sol += Jp * v2 + (v2 if has_r else 0.0)
            sol += Jp * v2 + (v2 if has_r else 0.0)
            sol += Jp * v1 + (Jp - 1) * v2
    t = thomas_flops(sizes[-1], n, d)
    return dict(factor=fac + t["factor"], solve=sol + t["solve"])
