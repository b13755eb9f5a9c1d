"""Partitioned solve of one SPD block-tridiagonal system over G ranks.

The separator / interior partition of Sec. 3.1 (Eq. 2-4), applied once at
the top level: the N blocks are cut into G contiguous chunks and the last
block of every chunk but the last is a separator.  Rank g eliminates the
interior of its chunk (its blocks between the left and right separators) and
contributes, for Eq. 5 with that interior as A_uu,

    S_LL = A_left^T (A_I^-1)_{first,first} A_left     (to its left separator)
    S_RR = A_right (A_I^-1)_{last,last} A_right^T     (to its right separator)
    S_RL = A_right (A_I^-1)_{last,first} A_left       (their new coupling)
    b_L  = A_left^T (A_I^-1 B_I)_first,   b_R = A_right (A_I^-1 B_I)_last

together with its separator's own diagonal block and right-hand side.  One
all-gather exchanges these (4 n^2 + 3 n d numbers per rank); every rank
assembles the reduced system of the G - 1 separators,

    D_g = A_{s_g s_g} - S_RR(g) - S_LL(g + 1),   E_g = -S_RL(g + 1),
    b_g = B_{s_g} - b_R(g) - b_L(g + 1),

solves it redundantly, and back-solves its interior
X_I = A_I^-1 (B_I - E_first A_left x_left - E_last A_right^T x_right).

The elimination, back-solve and reduced solve are passed in (on a GPU: the
library's bdss_chunk_reduce / bdss_chunk_backsolve and a solver of the
reduced system), and so is the all-gather (torch.distributed, or a list when
one process plays every rank in turn).  This module holds the partition and
the exchange only.
"""
from __future__ import annotations

import numpy as np


def chunk_bounds(N: int, G: int):
    """[(start, end)] of G contiguous chunks covering 0..N-1.  Every chunk but
    the last holds at least two blocks (an interior block and its separator
    end - 1); the last at least one.  Needs N >= 2 G - 1."""
    if G < 1 or N < 2 * G - 1:
        raise ValueError(f"cannot cut N = {N} blocks into {G} chunks with separators")
    sizes = [2] * (G - 1) + [1]
    extra = N - (2 * G - 1)
    for g in range(G):
        sizes[g] += extra // G + (1 if g < extra % G else 0)
    out, s = [], 0
    for sz in sizes:
        out.append((s, s + sz))
        s += sz
    return out


def chunk_layout(N: int, G: int, g: int):
    """Interior range, left separator, right separator of chunk g
    (separators are None where absent)."""
    start, end = chunk_bounds(N, G)[g]
    right = end - 1 if g < G - 1 else None
    interior = (start, end - 1) if right is not None else (start, end)
    left = start - 1 if g > 0 else None
    return interior, left, right


def _pack(n, d, S, bh, D, b):
    """One rank's message: S (3, n, n), b_hat (2, n, d), its separator's
    diagonal block D (n, n) and right-hand side b (n, d) (zeros if none)."""
    return np.concatenate([np.asarray(S, dtype=np.float64).ravel(), np.asarray(bh, dtype=np.float64).ravel(),
                           np.asarray(D, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()])


def _unpack(msg, n, d):
    o = 0
    S = msg[o:o + 3 * n * n].reshape(3, n, n)
    o += 3 * n * n
    bh = msg[o:o + 2 * n * d].reshape(2, n, d)
    o += 2 * n * d
    D = msg[o:o + n * n].reshape(n, n)
    o += n * n
    b = msg[o:o + n * d].reshape(n, d)
    return S, bh, D, b


def reduced_system(msgs, n, d):
    """Assemble the block-tridiagonal reduced system of the G - 1 separators
    (Eq. 5 per interior, summed) from the G gathered messages: returns
    (D (G-1, n, n), E (G-2, n, n), b (G-1, n, d))."""
    G = len(msgs)
    parts = [_unpack(m, n, d) for m in msgs]
    D = np.empty((G - 1, n, n))
    E = np.empty((max(G - 2, 0), n, n))
    b = np.empty((G - 1, n, d))
    for g in range(G - 1):
        S_g, bh_g, Dg, bg = parts[g]
        S_n, bh_n, _, _ = parts[g + 1]
        D[g] = Dg - S_g[1] - S_n[0]
        b[g] = bg - bh_g[1] - bh_n[0]
        if g + 1 < G - 1:
            E[g] = -parts[g + 1][0][2]
    return D, E, b


def chunk_message(A_diag, A_sub, B, G, rank, eliminate):
    """Phase 1 of rank `rank`: eliminate its chunk interior and return the
    message it contributes to the exchange (4 n^2 + 3 n d numbers)."""
    A_diag, A_sub, B = np.asarray(A_diag), np.asarray(A_sub), np.asarray(B)
    N, n, _ = A_diag.shape
    d = B.shape[-1]
    (i0, i1), left, right = chunk_layout(N, G, rank)
    A_left = A_sub[i0 - 1] if left is not None else None
    A_right = A_sub[i1 - 1] if right is not None else None
    S, bh = eliminate(A_diag[i0:i1], A_sub[i0:i1 - 1], A_left, A_right, B[i0:i1])
    D = A_diag[right] if right is not None else np.zeros((n, n))
    bs = B[right] if right is not None else np.zeros((n, d))
    return _pack(n, d, S, bh, D, bs)


def chunk_finish(A_sub, B, G, rank, msgs, backsolve, reduced_solve):
    """Phase 2 of rank `rank`, given every rank's message: solve the reduced
    system of the separators (redundantly on every rank) and back-solve the
    chunk.  Returns ((start, end), X of the chunk's blocks)."""
    A_sub, B = np.asarray(A_sub), np.asarray(B)
    N, n, d = B.shape
    (i0, i1), left, right = chunk_layout(N, G, rank)
    A_left = A_sub[i0 - 1] if left is not None else None
    A_right = A_sub[i1 - 1] if right is not None else None
    if G > 1:
        Dr, Er, br = reduced_system(msgs, n, d)
        xs = np.asarray(reduced_solve(Dr, Er, br))
    else:
        xs = np.zeros((0, n, d))
    x_left = xs[rank - 1] if left is not None else None
    x_right = xs[rank] if right is not None else None
    X_I = np.asarray(backsolve(B[i0:i1], A_left, A_right, x_left, x_right))
    start, end = chunk_bounds(N, G)[rank]
    X = np.empty((end - start, n, d))
    X[:i1 - i0] = X_I
    if right is not None:
        X[-1] = x_right
    return (start, end), X


def partitioned_solve(A_diag, A_sub, B, G, rank, eliminate, backsolve, reduced_solve, allgather):
    """This rank's share of the partitioned solve: eliminate, one all-gather,
    reduced solve, back-solve.  Returns ((start, end), X_chunk): the solution
    of its chunk's blocks (interior and its separator).

    eliminate(A_diag_I, A_sub_I, A_left, A_right, B_I) -> (S, b_hat);
    backsolve(B_I, A_left, A_right, x_left, x_right) -> X_I;
    reduced_solve(D, E, b) -> x (G-1, n, d);  allgather(msg) -> [msg of rank 0..G-1].
    Arrays are numpy (host); A_left / A_right are None where absent."""
    msg = chunk_message(A_diag, A_sub, B, G, rank, eliminate)
    return chunk_finish(A_sub, B, G, rank, allgather(msg), backsolve, reduced_solve)


def torch_allgather(group=None):
    """All-gather of one float64 message per rank over torch.distributed
    (gloo: host tensors; NCCL: the caller's current CUDA device)."""
    import torch
    import torch.distributed as dist

    def gather(msg):
        backend = dist.get_backend(group)
        dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
        t = torch.from_numpy(np.ascontiguousarray(msg)).to(dev)
        out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
        dist.all_gather(out, t, group=group)
        return [o.cpu().numpy() for o in out]
    return gather


def gpu_chunk_ops(n, d, stream=None):
    """eliminate / backsolve / reduced_solve through the library (FP64) on
    the current GPU; one handle per call of eliminate, kept for the
    back-solve that follows it."""
    import torch

    from .solver import Solver
    state = {}

    def dev(a):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda")

    def eliminate(Ad, As, A_left, A_right, B_I):
        Ni = Ad.shape[0]
        if "solver" in state:
            state["solver"].close()
        sol = Solver(Ni, n, d_max=max(d, min(n, 64)), stream=stream)
        state["solver"] = sol
        state["blocks"] = (dev(Ad), dev(As if Ni > 1 else np.zeros((1, n, n))), dev(A_left), dev(A_right))
        S, bh = sol.chunk_reduce(state["blocks"][0], state["blocks"][1], state["blocks"][2], state["blocks"][3],
                                 dev(B_I))
        return S.cpu().numpy(), bh.cpu().numpy()

    def backsolve(B_I, A_left, A_right, x_left, x_right):
        sol = state["solver"]
        X = sol.chunk_backsolve(dev(B_I), state["blocks"][2], state["blocks"][3], dev(x_left), dev(x_right))
        out = X.cpu().numpy()
        sol.close()
        del state["solver"]
        return out

    def reduced_solve(D, E, b):
        Gm = D.shape[0]
        sol = Solver(Gm, n, d_max=d, stream=stream)
        X = sol.factor_solve(dev(D), dev(E if Gm > 1 else np.zeros((1, n, n))), dev(b))
        out = X.cpu().numpy()
        sol.close()
        return out
    return eliminate, backsolve, reduced_solve
