"""The benchmark's flop accounting against the oracle's tally and a direct
count of the cyclic-reduction schedule."""
import pytest

from paper_2509_03015_gb300 import accounting


@pytest.mark.parametrize("N,n,d", [(1, 1, 1), (2, 3, 1), (7, 5, 2), (64, 8, 1), (16384, 64, 4)])
def test_thomas_matches_oracle_tally(oracle_mod, N, n, d):
    t = oracle_mod.tally(N, n, d)
    a = accounting.thomas_flops(N, n, d)
    assert abs(a["factor"] - t["factor"]) <= 1e-12 * t["factor"]
    assert abs(a["solve"] - t["solve"]) <= 1e-12 * t["solve"]


def test_levels():
    assert accounting.levels(1) == [1]
    assert accounting.levels(2) == [2, 1]
    assert accounting.levels(9) == [9, 5, 3, 2, 1]
    assert accounting.levels(16384)[-2:] == [2, 1] and len(accounting.levels(16384)) == 15


def test_cr_flops_small_cases():
    n, d = 4, 2
    c = accounting.chol_flops(n)
    # N = 1: the top block only
    assert accounting.cr_flops(1, n, d) == dict(factor=c, solve=2 * n * n * d)
    # N = 2: block 1 eliminated with one coupling; separator 0 gets one update
    f = accounting.cr_flops(2, n, d)
    assert f["factor"] == c + n ** 3 + n * n * (n + 1) + c
    assert f["solve"] == (n * n * d + 2 * n * n * d + n * n * d) + 2 * n * n * d + 2 * n * n * d


def test_cr_over_thomas_ratio():
    # cyclic reduction executes ~ (n^3/3 + 6 n^3) / (n^3/3 + 2 n^3) = 2.7x the
    # block-Thomas factor flops for large N
    r = accounting.cr_flops(16384, 64, 4)["factor"] / accounting.thomas_flops(16384, 64, 4)["factor"]
    assert 2.6 < r < 2.75


@pytest.mark.parametrize("N,n", [(1, 4), (2, 3), (9, 5), (100, 7)])
def test_tc_tile_flops_is_the_separator_part_of_cr(N, n):
    """The tensor-core Schur products are cr_flops' factor count minus the
    eliminated blocks' Cholesky and coupling solves and the top Cholesky."""
    elim = sum(chol + (1 + (1 if j + 1 < Nl else 0)) * n ** 3
               for Nl in accounting.levels(N)[:-1] for j in range(1, Nl, 2)
               for chol in [accounting.chol_flops(n)])
    expect = accounting.cr_flops(N, n, 1)["factor"] - elim - accounting.chol_flops(n)
    assert abs(accounting.tc_tile_flops(N, n) - expect) <= 1e-9 * max(expect, 1.0)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 9, 33, 100, 1000, 16384])
@pytest.mark.parametrize("n,d", [(1, 1), (4, 2), (64, 4)])
def test_segment_flops_J1_is_cyclic_reduction(N, n, d):
    """Segments of one block with separators at the even positions are the
    odd-even cyclic reduction the kernels run: the two tallies agree."""
    a = accounting.segment_flops(N, n, d, J=1)
    b = accounting.cr_flops(N, n, d)
    assert a["factor"] == pytest.approx(b["factor"], rel=1e-12)
    assert a["solve"] == pytest.approx(b["solve"], rel=1e-12)


@pytest.mark.parametrize("N,n,d", [(1, 3, 1), (7, 5, 2), (100, 8, 1), (16384, 64, 4)])
def test_segment_flops_serial_crossover_is_block_thomas(N, n, d):
    """N <= N_*: no recursion, the serial sweep of Algorithm 1 with K = 1."""
    assert accounting.segment_flops(N, n, d, J=3, n_star=N) == accounting.thomas_flops(N, n, d)


@pytest.mark.parametrize("J", [1, 2, 3, 7, 15, 63])
def test_segments_do_not_cut_the_arithmetic(J):
    """The paper's segment form does not lower the flops of cyclic reduction:
    eliminating an interior block of a segment costs chol + 6 n^3 (its sweep,
    the fill of the left coupling, the separator update) exactly as one CR
    elimination does.  Over all levels N - 1 blocks are eliminated either way,
    so for large N both tallies approach (N - 1)(n^3/3 + 6 n^3) and exceed the
    block-Thomas tally by about (6 + 1/3) / (2 + 1/3) = 2.7x."""
    N, n, d = 16384, 64, 4
    seg = accounting.segment_flops(N, n, d, J)["factor"]
    cr = accounting.cr_flops(N, n, d)["factor"]
    th = accounting.thomas_flops(N, n, d)["factor"]
    per_block = (N - 1) * (n ** 3 / 3 + 6 * n ** 3)
    assert abs(seg - per_block) / per_block < 0.02
    assert abs(seg - cr) / cr < 0.02
    assert 2.6 < seg / th < 2.75


def test_segment_levels():
    assert accounting.segment_levels(9, 3) == [9, 3, 1]
    assert accounting.segment_levels(9, 1) == accounting.levels(9)
    assert accounting.segment_levels(100, 1, n_star=16) == [100, 50, 25, 13]


def test_emu_schur_mma_flops_counts_tiles_by_brute_force():
    """Rounds of the digit-slice Schur engine: every 128 x 16 tile of D that
    touches the lower triangle once per eliminated neighbour, every tile of E
    once when the next separator exists; ten 128 x 160 x np products each."""
    for N, n in [(2, 96), (3, 200), (9, 256), (64, 130)]:
        np_ = -(-n // 64) * 64
        tiles_lower = sum(1 for r0 in range(0, n, 128) for c0 in range(0, n, 16)
                          if any(c <= r for r in range(r0, min(n, r0 + 128)) for c in range(c0, min(n, c0 + 16))))
        tiles_all = len(range(0, n, 128)) * len(range(0, n, 16))
        rounds = 0
        for Nl in accounting.levels(N)[:-1]:
            for s in range(0, Nl, 2):
                rounds += tiles_lower * ((s >= 2) + (s + 1 < Nl)) + tiles_all * (s + 2 < Nl)
        assert accounting.emu_schur_mma_flops(N, n) == rounds * 2.0 * 10 * 128 * 160 * np_


def test_emu_wslice_bytes_one_level():
    # N = 2: one coupling block, read as FP64 and written as ten BF16 planes
    assert accounting.emu_wslice_bytes(2, 256) == 8.0 * 256 * 256 + 20.0 * 256 * 256
