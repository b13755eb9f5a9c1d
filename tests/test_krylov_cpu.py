"""Host-side checks of the CG refinement: the ill-conditioned generator's
spectrum and the C-ABI argument checks (no GPU)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2509_03015_gb300 import inputs


@pytest.mark.parametrize("N,n", [(16, 3), (64, 4)])
def test_laplace_btd_smallest_eigenvalue_is_the_laplacian_one(N, n):
    s = inputs.laplace_btd(N, n, 1, seed=0)
    blk = oracle.dense_blocks(s["A_diag"], s["A_sub"])
    A = np.block([[blk(r, c) for c in range(N)] for r in range(N)])
    w = np.linalg.eigvalsh(A)
    assert w[0] > 0
    np.testing.assert_allclose(w[0], 4 * np.sin(np.pi / (2 * (N + 1))) ** 2, rtol=1e-9)


def test_refine_options_and_stats_reject_bad_arguments():
    from paper_2509_03015_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    assert lib.bdss_set_option(None, 7, 1) == 1
    assert lib.bdss_set_option(None, 8, 10) == 1
    p, c = ctypes.c_int32(), ctypes.c_int32()
    assert lib.bdss_last_refine_stats(None, ctypes.byref(p), ctypes.byref(c)) == 1
    assert _lib.OPTIONS["refine_krylov"] == 7 and _lib.OPTIONS["max_krylov_iters"] == 8


def test_illcond_generator_condition_number():
    """The shifted-factorisation test input: kappa within a factor 4 of the
    requested value (the couplings move eigenvalues by at most a quarter of
    the smallest block eigenvalue each way)."""
    from tests._helpers import dense_A
    s = inputs.illcond_btd(6, 5, 1, seed=3, kappa=1e9)
    ev = np.linalg.eigvalsh(dense_A(s["A_diag"], s["A_sub"]))
    assert ev.min() > 0
    k = ev.max() / ev.min()
    assert 0.25e9 <= k <= 4e9
