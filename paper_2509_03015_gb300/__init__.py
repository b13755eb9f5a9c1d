"""GB300 (sm_103a) solver for SPD block-tridiagonal systems A X = B by odd-even
block cyclic reduction -- the recursive Schur-complement method of
arXiv 2509.03015 (Sec. 3) with interior segments of length one, every level
fused into one persistent kernel.

The compute path is the C-ABI library libbdss.so (include/bdss.h) built from
csrc/; this package only marshals arguments to it.
"""
from ._lib import BDSSError, load  # noqa: F401


def __getattr__(name):
    # torch-facing binding, imported lazily so that the C-ABI layer and the
    # input generators load without torch
    if name in ("Solver", "solve", "BlockTriSolve", "block_tri_solve", "BatchSolver",
                "kalman_assemble"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
