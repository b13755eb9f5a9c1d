"""GPU check of the phase trace: a persistent factor+solve records one
release stamp per grid barrier it ran, in time order, and the solve-only
pass records its own (shorter) set."""
import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_trace_stamps_every_barrier(precision):
    from paper_2509_03015_gb300 import Solver
    s = inputs.kalman_btd(1000, 16, 8, 2, 0.95, 3)
    dev = torch.device("cuda:0")
    Ad, As, B = (torch.from_numpy(np.ascontiguousarray(s[k])).to(dev) for k in ("A_diag", "A_sub", "B"))
    sol = Solver(1000, 16, d_max=2, precision=precision)
    try:
        sol.factor(Ad, As)
        L = sol.plan_levels
        assert L == 10
        stamps = sol.trace()
        assert len(stamps) == 1 + 2 * L                       # start-up + (A, B) per level
        assert all(b >= a for a, b in zip(stamps, stamps[1:]))
        if precision == "fp64":
            _, bars = sol.launch_stats()
            assert bars == len(stamps)
        sol.solve(B)
        stamps = sol.trace()
        # start-up, (A, B) per level, after the top block, downward levels L-1..1
        assert len(stamps) == 1 + 2 * L + 1 + (L - 1)
        assert all(b >= a for a, b in zip(stamps, stamps[1:]))
        assert stamps[-1] - stamps[0] < 10_000_000_000
    finally:
        sol.close()


@pytest.mark.parametrize("n,precision", [(64, "fp64"), (64, "fp32_ir"), (256, "fp64"), (256, "fp32_ir"),
                                         (256, "tf32_ir")])
def test_launch_config_is_resident(n, precision):
    # the persistent grid must fit on the GPU at once (cooperative launch):
    # at least one CTA per SM, with the shared memory the occupancy
    # calculator was given
    from paper_2509_03015_gb300 import Solver
    sol = Solver(64, n, d_max=16 if n == 256 else 4, precision=precision)
    try:
        per_sm, sms, smem = sol.launch_config()
        props = torch.cuda.get_device_properties(0)
        assert sms == props.multi_processor_count
        assert 1 <= per_sm <= 8 and 0 < smem <= 232448
        print(f"n={n} {precision}: {per_sm} CTAs/SM, {smem} B shared memory")
    finally:
        sol.close()
