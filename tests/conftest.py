import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def mixed_workload_oracle(oracle_mod):
    """The N = 4096, n = 256, d = 16 Kalman workload (rho = 0.99) and the
    oracle's X for it, computed once per session (about a minute on one
    core) for every test that checks a result of that workload."""
    from paper_2509_03015_gb300 import inputs
    s = inputs.workload("kalman-N4096-n256-d16-rho0.99")
    return s, oracle_mod.solve_system(s["A_diag"], s["A_sub"], s["B"])
