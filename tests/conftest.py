import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def small_biharmonic():
    """Oracle hierarchy of the 16x16-patch biharmonic p=3 problem (4 levels), seed-0 Fourier RHS."""
    from oracle import pum
    import pum_inputs as pin
    pr = pin.SMALL_BIHARMONIC
    f = pum.fourier_source(pin.fourier_coefficients(pr.rhs_seed), pr.rhs_decay)
    return pum.build_hierarchy(pr.finest_m, pr.p, pr.equation, pr.n_levels, f=f, constants=pr.nitsche)
