import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def geom():
    import velo_synth
    return velo_synth.geometry()


@pytest.fixture(scope="session")
def cfg0_events():
    import velo_synth
    return velo_synth.generate(velo_synth.config(0))


@pytest.fixture(scope="session")
def cfg0_oracle(geom, cfg0_events):
    import oracle
    return oracle.reconstruct(geom, cfg0_events, n_threads=os.cpu_count() or 1)
