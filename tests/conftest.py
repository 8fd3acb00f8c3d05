import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def tiny_scene():
    from paper_2302_12249_b300 import synth
    return synth.make_scene("tiny")


@pytest.fixture(scope="session")
def tiny_oscene(tiny_scene):
    import oracle
    return oracle.OracleScene(tiny_scene)


@pytest.fixture(scope="session")
def paper_scene():
    """The paper-scale synthetic scene (host arrays), built once per session."""
    from paper_2302_12249_b300 import synth
    return synth.make_scene("paper")
