"""Shared fixtures.  Tests marked ``gpu`` need a CUDA device and call the
CUDA library through its C-ABI; every other test runs on the CPU."""
import os
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if REPO not in sys.path:
    sys.path.insert(0, REPO)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def synth_mod():
    from paper_1805_07920_gb300 import synth
    return synth


@pytest.fixture(scope="session")
def tiny_scene(synth_mod):
    return synth_mod.make_scene("tiny")


@pytest.fixture(scope="session")
def medium_scene(synth_mod):
    return synth_mod.make_scene("medium")
