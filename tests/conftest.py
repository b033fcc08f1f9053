"""Shared fixtures. The ``gpu`` marker (registered in pytest.ini) tags tests that need a
CUDA device; everything else runs on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def single_object():
    from paper_2312_08715_gb300 import synth
    return synth.single_object_workload(0)


@pytest.fixture(scope="session")
def tabletop():
    from paper_2312_08715_gb300 import synth
    return synth.tabletop_workload(0)
