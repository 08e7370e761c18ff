import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


_PROBLEMS = {}


def oracle_problem(name, primal=None):
    """Session-cached oracle Problem for a named synthetic workload."""
    import synth
    from oracle.bidomain import Problem
    key = (name, primal)
    if key not in _PROBLEMS:
        w = synth.workload(name)
        if primal is not None:
            w["primal"] = primal
        _PROBLEMS[key] = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU,
                                 synth.stimulus(w))
    return _PROBLEMS[key]


@pytest.fixture
def problem():
    return oracle_problem
