import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def app_d_circuit():
    """The two-qubit example of Eq. ex_circ / App. D: H on both, CZ, H on both."""
    import qgm_inputs as qi
    G = qi.Gate
    return qi.circuit_from_gates(2, [G(qi.GATE_H, 0, 0), G(qi.GATE_H, 0, 1),
                                     G(qi.GATE_CZ, 1, 0, 1),
                                     G(qi.GATE_H, 2, 0), G(qi.GATE_H, 2, 1)])


@pytest.fixture
def app_d():
    return app_d_circuit()
