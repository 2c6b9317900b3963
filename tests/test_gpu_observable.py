"""Expectation values of Pauli strings on the GPU (Sec. III) against the
FP64 oracle (needs a GB300).  The library keeps the light cone of the
observable and computes one amplitude of W = V, P, V^dagger; the oracle
applies P to the state vector.  Tolerance: FP32 elimination, |error| below
1e-5 (expectations are at most 1 in magnitude)."""
import numpy as np
import pytest

import qgm_inputs as qi
from oracle import observable as OB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_05384_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# Pauli strings with large |<P>| on these circuits (found by scanning all
# weight-2 and weight-3 strings with the oracle), and some with <P> = 0
P3 = ["IIIIIIIZX", "IIZIIYIII", "YIIXXIIII", "IZXIIZIII", "IIIIXIIII", "XIIIIIIIZ", "IIIIIIIII"]
P4 = ["IYIIXIIIIIIIIIII", "IIIXIIYIIIIIIIII", "IIIZIIYIIIIIIIII", "Z" + "I" * 14 + "Z",
      "I" * 15 + "Z"]


@pytest.mark.parametrize("executor", [1, 2, 3])
def test_expectations_3x3_d6(executor):
    from paper_1712_05384_gb300 import Circuit, observable
    c = qi.grid_circuit(3, 3, 6, 5)
    assert abs(OB.expectation(c, P3[0]) - 1) < 1e-12
    for pauli in P3:
        ref = OB.expectation(c, pauli)
        got = observable.expectation(Circuit.grid(3, 3, 6, 5), pauli, executor=executor)
        assert abs(got - ref) < 1e-5, (pauli, got, ref)


def test_expectations_4x4_d10():
    from paper_1712_05384_gb300 import Circuit, observable
    c = qi.grid_circuit(4, 4, 10, 0)
    for pauli in P4:
        ref = OB.expectation(c, pauli)
        got = observable.expectation(Circuit.grid(4, 4, 10, 0), pauli)
        assert abs(got - ref) < 1e-5, (pauli, got, ref)
