"""Writes the stored expected values under tests/golden/ -- calls only oracle/.

  python tests/golden/make_golden.py

moments_grid5x5_d20.json: exact output-distribution moments of the 5x5 grid,
depth-20 circuit (seed 0) from the FP64 state vector: sum_x p_x (= 1) and the
collision moment N sum_x p_x^2 (Porter-Thomas would give 2).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import qgm_inputs as qi  # noqa: E402
from oracle import statevector as sv  # noqa: E402


def main():
    c = qi.grid_circuit(5, 5, 20, 0)
    p = np.abs(sv.state(c)) ** 2
    out = {"circuit": "grid 5x5, depth 20, seed 0", "sum_p": float(p.sum()),
           "N_sum_p2": float((2 ** c.n) * (p ** 2).sum()),
           "source": "oracle/statevector.py (FP64)"}
    with open(os.path.join(HERE, "moments_grid5x5_d20.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
