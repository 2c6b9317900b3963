"""Writes the stored expected values under tests/golden/ -- calls only oracle/
and the seeded input generators (qgm_inputs).

  python tests/golden/make_golden.py [moments] [circuits] [amps5x9] [amps6x6]

moments_grid5x5_d20.json: exact output-distribution moments of the 5x5 grid,
depth-20 circuit (seed 0) from the FP64 state vector: sum_x p_x (= 1) and the
collision moment N sum_x p_x^2 (Porter-Thomas would give 2).

circuits_seed0.json: sha256 of the canonical gate list (kind, cycle, q0, q1,
theta, phi to 17 significant digits) of each workload's seed-0 circuit, with
its gate counts per kind, so that a change of the generator shows.

amps_grid5x9_d40.json: <x|C|0^n> of the 5x9, depth-40 circuit (seed 0) for
the first bitstrings of its seed-0 batch, by FP64 bucket elimination in plain
C (oracle/ve.c) in the oracle's min-fill order, sliced greedily
(oracle.order.slice_greedy) until the largest clique has at most 30
variables.  Hours of CPU time; written one bitstring at a time.

amps_grid6x6_d25.json: the same for 32 bitstrings of the 6x6 depth-25 batch
(unsliced).

grad_grid6x6_d20.json: the gradient of L = sum_x log |a_x|^2 over all 256
bitstrings of the parametrised 6x6 depth-20 batch (seed 0) with respect to
48 of its angles (24 RXY gates spread over the circuit, theta and phi), by
derivative insertion with the plain-C elimination: dL/dp = 2 Re sum_x
conj(a_x / |a_x|^2) da_x/dp (App. B's log-probability loss).
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import qgm_inputs as qi  # noqa: E402
from oracle import order as O  # noqa: E402
from oracle import statevector as sv  # noqa: E402
from oracle import ugm, vec  # noqa: E402


def moments():
    c = qi.grid_circuit(5, 5, 20, 0)
    p = np.abs(sv.state(c)) ** 2
    out = {"circuit": "grid 5x5, depth 20, seed 0", "sum_p": float(p.sum()),
           "N_sum_p2": float((2 ** c.n) * (p ** 2).sum()),
           "source": "oracle/statevector.py (FP64)"}
    with open(os.path.join(HERE, "moments_grid5x5_d20.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


def canonical_gates(c):
    return [(int(g.kind), int(g.cycle), int(g.q0), int(g.q1), f"{float(g.theta):.17g}", f"{float(g.phi):.17g}")
            for g in c.gates]


def circuits():
    out = {}
    for name, (rows, cols, depth, _, param) in sorted(qi.WORKLOADS.items()):
        c = qi.grid_circuit(rows, cols, depth, 0, param=param)
        gl = canonical_gates(c)
        h = hashlib.sha256(json.dumps(gl).encode()).hexdigest()
        kinds = {}
        for g in gl:
            kinds[str(g[0])] = kinds.get(str(g[0]), 0) + 1
        out[name] = {"sha256": h, "n_gates": len(gl), "by_kind": kinds}
    with open(os.path.join(HERE, "circuits_seed0.json"), "w") as f:
        json.dump({"source": "qgm_inputs.grid_circuit, seed 0", "circuits": out}, f, indent=1)
    print(out)


def amps(rows, cols, depth, count, max_clique, fname, threads=0):
    c = qi.grid_circuit(rows, cols, depth, 0)
    m = ugm.build(c)
    adj = O.graph(m)
    order, w = O.min_fill(adj)
    sl = O.slice_greedy(adj, order, max_clique=max_clique) if max_clique else []
    bits = qi.bitstrings(c.n, 1000, 0)[:count]
    path = os.path.join(HERE, fname)
    doc = {"circuit": f"grid {rows}x{cols}, depth {depth}, seed 0",
           "bitstrings": "the first entries of qgm_inputs.bitstrings(n, 1000, seed 0)",
           "source": "oracle/ve.c (FP64 bucket elimination), oracle.order.min_fill order, "
                     "oracle.order.slice_greedy slices",
           "max_clique_unsliced": w, "slice_vars": sl, "amplitudes": []}
    if os.path.exists(path):
        with open(path) as f:
            old = json.load(f)
        if old.get("slice_vars") == sl:
            doc["amplitudes"] = old["amplitudes"]
    pr = vec.Prepared(m)
    done = {int(a["x"]) for a in doc["amplitudes"]}
    for x in bits:
        if int(x) in done:
            continue
        t0 = time.time()
        a = vec.amplitude(c, int(x), order=order, slice_vars=sl, model=m, prepared=pr, threads=threads)
        doc["amplitudes"].append({"x": int(x), "re": a.real, "im": a.imag, "seconds": round(time.time() - t0, 1)})
        with open(path + ".tmp", "w") as f:
            json.dump(doc, f, indent=1)
        os.replace(path + ".tmp", path)
        print(f"x={int(x)} a={a!r} {time.time() - t0:.0f}s", flush=True)


def grad6x6():
    c = qi.grid_circuit(6, 6, 20, 0, param=True)
    m = ugm.build(c)
    pr = vec.Prepared(m)
    order, _ = O.min_fill(O.graph(m))
    bits = qi.bitstrings(c.n, 256, 0)
    a = np.array([vec.amplitude(c, int(x), order=order, model=m, prepared=pr) for x in bits])
    gbar = a / np.abs(a) ** 2
    n_gates = len(c.param_gates)
    gates = sorted(set(np.linspace(0, n_gates - 1, 24).round().astype(int).tolist()))
    out = []
    for p in gates:
        for which in (0, 1):
            da = np.array([vec.amplitude_derivative(c, int(x), p, which, order=order, model=m, prepared=pr)
                           for x in bits])
            out.append({"param": 2 * p + which, "gate": int(c.param_gates[p]),
                        "dL": float(2 * np.real(np.sum(np.conj(gbar) * da)))})
        print(p, out[-2:], flush=True)
    doc = {"circuit": "grid 6x6, depth 20, seed 0, parametrised (theta, phi per RXY gate)",
           "bitstrings": "qgm_inputs.bitstrings(36, 256, 0), all of them",
           "loss": "sum_x log |a_x|^2", "n_params": 2 * n_gates,
           "source": "oracle/ve.c by derivative insertion (oracle.vec.amplitude_derivative), min-fill order",
           "sum_log_p": float(np.sum(np.log(np.abs(a) ** 2))), "grad": out}
    with open(os.path.join(HERE, "grad_grid6x6_d20.json"), "w") as f:
        json.dump(doc, f, indent=1)


def main():
    what = sys.argv[1:] or ["moments", "circuits"]
    if "moments" in what:
        moments()
    if "circuits" in what:
        circuits()
    if "amps6x6" in what:
        amps(6, 6, 25, 32, 0, "amps_grid6x6_d25.json")
    if "grad6x6" in what:
        grad6x6()
    if "amps5x9" in what:
        amps(5, 9, 40, 4, 30, "amps_grid5x9_d40.json")


if __name__ == "__main__":
    main()
