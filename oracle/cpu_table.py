"""CPU timing table of the FP64 oracle (test infrastructure; the reported CPU
baseline): amplitudes/s of oracle/ve.c on each batch workload, with one
thread and with every host core (a pool of threads over bitstrings; for
5x9 depth 40, OpenMP inside each bucket), on bounded samples.

  python -m oracle.cpu_table [seconds_per_cell]

Prints one JSON object: host core count (os.cpu_count), and per workload and
thread count the rate, the sample (bitstrings done, or for 5x9 depth 40 one of
its 2^7 conditioned parts scaled to a whole amplitude) and the seconds spent.
"""
import json
import os
import sys
import time

import numpy as np

import qgm_inputs as qi

from . import order as O
from . import ugm, vec


def _rate(c, bits, threads, seconds):
    m = ugm.build(c)
    adj = O.graph(m)
    order, w = O.min_fill(adj)
    pr = vec.Prepared(m)
    if w > 31:
        sl = O.slice_greedy(adj, order, max_clique=30)
        fixed = np.full(m.n_vars, -1, dtype=np.int32)
        x = int(bits[0])
        for v in m.inputs:
            fixed[v] = 0
        for j, v in enumerate(m.outputs):
            fixed[v] = (x >> j) & 1
        for v in sl:
            fixed[v] = 0
        elim = np.array([v for v in order if v not in set(sl)], dtype=np.int32)
        out = np.zeros(2)
        t0 = time.perf_counter()
        vec.lib().ve_amplitude(m.n_vars, len(m.factors), pr.rank.ctypes.data, pr.off.ctypes.data,
                               pr.vars.ctypes.data, pr.toff.ctypes.data, pr.tables.ctypes.data, fixed.ctypes.data,
                               elim.ctypes.data, len(elim), threads, out.ctypes.data)
        dt = time.perf_counter() - t0
        return 1.0 / (dt * 2 ** len(sl)), f"one of {2 ** len(sl)} slices, scaled", dt
    t0 = time.perf_counter()
    done = 0
    if threads == 1:
        while done < len(bits) and time.perf_counter() - t0 < seconds:
            vec.amplitude(c, int(bits[done]), order=order, model=m, prepared=pr, threads=1)
            done += 1
    else:
        # a pool of host threads over bitstrings, in rounds of 4 per thread
        while done < len(bits) and time.perf_counter() - t0 < seconds:
            chunk = bits[done:done + 4 * threads]
            vec.amplitudes_parallel(c, chunk, order=order, model=m, prepared=pr, workers=threads)
            done += len(chunk)
    dt = time.perf_counter() - t0
    return done / dt, f"{done} bitstrings", dt


def main():
    seconds = float(sys.argv[1]) if len(sys.argv) > 1 else 10.0
    cores = os.cpu_count() or 1
    out = {"cores": cores, "oracle": "oracle/ve.c (FP64 bucket elimination, min-fill order)", "rows": []}
    for name, (rows, cols, depth, B, param) in sorted(qi.WORKLOADS.items()):
        if B == 0:
            continue
        c = qi.grid_circuit(rows, cols, depth, 0, param=param)
        bits = qi.bitstrings(c.n, B, 0)
        for threads in (1, cores):
            if rows * cols > 40 and threads == 1:
                continue  # a 5x9 depth-40 slice takes minutes on one thread
            rate, sample, dt = _rate(c, bits, threads, seconds)
            out["rows"].append({"workload": name, "threads": threads, "amplitudes_per_s": rate,
                                "sample": sample, "seconds": round(dt, 2)})
            print(json.dumps(out["rows"][-1]), file=sys.stderr, flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
