"""Error measures of amplitudes against the FP64 oracle, shared by the GPU
parity tests (not a test module).

The paper reports relative error per probability below 1e-5 in single
precision (Sec. II).  Relative error is undefined where the reference is
near zero, so three numbers are formed:
  rel        max |a - r| / |r| over |r| >= 2^{-n/2} (probability at least
             the uniform 2^{-n}; the measure the tests assert);
  rel_1e3    the same over |r| >= 1e-3 * 2^{-n/2} (the wider cut), with the
             count of amplitudes below that cut;
  abs        max |a - r| * 2^{n/2} over all amplitudes (error relative to
             the root-mean-square amplitude).
Every call prints all of them, so that a run with -s reports the wider cut
even where an FP32 absolute floor keeps it above the stated bound.
"""
import numpy as np


def measures(a, ref, n):
    a = np.asarray(a).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    d = np.abs(a - ref)
    rms = 2.0 ** (-n / 2)
    big = np.abs(ref) >= rms
    wide = np.abs(ref) >= 1e-3 * rms
    return {
        "rel": float(np.max(d[big] / np.abs(ref[big]))) if big.any() else 0.0,
        "rel_1e3": float(np.max(d[wide] / np.abs(ref[wide]))) if wide.any() else 0.0,
        "excluded_1e3": int((~wide).sum()),
        "abs": float(np.max(d) * 2.0 ** (n / 2)),
        "count": int(a.size),
    }


def errors(a, ref, n, label=""):
    m = measures(a, ref, n)
    print(f"[errors] {label} n={n} count={m['count']}: rel(|r|>=2^-n/2) {m['rel']:.2e}, "
          f"rel(|r|>=1e-3*2^-n/2) {m['rel_1e3']:.2e} ({m['excluded_1e3']} below), "
          f"abs*2^(n/2) {m['abs']:.2e}")
    return m["rel"], m["abs"]
