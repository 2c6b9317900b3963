"""Cross-entropy benchmarking and sampling from a computed set (oracle; test only).

App. B of the paper: S(p_exp, p_U) is estimated by -(1/m) sum_j log p_U(x_j)
over measured bitstrings (Eq. cee); the fidelity estimate is
alpha = (H0 - S) / (H0 - H(p_U)) (Eq. ae), with the Porter-Thomas values
H0 = log(2^n) + gamma and H(p_U) = log(2^n) - 1 + gamma (gamma: Euler's
constant).
App. C: sample m bitstrings from a computed set T of t amplitudes with the
normalised probabilities p~_j = p_j / sum_T p, here by inverse transform of
uniforms u_i (the i-th draw of SplitMix64(seed), top 53 bits); index j is
the first with cumulative p~ above u_i.
Parity: pinned (Euler's constant from exponential samples, alpha = 1 for
ideal samples of a Porter-Thomas set, inverse-transform frequencies;
tests/test_oracle_xeb.py).
"""
import math

import numpy as np

EULER_GAMMA = 0.5772156649015329


def stats(amps, n):
    p = np.abs(np.asarray(amps)) ** 2
    N = 2.0 ** n
    S = -np.mean(np.log(p))
    H0 = n * math.log(2) + EULER_GAMMA
    H = n * math.log(2) - 1 + EULER_GAMMA
    return {"cross_entropy": S, "alpha": (H0 - S) / (H0 - H), "mean_Np": np.mean(N * p),
            "second_moment": np.mean((N * p) ** 2)}


def uniforms(seed, m):
    import qgm_inputs as qi
    g = qi.SplitMix64(seed)
    return np.array([(g.next() >> 11) * 2.0 ** -53 for _ in range(m)])


def sample_from_set(amps, m, seed):
    p = np.abs(np.asarray(amps)) ** 2
    cdf = np.cumsum(p / p.sum())
    u = uniforms(seed, m)
    idx = np.searchsorted(cdf, u, side="right")
    return np.minimum(idx, len(p) - 1), u, cdf
