"""Pins for oracle/xeb.py (App. B, C)."""
import math

import numpy as np

from oracle import xeb


def test_euler_gamma_from_exponential_probabilities():
    # for N p ~ Exp(1) (Porter-Thomas), E[-log(N p)] = gamma
    rng = np.random.default_rng(0)
    Np = rng.exponential(size=400000)
    assert abs(np.mean(-np.log(Np)) - xeb.EULER_GAMMA) < 0.01
    assert abs(xeb.EULER_GAMMA - 0.5772156649015329) < 1e-15


def test_alpha_is_one_for_ideal_samples():
    # bitstrings drawn from p itself: S = H(p) -> alpha = 1 (Porter-Thomas set)
    n = 12
    rng = np.random.default_rng(1)
    p = rng.exponential(size=2 ** n)
    p /= p.sum()
    draws = rng.choice(2 ** n, size=200000, p=p)
    st = xeb.stats(np.sqrt(p[draws]), n)
    assert abs(st["alpha"] - 1) < 0.02
    # uniform (uncorrelated) samples: S = H0 -> alpha = 0
    st0 = xeb.stats(np.sqrt(p[rng.integers(0, 2 ** n, 200000)]), n)
    assert abs(st0["alpha"]) < 0.02


def test_sampling_frequencies_follow_normalised_probabilities():
    a = np.sqrt(np.array([0.1, 0.4, 0.2, 0.3]) * 7.0)
    idx, u, cdf = xeb.sample_from_set(a, 40000, seed=5)
    freq = np.bincount(idx, minlength=4) / 40000
    assert np.allclose(freq, [0.1, 0.4, 0.2, 0.3], atol=0.01)
    assert np.all(u >= 0) and np.all(u < 1)
    # inverse transform: cdf[idx-1] <= u < cdf[idx]
    lo = np.where(idx > 0, cdf[np.maximum(idx - 1, 0)], 0.0)
    assert np.all(lo <= u) and np.all(u < cdf[idx])
