"""Pins for the oracle's initial state (the model's priors, BPFA section;
readings 1 and 7 of the design notes).

* The initial dictionary is a draw from the atom prior d_k ~ N(0, I/P): for
  several patch sizes P, the entries scaled by sqrt(P) pass a
  Kolmogorov-Smirnov test against the standard normal, their variance is 1/P
  within its sampling error, and distinct atoms and pixels are uncorrelated.
  A wrong prior scale (1/P, or the prior variance taken as P) fails here.
* The initial noise precision is 1 / var(observed pixels) (population
  variance, FP64): checked against numpy, with its two limits -- a constant
  frame clamps the variance at 1e-12, and an empty mask (no variance at all)
  starts at 1.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O


@pytest.mark.parametrize("B", [(3, 3), (8, 8), (10, 10), (16, 16)])
def test_initial_dictionary_is_a_prior_draw(B):
    P = B[0] * B[1]
    K = max(8, 12800 // P)          # about 12,800 entries per seed
    samples = []
    for seed in range(4):
        prm = O.params((B[0] + 3, B[1] + 2), B, (1, 1), K, seed=seed)
        D = O.State(prm).D
        assert D.shape == (K, P)
        samples.append(D)
    z = np.concatenate([d.ravel() for d in samples]) * np.sqrt(P)
    n = z.size
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * np.sqrt(2.0 / n)
    # different seeds give different dictionaries
    assert not np.array_equal(samples[0], samples[1])
    # atoms (rows) and pixels (columns) are uncorrelated: neighbouring rows and
    # columns of one dictionary, correlation within 5 standard errors of 0
    D = samples[0]
    rows = np.corrcoef(D[:-1].ravel(), D[1:].ravel())[0, 1]
    cols = np.corrcoef(D[:, :-1].ravel(), D[:, 1:].ravel())[0, 1]
    assert abs(rows) < 5.0 / np.sqrt(D[:-1].size)
    assert abs(cols) < 5.0 / np.sqrt(D[:, :-1].size)


def test_initial_noise_precision_is_inverse_observed_variance():
    rng = np.random.default_rng(3)
    M = (37, 41)
    prm = O.params(M, (4, 4), (1, 1), 8)
    for frac in (0.05, 0.3, 1.0):
        x = rng.gamma(2.0, 0.2, size=M).astype(np.float32)
        mask = (rng.random(M) < frac).astype(np.uint8)
        want = 1.0 / max(np.var(x[mask == 1].astype(np.float64)), 1e-12)
        got = O.init_gamma_eps(prm, x, mask)
        assert abs(got / want - 1.0) < 1e-12, (frac, got, want)


def test_initial_noise_precision_limits():
    M = (20, 24)
    prm = O.params(M, (4, 4), (1, 1), 8)
    x = np.full(M, 0.375, np.float32)            # constant frame: variance 0, clamped
    mask = np.ones(M, np.uint8)
    assert O.init_gamma_eps(prm, x, mask) == pytest.approx(1e12, rel=1e-12)
    x = np.random.default_rng(0).random(M).astype(np.float32)
    assert O.init_gamma_eps(prm, x, np.zeros(M, np.uint8)) == 1.0   # nothing observed
    one = np.zeros(M, np.uint8)
    one[3, 5] = 1                                 # a single pixel: variance 0, clamped
    assert O.init_gamma_eps(prm, x, one) == pytest.approx(1e12, rel=1e-12)
