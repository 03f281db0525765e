"""Whole-sampler pin for the oracle: recovery of a planted sparse dictionary.

A frame is tiled with non-overlapping 8x8 patches (stride 8, so patches are
independent), each x_i = D* w_i + N(0, 0.1^2) with K = 16 unit-norm planted
atoms and exactly 3 active N(0, 1) weights per patch.  After 200 Gibbs
iterations the learned dictionary must contain every planted atom up to sign
and permutation (|cos| >= 0.95 for >= 90% of them), with about 3 active atoms
per patch, for the full mask and for a 50% random mask.
"""
import numpy as np
import pytest

import oracle as O


def _planted(frac, seed, K=16, side=8, grid=40, noise=0.1, active=3):
    rng = np.random.default_rng(seed)
    P = side * side
    Dt = rng.standard_normal((K, P))
    Dt /= np.linalg.norm(Dt, axis=1, keepdims=True)
    N = grid * grid
    W = np.zeros((N, K))
    for i in range(N):
        act = rng.choice(K, active, replace=False)
        W[i, act] = rng.standard_normal(active)
    X = W @ Dt + noise * rng.standard_normal((N, P))
    frame = X.reshape(grid, grid, side, side).transpose(0, 2, 1, 3).reshape(grid * side, grid * side)
    mask = (rng.random(frame.shape) < frac).astype(np.uint8)
    return Dt, frame.astype(np.float32), mask


@pytest.mark.parametrize("frac", [1.0, 0.5])
def test_planted_dictionary_is_recovered(frac):
    Dt, frame, mask = _planted(frac, seed=0)
    prm = O.params(frame.shape, (8, 8), (8, 8), 16, seed=0)
    st = O.learn(O.State(prm), frame, mask, 200)
    Dl = st.D / np.linalg.norm(st.D, axis=1, keepdims=True)
    best = np.abs(Dt @ Dl.T).max(axis=1)
    assert (best >= 0.95).mean() >= 0.9, np.sort(best)
    assert 2.5 < st.Z.sum(axis=1).mean() < 3.5


def test_stem_reconstruction_improves_with_iterations():
    """Integration sanity on the 128x128 STEM workload (not a pin): PSNR
    against the clean frame rises over the first iterations."""
    from paper_2311_15061_gb300 import synth
    x, clean = synth.stem_frame((128, 128), 0)
    m = synth.random_mask((128, 128), 0.25, 0)
    prm = O.params((128, 128), (8, 8), (1, 1), 64, seed=0)
    st = O.State(prm)
    scores = []
    O.learn(st, x, m, 6, callback=lambda s, _: scores.append(O.psnr(O.reconstruct(s), clean)))
    assert scores[-1] > scores[0] + 3.0
