"""Pins for the oracle's posterior-mean reconstruction (the reconstruction
the paper shows from its samples, "Time-To-Solution" section; the mean over
the last T samples of the chain).

* T copies of one sample give that sample's overlap-add reconstruction.
* Against the definition written out in numpy by another route: each
  sample's per-patch products D^T w_i placed at the patch's pixels by index
  arithmetic of numpy's own (np.add.at over sliding-window coordinates),
  divided by the coverage count, then averaged over the samples; 2-D and 3-D
  frames with strides.
* On a chain of the sampler, the mean of its last samples.
"""
import numpy as np
import pytest

import oracle as O


def _sample(prm, rng, density):
    st = O.State(prm)
    st.Z = (rng.random(st.Z.shape) < density).astype(np.uint8)
    st.S = rng.standard_normal(st.S.shape) * st.Z
    st.D = rng.standard_normal(st.D.shape)
    return st


def _numpy_mean(prm, states):
    M = tuple(prm.M[i] for i in range(prm.ndim))
    B = tuple(prm.B[i] for i in range(prm.ndim))
    S = tuple(prm.S[i] for i in range(prm.ndim))
    coords = np.indices(M).reshape(len(M), -1).T.reshape(M + (len(M),))
    win = np.lib.stride_tricks.sliding_window_view(coords, B, axis=tuple(range(len(M))))
    win = win[tuple(slice(None, None, s) for s in S)]          # patch grid x coordinate x B
    grid = win.shape[:len(M)]
    # pixel coordinates of every (patch, within-patch pixel), patches and
    # pixels in row-major order
    pix = np.moveaxis(win, len(M), -1).reshape(int(np.prod(grid)), int(np.prod(B)), len(M))
    flat = np.ravel_multi_index(tuple(pix[..., d] for d in range(len(M))), M)
    count = np.zeros(int(np.prod(M)))
    np.add.at(count, flat.ravel(), 1.0)
    acc = np.zeros(int(np.prod(M)))
    for st in states:
        Y = (st.Z * st.S) @ st.D                                 # N x P products D^T w_i
        frame = np.zeros(int(np.prod(M)))
        np.add.at(frame, flat.ravel(), Y.ravel())
        acc += np.where(count > 0, frame / np.maximum(count, 1), 0.0)
    return (acc / len(states)).reshape(M)


@pytest.mark.parametrize("M,B,S,K", [((23, 19), (4, 3), (1, 2), 6), ((7, 12, 10), (3, 4, 2), (2, 1, 2), 5),
                                     ((41,), (5,), (3,), 4)])
def test_mean_against_numpy_definition(M, B, S, K):
    prm = O.params(M, B, S, K)
    rng = np.random.default_rng(sum(M))
    states = [_sample(prm, rng, 0.3 + 0.1 * t) for t in range(4)]
    got = O.reconstruct_mean(states)
    want = _numpy_mean(prm, states)
    assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_mean_of_equal_samples_is_the_sample():
    prm = O.params((20, 22), (5, 4), (1, 1), 7)
    st = _sample(prm, np.random.default_rng(1), 0.4)
    one = O.reconstruct(st)
    mean = O.reconstruct_mean([st, st, st])
    assert np.abs(mean - one).max() <= 1e-14 * max(1.0, np.abs(one).max())


def test_mean_over_a_chain():
    from paper_2311_15061_gb300 import synth
    M = (40, 40)
    x, clean = synth.stem_frame(M, 0)
    mask = synth.random_mask(M, 0.3, 0)
    prm = O.params(M, (6, 6), (1, 1), 16, seed=3)
    kept = []
    O.learn(O.State(prm), x, mask, 6, callback=lambda st, stats: kept.append(st.copy()) if st.t >= 3 else None)
    assert len(kept) == 3
    want = sum(O.reconstruct(st) for st in kept) / 3.0
    assert np.abs(O.reconstruct_mean(kept) - want).max() <= 1e-13
