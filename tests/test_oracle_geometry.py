"""Geometry pins for the oracle (patch extraction, overlap counts, overlap-add).

* Overlap counts from the closed form equal a brute-force count over every
  patch's pixels, bit for bit, in 1 to 4 dimensions with strides > 1.
* sum_i |Omega_i| = sum_q m_q c_q (each observed pixel is seen once per
  covering patch) -- an integer identity.
* Overlap-add of patches reconstructed exactly (a permutation dictionary with
  weights chosen so that D w_i equals the extracted patch) returns the frame.
"""
import itertools

import numpy as np
import pytest

import oracle as O

GEOMS = [
    ((17,), (4,), (1,)),
    ((19,), (5,), (2,)),
    ((12, 15), (3, 4), (1, 1)),
    ((13, 16), (3, 4), (2, 3)),
    ((8, 9, 10), (2, 3, 4), (3, 2, 2)),
    ((5, 6, 7, 4), (2, 3, 2, 2), (1, 3, 5, 2)),
]


def _brute(M, B, S):
    counts = np.zeros(M, dtype=np.int64)
    starts = [range(0, M[d] - B[d] + 1, S[d]) for d in range(len(M))]
    for t in itertools.product(*starts):
        sl = tuple(slice(t[d], t[d] + B[d]) for d in range(len(M)))
        counts[sl] += 1
    return counts


@pytest.mark.parametrize("M,B,S", GEOMS)
def test_overlap_counts_bit_exact(M, B, S):
    prm = O.params(M, B, S, 3)
    assert O.check(prm) == 0
    np.testing.assert_array_equal(O.overlap_counts(prm), _brute(M, B, S))


@pytest.mark.parametrize("M,B,S", GEOMS)
def test_patch_grid_matches_numpy_strided_view(M, B, S):
    """Origins + offsets address the same pixels as numpy's sliding windows."""
    prm = O.params(M, B, S, 3)
    frame = np.arange(int(np.prod(M)), dtype=np.int64).reshape(M)
    win = np.lib.stride_tricks.sliding_window_view(frame, B)
    win = win[tuple(slice(None, None, s) for s in S)]
    ref = win.reshape(-1, int(np.prod(B)))
    got = O.patch_origins(prm)[:, None] + O.pixel_offsets(prm)[None, :]
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("M,B,S", GEOMS)
def test_observed_count_identity(M, B, S):
    prm = O.params(M, B, S, 3)
    rng = np.random.default_rng(0)
    mask = (rng.random(M) < 0.3).astype(np.uint8)
    idx = O.patch_origins(prm)[:, None] + O.pixel_offsets(prm)[None, :]
    per_patch = mask.reshape(-1)[idx].sum()
    assert per_patch == int((mask.astype(np.int64) * O.overlap_counts(prm)).sum())


def test_invalid_geometry_rejected():
    assert O.check(O.params((10,), (4,), (4,), 2)) != 0   # (10-4) % 4 != 0
    assert O.check(O.params((10,), (11,), (1,), 2)) != 0  # patch larger than frame
    assert O.check(O.params((10,), (4,), (1,), 0)) != 0   # no atoms


@pytest.mark.parametrize("M,B,S", GEOMS[:5])
def test_overlap_add_of_exact_patches_returns_frame(M, B, S):
    P = int(np.prod(B))
    prm = O.params(M, B, S, P)
    rng = np.random.default_rng(1)
    frame = rng.random(M)
    perm = rng.permutation(P)
    D = np.zeros((P, P))
    D[np.arange(P), perm] = 1.0           # d_k = e_{perm[k]}: not symmetric
    idx = O.patch_origins(prm)[:, None] + O.pixel_offsets(prm)[None, :]
    patches = frame.reshape(-1)[idx]       # N x P
    # (D w)_p = sum_k D[k, p] w_k = w_{perm^-1(p)}  =>  w_k = x_{perm[k]}
    S_ = patches[:, perm]
    st = O.State(prm, D=D, Z=np.ones_like(S_, dtype=np.uint8), S=S_)
    rec = O.reconstruct(st)
    covered = O.overlap_counts(prm) > 0
    np.testing.assert_allclose(rec[covered], frame[covered], rtol=1e-14, atol=1e-15)
