"""GPU parity of the overlap-add reconstruction (a6) against the FP64 oracle.

The per-patch reconstructions y_i = D^T (z_i * s_i) run on the tensor cores
(tcgen05, TF32 head + tail split, FP32 accumulation in TMEM) for patches of
up to 256 pixels and on the FP32 ALU kernel above; the overlap-add gather
follows either.  The shapes cross every accumulator width the tensor-core
form allocates (patch sizes rounded up to 16, in 32, 64, 128 and 256 TMEM
columns), dictionaries whose size is not a multiple of the 8-atom block,
patch counts that leave a ragged last 128-patch tile and a ragged last warp,
1-D and 3-D frames, sparse, dense, all-zero and all-one codes, and weights
of very different magnitudes.  Tolerance: 1e-5 of the frame's largest
magnitude, the a6 tolerance of the other parity tests.
"""
import numpy as np
import pytest

import oracle as O
from parity_helpers import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_15061_gb300 import build
    build.build()


# (frame shape, patch shape, stride, K, code density)
CASES = [
    ((40, 36), (2, 2), (1, 1), 5, 0.5),          # P = 4: 16-wide tile, 32 columns; one partial block
    ((70, 65), (5, 6), (1, 1), 20, 0.3),         # P = 30
    ((96, 80), (8, 6), (1, 2), 24, 0.2),         # P = 48: 64 columns
    ((131, 127), (10, 10), (1, 1), 128, 0.1),    # P = 100: the benchmark patch, 112 of 128 columns
    ((65, 89), (11, 11), (2, 3), 33, 0.4),       # P = 121
    ((80, 77), (12, 12), (1, 1), 64, 0.25),      # P = 144: 256 columns
    ((60, 70), (16, 16), (2, 2), 40, 0.6),       # P = 256: the widest tensor-core tile
    ((50, 49), (17, 16), (3, 3), 12, 0.5),       # P = 272: the ALU kernel
    ((5002,), (64,), (3,), 16, 0.3),             # 1-D
    ((12, 14, 16), (4, 4, 4), (1, 2, 1), 24, 0.3),  # 3-D, P = 64
]


def _state(prm, density, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    st = O.State(prm)
    N, K = st.Z.shape
    P = st.D.shape[1]
    st.D = (rng.standard_normal((K, P)) / np.sqrt(P)).astype(np.float32).astype(np.float64)
    st.Z = (rng.random((N, K)) < density).astype(np.uint8)
    mag = scale * np.exp(rng.uniform(-4.0, 4.0, (N, K)))   # magnitudes over ~3.5 decades
    st.S = (rng.standard_normal((N, K)) * mag * st.Z).astype(np.float32).astype(np.float64)
    return st


def _check(prm, st, mask):
    ctx = gpu_context(prm, mask)
    ctx.sensai_set_state(D=st.D.astype(np.float32), Z=st.Z, S=st.S.astype(np.float32), gamma_s=1.0)
    rec = ctx.sensai_reconstruct()
    ctx.close()
    orec = O.reconstruct(st)
    assert rec.shape == orec.shape
    assert np.isfinite(rec).all()
    scale = max(np.abs(orec).max(), 1e-6)
    err = np.abs(rec - orec).max()
    assert err <= 1e-5 * scale, (err, scale)
    return rec, orec


@pytest.mark.parametrize("M,B,S,K,density", CASES)
def test_reconstruct_matches_oracle(M, B, S, K, density):
    from paper_2311_15061_gb300 import synth
    prm = O.params(M, B, S, K, seed=3)
    # the reconstruction does not read the mask; patches above 256 pixels get
    # a half mask so that each observes at most 256 pixels
    mask = np.ones(M, np.uint8) if np.prod(B) <= 256 else synth.random_mask(M, 0.5, 0)
    _check(prm, _state(prm, density, 11), mask)


def test_reconstruct_all_zero_codes_is_exactly_zero():
    M, B, S, K = (131, 127), (10, 10), (1, 1), 128
    prm = O.params(M, B, S, K, seed=3)
    st = _state(prm, 0.0, 5)
    rec, _ = _check(prm, st, np.ones(M, np.uint8))
    assert (rec == 0).all()


def test_reconstruct_dense_codes():
    M, B, S, K = (97, 101), (10, 10), (1, 1), 64
    prm = O.params(M, B, S, K, seed=3)
    _check(prm, _state(prm, 1.0, 6), np.ones(M, np.uint8))


def test_reconstruct_single_atom_is_the_atom_overlap_average():
    """K = 1, z = 1 and s = 1 everywhere: every pixel is the average of d_p over
    the patches covering it, a closed form the oracle does not need."""
    M, B, S, K = (40, 44), (8, 8), (1, 1), 1
    prm = O.params(M, B, S, K, seed=3)
    st = _state(prm, 1.0, 7)
    st.S = st.Z.astype(np.float64)
    rec, _ = _check(prm, st, np.ones(M, np.uint8))
    d = st.D[0].reshape(B).astype(np.float64)
    acc = np.zeros(M)
    cnt = np.zeros(M)
    for r in range(M[0] - B[0] + 1):
        for c in range(M[1] - B[1] + 1):
            acc[r:r + B[0], c:c + B[1]] += d
            cnt[r:r + B[0], c:c + B[1]] += 1
    np.testing.assert_allclose(rec, acc / cnt, rtol=0, atol=1e-5 * np.abs(d).max())


def test_reconstruct_is_deterministic():
    M, B, S, K = (131, 127), (10, 10), (1, 1), 128
    prm = O.params(M, B, S, K, seed=3)
    st = _state(prm, 0.1, 8)
    outs = []
    for _ in range(2):
        ctx = gpu_context(prm, np.ones(M, np.uint8))
        ctx.sensai_set_state(D=st.D.astype(np.float32), Z=st.Z, S=st.S.astype(np.float32), gamma_s=1.0)
        outs.append(ctx.sensai_reconstruct())
        outs.append(ctx.sensai_reconstruct())
        ctx.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)


# --- posterior-mean reconstruction over the last T samples (sensai_mean_*) ---

@pytest.mark.parametrize("M,B,S,K,T", [((128, 128), (8, 8), (1, 1), 64, 3),
                                       ((12, 14, 16), (4, 4, 4), (1, 2, 1), 24, 4)])
def test_posterior_mean_matches_oracle(M, B, S, K, T):
    """The last T samples of an oracle chain, pushed into the context one by
    one and added: the mean against the oracle's, 1e-5 of the largest value."""
    from parity_helpers import problem, round_state
    prm, x, clean, mask = problem(M, B, S, K, 0.25, seed=2)
    kept = []
    O.learn(O.State(prm), x, mask, T + 1,
            callback=lambda st, stats: kept.append(round_state(st.copy())) if st.t >= 1 else None)
    assert len(kept) == T
    ctx = gpu_context(prm, mask)
    ctx.sensai_mean_reset()
    for st in kept:
        ctx.sensai_set_state(D=st.D.astype(np.float32), Z=st.Z, S=st.S.astype(np.float32), gamma_s=st.gamma_s,
                             gamma_eps=st.gamma_eps, iter=st.t)
        ctx.sensai_mean_add()
    got = ctx.sensai_mean_read()
    ctx.close()
    want = O.reconstruct_mean(kept)
    assert np.abs(got - want).max() <= 1e-5 * max(np.abs(want).max(), 1e-6)


def test_posterior_mean_of_one_state_is_the_reconstruction_full_size():
    """512x512, K = 128: the mean of three adds of one state equals
    sensai_reconstruct bit for bit ((3 y) / 3 is exact in FP64 for an FP32 y);
    reading before any add after a reset is refused."""
    from paper_2311_15061_gb300 import sensai
    M, B, S, K = (512, 512), (10, 10), (1, 1), 128
    prm = O.params(M, B, S, K, seed=3)
    st = _state(prm, 0.3, 9)
    ctx = gpu_context(prm, np.ones(M, np.uint8))
    ctx.sensai_set_state(D=st.D.astype(np.float32), Z=st.Z, S=st.S.astype(np.float32), gamma_s=1.0)
    ctx.sensai_mean_reset()
    with pytest.raises(sensai.SensaiError) as err:
        ctx.sensai_mean_read()
    assert err.value.status == sensai.SENSAI_ESTATE
    for _ in range(3):
        ctx.sensai_mean_add()
    np.testing.assert_array_equal(ctx.sensai_mean_read(), ctx.sensai_reconstruct())
    ctx.close()


def test_posterior_mean_during_learning():
    """The intended use: learn, then add after each of the last T iterations;
    the mean is the average of the T reconstructions read one by one."""
    from parity_helpers import problem
    prm, x, clean, mask = problem((96, 80), (8, 8), (1, 1), 32, 0.25, seed=4)
    ctx = gpu_context(prm, mask)
    ctx.sensai_learn(x, 3)
    ctx.sensai_mean_reset()
    recs = []
    for _ in range(4):
        ctx.sensai_learn(None, 1)
        ctx.sensai_mean_add()
        recs.append(ctx.sensai_reconstruct().astype(np.float64))
    got = ctx.sensai_mean_read()
    ctx.close()
    want = np.mean(recs, axis=0)
    assert np.abs(got - want).max() <= 1e-6 * max(np.abs(want).max(), 1e-6)
