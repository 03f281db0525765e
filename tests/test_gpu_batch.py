"""GPU tests of batches (sensai_batch_*): many independent contexts learned
together under one captured CUDA graph.

* A batch of heterogeneous instances (1-D, 2-D and 3-D, different K, P,
  masks, strides, one streamed dictionary, one with two lanes per patch)
  ends bit for bit where sensai_learn on
  each instance alone ends: codes, dictionary, pi, gammas and reconstruction.
* Repeated replays advance the iteration index (3 + 2 batch iterations equal
  5 single ones), and tuning, whose trials are real iterations with narrower
  code-sweep grids, leaves the results unchanged.
* A context with the cooperative dictionary kernel, or listed twice, is
  rejected with EINVAL.
"""
import numpy as np
import pytest

from parity_helpers import problem

pytestmark = pytest.mark.gpu

CASES = [
    dict(M=(64, 64), B=(8, 8), S=(1, 1), K=32, frac=0.25, seed=0),
    dict(M=(96, 80), B=(6, 6), S=(1, 1), K=16, frac=0.1, seed=1),
    dict(M=(10, 24, 20), B=(2, 4, 4), S=(2, 1, 1), K=24, frac=0.3, seed=2),
    dict(M=(48, 48), B=(16, 16), S=(1, 1), K=256, frac=0.1, seed=3),   # streamed dictionary
    dict(M=(128, 96), B=(8, 8), S=(1, 1), K=64, frac=0.05, seed=4),
    dict(M=(333,), B=(9,), S=(2,), K=8, frac=0.4, seed=5),
    dict(M=(40, 40), B=(12, 12), S=(1, 1), K=16, frac=1.0, seed=6),   # |Omega_i| = 144: two lanes per patch
]


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_15061_gb300 import build
    build.build()
    from paper_2311_15061_gb300 import sensai
    return sensai


def _contexts(lib, extra_flags=0):
    out = []
    for c in CASES:
        prm, x, clean, mask = problem(c["M"], c["B"], c["S"], c["K"], c["frac"], seed=c["seed"])
        p = lib.make_params(c["M"], c["B"], c["S"], c["K"], seed=c["seed"],
                            flags=lib.SENSAI_FLAG_CHAIN_DICTIONARY | extra_flags)
        ctx = lib.Context(p, mask)
        ctx.sensai_set_frame(x)
        out.append(ctx)
    return out


def _state(ctx):
    g = ctx.sensai_get_state()
    g["rec"] = ctx.sensai_reconstruct()
    return g


def _assert_same(a, b):
    for key in ("D", "Z", "S", "pi", "rec"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    for key in ("gamma_s", "gamma_eps", "iter"):
        assert a[key] == b[key], key


def test_batch_equals_individual_learning(lib):
    batched, alone = _contexts(lib), _contexts(lib)
    b = lib.Batch(batched)
    b.sensai_batch_learn(3)
    b.sensai_batch_learn(2)
    b.close()
    for cb, ca in zip(batched, alone):
        ca.sensai_learn(None, 5)
        _assert_same(_state(cb), _state(ca))
    assert batched[3].sensai_get_stats().slices >= 2   # the streamed instance really streamed


@pytest.mark.parametrize("which", [0, 2])
def test_batch_member_matches_oracle(lib, which):
    """One batched Gibbs iteration of one member, from an oracle state,
    against the oracle: the codes by the flip rule and 1e-5 on s; the
    dictionary and then pi / gammas conditioned on the GPU's codes (and
    dictionary), so that a near-threshold flip does not change the path."""
    import oracle as O
    from parity_helpers import (D_TOL, S_TOL, compare_codes, dict_errors, oracle_state, push_state,
                                round_state)
    c = CASES[which]
    prm, x, clean, mask = problem(c["M"], c["B"], c["S"], c["K"], c["frac"], seed=c["seed"])
    st = oracle_state(prm, x, mask, 2)
    members = _contexts(lib)
    ctx = members[which]
    push_state(ctx, st, x)
    b = lib.Batch(members)
    b.sensai_batch_learn(1)
    b.close()
    g = ctx.sensai_get_state()
    assert g["iter"] == st.t + 1
    ost = st.copy()
    _, L = O.zs_sweep_subset(ost, x, mask, want_logodds=True)
    nflip, serr = compare_codes(st, g, ost, L)
    assert nflip <= max(3, 1e-4 * ost.Z.shape[0]), nflip
    assert serr <= S_TOL, serr
    od = round_state(O.State(prm, D=st.D, Z=g["Z"], S=g["S"].astype(np.float64), pi=st.pi,
                             gamma_s=st.gamma_s, gamma_eps=st.gamma_eps, t=st.t))
    O.d_sweep(od, x, mask)
    assert dict_errors(g["D"], od.D).max() <= D_TOL
    oh = round_state(O.State(prm, D=g["D"].astype(np.float64), Z=g["Z"], S=g["S"].astype(np.float64),
                             pi=st.pi, gamma_s=st.gamma_s, gamma_eps=st.gamma_eps, t=st.t))
    O.hyper(oh, x, mask)
    np.testing.assert_allclose(g["pi"], oh.pi, rtol=1e-9)
    # here the s^2 sum behind gamma_s is the sweep's own (FP32 per patch, over
    # K atoms), not a sum of pushed values: ~1e-7 relative per patch
    assert abs(g["gamma_s"] / oh.gamma_s - 1) <= 1e-6
    assert abs(g["gamma_eps"] / oh.gamma_eps - 1) <= 1e-5


def test_tuning_keeps_results(lib):
    batched, alone = _contexts(lib), _contexts(lib)
    b = lib.Batch(batched)
    div = b.sensai_batch_tune(1)
    assert div in (1, 2, 4, 8, 16)
    b.sensai_batch_learn(2)
    b.close()
    for cb, ca in zip(batched, alone):
        ca.sensai_learn(None, 5 * 2 + 2)
        _assert_same(_state(cb), _state(ca))


def test_batch_rejects_cooperative_duplicate_and_full_reading_contexts(lib):
    prm, x, clean, mask = problem((64, 64), (8, 8), (1, 1), 16, 0.25)
    coop = lib.Context(lib.make_params((64, 64), (8, 8), (1, 1), 16), mask)
    chain = lib.Context(lib.make_params((64, 64), (8, 8), (1, 1), 16, flags=lib.SENSAI_FLAG_CHAIN_DICTIONARY), mask)
    full = lib.Context(lib.make_params((64, 64), (8, 8), (1, 1), 16, flags=lib.SENSAI_FLAG_CHAIN_DICTIONARY
                                       | lib.SENSAI_FLAG_GAMMA_S_FULL), mask)
    for members in ([coop], [chain, chain], [chain, full]):
        with pytest.raises(lib.SensaiError) as err:
            lib.Batch(members)
        assert err.value.status == lib.SENSAI_EINVAL
