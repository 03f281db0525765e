"""GPU tests of the live serving engine (sensai_serve_start / sensai_submit_frame).

* A frame's result is bit-identical when served alone and when served among
  many concurrent frames of other sizes, masks and streams (continuous
  batching must not change results).
* A served frame equals sensai_inpaint on a context keyed by the frame's own
  seed h(h(h(seed) ^ stream) ^ frame), h = SplitMix64's finaliser (written out
  here from its published definition), and the oracle's inpainting with that
  key reaches the same PSNR within 0.1 dB on average.
* Memory-based admission: a budget that fits one large frame at a time still
  completes every frame with the same results; a frame larger than the engine
  accepts is rejected with EINVAL.
* A dictionary too large for shared memory (K = 256 atoms of 16x16 pixels)
  is streamed in slices when serving too, with the same results as
  sensai_inpaint.
"""
import threading

import numpy as np
import pytest

import oracle as O
from parity_helpers import gpu_context, problem, push_state

pytestmark = pytest.mark.gpu

MASK64 = (1 << 64) - 1


def _splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _frame_seed(seed, stream_id, frame_id):
    h = _splitmix64(seed)
    h = _splitmix64(h ^ (stream_id & 0xFFFFFFFF))
    return _splitmix64(h ^ frame_id)


@pytest.fixture(scope="module")
def learned():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_15061_gb300 import build
    build.build()
    from paper_2311_15061_gb300 import sensai
    prm, x, clean, mask = problem((128, 128), (8, 8), (1, 1), 32, 0.25, seed=0)
    # a = 0, b = 0: the defaults a = K, b = N / 8 taken per frame
    ctx = sensai.Context(sensai.make_params((128, 128), (8, 8), (1, 1), 32, seed=prm.seed), mask)
    ctx.sensai_learn(x, 6)
    st = ctx.sensai_get_state()
    return prm, ctx, st


def _frames(seed, shapes):
    from paper_2311_15061_gb300 import synth
    out = []
    for j, shp in enumerate(shapes):
        x, clean = synth.stem_frame(shp, seed + j, drift=(0.0, 0.3 * j))
        m = synth.random_mask(shp, 0.05 + 0.15 * ((j * 7) % 10) / 10.0, seed + j) if j % 2 == 0 \
            else synth.line_hop_mask(shp, 0.1, seed + j)
        out.append((x, clean, m))
    return out


def _serve(ctx, items, sweeps=3):
    """items: (stream_id, frame_id, x, mask); returns {(stream, frame): out}."""
    done = {}
    lock = threading.Lock()

    def on_done(fid, status, out):
        with lock:
            done[fid] = status

    outs = {}
    for sid, fid, x, m in items:
        outs[(sid, fid)] = ctx.sensai_submit_frame(sid, fid, x, m, sweeps, done=on_done)
    ctx.sensai_serve_drain()
    assert all(v == 0 for v in done.values()), done
    assert len(done) == len(items)
    return outs


def test_same_result_alone_and_in_the_mix(learned):
    prm, ctx, st = learned
    ctx.sensai_serve_start(slots=4, max_pixels=256 * 256)
    (x, clean, m), = _frames(40, [(160, 200)])
    alone = _serve(ctx, [(3, 77, x, m)])[(3, 77)].copy()
    others = _frames(50, [(256, 256), (96, 128), (200, 120), (256, 256), (64, 64), (128, 176)] * 2)
    items = [(j % 4, 1000 + j, ox, om) for j, (ox, oc, om) in enumerate(others)]
    items.insert(5, (3, 77, x, m))
    mixed = _serve(ctx, items)[(3, 77)]
    ctx.sensai_serve_stop()
    np.testing.assert_array_equal(alone, mixed)
    assert np.isfinite(alone).all()


def test_served_frame_equals_inpaint_and_tracks_oracle(learned):
    prm, ctx, st = learned
    ctx.sensai_serve_start(slots=2, max_pixels=128 * 128)
    frames = _frames(60, [(128, 128), (112, 96), (128, 128)])
    diffs = []
    for j, (x, clean, m) in enumerate(frames):
        served = _serve(ctx, [(1, j, x, m)])[(1, j)]
        fseed = _frame_seed(prm.seed, 1, j)
        p2, _, _, _ = problem(x.shape, (8, 8), (1, 1), 32, 0.2, seed=0)
        p2.seed = fseed
        c2 = gpu_context(p2, m)
        c2.sensai_set_state(D=st["D"], pi=st["pi"], gamma_s=st["gamma_s"], gamma_eps=st["gamma_eps"],
                            iter=st["iter"])
        ref = np.empty(x.shape, np.float32)
        c2.sensai_inpaint(x, 3, ref)
        c2.close()
        np.testing.assert_array_equal(served, ref)
        ost = O.State(p2, D=st["D"].astype(np.float64), pi=st["pi"], gamma_s=st["gamma_s"],
                      gamma_eps=st["gamma_eps"], t=st["iter"])
        O.inpaint_sweeps(ost, x, m, 3)
        diffs.append(O.psnr(served, clean) - O.psnr(O.reconstruct(ost), clean))
    ctx.sensai_serve_stop()
    assert abs(np.mean(diffs)) <= 0.1, diffs


def test_memory_admission_and_rejection(learned):
    from paper_2311_15061_gb300 import sensai
    prm, ctx, st = learned
    ctx.sensai_serve_start(slots=3, max_pixels=256 * 256)
    frames = _frames(70, [(256, 256), (128, 128), (256, 256)])
    items = [(0, j, x, m) for j, (x, c, m) in enumerate(frames)]
    free = _serve(ctx, items)
    ctx.sensai_serve_stop()
    # a budget that holds one 256x256 frame (~33 MB here) but not two
    ctx.sensai_serve_start(slots=3, max_pixels=256 * 256, memory_budget=36 * 1024 * 1024)
    tight = _serve(ctx, items)
    with pytest.raises(sensai.SensaiError) as err:
        big = np.zeros((300, 300), np.float32)
        ctx.sensai_submit_frame(0, 99, big, np.ones((300, 300), np.uint8), 3)
    assert err.value.status == sensai.SENSAI_EINVAL
    ctx.sensai_serve_stop()
    for key in free:
        np.testing.assert_array_equal(free[key], tight[key])


def test_serving_with_streamed_dictionary():
    from paper_2311_15061_gb300 import sensai, synth
    M, B, K = (48, 48), (16, 16), 256
    x, clean = synth.stem_frame(M, 3)
    mask = synth.random_mask(M, 0.15, 3)
    ctx = sensai.Context(sensai.make_params(M, B, (1, 1), K, seed=5), mask)
    ctx.sensai_learn(x, 2)
    assert ctx.sensai_get_stats().slices >= 2
    st = ctx.sensai_get_state()
    ctx.sensai_serve_start(slots=2, max_pixels=64 * 64, max_observed=96)
    frames = [(synth.stem_frame((56, 52), 10 + j)[0], synth.random_mask((56, 52), 0.12, 10 + j)) for j in range(3)]
    served = _serve(ctx, [(2, j, fx, fm) for j, (fx, fm) in enumerate(frames)])
    ctx.sensai_serve_stop()
    for j, (fx, fm) in enumerate(frames):
        p = sensai.make_params((56, 52), B, (1, 1), K, seed=_frame_seed(5, 2, j))
        c2 = sensai.Context(p, fm)
        c2.sensai_set_state(D=st["D"], pi=st["pi"], gamma_s=st["gamma_s"], gamma_eps=st["gamma_eps"], iter=st["iter"])
        ref = np.empty((56, 52), np.float32)
        c2.sensai_inpaint(fx, 3, ref)
        c2.close()
        np.testing.assert_array_equal(served[(2, j)], ref)


def test_serving_with_full_gamma_s_reading():
    """SENSAI_FLAG_GAMMA_S_FULL carries into serving: each served frame runs
    the prior-draw pass after its code sweeps and equals sensai_inpaint on a
    context with the same flag and the frame's seed."""
    from paper_2311_15061_gb300 import sensai, synth
    M, B, K = (48, 48), (8, 8), 32
    flags = sensai.SENSAI_FLAG_GAMMA_S_FULL
    x, clean = synth.stem_frame(M, 4)
    mask = synth.random_mask(M, 0.2, 4)
    ctx = sensai.Context(sensai.make_params(M, B, (1, 1), K, seed=6, flags=flags), mask)
    ctx.sensai_learn(x, 2)
    st = ctx.sensai_get_state()
    ctx.sensai_serve_start(slots=2, max_pixels=64 * 64, max_observed=64)
    frames = [(synth.stem_frame((52, 56), 20 + j)[0], synth.random_mask((52, 56), 0.15, 20 + j)) for j in range(3)]
    served = _serve(ctx, [(3, j, fx, fm) for j, (fx, fm) in enumerate(frames)])
    ctx.sensai_serve_stop()
    ctx.close()
    for j, (fx, fm) in enumerate(frames):
        for f, same in ((flags, True), (0, False)):
            p = sensai.make_params((52, 56), B, (1, 1), K, seed=_frame_seed(6, 3, j), flags=f)
            c2 = sensai.Context(p, fm)
            c2.sensai_set_state(D=st["D"], pi=st["pi"], gamma_s=st["gamma_s"], gamma_eps=st["gamma_eps"],
                                iter=st["iter"])
            ref = np.empty((52, 56), np.float32)
            c2.sensai_inpaint(fx, 3, ref)
            c2.close()
            if same:
                np.testing.assert_array_equal(served[(3, j)], ref)
            else:   # the default reading draws other gamma_s values, so other codes
                assert not np.array_equal(served[(3, j)], ref)
