"""GPU test of sensai_reconstruct_static, the reconstruction entry point that
allocates no device memory.

Some callers cannot allocate GPU memory: a plugin running inside a host
application whose memory pool owns the whole device, or a live-acquisition
callback with a hard time budget in which cudaMalloc (which may block and
synchronise the device) is not allowed.  They hand the library their own
device buffers; the only scratch, the per-patch reconstructions, sits in a
fixed 16 MiB static device array inside libsensai.

The test calls the entry point through the C ABI and compares its output with
the context-based sensai_reconstruct on the same dictionary and codes, within
the reconstruction tolerance of the other GPU tests (1e-5 of the frame's
largest value), on two calls in a row with different codes: the static
scratch keeps the previous call's contents, which must not leak into the next
result.  The file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sensai():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_15061_gb300 import build
    build.build()
    from paper_2311_15061_gb300 import sensai as s
    return s


@pytest.mark.parametrize("M,B,S,K", [
    ((96, 80), (8, 6), (1, 2), 24),          # 2-D, stride 2 on the last axis
    ((6, 20, 21), (2, 4, 3), (2, 2, 3), 7),  # 3-D, strides on every axis
    ((48, 40), (6, 5), (3, 5), 9),           # stride 5 on the last axis
    ((263, 263), (8, 8), (1, 1), 12),        # P * N = 4,194,304: the whole static scratch
])
def test_static_reconstruction_matches_context_path(sensai, M, B, S, K):
    import torch
    from paper_2311_15061_gb300 import synth
    mask = synth.random_mask(M, 0.3, 0)
    prm = sensai.make_params(M, B, S, K)
    ctx = sensai.Context(prm, mask)
    N, P = ctx.N, ctx.P
    rng = np.random.default_rng(7)
    out = torch.full(M, float("nan"), dtype=torch.float32, device="cuda")
    for call in range(2):
        D = (rng.standard_normal((K, P)) / np.sqrt(P)).astype(np.float32)
        Z = (rng.random((N, K)) < 0.2 + 0.3 * call).astype(np.uint8)
        Sv = (rng.standard_normal((N, K)) * Z).astype(np.float32)
        ctx.sensai_set_state(D=D, Z=Z, S=Sv, gamma_s=1.0)
        ref = ctx.sensai_reconstruct()
        Dt = torch.from_numpy(D).cuda()
        St = torch.from_numpy(Sv).cuda()
        sensai.sensai_reconstruct_static(prm, Dt, St, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1e-6), call
    ctx.close()


def test_static_reconstruction_rejects_oversized_problems(sensai):
    import torch
    prm = sensai.make_params((2100, 2100), (1, 1), (1, 1), 4)   # P * N = 4.41 M floats > 4.19 M
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):   # the binding checks the element counts first
        sensai.sensai_reconstruct_static(prm, small, small, small)
    import ctypes                     # the C side rejects the size before any launch
    p = small.data_ptr()
    st = sensai._lib.sensai_reconstruct_static(ctypes.byref(prm), p, p, p, None)
    assert st == sensai.SENSAI_EINVAL
    assert "static scratch" in sensai.sensai_last_error()


def test_static_reconstruction_rejects_host_memory(sensai):
    """Host pointers reach the C side only through the raw ABI (the binding
    refuses them earlier); the entry point rejects them without a launch."""
    import ctypes
    import torch
    M, B, S, K = (20, 18), (4, 3), (1, 1), 6
    prm = sensai.make_params(M, B, S, K)
    D = torch.zeros(K * 12, device="cuda")
    Sv = torch.zeros(17 * 16 * K, device="cuda")
    host_out = np.zeros(M, np.float32)
    st = sensai._lib.sensai_reconstruct_static(ctypes.byref(prm), D.data_ptr(), Sv.data_ptr(),
                                               host_out.ctypes.data, None)
    assert st == sensai.SENSAI_EINVAL
    assert "current device" in sensai.sensai_last_error()
