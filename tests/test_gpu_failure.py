"""Failure detection and checkpoint/resume on the GPU, with no GPU fault.

* Each kind of device-side wait (the dictionary kernel's grid barrier and the
  streamed sweep's mbarrier) is made to run out on a condition that nothing
  satisfies: it must give up within its ~1 s limit with SENSAI_ETIMEOUT, and
  the device must stay usable (a context learns and matches a fresh run
  afterwards).
* Checkpoint / resume: learning 3 iterations, exporting the state, importing
  it into a new context and learning 2 more gives bit for bit the state of 5
  uninterrupted iterations (the random numbers are counter-based).
* Allocation failures, injected on the host (SENSAI_FAULT=alloc:N fails the
  N-th device allocation of sensai_create as out of memory): every N gives
  ENOMEM until N exceeds the allocations made, nothing leaks, and a context
  created afterwards learns as a fresh one does.
"""
import time

import numpy as np
import pytest

from parity_helpers import gpu_context, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_15061_gb300 import build
    build.build()
    from paper_2311_15061_gb300 import sensai
    return sensai


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_gives_up_and_device_stays_usable(lib, which):
    t0 = time.perf_counter()
    assert lib.sensai_selftest_wait(which) == lib.SENSAI_ETIMEOUT
    dt = time.perf_counter() - t0
    assert dt < 30.0, dt
    prm, x, clean, mask = problem((48, 48), (8, 8), (1, 1), 16, 0.25, seed=1)
    a, b = gpu_context(prm, mask), gpu_context(prm, mask)
    a.sensai_learn(x, 2)
    b.sensai_learn(x, 2)
    np.testing.assert_array_equal(a.sensai_get_state()["D"], b.sensai_get_state()["D"])
    assert lib.sensai_selftest_wait(7) == lib.SENSAI_EINVAL


def test_checkpoint_resume_is_exact(lib):
    prm, x, clean, mask = problem((96, 96), (8, 8), (1, 1), 32, 0.2, seed=4)
    full = gpu_context(prm, mask)
    full.sensai_learn(x, 5)
    ref = full.sensai_get_state()
    first = gpu_context(prm, mask)
    first.sensai_learn(x, 3)
    ck = first.sensai_get_state()
    resumed = gpu_context(prm, mask)
    resumed.sensai_set_frame(x)
    resumed.sensai_set_state(D=ck["D"], Z=ck["Z"], S=ck["S"], pi=ck["pi"], gamma_s=ck["gamma_s"],
                             gamma_eps=ck["gamma_eps"], iter=ck["iter"])
    resumed.sensai_learn(None, 2)
    got = resumed.sensai_get_state()
    for key in ("D", "Z", "S", "pi"):
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
    assert got["gamma_s"] == ref["gamma_s"] and got["gamma_eps"] == ref["gamma_eps"] and got["iter"] == ref["iter"]


def test_injected_allocation_failures_free_everything(lib, monkeypatch):
    import torch
    prm, x, clean, mask = problem((64, 64), (8, 8), (1, 1), 16, 0.25, seed=2)
    ref = gpu_context(prm, mask)          # warm-up: the CUDA context and module loads
    ref.sensai_learn(x, 2)
    want = ref.sensai_get_state()
    ref.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for n in range(1, 200):
        monkeypatch.setenv("SENSAI_FAULT", f"alloc:{n}")
        try:
            ctx = gpu_context(prm, mask)
        except lib.SensaiError as err:
            assert err.status == lib.SENSAI_ENOMEM, (n, str(err))
            failed += 1
            continue
        ctx.close()                       # n is past the last allocation
        break
    else:
        raise AssertionError("creation never succeeded")
    assert failed >= 10, failed
    monkeypatch.delenv("SENSAI_FAULT")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < 64 << 20, (free0, free1)
    ctx = gpu_context(prm, mask)
    ctx.sensai_learn(x, 2)
    got = ctx.sensai_get_state()
    ctx.close()
    for key in ("D", "Z", "S"):
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)
