"""GPU test of the per-iteration metrics trace (sensai_trace): one JSON line
per Gibbs iteration whose draws, counts and PSNR equal what the context
reports after that iteration, and a chain that does not depend on tracing."""
import json

import numpy as np
import pytest

import oracle as O
from parity_helpers import gpu_context, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_15061_gb300 import build
    build.build()


def test_trace_lines_match_the_state(tmp_path):
    prm, x, clean, mask = problem((128, 128), (8, 8), (1, 1), 64, 0.25, 2)
    path = tmp_path / "trace.jsonl"
    ctx = gpu_context(prm, mask)
    ctx.sensai_trace(path, clean)
    ctx.sensai_learn(x, 3)
    st = ctx.sensai_get_state()
    stats = ctx.sensai_get_stats()
    rec = ctx.sensai_reconstruct()
    out = np.empty_like(x)
    ctx.sensai_inpaint(x, 2, out)
    ctx.sensai_trace(None)
    ctx.sensai_learn(x, 1)          # not traced
    ctx.close()
    lines = [json.loads(line) for line in open(path)]
    assert [ln["t"] for ln in lines] == [0, 1, 2, 3, 4]
    assert [ln["mode"] for ln in lines] == ["learn"] * 3 + ["inpaint"] * 2
    third = lines[2]
    assert third["gamma_s"] == st["gamma_s"] and third["gamma_eps"] == st["gamma_eps"]
    assert third["active"] == stats.n_active == int(st["Z"].sum())
    assert third["active_per_patch"] == pytest.approx(stats.n_active / st["Z"].shape[0], rel=1e-9)
    assert third["psnr_db"] == pytest.approx(O.psnr(rec, clean), abs=1e-9)
    assert lines[-1]["psnr_db"] == pytest.approx(O.psnr(out, clean), abs=1e-9)
    assert all(ln["wall_ms"] >= 0 for ln in lines)

    # the same chain without tracing
    ctx = gpu_context(prm, mask)
    ctx.sensai_learn(x, 3)
    ref = ctx.sensai_get_state()
    ctx.close()
    for key in ("D", "Z", "S", "pi"):
        np.testing.assert_array_equal(ref[key], st[key], err_msg=key)


def test_trace_without_ground_truth_and_bad_path(tmp_path):
    from paper_2311_15061_gb300 import sensai
    prm, x, clean, mask = problem((64, 64), (8, 8), (1, 1), 16, 0.25, 1)
    ctx = gpu_context(prm, mask)
    path = tmp_path / "t.jsonl"
    ctx.sensai_trace(path)
    ctx.sensai_learn(x, 2)
    ctx.sensai_trace(None)
    lines = [json.loads(line) for line in open(path)]
    assert len(lines) == 2 and all(ln["psnr_db"] is None for ln in lines)
    with pytest.raises(sensai.SensaiError) as err:
        ctx.sensai_trace(tmp_path / "missing_dir" / "t.jsonl")
    assert err.value.status == sensai.SENSAI_EINVAL
    ctx.close()
