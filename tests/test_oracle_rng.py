"""Pins for the oracle's random-number layer.

* Philox4x32-10 (Salmon et al., SC'11) equals Triton's independent Philox
  implementation, run in Triton's CPU interpreter, on random counters and keys.
* Box-Muller normals, Marsaglia-Tsang Gamma and the Gamma-ratio Beta match the
  textbook distributions (scipy.stats) by Kolmogorov-Smirnov and by moments.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle as O

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def kern(c_ptr, k_ptr, out_ptr, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c_ptr + 4 * i + 0); c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2); c3 = tl.load(c_ptr + 4 * i + 3)
    k0 = tl.load(k_ptr + 2 * i + 0); k1 = tl.load(k_ptr + 2 * i + 1)
    r0, r1, r2, r3 = tl.random.philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(out_ptr + 4 * i + 0, r0); tl.store(out_ptr + 4 * i + 1, r1)
    tl.store(out_ptr + 4 * i + 2, r2); tl.store(out_ptr + 4 * i + 3, r3)

inp = json.loads(sys.stdin.read())
ctr = torch.tensor(np.array(inp["ctr"], dtype=np.uint32).view(np.int32))
key = torch.tensor(np.array(inp["key"], dtype=np.uint32).view(np.int32))
ctr_u = ctr.view(torch.uint32) if hasattr(torch, "uint32") else ctr
key_u = key.view(torch.uint32) if hasattr(torch, "uint32") else key
out = torch.zeros_like(ctr_u)
kern[(1,)](ctr_u, key_u, out, len(inp["key"]) // 2)
print(json.dumps((out.view(torch.int32).numpy().view(np.uint32)).tolist()))
"""


def test_philox_matches_triton_interpreter():
    pytest.importorskip("triton")
    rng = np.random.default_rng(1234)
    n = 64
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(
        {"ctr": ctr.reshape(-1).tolist(), "key": key.reshape(-1).tolist()}),
        capture_output=True, text=True, env=env, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    ref = np.array(json.loads(res.stdout.strip().splitlines()[-1]), dtype=np.uint64).astype(np.uint32)
    ref = ref.reshape(n, 4)
    for j in range(n):
        np.testing.assert_array_equal(O.philox(ctr[j], key[j]), ref[j])


def test_philox_bits_are_balanced():
    # Every output bit of consecutive counters is set about half of the time.
    n = 20000
    outs = np.array([O.philox([j, 7, 3, 2], [11, 13]) for j in range(n)], dtype=np.uint64)
    bits = np.array([(outs >> b) & 1 for b in range(32)]).mean(axis=(1, 2))
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(4 * n))


def _normals(n, seed=5):
    return np.array([O.normal(seed, [j, 1, 2, O.TAG_D]) for j in range(n)])


def test_box_muller_is_standard_normal():
    x = _normals(100000)
    assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(x.mean()) < 5 / np.sqrt(len(x))
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / len(x))


def test_box_muller_pair_is_two_independent_normals():
    """The code draws' pair (cosine for the even atom, sine for the odd one):
    each component standard normal, uncorrelated, and their squared radius
    chi-square with 2 degrees of freedom (exponential, mean 2) -- which fails
    if both took the cosine or the radius were not shared."""
    n = 60000
    a = np.array([O.normal_pair(7, [j, 3, 5, O.TAG_ZS], 0) for j in range(n)])
    b = np.array([O.normal_pair(7, [j, 3, 5, O.TAG_ZS], 1) for j in range(n)])
    for x in (a, b):
        assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / np.sqrt(n)
    assert stats.kstest(a * a + b * b, stats.expon(scale=2.0).cdf).pvalue > 1e-3
    # independent of the words 0-1 normal of the same block
    c = np.array([O.normal(7, [j, 3, 5, O.TAG_ZS]) for j in range(n)])
    assert abs(np.corrcoef(a, c)[0, 1]) < 5 / np.sqrt(n)


@pytest.mark.parametrize("shape", [0.05, 0.3, 1.0, 2.5, 50.0, 3e4])
def test_gamma_matches_scipy(shape):
    n = 40000
    g = np.array([O.gamma(shape, 99, j, 0, 4, O.TAG_GS) for j in range(n)])
    assert np.all(g >= 0)
    assert stats.kstest(g, stats.gamma(shape).cdf).pvalue > 1e-3
    assert abs(g.mean() - shape) < 5 * np.sqrt(shape / n)


@pytest.mark.parametrize("ab", [(1.0, 5.0), (0.5, 0.5), (3.0, 2000.0), (40.0, 9.0)])
def test_beta_matches_scipy(ab):
    a, b = ab
    n = 30000
    x = np.array([O.beta(a, b, 3, j, 11) for j in range(n)])
    assert np.all((x >= 0) & (x <= 1))
    assert stats.kstest(x, stats.beta(a, b).cdf).pvalue > 1e-3
