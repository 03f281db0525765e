"""Host-side checks of the C ABI (no GPU needed).

* libsensai.so builds for sm_103a and exports exactly the entry points that
  include/sensai.h declares (and nothing else under the sensai_ prefix).
* Argument validation happens before any CUDA call: invalid geometry returns
  SENSAI_EINVAL with a message, on machines with or without a GPU.
* The binding's ctypes structures have the header's layout: a C program
  compiled against include/sensai.h prints every structure's size and field
  offsets, which must equal the ctypes ones; likewise the status codes, the
  flags and the slice-size encoding.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_15061_gb300 import build
    build.build()
    from paper_2311_15061_gb300 import sensai
    return sensai


def _declared():
    text = open(os.path.join(ROOT, "include", "sensai.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sensai_[a-z_]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        getattr(lib._lib, n)  # raises AttributeError when missing
    assert sorted(lib.EXPORTED) == names


def test_no_undeclared_sensai_exports(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.library_path()], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    exported = sorted({l.split()[-1] for l in out.stdout.splitlines() if " sensai_" in l})
    assert exported == _declared()


@pytest.mark.parametrize("M,B,S,K", [
    ((10,), (4,), (4,), 8),          # (M - B) not divisible by the stride
    ((10,), (11,), (1,), 8),         # patch larger than the frame
    ((10, 10), (3, 3), (1, 1), 0),   # no atoms
    ((40, 40), (33, 33), (1, 1), 4), # P > 1024
])
def test_invalid_geometry_is_rejected(lib, M, B, S, K):
    prm = lib.make_params(M, B, S, K)
    mask = np.ones(M, np.uint8)
    h = ctypes.c_void_p()
    st = lib._lib.sensai_create(ctypes.byref(prm), mask.ctypes.data, ctypes.byref(h))
    assert st == lib.SENSAI_EINVAL
    assert h.value is None
    assert lib.sensai_last_error()


def test_invalid_hyperparameters_rejected(lib):
    prm = lib.make_params((16, 16), (4, 4), (1, 1), 8, c=0.0)
    mask = np.ones((16, 16), np.uint8)
    h = ctypes.c_void_p()
    assert lib._lib.sensai_create(ctypes.byref(prm), mask.ctypes.data, ctypes.byref(h)) == lib.SENSAI_EINVAL
    for flags in (0x40, lib.SENSAI_SLICE_ATOMS(8)):   # an unknown bit; a slice size without streaming
        prm = lib.make_params((16, 16), (4, 4), (1, 1), 8, flags=flags)
        assert lib._lib.sensai_create(ctypes.byref(prm), mask.ctypes.data, ctypes.byref(h)) == lib.SENSAI_EINVAL
    # the dense-statistics form: K <= 128 only, and not together with the per-chain form
    for K, flags in ((129, lib.SENSAI_FLAG_DENSE_STATISTICS), (200, lib.SENSAI_FLAG_TF32_STATISTICS),
                     (8, lib.SENSAI_FLAG_DENSE_STATISTICS | lib.SENSAI_FLAG_CHAIN_DICTIONARY)):
        prm = lib.make_params((16, 16), (4, 4), (1, 1), K, flags=flags)
        assert lib._lib.sensai_create(ctypes.byref(prm), mask.ctypes.data, ctypes.byref(h)) == lib.SENSAI_EINVAL
        assert "dense-statistics" in lib.sensai_last_error()


def test_null_context_is_an_error_not_a_crash(lib):
    assert lib._lib.sensai_learn(None, None, 1, None) == lib.SENSAI_EINVAL
    lib._lib.sensai_destroy(None)


# --- sensai_reconstruct_static: the checks made before anything touches the device ---

def _fake_ptr():
    # never dereferenced: every case below is rejected during argument checks
    return ctypes.c_void_p(256)


@pytest.mark.parametrize("M,B,S,K,what", [
    ((70000, 70000), (1, 1), (1, 1), 4, "frame too large"),       # 4.9e9 pixels >= 2^31
    ((2100, 2100), (1, 1), (1, 1), 4, "static scratch"),          # P * N = 4.41 M floats > 4.19 M
    ((40, 40), (33, 33), (1, 1), 4, "exceeds 1024"),              # P = 1089
    ((10,), (4,), (4,), 8, "geometry"),                           # stride does not divide M - B
])
def test_static_reconstruction_rejects_before_device(lib, M, B, S, K, what):
    prm = lib.make_params(M, B, S, K)
    st = lib._lib.sensai_reconstruct_static(ctypes.byref(prm), _fake_ptr(), _fake_ptr(), _fake_ptr(), None)
    assert st == lib.SENSAI_EINVAL
    assert what in lib.sensai_last_error()


def test_static_reconstruction_binding_checks_counts(lib):
    """The C side gets bare pointers, so the binding checks every element count
    (an undersized tensor would be read or written past its end)."""
    import torch
    M, B, S, K = (20, 18), (4, 3), (1, 1), 6
    prm = lib.make_params(M, B, S, K)
    P, N = 12, 17 * 16
    good = dict(D=torch.zeros(K * P), S=torch.zeros(N * K), out=torch.zeros(M))
    for name in good:
        args = dict(good)
        args[name] = torch.zeros(good[name].numel() - 1)
        with pytest.raises(ValueError, match=name):
            lib.sensai_reconstruct_static(prm, args["D"], args["S"], args["out"])
    with pytest.raises(TypeError, match="CUDA"):   # right sizes, host memory
        lib.sensai_reconstruct_static(prm, good["D"], good["S"], good["out"])


STRUCTS = ("sensai_params", "sensai_state", "sensai_stats", "sensai_serve_params")


def test_struct_layouts_match_header(lib, tmp_path):
    """Size and every field offset of the C structures (compiled by the host C
    compiler against the header) equal the binding's ctypes structures."""
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sensai.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, *_ in getattr(lib, name)._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name in STRUCTS:
        cls = getattr(lib, name)
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, *_ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_constants_match_header(lib, tmp_path):
    """Status codes, SENSAI_FLAG_* values and SENSAI_SLICE_ATOMS(n) as the
    header defines them equal the binding's."""
    header = open(os.path.join(ROOT, "include", "sensai.h")).read()
    names = sorted(set(re.findall(r"\b(SENSAI_(?:FLAG_[A-Z0-9_]+|OK|E[A-Z]+))\b", header)))
    assert "SENSAI_FLAG_DENSE_STATISTICS" in names and "SENSAI_ETIMEOUT" in names
    slices = (0, 8, 16, 104, 256, 2040)
    lines = ["#include <stdio.h>", '#include "sensai.h"', "int main(void) {"]
    lines += [f'    printf("{n} %lld\\n", (long long)({n}));' for n in names]
    lines += [f'    printf("SLICE{n} %lld\\n", (long long)SENSAI_SLICE_ATOMS({n}));' for n in slices]
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "constants.c", tmp_path / "constants"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.split("\n") if line)
    for n in names:
        assert int(out[n]) == getattr(lib, n), n
    for n in slices:
        assert int(out[f"SLICE{n}"]) == lib.SENSAI_SLICE_ATOMS(n), n
