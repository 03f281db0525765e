"""FP64 CPU oracle for BPFA inpainting -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with the CUDA path.

``build()`` compiles ``bpfa_oracle.c`` with gcc (OpenMP, -O2, no fast-math)
into ``liboracle.so`` beside it; ``lib()`` loads it (building on first use) and
the wrappers below take and return NumPy arrays.

Parity pins (tests/test_oracle_*.py): Philox against Triton's Philox
(interpreter mode), sampler moments against closed forms, the z-posterior of
the sparse-code sweep against exact enumeration, the dictionary conditional
against ridge least squares, overlap counts against brute force, overlap-add
of extracted patches against the frame, planted-dictionary recovery.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bpfa_oracle.c")
_HDR = os.path.join(_HERE, "bpfa_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

TAG_INIT, TAG_ZS, TAG_D, TAG_PI_A, TAG_PI_B, TAG_GS, TAG_GE = 1, 2, 3, 4, 5, 6, 7


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, strict FP64)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("M", ctypes.c_int64 * 4),
        ("B", ctypes.c_int32 * 4),
        ("S", ctypes.c_int32 * 4),
        ("K", ctypes.c_int32),
        ("a", ctypes.c_double), ("b", ctypes.c_double),
        ("c", ctypes.c_double), ("d", ctypes.c_double),
        ("e", ctypes.c_double), ("f", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("flags", ctypes.c_int32),
    ]


FLAG_GAMMA_S_FULL = 4   # reading A of the gamma_s update (prior draws for inactive s)


def params(M, B, S, K, *, a=None, b=None, c=1e-6, d=1e-6, e=1e-6, f=1e-6, seed=0, flags=0):
    """Model parameters; defaults a = K, b = N/8 (N = number of patches)."""
    prm = Params()
    prm.ndim = len(M)
    for i in range(len(M)):
        prm.M[i], prm.B[i], prm.S[i] = int(M[i]), int(B[i]), int(S[i])
    prm.K = int(K)
    n = 1
    for i in range(len(M)):
        n *= (int(M[i]) - int(B[i])) // int(S[i]) + 1
    prm.a = float(K if a is None else a)
    prm.b = float(n / 8.0 if b is None else b)
    prm.c, prm.d, prm.e, prm.f = float(c), float(d), float(e), float(f)
    prm.seed = int(seed)
    prm.flags = int(flags)
    return prm


def _p(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = ctypes.CDLL(build())
    P = ctypes.POINTER
    dbl, i64, u8, f32, u32, i32 = (ctypes.c_double, ctypes.c_int64, ctypes.c_uint8,
                                   ctypes.c_float, ctypes.c_uint32, ctypes.c_int32)
    pp = P(Params)
    sig = {
        "orc_check": (ctypes.c_int, [pp]),
        "orc_num_patches": (i64, [pp]),
        "orc_patch_size": (i64, [pp]),
        "orc_frame_size": (i64, [pp]),
        "orc_philox": (None, [P(u32), P(u32), P(u32)]),
        "orc_normal": (dbl, [ctypes.c_uint64, P(u32)]),
        "orc_normal_pair": (dbl, [ctypes.c_uint64, P(u32), ctypes.c_int]),
        "orc_gamma": (dbl, [dbl, ctypes.c_uint64, u32, u32, u32, u32]),
        "orc_beta": (dbl, [dbl, dbl, ctypes.c_uint64, u32, u32]),
        "orc_overlap_counts": (None, [pp, P(i32)]),
        "orc_patch_origins": (None, [pp, P(i64)]),
        "orc_pixel_offsets": (None, [pp, P(i64)]),
        "orc_init_dictionary": (None, [pp, P(dbl)]),
        "orc_init_gamma_eps": (dbl, [pp, P(f32), P(u8)]),
        "orc_zs_sweep": (None, [pp, P(f32), P(u8), P(dbl), P(u8), P(dbl), P(dbl), dbl, dbl, i64, P(dbl)]),
        "orc_zs_sweep_subset": (None, [pp, P(f32), P(u8), P(dbl), P(u8), P(dbl), P(dbl), dbl, dbl, i64,
                                       P(i64), i64, P(dbl), P(dbl)]),
        "orc_d_sweep": (None, [pp, P(f32), P(u8), P(dbl), P(u8), P(dbl), dbl, i64]),
        "orc_hyper": (None, [pp, P(f32), P(u8), P(dbl), P(u8), P(dbl), P(dbl), P(dbl), P(dbl), i64, P(dbl)]),
        "orc_reconstruct": (None, [pp, P(dbl), P(u8), P(dbl), P(dbl)]),
        "orc_reconstruct_mean": (None, [pp, ctypes.c_int, P(dbl), P(u8), P(dbl), P(dbl)]),
        "orc_num_threads": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------- wrappers --

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def normal(seed, ctr):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    return lib().orc_normal(seed, _p(c, ctypes.c_uint32))


def normal_pair(seed, ctr, second):
    """Normal of the Box-Muller pair from words 2-3 of the block at ctr (the
    code draws' pair: cosine for the even atom, sine for the odd one)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    return lib().orc_normal_pair(seed, _p(c, ctypes.c_uint32), int(second))


def gamma(shape, seed, c0, c1, t, tag):
    return lib().orc_gamma(shape, seed, c0, c1, t, tag)


def beta(alpha, beta_, seed, c0, t):
    return lib().orc_beta(alpha, beta_, seed, c0, t)


def check(prm):
    return lib().orc_check(ctypes.byref(prm))


def num_patches(prm):
    return lib().orc_num_patches(ctypes.byref(prm))


def patch_size(prm):
    return lib().orc_patch_size(ctypes.byref(prm))


def overlap_counts(prm):
    shape = tuple(prm.M[i] for i in range(prm.ndim))
    out = np.zeros(shape, dtype=np.int32)
    lib().orc_overlap_counts(ctypes.byref(prm), _p(out, ctypes.c_int32))
    return out


def patch_origins(prm):
    out = np.zeros(num_patches(prm), dtype=np.int64)
    lib().orc_patch_origins(ctypes.byref(prm), _p(out, ctypes.c_int64))
    return out


def pixel_offsets(prm):
    out = np.zeros(patch_size(prm), dtype=np.int64)
    lib().orc_pixel_offsets(ctypes.byref(prm), _p(out, ctypes.c_int64))
    return out


class State:
    """Sampler state: D (K x P), Z (N x K uint8), S (N x K), pi, gamma_s, gamma_eps, t."""

    def __init__(self, prm, D=None, Z=None, S=None, pi=None, gamma_s=1.0, gamma_eps=None, t=0):
        N, P, K = num_patches(prm), patch_size(prm), prm.K
        self.prm = prm
        if D is None:
            D = np.zeros((K, P), dtype=np.float64)
            lib().orc_init_dictionary(ctypes.byref(prm), _p(D, ctypes.c_double))
        self.D = np.ascontiguousarray(D, dtype=np.float64).copy()
        self.Z = np.zeros((N, K), np.uint8) if Z is None else np.ascontiguousarray(Z, np.uint8).copy()
        self.S = np.zeros((N, K), np.float64) if S is None else np.ascontiguousarray(S, np.float64).copy()
        self.pi = np.full(K, 0.5) if pi is None else np.ascontiguousarray(pi, np.float64).copy()
        self.gamma_s = float(gamma_s)
        self.gamma_eps = gamma_eps
        self.t = int(t)

    def copy(self):
        return State(self.prm, self.D, self.Z, self.S, self.pi, self.gamma_s, self.gamma_eps, self.t)


def init_gamma_eps(prm, x, mask):
    x = np.ascontiguousarray(x, np.float32)
    m = np.ascontiguousarray(mask, np.uint8)
    return lib().orc_init_gamma_eps(ctypes.byref(prm), _p(x, ctypes.c_float), _p(m, ctypes.c_uint8))


def zs_sweep(st, x, mask):
    x = np.ascontiguousarray(x, np.float32)
    m = np.ascontiguousarray(mask, np.uint8)
    if st.gamma_eps is None:
        st.gamma_eps = init_gamma_eps(st.prm, x, m)
    stats = np.zeros(3)
    lib().orc_zs_sweep(ctypes.byref(st.prm), _p(x, ctypes.c_float), _p(m, ctypes.c_uint8),
                       _p(st.D, ctypes.c_double), _p(st.Z, ctypes.c_uint8), _p(st.S, ctypes.c_double),
                       _p(st.pi, ctypes.c_double), st.gamma_s, st.gamma_eps, st.t, _p(stats, ctypes.c_double))
    return stats


def zs_sweep_subset(st, x, mask, patches=None, want_logodds=False):
    """Sweep only ``patches`` (all if None); returns (stats, logodds or None)."""
    x = np.ascontiguousarray(x, np.float32)
    m = np.ascontiguousarray(mask, np.uint8)
    if st.gamma_eps is None:
        st.gamma_eps = init_gamma_eps(st.prm, x, m)
    stats = np.zeros(3)
    L = np.full(st.Z.shape, np.nan) if want_logodds else None
    idx = None if patches is None else np.ascontiguousarray(patches, np.int64)
    lib().orc_zs_sweep_subset(
        ctypes.byref(st.prm), _p(x, ctypes.c_float), _p(m, ctypes.c_uint8), _p(st.D, ctypes.c_double),
        _p(st.Z, ctypes.c_uint8), _p(st.S, ctypes.c_double), _p(st.pi, ctypes.c_double), st.gamma_s,
        st.gamma_eps, st.t, None if idx is None else _p(idx, ctypes.c_int64), -1 if idx is None else len(idx),
        None if L is None else _p(L, ctypes.c_double), _p(stats, ctypes.c_double))
    return stats, L


def d_sweep(st, x, mask):
    x = np.ascontiguousarray(x, np.float32)
    m = np.ascontiguousarray(mask, np.uint8)
    lib().orc_d_sweep(ctypes.byref(st.prm), _p(x, ctypes.c_float), _p(m, ctypes.c_uint8),
                      _p(st.D, ctypes.c_double), _p(st.Z, ctypes.c_uint8), _p(st.S, ctypes.c_double),
                      st.gamma_eps, st.t)


def hyper(st, x, mask):
    x = np.ascontiguousarray(x, np.float32)
    m = np.ascontiguousarray(mask, np.uint8)
    gs = ctypes.c_double(st.gamma_s)
    ge = ctypes.c_double(st.gamma_eps)
    stats = np.zeros(4)
    lib().orc_hyper(ctypes.byref(st.prm), _p(x, ctypes.c_float), _p(m, ctypes.c_uint8),
                    _p(st.D, ctypes.c_double), _p(st.Z, ctypes.c_uint8), _p(st.S, ctypes.c_double),
                    _p(st.pi, ctypes.c_double), ctypes.byref(gs), ctypes.byref(ge), st.t,
                    _p(stats, ctypes.c_double))
    st.gamma_s, st.gamma_eps = gs.value, ge.value
    return stats


def learn(st, x, mask, iters, callback=None):
    """``iters`` full Gibbs iterations: codes, dictionary, then pi / gammas."""
    for _ in range(iters):
        zs_sweep(st, x, mask)
        d_sweep(st, x, mask)
        stats = hyper(st, x, mask)
        if callback is not None:
            callback(st, stats)
        st.t += 1
    return st


def inpaint_sweeps(st, x, mask, sweeps):
    """Sparse coding with the dictionary held fixed: codes then pi / gammas."""
    for _ in range(sweeps):
        zs_sweep(st, x, mask)
        hyper(st, x, mask)
        st.t += 1
    return st


def reconstruct(st):
    shape = tuple(st.prm.M[i] for i in range(st.prm.ndim))
    out = np.zeros(shape, dtype=np.float64)
    lib().orc_reconstruct(ctypes.byref(st.prm), _p(st.D, ctypes.c_double), _p(st.Z, ctypes.c_uint8),
                          _p(st.S, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def reconstruct_mean(states):
    """Posterior-mean reconstruction: the mean of the overlap-add
    reconstructions of the given samples (states of one chain)."""
    prm = states[0].prm
    shape = tuple(prm.M[i] for i in range(prm.ndim))
    D = np.ascontiguousarray(np.stack([st.D for st in states]), np.float64)
    Z = np.ascontiguousarray(np.stack([st.Z for st in states]), np.uint8)
    S = np.ascontiguousarray(np.stack([st.S for st in states]), np.float64)
    out = np.zeros(shape, dtype=np.float64)
    lib().orc_reconstruct_mean(ctypes.byref(prm), len(states), _p(D, ctypes.c_double), _p(Z, ctypes.c_uint8),
                               _p(S, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def psnr(estimate, reference):
    """10 log10(1 / MSE) over all pixels, in FP64 (peak value 1)."""
    err = np.asarray(estimate, np.float64) - np.asarray(reference, np.float64)
    mse = float(np.mean(err * err))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def num_threads():
    return lib().orc_num_threads()
