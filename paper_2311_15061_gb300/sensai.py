"""Thin ctypes binding of libsensai.so (include/sensai.h).

Every function keeps its C name and only marshals arguments: NumPy arrays are
host buffers, CUDA torch tensors are device buffers (``data_ptr()``), streams
are ``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or ``None``
(legacy default stream).  All arithmetic runs in the library's CUDA kernels;
there is no CPU fallback.  Importing this module raises ``ImportError`` when
the library has not been built (``paper_2311_15061_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsensai.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libsensai.so not built at {_LIB_PATH}; run paper_2311_15061_gb300.build.build()")
_lib = ctypes.CDLL(_LIB_PATH)

SENSAI_OK, SENSAI_EINVAL, SENSAI_ENOMEM, SENSAI_ECUDA, SENSAI_ETIMEOUT, SENSAI_EBUSY, SENSAI_ESTATE = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EBUSY", "ESTATE"]

EXPORTED = [
    "sensai_create", "sensai_destroy", "sensai_set_frame", "sensai_reset", "sensai_learn",
    "sensai_inpaint", "sensai_sweep_codes", "sensai_draw_dictionary", "sensai_draw_hyper",
    "sensai_reconstruct", "sensai_mean_reset", "sensai_mean_add", "sensai_mean_read", "sensai_overlap_counts",
    "sensai_get_dictionary", "sensai_set_dictionary",
    "sensai_get_state", "sensai_set_state", "sensai_get_stats", "sensai_trace", "sensai_profile",
    "sensai_profile_read",
    "sensai_reconstruct_static", "sensai_serve_start", "sensai_submit_frame", "sensai_serve_drain",
    "sensai_serve_stop", "sensai_batch_create", "sensai_batch_learn", "sensai_batch_tune",
    "sensai_batch_destroy", "sensai_selftest_wait", "sensai_last_error",
]


class SensaiError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"sensai {STATUS_NAMES[status] if 0 <= status < 7 else status}: {message}")
        self.status = status


class sensai_params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("M", ctypes.c_int64 * 4),
        ("B", ctypes.c_int32 * 4),
        ("stride", ctypes.c_int32 * 4),
        ("K", ctypes.c_int32),
        ("a", ctypes.c_double), ("b", ctypes.c_double),
        ("c", ctypes.c_double), ("d", ctypes.c_double),
        ("e", ctypes.c_double), ("f", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("flags", ctypes.c_int32),
    ]


class sensai_state(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_void_p),
        ("Z", ctypes.c_void_p),
        ("S", ctypes.c_void_p),
        ("pi", ctypes.c_void_p),
        ("gamma_s", ctypes.c_double),
        ("gamma_eps", ctypes.c_double),
        ("iter", ctypes.c_int64),
    ]


class sensai_stats(ctypes.Structure):
    _fields_ = [
        ("iter", ctypes.c_int64),
        ("n_patches", ctypes.c_int64),
        ("patch_size", ctypes.c_int64),
        ("n_observed", ctypes.c_int64),
        ("n_active", ctypes.c_int64),
        ("max_observed", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("sum_s2", ctypes.c_double),
        ("sum_r2", ctypes.c_double),
        ("gamma_s", ctypes.c_double),
        ("gamma_eps", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
        ("changed_updates", ctypes.c_int64),
        ("changed_observed", ctypes.c_int64),
        ("active_draws", ctypes.c_int64),
        ("slice_atoms", ctypes.c_int32),
        ("slices", ctypes.c_int32),
        ("rebuild_observed", ctypes.c_int64),
        ("dictionary_form", ctypes.c_int32),
        ("dictionary_smem_kb", ctypes.c_int32),
    ]


class sensai_serve_params(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int32),
        ("max_pixels", ctypes.c_int64),
        ("memory_budget", ctypes.c_int64),
        ("max_observed", ctypes.c_int32),
    ]


DONE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32)

_vp, _i32, _st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
_SIG = {
    "sensai_create": (_st, [ctypes.POINTER(sensai_params), _vp, ctypes.POINTER(_vp)]),
    "sensai_destroy": (None, [_vp]),
    "sensai_set_frame": (_st, [_vp, _vp, _vp]),
    "sensai_reset": (_st, [_vp, _vp]),
    "sensai_learn": (_st, [_vp, _vp, _i32, _vp]),
    "sensai_inpaint": (_st, [_vp, _vp, _i32, _vp, _vp]),
    "sensai_sweep_codes": (_st, [_vp, _vp]),
    "sensai_draw_dictionary": (_st, [_vp, _vp]),
    "sensai_draw_hyper": (_st, [_vp, _vp]),
    "sensai_reconstruct": (_st, [_vp, _vp, _vp]),
    "sensai_mean_reset": (_st, [_vp, _vp]),
    "sensai_mean_add": (_st, [_vp, _vp]),
    "sensai_mean_read": (_st, [_vp, _vp, _vp]),
    "sensai_overlap_counts": (_st, [_vp, _vp, _vp]),
    "sensai_get_dictionary": (_st, [_vp, _vp]),
    "sensai_set_dictionary": (_st, [_vp, _vp]),
    "sensai_get_state": (_st, [_vp, ctypes.POINTER(sensai_state)]),
    "sensai_set_state": (_st, [_vp, ctypes.POINTER(sensai_state)]),
    "sensai_get_stats": (_st, [_vp, ctypes.POINTER(sensai_stats)]),
    "sensai_trace": (_st, [_vp, ctypes.c_char_p, _vp]),
    "sensai_profile": (_st, [_vp, _i32]),
    "sensai_profile_read": (_st, [_vp, _vp, _vp]),
    "sensai_reconstruct_static": (_st, [ctypes.POINTER(sensai_params), _vp, _vp, _vp, _vp]),
    "sensai_serve_start": (_st, [_vp, ctypes.POINTER(sensai_serve_params)]),
    "sensai_submit_frame": (_st, [_vp, _i32, ctypes.c_uint64, _vp, _vp, _vp, _i32, _vp, DONE_FN, _vp]),
    "sensai_serve_drain": (_st, [_vp]),
    "sensai_serve_stop": (_st, [_vp]),
    "sensai_batch_create": (_st, [_vp, _i32, ctypes.POINTER(_vp)]),
    "sensai_batch_learn": (_st, [_vp, _i32, _vp]),
    "sensai_batch_tune": (_st, [_vp, _i32, _vp, ctypes.POINTER(_i32)]),
    "sensai_batch_destroy": (None, [_vp]),
    "sensai_selftest_wait": (_st, [_i32]),
    "sensai_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def library_path():
    return _LIB_PATH


def _check(status):
    if status != SENSAI_OK:
        raise SensaiError(status, _lib.sensai_last_error().decode())


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _buf(a, dtype, count=None, name="buffer"):
    """Pointer to a contiguous NumPy array (host) or torch tensor (host/device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{name}: need a C-contiguous {np.dtype(dtype)} array")
        if count is not None and a.size != count:
            raise ValueError(f"{name}: need {count} elements, got {a.size}")
        return a.ctypes.data
    import torch  # only for tensors
    tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.int32: torch.int32,
           np.float64: torch.float64}[np.dtype(dtype).type]
    if a.dtype != tdt or not a.is_contiguous():
        raise TypeError(f"{name}: need a contiguous {tdt} tensor")
    if count is not None and a.numel() != count:
        raise ValueError(f"{name}: need {count} elements, got {a.numel()}")
    return a.data_ptr()


SENSAI_FLAG_STREAM_DICTIONARY = 0x1
SENSAI_FLAG_CHAIN_DICTIONARY = 0x2
SENSAI_FLAG_GAMMA_S_FULL = 0x4   # reading A of the gamma_s update: prior draws for inactive weights
SENSAI_FLAG_DENSE_STATISTICS = 0x8      # the dense-statistics (tensor-core Gram) form of the dictionary draw
SENSAI_FLAG_TF32_STATISTICS = 0x10      # TF32-level dense statistics (one tensor-core pass)


def SENSAI_SLICE_ATOMS(n):
    """flags bits fixing the streamed dictionary slice at n atoms (n a multiple of 8)."""
    return ((int(n) // 8) & 0xFF) << 8


def make_params(M, B, stride, K, *, a=0.0, b=0.0, c=1e-6, d=1e-6, e=1e-6, f=1e-6, seed=0, flags=0):
    """sensai_params for frame shape M, patch shape B, stride, K atoms
    (a <= 0 -> K, b <= 0 -> N/8)."""
    prm = sensai_params()
    prm.ndim = len(M)
    for i in range(len(M)):
        prm.M[i], prm.B[i], prm.stride[i] = int(M[i]), int(B[i]), int(stride[i])
    prm.K = int(K)
    prm.a, prm.b, prm.c, prm.d, prm.e, prm.f = map(float, (a, b, c, d, e, f))
    prm.seed = int(seed)
    prm.flags = int(flags)
    return prm


class Context:
    """Owns one sensai_ctx; the methods map one to one onto the C entry points."""

    def __init__(self, params, mask):
        self.params = params
        self.shape = tuple(params.M[i] for i in range(params.ndim))
        self.nframe = int(np.prod(self.shape))
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        if m.size != self.nframe:
            raise ValueError("mask size does not match the frame shape")
        h = ctypes.c_void_p()
        _check(_lib.sensai_create(ctypes.byref(params), m.ctypes.data, ctypes.byref(h)))
        self._h = h
        st = self.sensai_get_stats()
        self.N, self.P, self.K = st.n_patches, st.patch_size, st.K

    def close(self):
        if getattr(self, "_h", None):
            _lib.sensai_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- entry points ------------------------------------------------------
    def sensai_set_frame(self, frame, stream=None):
        _check(_lib.sensai_set_frame(self._h, _buf(frame, np.float32, self.nframe, "frame"), _stream(stream)))

    def sensai_reset(self, stream=None):
        _check(_lib.sensai_reset(self._h, _stream(stream)))

    def sensai_learn(self, frame, iters, stream=None):
        _check(_lib.sensai_learn(self._h, _buf(frame, np.float32, self.nframe, "frame"), int(iters), _stream(stream)))

    def sensai_inpaint(self, frame, sweeps, out=None, stream=None):
        _check(_lib.sensai_inpaint(self._h, _buf(frame, np.float32, self.nframe, "frame"), int(sweeps),
                                   _buf(out, np.float32, self.nframe, "out"), _stream(stream)))

    def sensai_sweep_codes(self, stream=None):
        _check(_lib.sensai_sweep_codes(self._h, _stream(stream)))

    def sensai_draw_dictionary(self, stream=None):
        _check(_lib.sensai_draw_dictionary(self._h, _stream(stream)))

    def sensai_draw_hyper(self, stream=None):
        _check(_lib.sensai_draw_hyper(self._h, _stream(stream)))

    def sensai_reconstruct(self, out=None, stream=None):
        host = out is None
        if host:
            out = np.empty(self.shape, dtype=np.float32)
        _check(_lib.sensai_reconstruct(self._h, _buf(out, np.float32, self.nframe, "out"), _stream(stream)))
        return out

    def sensai_mean_reset(self, stream=None):
        _check(_lib.sensai_mean_reset(self._h, _stream(stream)))

    def sensai_mean_add(self, stream=None):
        _check(_lib.sensai_mean_add(self._h, _stream(stream)))

    def sensai_mean_read(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        _check(_lib.sensai_mean_read(self._h, _buf(out, np.float32, self.nframe, "out"), _stream(stream)))
        return out

    def sensai_overlap_counts(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.int32)
        _check(_lib.sensai_overlap_counts(self._h, _buf(out, np.int32, self.nframe, "out"), _stream(stream)))
        return out

    def sensai_get_dictionary(self):
        D = np.empty((self.K, self.P), dtype=np.float32)
        _check(_lib.sensai_get_dictionary(self._h, D.ctypes.data))
        return D

    def sensai_set_dictionary(self, D):
        D = np.ascontiguousarray(D, dtype=np.float32)
        _check(_lib.sensai_set_dictionary(self._h, _buf(D, np.float32, self.K * self.P, "D")))

    def sensai_get_state(self):
        D = np.empty((self.K, self.P), np.float32)
        Z = np.empty((self.N, self.K), np.uint8)
        S = np.empty((self.N, self.K), np.float32)
        pi = np.empty(self.K, np.float64)
        st = sensai_state(D.ctypes.data, Z.ctypes.data, S.ctypes.data, pi.ctypes.data, 0.0, 0.0, 0)
        _check(_lib.sensai_get_state(self._h, ctypes.byref(st)))
        return {"D": D, "Z": Z, "S": S, "pi": pi, "gamma_s": st.gamma_s,
                "gamma_eps": st.gamma_eps, "iter": st.iter}

    def sensai_set_state(self, D=None, Z=None, S=None, pi=None, gamma_s=1.0, gamma_eps=0.0, iter=0):
        keep = []

        def host(a, dt, n, name):
            if a is None:
                return None
            arr = np.ascontiguousarray(a, dtype=dt)
            keep.append(arr)
            return _buf(arr, dt, n, name)

        st = sensai_state(host(D, np.float32, self.K * self.P, "D"), host(Z, np.uint8, self.N * self.K, "Z"),
                          host(S, np.float32, self.N * self.K, "S"), host(pi, np.float64, self.K, "pi"),
                          float(gamma_s), float(gamma_eps), int(iter))
        _check(_lib.sensai_set_state(self._h, ctypes.byref(st)))

    # -- live serving -------------------------------------------------------
    def sensai_serve_start(self, slots=4, max_pixels=1 << 20, memory_budget=0, max_observed=64):
        """Start the serving engine on this context's current dictionary, pi
        and precisions."""
        import threading
        sp = sensai_serve_params(int(slots), int(max_pixels), int(memory_budget), int(max_observed))
        self._serve_lock = threading.Lock()
        self._pending = {}
        self._cb = DONE_FN(self._on_done)
        _check(_lib.sensai_serve_start(self._h, ctypes.byref(sp)))

    def _on_done(self, user, frame_id, status):
        with self._serve_lock:
            entry = self._pending.pop(int(user), None)
        if entry is not None and entry[0] is not None:
            entry[0](int(frame_id), int(status), entry[1])

    def sensai_submit_frame(self, stream_id, frame_id, frame, mask, sweeps, out=None, done=None):
        """Queue one host frame (any shape valid for the patch geometry).
        ``done(frame_id, status, out)`` runs on a worker thread when the
        reconstruction is in ``out``.  Returns ``out``."""
        frame = np.ascontiguousarray(frame, dtype=np.float32)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        if frame.shape != mask.shape:
            raise ValueError("frame and mask shapes differ")
        if out is None:
            out = np.empty(frame.shape, dtype=np.float32)
        M = (ctypes.c_int64 * 4)(*([int(v) for v in frame.shape] + [0] * (4 - frame.ndim)))
        with self._serve_lock:
            self._serial = getattr(self, "_serial", 0) + 1
            token = self._serial
            self._pending[token] = (done, out, frame, mask, M)
        st = _lib.sensai_submit_frame(self._h, int(stream_id), int(frame_id), frame.ctypes.data, mask.ctypes.data,
                                      ctypes.addressof(M), int(sweeps), out.ctypes.data, self._cb, token)
        if st != SENSAI_OK:
            with self._serve_lock:
                self._pending.pop(token, None)
            _check(st)
        return out

    def sensai_serve_drain(self):
        _check(_lib.sensai_serve_drain(self._h))

    def sensai_serve_stop(self):
        _check(_lib.sensai_serve_stop(self._h))

    def sensai_trace(self, path, clean=None):
        """Append one JSON line of metrics per Gibbs iteration to ``path``
        (None stops); ``clean`` (a float32 frame, host or device) adds the
        PSNR of the current reconstruction."""
        arr = np.ascontiguousarray(clean, np.float32) if isinstance(clean, np.ndarray) else clean
        c = None if arr is None else _buf(arr, np.float32, self.nframe, "clean")
        _check(_lib.sensai_trace(self._h, None if path is None else str(path).encode(), c))

    def sensai_profile(self, enable):
        _check(_lib.sensai_profile(self._h, int(enable)))

    def sensai_profile_read(self):
        """Per-phase (ms, count) for codes, dictionary, hyper, reconstruction."""
        ms = np.zeros(4, np.float64)
        cnt = np.zeros(4, np.int64)
        _check(_lib.sensai_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data))
        names = ("codes", "dictionary", "hyper", "reconstruct")
        return {n: (float(ms[i]), int(cnt[i])) for i, n in enumerate(names)}

    def sensai_get_stats(self):
        st = sensai_stats()
        _check(_lib.sensai_get_stats(self._h, ctypes.byref(st)))
        return st


def _static_sizes(params):
    """(P, N, frame pixels) of a sensai_params, as the C side computes them."""
    P = N = nframe = 1
    for d in range(params.ndim):
        M, B, S = int(params.M[d]), int(params.B[d]), int(params.stride[d])
        if M < 1 or B < 1 or B > M or S < 1 or (M - B) % S:
            raise ValueError(f"dimension {d}: invalid frame / patch / stride geometry")
        P *= B
        N *= (M - B) // S + 1
        nframe *= M
    return P, N, nframe


def sensai_reconstruct_static(params, D, S, out, stream=None):
    """Overlap-add reconstruction without any device allocation (device
    tensors on the current device: D K x P, S N x K patch-major, out the
    frame shape).  The element counts are checked here, since the C side
    receives bare pointers."""
    P, N, nframe = _static_sizes(params)
    K = int(params.K)
    counts = (("D", D, K * P), ("S", S, N * K), ("out", out, nframe))
    for name, t, n in counts:
        if not hasattr(t, "numel"):
            raise TypeError(f"{name}: need a CUDA float32 tensor")
        if t.numel() != n:
            raise ValueError(f"{name}: need {n} elements, got {t.numel()}")
    import torch
    for name, t, _ in counts:
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise TypeError(f"{name}: need a CUDA float32 tensor on the current device")
    _check(_lib.sensai_reconstruct_static(ctypes.byref(params), _buf(D, np.float32, K * P, "D"),
                                          _buf(S, np.float32, N * K, "S"), _buf(out, np.float32, nframe, "out"),
                                          _stream(stream)))


def sensai_last_error():
    return _lib.sensai_last_error().decode()


class Batch:
    """Owns one sensai_batch over Context objects (kept alive here)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (_vp * len(self.contexts))(*[c._h for c in self.contexts])
        h = _vp()
        _check(_lib.sensai_batch_create(arr, len(self.contexts), ctypes.byref(h)))
        self._h = h

    def sensai_batch_learn(self, iters, stream=None):
        _check(_lib.sensai_batch_learn(self._h, int(iters), _stream(stream)))

    def sensai_batch_tune(self, iters_per_trial=1, stream=None):
        d = _i32(0)
        _check(_lib.sensai_batch_tune(self._h, int(iters_per_trial), _stream(stream), ctypes.byref(d)))
        return d.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.sensai_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sensai_selftest_wait(which):
    """Status of the bounded-wait self-test (SENSAI_ETIMEOUT is the expected result)."""
    return _lib.sensai_selftest_wait(int(which))
