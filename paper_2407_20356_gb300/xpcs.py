"""ctypes binding of libxpcs.so: the C ABI of include/xpcs.h, name for name.

Argument marshalling only.  Device buffers may be passed as torch CUDA tensors or raw
integer device addresses; host buffers as numpy arrays.  Every step of the computation
runs in the library's CUDA kernels; there is no fallback of any kind: if the library is
missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libxpcs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with paper_2407_20356_gb300._build.build_library() "
        "(or __graft_entry__.build()); this package has no CPU fallback")
_lib = C.CDLL(LIB_PATH)

XPCS_OK, XPCS_EINVAL, XPCS_ENOMEM, XPCS_ECUDA, XPCS_ETIMEOUT, XPCS_EBUSY, XPCS_ERANGE, XPCS_ENOTSUP = range(8)
STATUS_NAMES = ["XPCS_OK", "XPCS_EINVAL", "XPCS_ENOMEM", "XPCS_ECUDA", "XPCS_ETIMEOUT", "XPCS_EBUSY",
                "XPCS_ERANGE", "XPCS_ENOTSUP"]
XPCS_U8, XPCS_U16 = 0, 1
XPCS_PREC_FP16, XPCS_PREC_BF16, XPCS_PREC_BF16X3 = 0, 1, 2
PRECISIONS = {"fp16": XPCS_PREC_FP16, "bf16": XPCS_PREC_BF16, "bf16x3": XPCS_PREC_BF16X3}
XPCS_NORM_MEAN, XPCS_NORM_FROB, XPCS_NORM_EQ12 = 0, 1, 2
NORMS = {"mean": XPCS_NORM_MEAN, "frob": XPCS_NORM_FROB, "eq12": XPCS_NORM_EQ12}
SCHEDULES = ("tiles", "tile_pairs")  # two-time kernel schedules (codes 0, 1)
XPCS_QMEAN_COMPRESSED, XPCS_QMEAN_EXACT_RAW = 0, 1
QMEANS = {"compressed": XPCS_QMEAN_COMPRESSED, "exact_raw": XPCS_QMEAN_EXACT_RAW}


class XpcsOptions(C.Structure):
    """xpcs_options: precision, normalisation and ring sums of the compressed calls."""
    _fields_ = [("precision", C.c_int), ("norm", C.c_int), ("qmean", C.c_int)]

vp = C.c_void_p
i64 = C.c_int64
_SIGS = {
    "xpcs_version": (C.c_int, []),
    "xpcs_create": (C.c_int, [C.c_int, C.c_size_t, vp, C.POINTER(vp)]),
    "xpcs_destroy": (C.c_int, [vp]),
    "xpcs_last_error": (C.c_char_p, [vp]),
    "xpcs_set_async": (C.c_int, [vp, C.c_int]),
    "xpcs_synchronize": (C.c_int, [vp]),
    "xpcs_device_bytes": (C.c_size_t, [vp]),
    "xpcs_launch_count": (C.c_uint64, [vp]),
    "xpcs_profile_enable": (C.c_int, [vp, C.c_int]),
    "xpcs_profile_count": (C.c_int, [vp]),
    "xpcs_profile_get": (C.c_int, [vp, C.c_int, C.c_char_p, C.c_size_t, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64)]),
    "xpcs_rings_create": (C.c_int, [vp, vp, i64, C.c_int, C.POINTER(vp)]),
    "xpcs_rings_destroy": (C.c_int, [vp]),
    "xpcs_rings_sizes": (C.c_int, [vp, vp]),
    "xpcs_ring_sums": (C.c_int, [vp, vp, vp, C.c_int, i64, vp]),
    "xpcs_twotime_raw": (C.c_int, [vp, vp, vp, C.c_int, i64, vp, vp, vp, vp]),
    "xpcs_twotime_raw_norm": (C.c_int, [vp, vp, vp, C.c_int, i64, C.c_int, vp, vp, vp, vp]),
    "xpcs_fit_basis": (C.c_int, [vp, vp, vp, C.c_int, i64, C.c_int, C.POINTER(vp), vp]),
    "xpcs_basis_import": (C.c_int, [vp, vp, vp, C.c_int, C.POINTER(vp)]),
    "xpcs_basis_export": (C.c_int, [vp, vp, vp, vp, vp]),
    "xpcs_basis_rank": (C.c_int, [vp, C.POINTER(C.c_int)]),
    "xpcs_rank_from_spectrum": (C.c_int, [vp, C.c_int, C.c_double]),
    "xpcs_stream_row_tile": (C.c_int, [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]),
    "xpcs_basis_destroy": (C.c_int, [vp]),
    "xpcs_encode": (C.c_int, [vp, vp, vp, C.c_int, i64, vp]),
    "xpcs_twotime": (C.c_int, [vp, vp, vp, i64, C.c_int, vp, vp, vp]),
    "xpcs_twotime_norm": (C.c_int, [vp, vp, vp, i64, C.c_int, C.c_int, vp, vp, vp]),
    "xpcs_twotime_opts": (C.c_int, [vp, vp, vp, i64, C.POINTER(XpcsOptions), vp, vp, vp, vp]),
    "xpcs_encode_sums": (C.c_int, [vp, vp, vp, C.c_int, i64, vp, vp]),
    "xpcs_encode_host": (C.c_int, [vp, vp, vp, C.c_int, i64, vp]),
    "xpcs_raw_stream_open": (C.c_int, [vp, vp, i64, C.c_int, C.POINTER(vp)]),
    "xpcs_raw_stream_push_device": (C.c_int, [vp, vp, i64]),
    "xpcs_raw_stream_read_g2": (C.c_int, [vp, vp, vp]),
    "xpcs_raw_stream_frames": (i64, [vp]),
    "xpcs_raw_stream_close": (C.c_int, [vp]),
    "xpcs_stream_open_opts": (C.c_int, [vp, vp, i64, C.c_int, C.c_int, C.POINTER(XpcsOptions), C.POINTER(vp)]),
    "xpcs_autotune_twotime": (C.c_int, [vp, vp, vp, i64, C.c_int, vp, vp, vp, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "xpcs_autotune_twotime_raw": (C.c_int, [vp, vp, vp, C.c_int, i64, vp, vp, vp, vp, C.c_int,
                                            C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "xpcs_set_timeout": (C.c_int, [vp, C.c_int]),
    "xpcs_twotime_config": (C.c_int, [vp, C.c_int, C.c_int]),
    "xpcs_get_timeout": (C.c_int, [vp]),
    "xpcs_g2": (C.c_int, [vp, vp, C.c_int, i64, vp, vp]),
    "xpcs_fit_relaxation": (C.c_int, [vp, vp, C.c_int, i64, i64, i64, C.c_double, C.c_double, vp]),
    "xpcs_twotime_stats": (C.c_int, [vp, vp, C.c_int, i64, vp, vp]),
    "xpcs_peak_visibility": (C.c_int, [vp, vp, C.c_int, i64, i64, i64, i64, i64, vp, C.c_double, vp, vp]),
    "xpcs_selftest_timeout": (C.c_int, [vp, C.c_int]),
    "xpcs_capture_begin": (C.c_int, [vp]),
    "xpcs_capture_end": (C.c_int, [vp, C.POINTER(vp)]),
    "xpcs_graph_launch": (C.c_int, [vp, vp]),
    "xpcs_graph_kernels": (C.c_uint64, [vp]),
    "xpcs_graph_destroy": (C.c_int, [vp]),
    "xpcs_g2_noalloc": (C.c_int, [vp, vp, C.c_int, i64, vp, vp]),
    "xpcs_stream_open": (C.c_int, [vp, vp, i64, C.c_int, C.c_int, C.POINTER(vp)]),
    "xpcs_stream_push": (C.c_int, [vp, vp, i64, C.POINTER(C.c_uint64)]),
    "xpcs_stream_push_device": (C.c_int, [vp, vp, i64, C.POINTER(C.c_uint64)]),
    "xpcs_stream_push_device_at": (C.c_int, [vp, vp, i64, vp, C.POINTER(C.c_uint64)]),
    "xpcs_clock_ns": (i64, []),
    "xpcs_stream_poll": (C.c_int, [vp, C.c_uint64, C.c_int]),
    "xpcs_stream_read_g2": (C.c_int, [vp, vp, vp]),
    "xpcs_stream_frames": (i64, [vp]),
    "xpcs_stream_latency": (C.c_int, [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "xpcs_stream_close": (C.c_int, [vp]),
    "xpcs_stream_checkpoint_size": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
    "xpcs_stream_checkpoint": (C.c_int, [vp, vp, C.c_size_t]),
    "xpcs_stream_restore": (C.c_int, [vp, vp, C.c_size_t]),
    "xpcs_server_create": (C.c_int, [vp, C.POINTER(vp)]),
    "xpcs_server_open": (C.c_int, [vp, vp, i64, C.c_int, C.c_int, C.c_int, C.POINTER(vp)]),
    "xpcs_server_submit": (C.c_int, [vp, vp, vp, i64, C.POINTER(C.c_uint64)]),
    "xpcs_server_submit_device": (C.c_int, [vp, vp, vp, i64, C.POINTER(C.c_uint64)]),
    "xpcs_server_poll": (C.c_int, [vp, vp, C.c_uint64, C.c_int]),
    "xpcs_server_read_g2": (C.c_int, [vp, vp, vp, vp]),
    "xpcs_server_latency": (C.c_int, [vp, vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "xpcs_server_close": (C.c_int, [vp, vp]),
    "xpcs_server_batches": (C.c_uint64, [vp]),
    "xpcs_server_destroy": (C.c_int, [vp]),
}


def declared_symbols():
    """Names of the entry points this binding declares."""
    return list(_SIGS)


for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class XpcsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _ptr(x):
    """Device or host address of a tensor/array/int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _dtype_code(x):
    s = str(getattr(x, "dtype", x))
    if "uint8" in s:
        return XPCS_U8
    if "uint16" in s:
        return XPCS_U16
    raise TypeError(f"counts must be uint8 or uint16, got {s}")


class Context:
    """An xpcs_ctx: device, CUDA stream, device-memory budget."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, stream=None):
        h = vp()
        self.h = None
        self._children = weakref.WeakSet()
        st = _lib.xpcs_create(device, hbm_budget, stream, C.byref(h))
        if st != XPCS_OK:
            raise XpcsError(st, "xpcs_create failed")
        self.h = h

    def _adopt(self, child):
        self._children.add(child)

    def check(self, st):
        if st != XPCS_OK:
            raise XpcsError(st, _lib.xpcs_last_error(self.h).decode())

    _CLOSE_ORDER = {"Server": 0, "Graph": 1, "Stream": 2, "RawStream": 2, "Basis": 3, "Rings": 4}

    def close(self):
        """Destroy the context after every handle created on it, each handle before the
        ones it uses: servers and graphs, then streams, bases and ring plans."""
        if self.h:
            for ch in sorted(self._children, key=lambda c: self._CLOSE_ORDER.get(type(c).__name__, 0)):
                ch.close()
            _lib.xpcs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_async(self, on: bool):
        self.check(_lib.xpcs_set_async(self.h, 1 if on else 0))

    def set_timeout(self, timeout_ms: int):
        """Limit (ms) of the bounded device waits of this context's kernels and of the streams
        opened on it afterwards; 0 restores the default."""
        self.check(_lib.xpcs_set_timeout(self.h, int(timeout_ms)))

    def timeout(self) -> int:
        return int(_lib.xpcs_get_timeout(self.h))

    def twotime_config(self, tiles: int = 0, schedule="tiles"):
        """Fix the two-time kernel's configuration (tiles per work item, schedule name or
        code); tiles = 0 returns to the autotuned or default choice."""
        sc = SCHEDULES.index(schedule) if isinstance(schedule, str) else int(schedule)
        self.check(_lib.xpcs_twotime_config(self.h, int(tiles), sc))

    def synchronize(self):
        self.check(_lib.xpcs_synchronize(self.h))

    def device_bytes(self) -> int:
        return int(_lib.xpcs_device_bytes(self.h))

    def launch_count(self) -> int:
        return int(_lib.xpcs_launch_count(self.h))

    def profile_enable(self, on: bool = True):
        self.check(_lib.xpcs_profile_enable(self.h, 1 if on else 0))

    def profile(self) -> dict:
        """{site name: (total ms, launches)} of the timed launch sites."""
        out = {}
        for i in range(_lib.xpcs_profile_count(self.h)):
            buf = C.create_string_buffer(64)
            ms = C.c_double()
            n = C.c_int64()
            self.check(_lib.xpcs_profile_get(self.h, i, buf, 64, C.byref(ms), C.byref(n)))
            out[buf.value.decode()] = (ms.value, n.value)
        return out


class Rings:
    def __init__(self, ctx: Context, qmap, M: int, n_q: int):
        h = vp()
        ctx.check(_lib.xpcs_rings_create(ctx.h, _ptr(qmap), M, n_q, C.byref(h)))
        self.ctx, self.h, self.M, self.n_q = ctx, h, M, n_q
        ctx._adopt(self)

    def sizes(self) -> np.ndarray:
        out = np.zeros(self.n_q, dtype=np.int64)
        self.ctx.check(_lib.xpcs_rings_sizes(self.h, out.ctypes.data))
        return out

    def close(self):
        if self.h and self.ctx.h:
            _lib.xpcs_rings_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Basis:
    def __init__(self, ctx: Context, rings: Rings, h, k: int):
        self.ctx, self.rings, self.h, self.k = ctx, rings, h, k
        ctx._adopt(self)

    def export(self):
        M, n_q, k = self.rings.M, self.rings.n_q, self.k
        B = np.empty((M, k))
        G = np.empty((n_q, k, k))
        s = np.empty((n_q, k))
        self.ctx.check(_lib.xpcs_basis_export(self.ctx.h, self.h, B.ctypes.data, G.ctypes.data, s.ctypes.data))
        return B, G, s

    def close(self):
        if self.h and self.ctx.h:
            _lib.xpcs_basis_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def xpcs_version() -> int:
    return int(_lib.xpcs_version())


def xpcs_rings_create(ctx: Context, qmap, M: int, n_q: int) -> Rings:
    return Rings(ctx, qmap, M, n_q)


def xpcs_ring_sums(ctx: Context, rings: Rings, X, T: int, S_out, dtype=None):
    ctx.check(_lib.xpcs_ring_sums(ctx.h, rings.h, _ptr(X), _dtype_code(dtype or X), T, _ptr(S_out)))


def _norm_code(norm) -> int:
    return NORMS[norm] if isinstance(norm, str) else int(norm)


def xpcs_twotime_raw(ctx: Context, rings: Rings, X, T: int, C_out=None, N_out=None, g2_out=None, count_out=None,
                     dtype=None, norm="mean"):
    if _norm_code(norm) != XPCS_NORM_MEAN:
        return xpcs_twotime_raw_norm(ctx, rings, X, T, norm, C_out, N_out, g2_out, count_out, dtype)
    ctx.check(_lib.xpcs_twotime_raw(ctx.h, rings.h, _ptr(X), _dtype_code(dtype or X), T, _ptr(C_out),
                                    _ptr(N_out), _ptr(g2_out), _ptr(count_out)))


def xpcs_twotime_raw_norm(ctx: Context, rings: Rings, X, T: int, norm, C_out=None, N_out=None, g2_out=None,
                          count_out=None, dtype=None):
    ctx.check(_lib.xpcs_twotime_raw_norm(ctx.h, rings.h, _ptr(X), _dtype_code(dtype or X), T, _norm_code(norm),
                                         _ptr(C_out), _ptr(N_out), _ptr(g2_out), _ptr(count_out)))


def xpcs_fit_basis(ctx: Context, rings: Rings, F, n_fit: int, k: int, sigma_host=None, dtype=None) -> Basis:
    h = vp()
    ctx.check(_lib.xpcs_fit_basis(ctx.h, rings.h, _ptr(F), _dtype_code(dtype or F), n_fit, k, C.byref(h),
                                  _ptr(sigma_host)))
    return Basis(ctx, rings, h, k)


def xpcs_basis_import(ctx: Context, rings: Rings, B_host: np.ndarray) -> Basis:
    B_host = np.ascontiguousarray(B_host, dtype=np.float64)
    assert B_host.shape[0] == rings.M
    h = vp()
    ctx.check(_lib.xpcs_basis_import(ctx.h, rings.h, B_host.ctypes.data, B_host.shape[1], C.byref(h)))
    return Basis(ctx, rings, h, B_host.shape[1])


def xpcs_rank_from_spectrum(sigma, factor: float = 2.0) -> int:
    """K = number of spectrum values >= factor * the smallest one within the numerical rank."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    K = _lib.xpcs_rank_from_spectrum(sigma.ctypes.data, sigma.size, float(factor))
    if K < 0:
        raise XpcsError(XPCS_EINVAL, "xpcs_rank_from_spectrum: bad spectrum or factor")
    return K


def xpcs_stream_row_tile(n_q: int, k: int, b: int) -> dict:
    """Row-update configuration of a stream step of b frames (host-side, no device)."""
    out = [C.c_int() for _ in range(4)]
    st = _lib.xpcs_stream_row_tile(n_q, k, b, *[C.byref(o) for o in out])
    if st != XPCS_OK:
        raise XpcsError(st, "xpcs_stream_row_tile")
    return dict(zip(("lags", "w_stages", "epilogue", "smem_bytes"), (o.value for o in out)))


def xpcs_encode(ctx: Context, basis: Basis, X, T: int, A_out, dtype=None):
    ctx.check(_lib.xpcs_encode(ctx.h, basis.h, _ptr(X), _dtype_code(dtype or X), T, _ptr(A_out)))


def xpcs_encode_host(ctx: Context, basis: Basis, X_host, T: int, A_out, dtype=None):
    """Encode frames in (pinned) host memory, the host-to-device copy overlapped with the encode."""
    ctx.check(_lib.xpcs_encode_host(ctx.h, basis.h, _ptr(X_host), _dtype_code(dtype or X_host), T, _ptr(A_out)))


def xpcs_encode_sums(ctx: Context, basis: Basis, X, T: int, A_out, S_out, dtype=None):
    """Encode and also capture the exact ring sums of the raw frames (S_out: n_q x T int64)."""
    ctx.check(_lib.xpcs_encode_sums(ctx.h, basis.h, _ptr(X), _dtype_code(dtype or X), T, _ptr(A_out), _ptr(S_out)))


def _options(prec="fp16", norm="mean", qmean="compressed") -> XpcsOptions:
    return XpcsOptions(PRECISIONS[prec] if isinstance(prec, str) else int(prec), _norm_code(norm),
                       QMEANS[qmean] if isinstance(qmean, str) else int(qmean))


def xpcs_twotime_opts(ctx: Context, basis: Basis, A, T: int, prec="fp16", norm="mean", qmean="compressed",
                      S_raw=None, C_out=None, g2_out=None, count_out=None):
    """Compressed two-time with every option; qmean="exact_raw" takes the raw ring sums S_raw."""
    o = _options(prec, norm, qmean)
    ctx.check(_lib.xpcs_twotime_opts(ctx.h, basis.h, _ptr(A), T, C.byref(o), _ptr(S_raw), _ptr(C_out), _ptr(g2_out),
                                     _ptr(count_out)))


def xpcs_twotime(ctx: Context, basis: Basis, A, T: int, prec="fp16", C_out=None, g2_out=None, count_out=None,
                 norm="mean"):
    if _norm_code(norm) != XPCS_NORM_MEAN:
        return xpcs_twotime_norm(ctx, basis, A, T, prec, norm, C_out, g2_out, count_out)
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    ctx.check(_lib.xpcs_twotime(ctx.h, basis.h, _ptr(A), T, p, _ptr(C_out), _ptr(g2_out), _ptr(count_out)))


def _tune_result(tiles, sched, ms) -> dict:
    return {"tiles_per_item": tiles.value, "schedule": SCHEDULES[sched.value], "pairs": sched.value == 1,
            "ms": ms.value}


def xpcs_autotune_twotime(ctx: Context, basis: Basis, A, T: int, prec="bf16x3", C_out=None, g2_out=None,
                          count_out=None, reps: int = 2) -> dict:
    """Time the two-time kernel's configurations on these arguments, keep the fastest."""
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    tiles, sched, ms = C.c_int(), C.c_int(), C.c_double()
    ctx.check(_lib.xpcs_autotune_twotime(ctx.h, basis.h, _ptr(A), T, p, _ptr(C_out), _ptr(g2_out), _ptr(count_out),
                                         reps, C.byref(tiles), C.byref(sched), C.byref(ms)))
    return _tune_result(tiles, sched, ms)


def xpcs_autotune_twotime_raw(ctx: Context, rings: Rings, X, T: int, C_out=None, N_out=None, g2_out=None,
                              count_out=None, reps: int = 2, dtype=None) -> dict:
    """The autotuner for the raw two-time call."""
    tiles, sched, ms = C.c_int(), C.c_int(), C.c_double()
    ctx.check(_lib.xpcs_autotune_twotime_raw(ctx.h, rings.h, _ptr(X), _dtype_code(dtype or X), T, _ptr(C_out),
                                             _ptr(N_out), _ptr(g2_out), _ptr(count_out), reps, C.byref(tiles),
                                             C.byref(sched), C.byref(ms)))
    return _tune_result(tiles, sched, ms)


def xpcs_twotime_norm(ctx: Context, basis: Basis, A, T: int, prec, norm, C_out=None, g2_out=None, count_out=None):
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    ctx.check(_lib.xpcs_twotime_norm(ctx.h, basis.h, _ptr(A), T, p, _norm_code(norm), _ptr(C_out), _ptr(g2_out),
                                     _ptr(count_out)))


class Graph:
    """A captured sequence of library calls on a context (xpcs_capture_begin/end)."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        ctx._adopt(self)

    def launch(self):
        self.ctx.check(_lib.xpcs_graph_launch(self.ctx.h, self.h))

    def kernels(self) -> int:
        return int(_lib.xpcs_graph_kernels(self.h))

    def close(self):
        if self.h and self.ctx.h:
            _lib.xpcs_graph_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def xpcs_capture_begin(ctx: Context):
    ctx.check(_lib.xpcs_capture_begin(ctx.h))


def xpcs_capture_end(ctx: Context) -> Graph:
    h = vp()
    ctx.check(_lib.xpcs_capture_end(ctx.h, C.byref(h)))
    return Graph(ctx, h)


def xpcs_fit_relaxation(ctx: Context, g2, n_q: int, T: int, tau_lo: int, tau_hi: int, t0_min: float,
                        t0_max: float, params_out):
    ctx.check(_lib.xpcs_fit_relaxation(ctx.h, _ptr(g2), n_q, T, tau_lo, tau_hi, float(t0_min), float(t0_max),
                                       _ptr(params_out)))


def xpcs_twotime_stats(ctx: Context, C_in, n_q: int, T: int, mean_out, std_out=None):
    ctx.check(_lib.xpcs_twotime_stats(ctx.h, _ptr(C_in), n_q, T, _ptr(mean_out), _ptr(std_out)))


def xpcs_peak_visibility(ctx: Context, g2, n_q: int, T: int, peak_lo: int, peak_hi: int, bg_lo: int, bg_hi: int,
                         vis_out, ttc_std=None, factor: float = 2.0, flag_out=None):
    ctx.check(_lib.xpcs_peak_visibility(ctx.h, _ptr(g2), n_q, T, peak_lo, peak_hi, bg_lo, bg_hi, _ptr(ttc_std),
                                        float(factor), _ptr(vis_out), _ptr(flag_out)))


def xpcs_g2(ctx: Context, C_in, n_q: int, T: int, g2_out, count_out=None):
    ctx.check(_lib.xpcs_g2(ctx.h, _ptr(C_in), n_q, T, _ptr(g2_out), _ptr(count_out)))


def xpcs_selftest_timeout(ctx: Context, limit_ms: int):
    """Run a bounded device wait that nothing satisfies; raises XpcsError(XPCS_ETIMEOUT).
    limit_ms = 0 waits through the library's own bounded wait with the context's limit."""
    ctx.check(_lib.xpcs_selftest_timeout(ctx.h, limit_ms))


def clock_ns() -> int:
    """The library's host steady clock (ns), in which stream latencies are measured."""
    return int(_lib.xpcs_clock_ns())


G2_NOALLOC_MAX_CELLS = 1 << 20  # n_q * T limit of xpcs_g2_noalloc (its fixed scratch)
G2_MAX_RINGS = 65535  # n_q limit of xpcs_g2 and xpcs_g2_noalloc


def xpcs_g2_noalloc(ctx: Context, C_in, n_q: int, T: int, g2_out, count_out=None):
    """xpcs_g2 with its scratch in a fixed per-device array: allocates no device memory."""
    ctx.check(_lib.xpcs_g2_noalloc(ctx.h, _ptr(C_in), n_q, T, _ptr(g2_out), _ptr(count_out)))


class RawStream:
    """An xpcs_raw_stream: every pushed frame's exact raw two-time row folded into g2."""

    def __init__(self, ctx: Context, rings: Rings, history: int, dtype="uint16"):
        h = vp()
        st = _lib.xpcs_raw_stream_open(ctx.h, rings.h, history, _dtype_code(dtype), C.byref(h))
        if st != XPCS_OK:
            raise XpcsError(st, _lib.xpcs_last_error(ctx.h).decode())
        self.ctx, self.rings, self.h, self.W = ctx, rings, h, history
        self.n_q = rings.n_q
        ctx._adopt(self)

    def push(self, frames_dev):
        """Push device frames (n x M tensor); returns once they are folded in."""
        self.ctx.check(_lib.xpcs_raw_stream_push_device(self.h, _ptr(frames_dev), int(frames_dev.shape[0])))

    def read_g2(self):
        g2 = np.empty((self.n_q, self.W), dtype=np.float64)
        cnt = np.empty((self.n_q, self.W), dtype=np.int64)
        self.ctx.check(_lib.xpcs_raw_stream_read_g2(self.h, g2.ctypes.data, cnt.ctypes.data))
        return g2, cnt

    def frames(self) -> int:
        return int(_lib.xpcs_raw_stream_frames(self.h))

    def close(self):
        if self.h:
            _lib.xpcs_raw_stream_close(self.h)
            self.h = None


class Stream:
    """An xpcs_stream: online encode + two-time row update of every pushed frame.

    prec: "bf16x3" (coefficient rows as bf16 hi | lo pieces, three products) or "fp16"
    (one f16 product, half the history bytes; about 2^-11 relative per row)."""

    def __init__(self, ctx: Context, basis: Basis, history: int, max_batch: int, dtype="uint16", qmean="compressed",
                 prec="bf16x3"):
        h = vp()
        o = _options(prec=prec, qmean=qmean)
        st = _lib.xpcs_stream_open_opts(ctx.h, basis.h, history, max_batch, _dtype_code(dtype), C.byref(o),
                                        C.byref(h))
        if st != XPCS_OK:
            raise XpcsError(st, _lib.xpcs_last_error(ctx.h).decode())
        self.ctx, self.basis, self.h, self.W = ctx, basis, h, history
        self.n_q = basis.rings.n_q
        ctx._adopt(self)

    def push(self, frames) -> int:
        """Push frames (host numpy array or device tensor, n x M); returns the ticket."""
        t = C.c_uint64()
        n = int(frames.shape[0])
        on_device = hasattr(frames, "is_cuda") and frames.is_cuda
        f = _lib.xpcs_stream_push_device if on_device else _lib.xpcs_stream_push
        self.ctx.check(f(self.h, _ptr(frames), n, C.byref(t)))
        return t.value

    def push_at(self, frames, arrive_ns) -> int:
        """Push device frames (n x M) with their arrival times (n int64 values of clock_ns())."""
        t = C.c_uint64()
        arr = np.ascontiguousarray(arrive_ns, dtype=np.int64)
        n = int(frames.shape[0])
        assert arr.shape == (n,)
        self.ctx.check(_lib.xpcs_stream_push_device_at(self.h, _ptr(frames), n, arr.ctypes.data, C.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0) -> bool:
        st = _lib.xpcs_stream_poll(self.h, ticket, timeout_ms)
        if st == XPCS_EBUSY:
            return False
        self.ctx.check(st)
        return True

    def read_g2(self):
        g2 = np.empty((self.n_q, self.W))
        cnt = np.empty((self.n_q, self.W), dtype=np.int64)
        self.ctx.check(_lib.xpcs_stream_read_g2(self.h, g2.ctypes.data, cnt.ctypes.data))
        return g2, cnt

    def frames(self) -> int:
        return int(_lib.xpcs_stream_frames(self.h))

    def latency(self, reset: bool = False) -> dict:
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        n = C.c_int64()
        self.ctx.check(_lib.xpcs_stream_latency(self.h, 1 if reset else 0, C.byref(a), C.byref(b), C.byref(c),
                                                C.byref(n)))
        return {"p50_us": a.value, "p99_us": b.value, "max_us": c.value, "batches": n.value}

    def checkpoint(self) -> np.ndarray:
        """The stream's state as bytes (waits for its queued batches)."""
        n = C.c_size_t()
        self.ctx.check(_lib.xpcs_stream_checkpoint_size(self.h, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self.ctx.check(_lib.xpcs_stream_checkpoint(self.h, buf.ctypes.data, n.value))
        return buf

    def restore(self, buf: np.ndarray):
        """Continue from a checkpoint (this stream must be fresh, same basis and shape)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self.ctx.check(_lib.xpcs_stream_restore(self.h, buf.ctypes.data, buf.size))

    def close(self):
        if self.h and self.ctx.h:
            _lib.xpcs_stream_close(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """An xpcs_server: a scheduler thread serving several streams with continuous batching."""

    def __init__(self, ctx: Context):
        h = vp()
        ctx.check(_lib.xpcs_server_create(ctx.h, C.byref(h)))
        self.ctx, self.h = ctx, h
        self.streams = {}
        ctx._adopt(self)

    def open(self, basis: Basis, history: int, max_batch: int, dtype="uint16", wait_ms: int = 0):
        """Open a stream; returns its handle (an int key), or raises XpcsError (XPCS_EBUSY)."""
        h = vp()
        st = _lib.xpcs_server_open(self.h, basis.h, history, max_batch, _dtype_code(dtype), wait_ms, C.byref(h))
        if st != XPCS_OK:
            raise XpcsError(st, _lib.xpcs_last_error(self.ctx.h).decode())
        self.streams[h.value] = (basis.rings.n_q, history)
        return h.value

    def submit(self, s: int, frames) -> int:
        t = C.c_uint64()
        self.ctx.check(_lib.xpcs_server_submit(self.h, s, _ptr(frames), int(frames.shape[0]), C.byref(t)))
        return t.value

    def submit_device(self, s: int, frames) -> int:
        """Queue device frames by pointer; they must stay unchanged until the ticket completes."""
        t = C.c_uint64()
        self.ctx.check(_lib.xpcs_server_submit_device(self.h, s, _ptr(frames), int(frames.shape[0]), C.byref(t)))
        return t.value

    def poll(self, s: int, ticket: int, timeout_ms: int = 0) -> bool:
        st = _lib.xpcs_server_poll(self.h, s, ticket, timeout_ms)
        if st == XPCS_EBUSY:
            return False
        self.ctx.check(st)
        return True

    def read_g2(self, s: int):
        n_q, W = self.streams[s]
        g2 = np.empty((n_q, W))
        cnt = np.empty((n_q, W), dtype=np.int64)
        self.ctx.check(_lib.xpcs_server_read_g2(self.h, s, g2.ctypes.data, cnt.ctypes.data))
        return g2, cnt

    def latency(self, s: int, reset: bool = False) -> dict:
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        n = C.c_int64()
        self.ctx.check(_lib.xpcs_server_latency(self.h, s, 1 if reset else 0, C.byref(a), C.byref(b), C.byref(c),
                                                C.byref(n)))
        return {"p50_us": a.value, "p99_us": b.value, "max_us": c.value, "frames": n.value}

    def close_stream(self, s: int):
        self.ctx.check(_lib.xpcs_server_close(self.h, s))
        self.streams.pop(s, None)

    def batches(self) -> int:
        return int(_lib.xpcs_server_batches(self.h))

    def close(self):
        if self.h and self.ctx.h:
            _lib.xpcs_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

