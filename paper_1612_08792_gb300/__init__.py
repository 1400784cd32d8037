"""GB300-native GMM superpixels (Ban, Liu, Cao, arXiv 1612.08792).

Thin Python binding over the C ABI of ``libgmmsp.so`` (``include/gmmsp.h``).
Every function of the C ABI is exposed under the same name and only
marshals arguments: images, labels and streams are passed as raw device
pointers taken from torch tensors; every step of the computation runs in
the library's CUDA kernels.  There is no CPU fallback: if the library has
not been built, or no CUDA device is present, calls raise.

Convenience layer: :class:`Superpixels` owns one context and offers
``em_iters`` / ``labels`` / ``segment`` on torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

__all__ = [
    "GMMSP_RGB8", "GMMSP_LAB32", "GMMSP_PREC_MIXED", "GMMSP_PREC_FP32", "GmmspError",
    "gmmsp_params", "load_library", "library_path", "Superpixels",
    "gmmsp_default_params", "gmmsp_init", "gmmsp_reinit", "gmmsp_em_iters", "gmmsp_labels",
    "gmmsp_segment", "gmmsp_get_lab", "gmmsp_get_grid", "gmmsp_get_params", "gmmsp_set_params", "gmmsp_get_stats",
    "gmmsp_profile_kernel", "gmmsp_probe_peaks", "gmmsp_probe_fp64_helpers", "gmmsp_set_timing", "gmmsp_get_timing", "gmmsp_set_launch", "gmmsp_get_launch",
    "gmmsp_autotune", "gmmsp_segment_lab_noalloc", "gmmsp_last_error", "SuperpixelsBatch", "gmmsp_bounds_status",
    "gmmsp_batch_create", "gmmsp_batch_segment", "gmmsp_batch_get_params", "gmmsp_batch_autotune",
    "gmmsp_batch_set_launch", "gmmsp_batch_set_tuning", "gmmsp_batch_info", "gmmsp_batch_destroy", "gmmsp_status_string", "gmmsp_destroy",
    "gmmsp_batch_get_tuning", "gmmsp_batch_set_first_pass", "gmmsp_batch_get_first_pass",
    "gmmsp_batch_first_pass_partials", "gmmsp_batch_set_init_net", "gmmsp_batch_lab", "gmmsp_batch_targets", "gmmsp_batch_get_lab",
    "gmmsp_net_param_count", "gmmsp_net_create", "gmmsp_net_set_weights", "gmmsp_net_get_weights",
    "gmmsp_net_forward", "gmmsp_net_grad", "gmmsp_net_adam", "gmmsp_net_train_step", "gmmsp_net_get_activation",
    "gmmsp_net_check", "gmmsp_net_destroy", "gmmsp_net_get_adam", "gmmsp_net_set_adam", "gmmsp_set_init", "gmmsp_init_from_net", "gmmsp_tc_wait_selftest",
    "GMMSP_OK", "GMMSP_E_INVALID", "GMMSP_E_CUDA", "GMMSP_E_NOMEM", "GMMSP_E_NUMERIC", "GMMSP_E_TIMEOUT",
    "GMMSP_E_STATE", "gmmsp_segmentation_metrics", "gmmsp_enforce_connectivity", "gmmsp_connectivity",
    "gmmsp_batch_connectivity", "gmmsp_segmentation_metrics_many", "GMMSP_GRAY8", "GMMSP_COLOUR_FULL", "GMMSP_COLOUR_SPLIT", "GMMSP_COLOUR_GRAY",
]

GMMSP_RGB8, GMMSP_LAB32, GMMSP_GRAY8 = 0, 1, 2
GMMSP_COLOUR_FULL, GMMSP_COLOUR_SPLIT, GMMSP_COLOUR_GRAY = 0, 1, 2
_COLOUR = {"full": GMMSP_COLOUR_FULL, "split": GMMSP_COLOUR_SPLIT, "gray": GMMSP_COLOUR_GRAY}


def colour_model(colour) -> int:
    """GMMSP_COLOUR_* from a name ("full", "split", "gray") or the constant itself."""
    c = _COLOUR.get(colour, None) if isinstance(colour, str) else int(colour)
    if c not in (GMMSP_COLOUR_FULL, GMMSP_COLOUR_SPLIT, GMMSP_COLOUR_GRAY):
        raise ValueError(f"unknown colour model {colour!r}")
    return c

GMMSP_PREC_MIXED, GMMSP_PREC_FP32 = 0, 1
GMMSP_OK, GMMSP_E_INVALID, GMMSP_E_CUDA, GMMSP_E_NOMEM, GMMSP_E_NUMERIC, GMMSP_E_TIMEOUT, GMMSP_E_STATE = range(7)
STATUS = {0: "GMMSP_OK", 1: "GMMSP_E_INVALID", 2: "GMMSP_E_CUDA", 3: "GMMSP_E_NOMEM",
          4: "GMMSP_E_NUMERIC", 5: "GMMSP_E_TIMEOUT", 6: "GMMSP_E_STATE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The library to load: GMMSP_LIBRARY if set (e.g. the bounds-checked build,
    _build/libgmmsp_checked.so), else _build/libgmmsp.so."""
    return os.environ.get("GMMSP_LIBRARY") or os.path.join(_HERE, "_build", "libgmmsp.so")


class GmmspError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {message}")


class gmmsp_params(ctypes.Structure):
    """Mirror of the C struct ``gmmsp_params`` (include/gmmsp.h)."""
    _fields_ = [("spacing", ctypes.c_int), ("K", ctypes.c_int), ("eps_s", ctypes.c_float),
                ("eps_c", ctypes.c_float), ("lambda_c", ctypes.c_float),
                ("input_format", ctypes.c_int), ("precision", ctypes.c_int), ("colour_model", ctypes.c_int)]


def load_library(path: str | None = None):
    """Loads libgmmsp.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libgmmsp.so not found at {path}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        pint = ctypes.POINTER(ctypes.c_int)
        pll = ctypes.POINTER(ctypes.c_longlong)
        sig = {
            "gmmsp_default_params": (None, [ctypes.POINTER(gmmsp_params)]),
            "gmmsp_init": (I, [PP, P, I, I, I, ctypes.POINTER(gmmsp_params), P]),
            "gmmsp_reinit": (I, [P, P, I]),
            "gmmsp_em_iters": (I, [P, I, P]),
            "gmmsp_labels": (I, [P, P, P]),
            "gmmsp_segment": (I, [P, P, I, I, P, P]),
            "gmmsp_get_lab": (I, [P, P]),
            "gmmsp_get_grid": (I, [P, pint, pint, pint, pint]),
            "gmmsp_get_params": (I, [P, P, P, P]),
            "gmmsp_set_params": (I, [P, P, P, P]),
            "gmmsp_get_stats": (I, [P, pll, pll, pll]),
            "gmmsp_profile_kernel": (I, [P, I, I, P, P, ctypes.c_ulonglong, ctypes.POINTER(D)]),
            "gmmsp_set_timing": (I, [P, I]),
            "gmmsp_get_timing": (I, [P, P, I, pint]),
            "gmmsp_set_launch": (I, [P, I]),
            "gmmsp_get_launch": (I, [P, pint]),
            "gmmsp_autotune": (I, [P, I, pint, P]),
            "gmmsp_last_error": (ctypes.c_char_p, [P]),
            "gmmsp_status_string": (ctypes.c_char_p, [I]),
            "gmmsp_destroy": (None, [P]),
            "gmmsp_bounds_status": (I, [pint, ctypes.POINTER(ctypes.c_ulonglong)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


BOUNDS_SITES = {1: "gp", 2: "pixel_x", 3: "pixel_y", 4: "partial_write", 5: "partial_read", 6: "theta",
                7: "label", 8: "label_value", 9: "cell_ll", 10: "batch_image", 11: "batch_item"}


def gmmsp_bounds_status():
    """(checked, first violation or None): whether this library was built with
    GMMSP_CHECK_BOUNDS and, if so, the first out-of-range index its EM kernels met
    since the last call, as {"site": name, "index": i} (reading clears it)."""
    checked, code = ctypes.c_int(), ctypes.c_ulonglong()
    st = load_library().gmmsp_bounds_status(ctypes.byref(checked), ctypes.byref(code))
    if st != 0:
        raise GmmspError(st, "bounds status")
    return bool(checked.value), bounds_decode(code.value)


def bounds_decode(code: int):
    """A gmmsp_bounds_status word -> None or {"site", "index"} (index sign-extended from 40 bits)."""
    if not code:
        return None
    site = (code >> 40) & 0x7FFFFF
    idx = code & ((1 << 40) - 1)
    if idx >= 1 << 39:
        idx -= 1 << 40
    return {"site": BOUNDS_SITES.get(site, site), "index": idx}


def _check(ctx, st: int):
    if st != 0:
        msg = ""
        if ctx:
            msg = (load_library().gmmsp_last_error(ctx) or b"").decode()
        raise GmmspError(st, msg)


def _dptr(t) -> int:
    """Device pointer of a CUDA torch tensor (or an int address)."""
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor (device memory)")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


# ------------------------------------------------------------------ C ABI, same names
def gmmsp_default_params() -> gmmsp_params:
    p = gmmsp_params()
    load_library().gmmsp_default_params(ctypes.byref(p))
    return p


def gmmsp_init(image, width: int, height: int, pitch_bytes: int, params: gmmsp_params, stream=None):
    ctx = ctypes.c_void_p()
    st = load_library().gmmsp_init(ctypes.byref(ctx), _dptr(image), int(width), int(height),
                                   int(pitch_bytes), ctypes.byref(params), _stream_handle(stream))
    _check(None, st)
    return ctx


def gmmsp_reinit(ctx, image, pitch_bytes: int) -> None:
    _check(ctx, load_library().gmmsp_reinit(ctx, _dptr(image), int(pitch_bytes)))


def gmmsp_em_iters(ctx, iters: int, want_loglik: bool = False):
    ll = np.zeros(max(iters, 1), dtype=np.float64) if want_loglik else None
    _check(ctx, load_library().gmmsp_em_iters(
        ctx, int(iters), ll.ctypes.data_as(ctypes.c_void_p) if ll is not None else None))
    return ll[:iters] if ll is not None else None


def gmmsp_labels(ctx, labels, want_loglik: bool = False):
    ll = np.zeros(1, dtype=np.float64) if want_loglik else None
    _check(ctx, load_library().gmmsp_labels(
        ctx, _dptr(labels), ll.ctypes.data_as(ctypes.c_void_p) if ll is not None else None))
    return float(ll[0]) if ll is not None else None


def gmmsp_segment(ctx, image, pitch_bytes: int, iters: int, labels, want_loglik: bool = False):
    ll = np.zeros(iters + 1, dtype=np.float64) if want_loglik else None
    _check(ctx, load_library().gmmsp_segment(
        ctx, _dptr(image), int(pitch_bytes), int(iters), _dptr(labels),
        ll.ctypes.data_as(ctypes.c_void_p) if ll is not None else None))
    return ll


def gmmsp_get_lab(ctx, H: int, W: int):
    out = np.zeros((H, W, 3), dtype=np.float32)
    _check(ctx, load_library().gmmsp_get_lab(ctx, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def gmmsp_get_grid(ctx):
    v, nx, ny, K = (ctypes.c_int() for _ in range(4))
    _check(ctx, load_library().gmmsp_get_grid(ctx, ctypes.byref(v), ctypes.byref(nx),
                                              ctypes.byref(ny), ctypes.byref(K)))
    return v.value, nx.value, ny.value, K.value


def gmmsp_get_params(ctx):
    K = gmmsp_get_grid(ctx)[3]
    mu, cs, cc = np.zeros((K, 5)), np.zeros((K, 3)), np.zeros((K, 6))
    _check(ctx, load_library().gmmsp_get_params(ctx, mu.ctypes.data_as(ctypes.c_void_p),
                                                cs.ctypes.data_as(ctypes.c_void_p),
                                                cc.ctypes.data_as(ctypes.c_void_p)))
    return mu, cs, cc


def gmmsp_set_params(ctx, mu, cs, cc) -> None:
    K = gmmsp_get_grid(ctx)[3]
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(K, 5)
    cs = np.ascontiguousarray(cs, dtype=np.float64).reshape(K, 3)
    cc = np.ascontiguousarray(cc, dtype=np.float64).reshape(K, 6)
    _check(ctx, load_library().gmmsp_set_params(ctx, mu.ctypes.data_as(ctypes.c_void_p),
                                                cs.ctypes.data_as(ctypes.c_void_p),
                                                cc.ctypes.data_as(ctypes.c_void_p)))


def gmmsp_get_stats(ctx):
    d, rs, rc = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(ctx, load_library().gmmsp_get_stats(ctx, ctypes.byref(d), ctypes.byref(rs), ctypes.byref(rc)))
    return d.value, rs.value, rc.value


GMMSP_KERNEL_EM_PASS, GMMSP_KERNEL_LABELS, GMMSP_KERNEL_FINALIZE = 0, 1, 2


def gmmsp_set_timing(ctx, enable: bool) -> None:
    _check(ctx, load_library().gmmsp_set_timing(ctx, int(bool(enable))))


def gmmsp_get_timing(ctx):
    buf = np.zeros(4096)
    n = ctypes.c_int()
    _check(ctx, load_library().gmmsp_get_timing(ctx, buf.ctypes.data_as(ctypes.c_void_p), 4096,
                                                ctypes.byref(n)))
    return buf[:min(n.value, 4096)].copy()


def gmmsp_set_launch(ctx, warps_per_cell: int) -> None:
    _check(ctx, load_library().gmmsp_set_launch(ctx, int(warps_per_cell)))


def gmmsp_get_launch(ctx) -> int:
    w = ctypes.c_int()
    _check(ctx, load_library().gmmsp_get_launch(ctx, ctypes.byref(w)))
    return w.value


def gmmsp_autotune(ctx, reps: int = 5):
    best = ctypes.c_int()
    times = np.zeros(3)
    _check(ctx, load_library().gmmsp_autotune(ctx, int(reps), ctypes.byref(best),
                                              times.ctypes.data_as(ctypes.c_void_p)))
    return best.value, dict(zip((1, 2, 4), times.tolist()))


def gmmsp_profile_kernel(ctx, which: int, reps: int, labels=None, flush=None) -> float:
    ms = ctypes.c_double()
    fptr = _dptr(flush) if flush is not None else None
    fbytes = int(flush.numel() * flush.element_size()) if flush is not None else 0
    _check(ctx, load_library().gmmsp_profile_kernel(
        ctx, int(which), int(reps), _dptr(labels) if labels is not None else None, fptr, fbytes,
        ctypes.byref(ms)))
    return ms.value


class gmmsp_peaks(ctypes.Structure):
    """Mirror of ``gmmsp_peaks`` (include/gmmsp_probe.h)."""
    _fields_ = [("sm_count", ctypes.c_int), ("clock_mhz", ctypes.c_int),
                ("fp32_fma_tflops", ctypes.c_double), ("fp64_fma_tflops", ctypes.c_double),
                ("fp64_fma_tflops_lane1", ctypes.c_double), ("mufu_ex2_tops", ctypes.c_double),
                ("fp32_fma_latency_clk", ctypes.c_double), ("fp64_fma_latency_clk", ctypes.c_double),
                ("fp32x2_fma_tflops", ctypes.c_double)]


def gmmsp_probe_peaks() -> dict:
    lib = load_library()
    f = lib.gmmsp_probe_peaks
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(gmmsp_peaks), ctypes.c_char_p, ctypes.c_int]
    out = gmmsp_peaks()
    err = ctypes.create_string_buffer(256)
    st = f(ctypes.byref(out), err, 256)
    if st != 0:
        raise GmmspError(2, err.value.decode())
    return {name: getattr(out, name) for name, _ in gmmsp_peaks._fields_}


def gmmsp_probe_fp64_helpers(x):
    """The finalize's FP64 reciprocal, square root and log2 helpers on a float64 CUDA tensor x:
    returns (1/x, sqrt(x), log2(x)) as CUDA tensors (float64, float64, float32)."""
    import torch
    lib = load_library()
    f = lib.gmmsp_probe_fp64_helpers
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
    x = x.contiguous()
    rcp, sq = torch.empty_like(x), torch.empty_like(x)
    lg = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    err = ctypes.create_string_buffer(256)
    st = f(_dptr(x), int(x.numel()), _dptr(rcp), _dptr(sq), _dptr(lg),
           _stream_handle(torch.cuda.current_stream()), err, 256)
    if st != 0:
        raise GmmspError(st, err.value.decode())
    return rcp, sq, lg


def gmmsp_segment_lab_noalloc(lab, width: int, height: int, pitch_bytes: int, params: gmmsp_params,
                              iters: int, labels, stream=None) -> None:
    """Allocation-free pipeline on a CIELAB float32 image (see include/gmmsp.h)."""
    lib = load_library()
    f = lib.gmmsp_segment_lab_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(gmmsp_params),
                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
    err = ctypes.create_string_buffer(256)
    st = f(_dptr(lab), int(width), int(height), int(pitch_bytes), ctypes.byref(params), int(iters),
           _dptr(labels), _stream_handle(stream), err, 256)
    if st != 0:
        raise GmmspError(st, err.value.decode())



def _batch_lib():
    lib = load_library()
    if not getattr(lib, "_batch_sigs", False):
        P, I = ctypes.c_void_p, ctypes.c_int
        PP = ctypes.POINTER(ctypes.c_void_p)
        pint = ctypes.POINTER(ctypes.c_int)
        sig = {
            "gmmsp_batch_create": (I, [PP, I, P, P, ctypes.POINTER(gmmsp_params), P]),
            "gmmsp_batch_segment": (I, [P, P, P, I, P, P]),
            "gmmsp_batch_get_params": (I, [P, I, P, P, P]),
            "gmmsp_batch_autotune": (I, [P, P, P, P, I, pint, P]),
            "gmmsp_batch_set_launch": (I, [P, I]),
            "gmmsp_batch_set_tuning": (I, [P, I, I]),
            "gmmsp_batch_info": (I, [P, ctypes.POINTER(ctypes.c_longlong), pint, pint]),
            "gmmsp_batch_get_lab": (I, [P, I, P]),
            "gmmsp_batch_get_tuning": (I, [P, pint, pint, P]),
            "gmmsp_batch_set_first_pass": (I, [P, I]),
            "gmmsp_batch_get_first_pass": (I, [P, pint, P]),
            "gmmsp_batch_first_pass_partials": (I, [P, P, P, P, I, I, P, P]),
            "gmmsp_batch_last_error": (ctypes.c_char_p, [P]),
            "gmmsp_batch_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        lib._batch_sigs = True
    return lib


def _bcheck(b, st):
    if st != 0:
        msg = (_batch_lib().gmmsp_batch_last_error(b) or b"").decode() if b else ""
        raise GmmspError(st, msg)


def gmmsp_batch_create(widths, heights, params: gmmsp_params, stream=None):
    n = len(widths)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    h = np.ascontiguousarray(heights, dtype=np.int32)
    out = ctypes.c_void_p()
    _bcheck(None, _batch_lib().gmmsp_batch_create(ctypes.byref(out), n, w.ctypes.data_as(ctypes.c_void_p),
                                                  h.ctypes.data_as(ctypes.c_void_p), ctypes.byref(params),
                                                  _stream_handle(stream)))
    return out


def _ptr_array(tensors):
    """A C array of device addresses: from tensors (or addresses), or passed through when it is
    one already (callers that keep their arrays skip rebuilding them on every call)."""
    if isinstance(tensors, ctypes.Array):
        return tensors
    return (ctypes.c_void_p * len(tensors))(*[_dptr(t) for t in tensors])


def gmmsp_batch_segment(b, images, pitches, iters, labels, want_loglik=False):
    n = len(images)
    pit = np.ascontiguousarray(pitches, dtype=np.int32)
    ll = np.zeros(n) if want_loglik else None
    _bcheck(b, _batch_lib().gmmsp_batch_segment(b, _ptr_array(images), pit.ctypes.data_as(ctypes.c_void_p),
                                                int(iters), _ptr_array(labels),
                                                ll.ctypes.data_as(ctypes.c_void_p) if ll is not None else None))
    return ll


def gmmsp_batch_get_params(b, i, K):
    mu, cs, cc = np.zeros((K, 5)), np.zeros((K, 3)), np.zeros((K, 6))
    _bcheck(b, _batch_lib().gmmsp_batch_get_params(b, int(i), mu.ctypes.data_as(ctypes.c_void_p),
                                                   cs.ctypes.data_as(ctypes.c_void_p),
                                                   cc.ctypes.data_as(ctypes.c_void_p)))
    return mu, cs, cc


def gmmsp_batch_autotune(b, images, pitches, labels, reps=3):
    pit = np.ascontiguousarray(pitches, dtype=np.int32)
    best = ctypes.c_int()
    times = np.zeros(5)
    _bcheck(b, _batch_lib().gmmsp_batch_autotune(b, _ptr_array(images), pit.ctypes.data_as(ctypes.c_void_p),
                                                 _ptr_array(labels), int(reps), ctypes.byref(best),
                                                 times.ctypes.data_as(ctypes.c_void_p)))
    return best.value, dict(zip((3, 4, 5, 6, 7), times.tolist()))


def gmmsp_batch_first_pass_partials(b, images, pitches, labels, blocks_per_sm: int, diagonal: bool):
    """One E + M pass from the start; the per-cell partials as a (cells, 136) float32 array."""
    lib = _batch_lib()
    nf = ctypes.c_longlong()
    _bcheck(b, lib.gmmsp_batch_first_pass_partials(b, None, None, None, int(blocks_per_sm), int(bool(diagonal)),
                                                   None, ctypes.byref(nf)))
    out = np.empty(nf.value, dtype=np.float32)
    pit = np.ascontiguousarray(pitches, dtype=np.int32)
    _bcheck(b, lib.gmmsp_batch_first_pass_partials(b, _ptr_array(images), pit.ctypes.data_as(ctypes.c_void_p),
                                                   _ptr_array(labels), int(blocks_per_sm), int(bool(diagonal)),
                                                   out.ctypes.data_as(ctypes.c_void_p), None))
    return out.reshape(-1, 136)


def gmmsp_batch_set_launch(b, blocks_per_sm: int) -> None:
    _bcheck(b, _batch_lib().gmmsp_batch_set_launch(b, int(blocks_per_sm)))


def gmmsp_batch_set_tuning(b, blocks_per_sm: int, finalize16: bool) -> None:
    _bcheck(b, _batch_lib().gmmsp_batch_set_tuning(b, int(blocks_per_sm), 1 if finalize16 else 0))


def gmmsp_batch_info(b):
    pix, K, cells = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
    _bcheck(b, _batch_lib().gmmsp_batch_info(b, ctypes.byref(pix), ctypes.byref(K), ctypes.byref(cells)))
    return pix.value, K.value, cells.value


def gmmsp_batch_get_lab(b, i, H, W):
    out = np.zeros((H, W, 3), dtype=np.float32)
    _bcheck(b, _batch_lib().gmmsp_batch_get_lab(b, int(i), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def gmmsp_batch_set_first_pass(b, blocks_per_sm: int) -> None:
    """Blocks per SM of a segment's first E + M pass (0: as the other passes)."""
    _bcheck(b, _batch_lib().gmmsp_batch_set_first_pass(b, int(blocks_per_sm)))


def gmmsp_batch_get_first_pass(b):
    """(blocks per SM in effect, {6: ms, 7: ms} of the autotuned diagonal kernels)."""
    bps = ctypes.c_int()
    ms = np.zeros(2)
    _bcheck(b, _batch_lib().gmmsp_batch_get_first_pass(b, ctypes.byref(bps), ms.ctypes.data_as(ctypes.c_void_p)))
    return bps.value, {6: float(ms[0]), 7: float(ms[1])}


def gmmsp_batch_get_tuning(b):
    bps, f16 = ctypes.c_int(), ctypes.c_int()
    ms = np.zeros(2)
    _bcheck(b, _batch_lib().gmmsp_batch_get_tuning(b, ctypes.byref(bps), ctypes.byref(f16),
                                                   ms.ctypes.data_as(ctypes.c_void_p)))
    first, first_ms = gmmsp_batch_get_first_pass(b)
    return {"blocks_per_sm": bps.value, "finalize16": bool(f16.value),
            "finalize_ms": {"16_lanes": float(ms[0]), "thread_per_superpixel": float(ms[1])},
            "first_pass_blocks_per_sm": first,
            "first_pass_diag_ms": {str(k): v for k, v in first_ms.items()}}


def gmmsp_batch_destroy(b) -> None:
    _batch_lib().gmmsp_batch_destroy(b)


def _net_lib():
    lib = load_library()
    if not getattr(lib, "_net_sigs", False):
        P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        PP = ctypes.POINTER(ctypes.c_void_p)
        LL = ctypes.c_longlong
        PD = ctypes.POINTER(ctypes.c_double)
        sig = {
            "gmmsp_net_param_count": (LL, []),
            "gmmsp_net_create": (I, [PP, I, P]),
            "gmmsp_net_set_weights": (I, [P, P, LL]),
            "gmmsp_net_get_weights": (I, [P, P, LL]),
            "gmmsp_net_get_adam": (I, [P, P, P, LL, ctypes.POINTER(LL)]),
            "gmmsp_net_set_adam": (I, [P, P, P, LL, LL]),
            "gmmsp_net_forward": (I, [P, P, I, I, I, P]),
            "gmmsp_net_grad": (I, [P, P, I, I, I, P, P, PD]),
            "gmmsp_net_adam": (I, [P, F, F, F, F]),
            "gmmsp_net_train_step": (I, [P, P, I, I, I, P, F, PD]),
            "gmmsp_net_check": (I, [P]),
            "gmmsp_net_get_activation": (I, [P, I, P, LL]),
            "gmmsp_tc_wait_selftest": (I, [I, P]),
            "gmmsp_net_last_error": (ctypes.c_char_p, [P]),
            "gmmsp_net_destroy": (None, [P]),
            "gmmsp_init_from_net": (I, [P, P]),
            "gmmsp_set_init": (I, [P, P, P]),
            "gmmsp_batch_set_init_net": (I, [P, P]),
            "gmmsp_batch_lab": (I, [P, PP]),
            "gmmsp_batch_targets": (I, [P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        lib._net_sigs = True
    return lib


def _ncheck(n, st):
    if st != 0:
        msg = (_net_lib().gmmsp_net_last_error(n) or b"").decode() if n else ""
        raise GmmspError(st, msg)


def gmmsp_net_param_count() -> int:
    return int(_net_lib().gmmsp_net_param_count())


def gmmsp_net_create(spacing: int, stream=None):
    out = ctypes.c_void_p()
    _ncheck(None, _net_lib().gmmsp_net_create(ctypes.byref(out), int(spacing), _stream_handle(stream)))
    return out


def gmmsp_net_set_weights(n, weights) -> None:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _ncheck(n, _net_lib().gmmsp_net_set_weights(n, w.ctypes.data_as(ctypes.c_void_p), w.size))


def gmmsp_net_get_weights(n):
    w = np.zeros(gmmsp_net_param_count(), dtype=np.float32)
    _ncheck(n, _net_lib().gmmsp_net_get_weights(n, w.ctypes.data_as(ctypes.c_void_p), w.size))
    return w


def gmmsp_net_get_adam(n):
    """(m, v, step): the Adam moments (float32 host arrays) and the step count."""
    m = np.zeros(gmmsp_net_param_count(), dtype=np.float32)
    v = np.zeros_like(m)
    step = ctypes.c_longlong()
    _ncheck(n, _net_lib().gmmsp_net_get_adam(n, m.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p),
                                             m.size, ctypes.byref(step)))
    return m, v, int(step.value)


def gmmsp_net_set_adam(n, m, v, step: int) -> None:
    m = np.ascontiguousarray(m, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    if m.shape != v.shape:
        raise ValueError("m and v must have one shape")
    _ncheck(n, _net_lib().gmmsp_net_set_adam(n, m.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p),
                                             m.size, int(step)))


def gmmsp_net_forward(n, lab, B: int, W: int, H: int, out) -> None:
    """lab: B images of CIELAB planes, a float32 CUDA tensor (kept referenced while the work is
    queued) or a device address the caller keeps alive until the work has run."""
    _ncheck(n, _net_lib().gmmsp_net_forward(n, _dptr(lab), int(B), int(W), int(H), _dptr(out)))


def gmmsp_net_grad(n, lab, B: int, W: int, H: int, target, want_grad: bool = True):
    g = np.zeros(gmmsp_net_param_count(), dtype=np.float32) if want_grad else None
    loss = ctypes.c_double()
    _ncheck(n, _net_lib().gmmsp_net_grad(n, _dptr(lab), int(B), int(W), int(H), _dptr(target),
                                         g.ctypes.data_as(ctypes.c_void_p) if g is not None else None,
                                         ctypes.byref(loss)))
    return loss.value, g


def gmmsp_net_adam(n, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    _ncheck(n, _net_lib().gmmsp_net_adam(n, lr, beta1, beta2, eps))


def gmmsp_net_train_step(n, lab, B: int, W: int, H: int, target, lr: float,
                         want_loss: bool = True):
    loss = ctypes.c_double()
    _ncheck(n, _net_lib().gmmsp_net_train_step(n, _dptr(lab), int(B), int(W), int(H), _dptr(target),
                                               float(lr), ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def gmmsp_net_get_activation(n, layer: int, cells: int):
    a = np.zeros((cells, 32), dtype=np.float32)
    _ncheck(n, _net_lib().gmmsp_net_get_activation(n, int(layer), a.ctypes.data_as(ctypes.c_void_p), a.size))
    return a


def gmmsp_tc_wait_selftest(max_tries: int = 1024, stream=None) -> int:
    """Status of the bounded-wait self-test (GMMSP_E_TIMEOUT = 5 is the expected outcome)."""
    return int(_net_lib().gmmsp_tc_wait_selftest(int(max_tries), _stream_handle(stream)))


def gmmsp_net_check(n) -> None:
    _ncheck(n, _net_lib().gmmsp_net_check(n))


def gmmsp_net_destroy(n) -> None:
    _net_lib().gmmsp_net_destroy(n)


def gmmsp_init_from_net(ctx, n) -> None:
    _check(ctx, _net_lib().gmmsp_init_from_net(ctx, n))


def gmmsp_set_init(ctx, dmu, logeig) -> None:
    """theta_0 from (K, 5) float32 CUDA arrays of mean offsets and log-eigenvalues (see gmmsp_cnn.h)."""
    for t in (dmu, logeig):
        if t.dim() != 2 or t.shape[1] != 5 or not t.is_contiguous():
            raise ValueError("dmu and logeig must be contiguous (K, 5) arrays")
    _check(ctx, _net_lib().gmmsp_set_init(ctx, _dptr(dmu), _dptr(logeig)))


def gmmsp_batch_set_init_net(b, n) -> None:
    _bcheck(b, _net_lib().gmmsp_batch_set_init_net(b, n))


def gmmsp_batch_lab(b) -> int:
    p = ctypes.c_void_p()
    _bcheck(b, _net_lib().gmmsp_batch_lab(b, ctypes.byref(p)))
    return int(p.value or 0)


def gmmsp_batch_targets(b, target) -> None:
    _bcheck(b, _net_lib().gmmsp_batch_targets(b, _dptr(target)))


class gmmsp_seg_metrics(ctypes.Structure):
    _fields_ = [("br", ctypes.c_double), ("ue", ctypes.c_double), ("asa", ctypes.c_double),
                ("br_recovered", ctypes.c_longlong), ("br_total", ctypes.c_longlong),
                ("ue_sum", ctypes.c_longlong), ("asa_sum", ctypes.c_longlong)]


def gmmsp_segmentation_metrics(labels, gt, K: int, G: int, radius: int = 2, eps: float = 0.05, stream=None):
    """BR, UE (Eq. ue) and ASA (Eq. asa) of an (H, W) int32 CUDA label map against an
    (H, W) int32 CUDA ground truth with ids in [0, G); synchronises."""
    lib = load_library()
    f = lib.gmmsp_segmentation_metrics
    if not getattr(f, "_sig", False):
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      ctypes.c_int, ctypes.c_double, ctypes.POINTER(gmmsp_seg_metrics), ctypes.c_void_p]
        f._sig = True
    H, W = int(labels.shape[0]), int(labels.shape[1])
    if tuple(gt.shape) != (H, W) or not labels.is_contiguous() or not gt.is_contiguous():
        raise ValueError("labels and gt must be contiguous (H, W) maps of one size")
    out = gmmsp_seg_metrics()
    st = f(_dptr(labels), _dptr(gt), W, H, int(K), int(G), int(radius), float(eps), ctypes.byref(out),
           _stream_handle(stream))
    if st != 0:
        raise GmmspError(st, "segmentation metrics failed (bad arguments or ids out of range)")
    return {k: getattr(out, k) for k, _ in gmmsp_seg_metrics._fields_}


def gmmsp_segmentation_metrics_many(labels, gts, Ks, Gs, radius: int = 2, eps: float = 0.05, stream=None):
    """The metrics of several (labels, gt) pairs in one call (lists of (H, W) int32 CUDA maps;
    Ks, Gs: per-image superpixel and segment counts, or one int for all); synchronises."""
    lib = load_library()
    f = lib.gmmsp_segmentation_metrics_many
    n = len(labels)
    if not getattr(f, "_sig", False):
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                      ctypes.POINTER(gmmsp_seg_metrics), ctypes.c_void_p]
        f._sig = True
    if len(gts) != n or n < 1:
        raise ValueError("one ground truth per label map")
    Ks = [int(Ks)] * n if isinstance(Ks, int) else [int(k) for k in Ks]
    Gs = [int(Gs)] * n if isinstance(Gs, int) else [int(g) for g in Gs]
    for l, g in zip(labels, gts):
        if tuple(g.shape) != tuple(l.shape) or not l.is_contiguous() or not g.is_contiguous():
            raise ValueError("labels and gt must be contiguous (H, W) maps of one size")
    Ws = np.array([int(l.shape[1]) for l in labels], dtype=np.int32)
    Hs = np.array([int(l.shape[0]) for l in labels], dtype=np.int32)
    Ka, Ga = np.array(Ks, dtype=np.int32), np.array(Gs, dtype=np.int32)
    out = (gmmsp_seg_metrics * n)()
    st = f(n, _ptr_array(labels), _ptr_array(gts), Ws.ctypes.data_as(ctypes.c_void_p),
           Hs.ctypes.data_as(ctypes.c_void_p), Ka.ctypes.data_as(ctypes.c_void_p), Ga.ctypes.data_as(ctypes.c_void_p),
           int(radius), float(eps), out, _stream_handle(stream))
    if st != 0:
        raise GmmspError(st, "segmentation metrics failed (bad arguments or ids out of range)")
    return [{k: getattr(o, k) for k, _ in gmmsp_seg_metrics._fields_} for o in out]


class gmmsp_conn_stats(ctypes.Structure):
    _fields_ = [("components", ctypes.c_longlong), ("small", ctypes.c_longlong), ("merged", ctypes.c_longlong)]


def _conn_lib():
    lib = load_library()
    if not getattr(lib, "_conn_sigs", False):
        P, I = ctypes.c_void_p, ctypes.c_int
        PS = ctypes.POINTER(gmmsp_conn_stats)
        for name, args in {"gmmsp_enforce_connectivity": [P, P, I, I, I, PS, P],
                           "gmmsp_connectivity": [P, P, PS],
                           "gmmsp_batch_connectivity": [P, P, PS]}.items():
            f = getattr(lib, name)
            f.restype = I
            f.argtypes = args
        lib._conn_sigs = True
    return lib


def _stats(st):
    return {"components": st.components, "small": st.small, "merged": st.merged}


def gmmsp_enforce_connectivity(labels, lab_planes, W: int, H: int, K: int, stream=None):
    """Algorithm 1, step 8 on an (H, W) int32 CUDA label map (rewritten in place);
    lab_planes: the CIELAB image as (3, H, W) float32 CUDA planes (or their address)."""
    st = gmmsp_conn_stats()
    r = _conn_lib().gmmsp_enforce_connectivity(_dptr(labels), _dptr(lab_planes), int(W), int(H), int(K),
                                               ctypes.byref(st), _stream_handle(stream))
    if r != 0:
        raise GmmspError(r, "connectivity post-processing failed")
    return _stats(st)


def gmmsp_connectivity(ctx, labels):
    st = gmmsp_conn_stats()
    _check(ctx, _conn_lib().gmmsp_connectivity(ctx, _dptr(labels), ctypes.byref(st)))
    return _stats(st)


def gmmsp_batch_connectivity(b, labels):
    st = gmmsp_conn_stats()
    _bcheck(b, _conn_lib().gmmsp_batch_connectivity(b, _ptr_array(labels), ctypes.byref(st)))
    return _stats(st)


class SuperpixelsBatch:
    """A batch context over lists of (H, W, 3) uint8 RGB (or float32 CIELAB, or (H, W)
    uint8 grey-level with gray_input) CUDA tensors.  colour: "full", "split" or "gray"."""

    def __init__(self, shapes, K: int = 0, spacing: int = 0, eps_s: float = 2.0, eps_c: float = 8.0,
                 lambda_c: float = 8.0, precision: int = GMMSP_PREC_MIXED, lab_input: bool = False,
                 stream=None, colour="full", gray_input: bool = False):
        import torch
        p = gmmsp_default_params()
        p.spacing, p.K, p.eps_s, p.eps_c, p.lambda_c = int(spacing), int(K), eps_s, eps_c, lambda_c
        p.input_format = GMMSP_GRAY8 if gray_input else (GMMSP_LAB32 if lab_input else GMMSP_RGB8)
        p.precision = int(precision)
        p.colour_model = colour_model(colour)
        self.params = (int(spacing), int(K), int(p.colour_model), int(precision))
        self.shapes = [(int(h), int(w)) for (h, w) in shapes]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.b = gmmsp_batch_create([w for _, w in self.shapes], [h for h, _ in self.shapes], p, self.stream)
        # the labels of all images in one buffer (image after image), one view per image
        self.labels_buffer = torch.empty(sum(h * w for h, w in self.shapes), dtype=torch.int32, device="cuda")
        self.labels, off = [], 0
        for h, w in self.shapes:
            self.labels.append(self.labels_buffer[off:off + h * w].view(h, w))
            off += h * w
        self._label_ptrs = _ptr_array(self.labels)

    @staticmethod
    def _pitch(t) -> int:
        return int(t.stride(0) * t.element_size())

    def segment(self, images, iters: int = 10, want_loglik: bool = False):
        ll = gmmsp_batch_segment(self.b, images, [self._pitch(t) for t in images], iters, self._label_ptrs,
                                 want_loglik)
        return (self.labels, ll) if want_loglik else self.labels

    def segment_stacked(self, images, iters: int = 10, want_loglik: bool = False):
        """segment() for a batch of images of one size given as one (n, H, W, C) (or, for
        grey levels, (n, H, W)) CUDA tensor whose rows are packed (each image's H rows
        pitch bytes apart): the image addresses are computed from its strides instead of
        being gathered from n tensors."""
        n = len(self.shapes)
        if images.shape[0] != n or any(sh != tuple(images.shape[1:3]) for sh in self.shapes):
            raise ValueError("segment_stacked wants one (n, H, W[, C]) tensor of the batch's (single) size")
        es = images.element_size()
        base = images.data_ptr()
        ptrs = (ctypes.c_void_p * n)(*[base + i * images.stride(0) * es for i in range(n)])
        pitches = np.full(n, images.stride(1) * es, dtype=np.int32)
        ll = gmmsp_batch_segment(self.b, ptrs, pitches, iters, self._label_ptrs, want_loglik)
        return (self.labels, ll) if want_loglik else self.labels

    def autotune(self, images, reps: int = 3, cache: str | None = None):
        """Times the E + M pass variants and the finalize variants and keeps the fastest;
        returns (blocks per SM, {blocks per SM: ms}).  With `cache` (a JSON file path) a
        tuning stored there for this GPU and batch shape is applied without timing, and a
        new tuning is stored."""
        key = None
        if cache:
            import torch
            from . import tuning_cache
            spacing, K, colour, precision = self.params
            key = tuning_cache.batch_key(torch.cuda.get_device_name(), self.shapes, spacing, K, colour, precision)
            hit = tuning_cache.lookup(cache, key)
            if hit is not None:
                gmmsp_batch_set_tuning(self.b, hit["blocks_per_sm"], hit["finalize16"])
                gmmsp_batch_set_first_pass(self.b, hit.get("first_pass_blocks_per_sm", 0))
                return hit["blocks_per_sm"], {int(k): float(v) for k, v in hit.get("em_pass_ms", {}).items()}
        best, times = gmmsp_batch_autotune(self.b, images, [self._pitch(t) for t in images], self.labels, reps)
        if key is not None:
            from . import tuning_cache
            t = self.tuning()
            tuning_cache.store(cache, key, {"blocks_per_sm": int(best), "finalize16": bool(t["finalize16"]),
                                            "first_pass_blocks_per_sm": int(t["first_pass_blocks_per_sm"]),
                                            "em_pass_ms": {str(k): v for k, v in times.items()},
                                            "finalize_ms": t["finalize_ms"]})
        return best, times

    def first_pass_partials(self, images, blocks_per_sm: int, diagonal: bool):
        """The per-cell partials of one E + M pass from the start (a check of the first-pass kernels)."""
        return gmmsp_batch_first_pass_partials(self.b, images, [self._pitch(t) for t in images], self.labels,
                                               blocks_per_sm, diagonal)

    def set_launch(self, blocks_per_sm: int, first_pass: int | None = None) -> None:
        """Blocks per SM of the E + M pass; `first_pass` that of a segment's first pass
        (None keeps the current choice, 0 follows `blocks_per_sm`)."""
        gmmsp_batch_set_launch(self.b, blocks_per_sm)
        if first_pass is not None:
            gmmsp_batch_set_first_pass(self.b, first_pass)

    def info(self):
        return gmmsp_batch_info(self.b)

    def tuning(self):
        return gmmsp_batch_get_tuning(self.b)

    def connectivity(self):
        """Algorithm 1, step 8 on the labels of the last segment (in place); totals."""
        return gmmsp_batch_connectivity(self.b, self.labels)

    def get_params(self, i: int, K: int):
        return gmmsp_batch_get_params(self.b, i, K)

    def get_lab(self, i: int):
        """Image i's CIELAB colours (H, W, 3) float32 as the last segment converted them."""
        H, W = self.shapes[i]
        return gmmsp_batch_get_lab(self.b, i, H, W)

    def set_init_net(self, net) -> None:
        """Start every later segment from the network's theta_0 (None: the paper's start)."""
        gmmsp_batch_set_init_net(self.b, net.n if net is not None else None)
        self._net = net

    def lab_ptr(self) -> int:
        """Device address of the batch's CIELAB planes (filled by segment)."""
        return gmmsp_batch_lab(self.b)

    def targets(self, out) -> None:
        """Training targets from the current theta into out (float32 CUDA, B K x 10)."""
        gmmsp_batch_targets(self.b, out)

    def close(self) -> None:
        if getattr(self, "b", None):
            gmmsp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gmmsp_last_error(ctx) -> str:
    return (load_library().gmmsp_last_error(ctx) or b"").decode()


def gmmsp_status_string(status: int) -> str:
    return load_library().gmmsp_status_string(int(status)).decode()


def gmmsp_destroy(ctx) -> None:
    load_library().gmmsp_destroy(ctx)


# ------------------------------------------------------------------ convenience
@dataclass
class Grid:
    v: int
    nx: int
    ny: int
    K: int


class Superpixels:
    """One library context over (H, W, 3) uint8 RGB or float32 CIELAB CUDA tensors, or
    (H, W) uint8 grey levels (grayscale colour model).  colour: "full", "split" or "gray"."""

    def __init__(self, image, K: int = 0, spacing: int = 0, eps_s: float = 2.0, eps_c: float = 8.0,
                 lambda_c: float = 8.0, precision: int = GMMSP_PREC_MIXED, stream=None, colour="full"):
        import torch
        if image.dim() == 2 and image.dtype == torch.uint8:
            fmt = GMMSP_GRAY8
        elif image.dim() != 3 or image.shape[2] != 3:
            raise ValueError("image must be (H, W, 3), or (H, W) uint8 grey levels")
        elif image.dtype == torch.uint8:
            fmt = GMMSP_RGB8
        elif image.dtype == torch.float32:
            fmt = GMMSP_LAB32
        else:
            raise ValueError("image must be uint8 sRGB or float32 CIELAB")
        p = gmmsp_default_params()
        p.spacing, p.K, p.eps_s, p.eps_c, p.lambda_c = int(spacing), int(K), eps_s, eps_c, lambda_c
        p.input_format, p.precision = fmt, int(precision)
        p.colour_model = colour_model(colour)
        self.H, self.W = int(image.shape[0]), int(image.shape[1])
        self.format = fmt
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = gmmsp_init(image, self.W, self.H, self._pitch(image), p, self.stream)
        self.grid = Grid(*gmmsp_get_grid(self.ctx))

    @staticmethod
    def _pitch(image) -> int:
        if image.dim() == 2:
            if image.stride(1) != 1:
                raise ValueError("grey-level rows must be packed (stride (pitch, 1))")
        elif image.stride(2) != 1 or image.stride(1) != 3:
            raise ValueError("image rows must be packed (stride (pitch, 3, 1))")
        return int(image.stride(0) * image.element_size())

    def reinit(self, image) -> None:
        gmmsp_reinit(self.ctx, image, self._pitch(image))

    def em_iters(self, iters: int, want_loglik: bool = False):
        return gmmsp_em_iters(self.ctx, iters, want_loglik)

    def labels(self, out=None, want_loglik: bool = False):
        import torch
        if out is None:
            out = torch.empty((self.H, self.W), dtype=torch.int32, device="cuda")
        ll = gmmsp_labels(self.ctx, out, want_loglik)
        return (out, ll) if want_loglik else out

    def segment(self, image, iters: int = 10, out=None, want_loglik: bool = False):
        import torch
        if out is None:
            out = torch.empty((self.H, self.W), dtype=torch.int32, device="cuda")
        ll = gmmsp_segment(self.ctx, image, self._pitch(image), iters, out, want_loglik)
        return (out, ll) if want_loglik else out

    def segment_host(self, image_host, labels_host, iters: int = 10, dev_image=None, dev_labels=None,
                     want_loglik: bool = False):
        """Host buffers in, host labels out: H2D copy, the graph-captured pipeline, D2H copy.

        image_host / labels_host should be pinned CPU tensors; dev_image / dev_labels
        are reusable device staging buffers (allocated on first use).
        """
        import torch
        with torch.cuda.stream(self.stream):
            if dev_image is None:
                dev_image = torch.empty_like(image_host, device="cuda")
            if dev_labels is None:
                dev_labels = torch.empty((self.H, self.W), dtype=torch.int32, device="cuda")
            dev_image.copy_(image_host, non_blocking=True)
            ll = gmmsp_segment(self.ctx, dev_image, self._pitch(dev_image), iters, dev_labels, want_loglik)
            labels_host.copy_(dev_labels, non_blocking=True)
        self.stream.synchronize()
        return ll

    def set_timing(self, enable: bool) -> None:
        gmmsp_set_timing(self.ctx, enable)

    def get_timing(self):
        return gmmsp_get_timing(self.ctx)

    def set_launch(self, warps_per_cell: int) -> None:
        gmmsp_set_launch(self.ctx, warps_per_cell)

    def get_launch(self) -> int:
        return gmmsp_get_launch(self.ctx)

    def autotune(self, reps: int = 5):
        return gmmsp_autotune(self.ctx, reps)

    def profile_kernel(self, which: int, reps: int = 20, labels=None, flush=None) -> float:
        return gmmsp_profile_kernel(self.ctx, which, reps, labels, flush)

    def get_lab(self):
        return gmmsp_get_lab(self.ctx, self.H, self.W)

    def connectivity(self, labels):
        """Algorithm 1, step 8 on `labels` (from this context's last labels / segment), in place."""
        return gmmsp_connectivity(self.ctx, labels)

    def init_from_net(self, net) -> None:
        """Replace theta by the network's theta_0 for the current image."""
        gmmsp_init_from_net(self.ctx, net.n)

    def set_init(self, dmu, logeig) -> None:
        """Replace theta by theta_0 from per-superpixel predictions: (K, 5) float32 CUDA
        arrays of mean offsets and log covariance diagonals (include/gmmsp_cnn.h)."""
        if dmu.shape[0] != self.grid.K or logeig.shape[0] != self.grid.K:
            raise ValueError("one row per superpixel")
        gmmsp_set_init(self.ctx, dmu, logeig)

    def get_params(self):
        return gmmsp_get_params(self.ctx)

    def set_params(self, mu, cs, cc) -> None:
        gmmsp_set_params(self.ctx, mu, cs, cc)

    def stats(self):
        return gmmsp_get_stats(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            gmmsp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
