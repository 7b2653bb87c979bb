"""Python binding of the GB300 optical-flow velocimetry library (libofv.so).

Argument marshalling only: every step of the estimator runs in the CUDA
kernels behind the C ABI declared in ``include/ofv.h``.  Functions carry the
C names.  Device buffers are passed as torch CUDA tensors (or raw integer
addresses); streams as ``torch.cuda.Stream`` objects (or raw handles); the
current torch stream is used when none is given.

Importing this package loads libofv.so and raises if it is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "OfvError", "Params", "ofv_default_params", "ofv_create", "ofv_destroy", "ofv_set_prefilter", "ofv_set_mask",
    "ofv_compute", "ofv_compute_host", "ofv_compute_sequence", "ofv_compute_sequence_host",
    "ofv_compute_noalloc", "ofv_compute_strips", "ofv_strip_plan", "ofv_compute_batched", "ofv_batch_tuning",
    "ofv_graph_create",
    "ofv_graph_create_batched", "ofv_graph_launch", "ofv_graph_destroy", "ofv_backward", "ofv_vorticity", "ofv_recirculation_area", "ofv_probe",
    "ofv_debug_fail_alloc", "ofv_debug_poison", "ofv_debug_reciprocal", "ofv_level_shape",
    "ofv_read_level",
    "ofv_profile_enable", "ofv_profile_read", "ofv_last_error", "ofv_status_string", "ofv_version",
    "Flow", "lib_path", "EXPORTED_SYMBOLS",
]

OFV_OK, OFV_ERR_INVALID_ARG, OFV_ERR_SHAPE, OFV_ERR_ALLOC, OFV_ERR_CUDA, OFV_ERR_TIMEOUT, OFV_ERR_UNSUPPORTED = range(7)
OFV_IN_U8, OFV_IN_U16, OFV_IN_F32 = range(3)
OFV_STORE_F32, OFV_STORE_F16, OFV_STORE_BF16 = range(3)
OFV_PATH_FUSED, OFV_PATH_PLAIN, OFV_PATH_TILE = range(3)
OFV_WINDOW_BOX, OFV_WINDOW_GAUSS = range(2)
OFV_K_INGEST, OFV_K_REDUCE, OFV_K_ITERATE, OFV_K_COUNT = range(4)
OFV_NOALLOC_SCRATCH_BYTES = 64 << 20

EXPORTED_SYMBOLS = [
    "ofv_default_params", "ofv_create", "ofv_destroy", "ofv_set_prefilter", "ofv_set_mask", "ofv_compute",
    "ofv_compute_host", "ofv_compute_sequence", "ofv_compute_sequence_host", "ofv_compute_noalloc",
    "ofv_graph_create", "ofv_graph_create_batched", "ofv_graph_launch",
    "ofv_graph_destroy", "ofv_compute_batched", "ofv_batch_tuning", "ofv_queue_selftest", "ofv_backward",
    "ofv_compute_strips", "ofv_strip_plan",
    "ofv_vorticity", "ofv_recirculation_area", "ofv_probe", "ofv_debug_fail_alloc", "ofv_debug_poison",
    "ofv_debug_reciprocal", "ofv_level_shape",
    "ofv_read_level",
    "ofv_profile_enable", "ofv_profile_read", "ofv_last_error", "ofv_status_string", "ofv_version",
]


class OfvError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {_status_name(status)}: {message}")


class Params(ctypes.Structure):
    """Mirror of ofv_params (include/ofv.h)."""
    _fields_ = [
        ("levels_psl", ctypes.c_int), ("kernel_radius", ctypes.c_int), ("iterations", ctypes.c_int),
        ("norm_radius", ctypes.c_int), ("input", ctypes.c_int), ("bit_depth", ctypes.c_int),
        ("storage", ctypes.c_int), ("path", ctypes.c_int), ("prefilter", ctypes.c_int),
        ("det_rel_eps", ctypes.c_float), ("det_abs_eps", ctypes.c_float), ("norm_eps", ctypes.c_float),
        ("max_batch", ctypes.c_int),
        ("window", ctypes.c_int), ("window_sigma", ctypes.c_float), ("increment_form", ctypes.c_int),
        ("warm_start", ctypes.c_int), ("tile_edge", ctypes.c_int),
    ]


class StripRows(ctypes.Structure):
    """Mirror of ofv_strip_rows (include/ofv.h)."""
    _fields_ = [(n, ctypes.c_int) for n in ("own_row0", "own_row1", "img_row0", "img_row1", "fld_row0", "fld_row1",
                                            "up_row0", "up_row1", "ingest_row0", "ingest_row1")]


def _load_library():
    path = _build.build_library()  # no-op when the library is up to date
    lib = ctypes.CDLL(path)
    P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    sig = {
        "ofv_default_params": ([ctypes.POINTER(Params)], None),
        "ofv_create": ([I, I, ctypes.POINTER(Params), ctypes.POINTER(P)], I),
        "ofv_destroy": ([P], I),
        "ofv_set_prefilter": ([P, P, P], I),
        "ofv_set_mask": ([P, P, P], I),
        "ofv_compute": ([P, P, P, P, P, P], I),
        "ofv_compute_host": ([P, P, P, P, P, P], I),
        "ofv_compute_sequence": ([P, I, P, Z, P, P, Z, P], I),
        "ofv_compute_sequence_host": ([P, I, P, Z, P, P, Z, P], I),
        "ofv_compute_noalloc": ([I, I, ctypes.POINTER(Params), P, P, P, P, P, P], I),
        "ofv_graph_create": ([P, P, P, P, P, ctypes.POINTER(P)], I),
        "ofv_graph_create_batched": ([P, I, P, ctypes.POINTER(P)], I),
        "ofv_graph_launch": ([P, P], I),
        "ofv_graph_destroy": ([P], I),
        "ofv_compute_batched": ([P, I, P, P], I),
        "ofv_compute_strips": ([P, I, I, P, P, P, P, P], I),
        "ofv_strip_plan": ([I, I, ctypes.POINTER(Params), I, I, I, I, ctypes.POINTER(StripRows)], I),
        "ofv_batch_tuning": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I)], I),
        "ofv_queue_selftest": ([I, ctypes.POINTER(I)], I),
        "ofv_backward": ([P, P, P, P, P, P, P, P, P], I),
        "ofv_vorticity": ([I, I, I, P, P, Z, P, P], I),
        "ofv_recirculation_area": ([I, I, I, P, Z, P, P, P], I),
        "ofv_probe": ([I, I, I, P, P, Z, I, P, P, P], I),
        "ofv_debug_fail_alloc": ([I], None),
        "ofv_debug_poison": ([P, P], I),
        "ofv_debug_reciprocal": ([P, P, I, P], I),
        "ofv_level_shape": ([P, I, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "ofv_read_level": ([P, I, I, P, P], I),
        "ofv_profile_enable": ([P, I], I),
        "ofv_profile_read": ([P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_double)], I),
        "ofv_last_error": ([], ctypes.c_char_p),
        "ofv_status_string": ([I], ctypes.c_char_p),
        "ofv_version": ([], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib, path


_lib, lib_path = _load_library()


def _status_name(st: int) -> str:
    return _lib.ofv_status_string(st).decode()


def _check(st: int, where: str):
    if st != OFV_OK:
        raise OfvError(st, where, _lib.ofv_last_error().decode())


def _addr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy array (host)
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# --- C names ----------------------------------------------------------------
def ofv_default_params(**overrides) -> Params:
    p = Params()
    _lib.ofv_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"ofv_params has no field {k}")
        setattr(p, k, v)
    return p


def ofv_create(H: int, W: int, params: Params | None = None) -> int:
    params = params or ofv_default_params()
    h = ctypes.c_void_p()
    _check(_lib.ofv_create(H, W, ctypes.byref(params), ctypes.byref(h)), "ofv_create")
    return h.value


def ofv_destroy(h: int):
    _check(_lib.ofv_destroy(h), "ofv_destroy")


def ofv_set_prefilter(h: int, w25, stream=None):
    _check(_lib.ofv_set_prefilter(h, _addr(w25), _stream(stream)), "ofv_set_prefilter")


def ofv_set_mask(h: int, mask, stream=None):
    """Region mask (H x W uint8 device tensor, nonzero = valid), or None to clear."""
    _check(_lib.ofv_set_mask(h, _addr(mask), _stream(stream)), "ofv_set_mask")


def ofv_compute(h: int, I1, I2, u, v, stream=None):
    _check(_lib.ofv_compute(h, _addr(I1), _addr(I2), _addr(u), _addr(v), _stream(stream)), "ofv_compute")


def ofv_compute_host(h: int, I1, I2, u, v, stream=None):
    _check(_lib.ofv_compute_host(h, _addr(I1), _addr(I2), _addr(u), _addr(v), _stream(stream)),
           "ofv_compute_host")


def ofv_compute_sequence(h: int, n_frames: int, frames, frame_stride_bytes: int, u, v, field_stride: int,
                         stream=None):
    _check(_lib.ofv_compute_sequence(h, n_frames, _addr(frames), frame_stride_bytes, _addr(u), _addr(v),
                                     field_stride, _stream(stream)), "ofv_compute_sequence")


def ofv_compute_sequence_host(h: int, n_frames: int, frames, frame_stride_bytes: int, u, v, field_stride: int,
                              stream=None):
    """frames, u, v are host buffers (pinned torch tensors or numpy arrays)."""
    _check(_lib.ofv_compute_sequence_host(h, n_frames, _addr(frames), frame_stride_bytes, _addr(u), _addr(v),
                                          field_stride, _stream(stream)), "ofv_compute_sequence_host")


def ofv_compute_noalloc(H: int, W: int, params: Params, w25, I1, I2, u, v, stream=None):
    """Same field as ofv_create + ofv_compute, for callers that must not
    allocate device memory: the workspace is the library's fixed scratch
    array (OFV_NOALLOC_SCRATCH_BYTES).  See include/ofv.h for its limits."""
    _check(_lib.ofv_compute_noalloc(H, W, ctypes.byref(params), _addr(w25), _addr(I1), _addr(I2), _addr(u),
                                    _addr(v), _stream(stream)), "ofv_compute_noalloc")


def ofv_compute_strips(h: int, nstrips: int, max_disp: int, I1, I2, u, v, stream=None):
    """One field computed as nstrips horizontal strips with their own
    workspaces and halo exchanges (the multi-GPU decomposition, run on the
    handle's device); bitwise ofv_compute's field while warps stay within
    max_disp px."""
    _check(_lib.ofv_compute_strips(h, nstrips, max_disp, _addr(I1), _addr(I2), _addr(u), _addr(v), _stream(stream)),
           "ofv_compute_strips")


def ofv_strip_plan(H: int, W: int, params: Params, nstrips: int, max_disp: int, level: int, strip: int) -> dict:
    """Rows strip `strip` works on at `level` (host only): own, img, fld, up
    and ingest as (first, end) pairs."""
    r = StripRows()
    _check(_lib.ofv_strip_plan(H, W, ctypes.byref(params), nstrips, max_disp, level, strip, ctypes.byref(r)),
           "ofv_strip_plan")
    return {k: (getattr(r, k + "_row0"), getattr(r, k + "_row1")) for k in ("own", "img", "fld", "up", "ingest")}


def ofv_backward(h: int, I1, I2, gu, gv, gI1, gI2, gw25=None, stream=None):
    """Reverse mode: gI1, gI2 (H x W float32) and gw25 (25 float32, or None)
    receive dL/dI1, dL/dI2, dL/dw for dL/du = gu, dL/dv = gv."""
    _check(_lib.ofv_backward(h, _addr(I1), _addr(I2), _addr(gu), _addr(gv), _addr(gI1), _addr(gI2), _addr(gw25),
                             _stream(stream)), "ofv_backward")


def ofv_vorticity(H: int, W: int, n: int, u, v, field_stride: int, omega, stream=None):
    """omega = dv/dx - du/dy of n fields (device)."""
    _check(_lib.ofv_vorticity(H, W, n, _addr(u), _addr(v), field_stride, _addr(omega), _stream(stream)),
           "ofv_vorticity")


def ofv_probe(H: int, W: int, n: int, u, v, field_stride: int, npts: int, xy, out, stream=None):
    """(u, v) of n fields at npts points xy (npts x 2 float32, device) into
    out (n x npts x 2 float32, device), bilinear, clamp-to-edge."""
    _check(_lib.ofv_probe(H, W, n, _addr(u), _addr(v), field_stride, npts, _addr(xy), _addr(out), _stream(stream)),
           "ofv_probe")


def ofv_debug_fail_alloc(n: int):
    """Make the n-th device allocation of the library from now on fail (n <= 0 cancels)."""
    _lib.ofv_debug_fail_alloc(n)


def ofv_debug_poison(h: int, stream=None):
    """Fill the handle's scratch with NaN bytes (state is kept)."""
    _check(_lib.ofv_debug_poison(h, _stream(stream)), "ofv_debug_poison")


def ofv_debug_reciprocal(x, y, n: int, stream=None):
    """y[i] = 1/x[i] as the forward solve forms it (device float arrays)."""
    _check(_lib.ofv_debug_reciprocal(_addr(x), _addr(y), n, _stream(stream)), "ofv_debug_reciprocal")


def ofv_recirculation_area(H: int, W: int, n: int, u, field_stride: int, mask, counts, stream=None):
    """counts[k] (device uint64 / int64) = pixels of field k in the mask where u < 0."""
    _check(_lib.ofv_recirculation_area(H, W, n, _addr(u), field_stride, _addr(mask), _addr(counts),
                                       _stream(stream)), "ofv_recirculation_area")


class Pair(ctypes.Structure):
    """Mirror of ofv_pair (include/ofv.h)."""
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("I1", ctypes.c_void_p), ("I2", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("v", ctypes.c_void_p)]


def _pair_array(pairs):
    arr = (Pair * len(pairs))()
    for k, p in enumerate(pairs):
        if isinstance(p, Pair):
            arr[k] = p
        else:
            I1, I2, u, v = p
            H, W = I1.shape[-2], I1.shape[-1]
            arr[k] = Pair(H, W, _addr(I1), _addr(I2), _addr(u), _addr(v))
    return arr


def ofv_compute_batched(h: int, pairs, stream=None):
    """pairs: sequence of (I1, I2, u, v) CUDA tensors (each H x W) or Pair
    structures; all pairs of the batch run in one persistent launch."""
    arr = _pair_array(pairs)
    _check(_lib.ofv_compute_batched(h, len(pairs), ctypes.cast(arr, ctypes.c_void_p), _stream(stream)),
           "ofv_compute_batched")


def ofv_graph_create_batched(h: int, pairs) -> int:
    """Record ofv_compute_batched(h, pairs) for these fixed buffers as a CUDA
    graph (it owns its workspace); replay it with ofv_graph_launch."""
    arr = _pair_array(pairs)
    g = ctypes.c_void_p()
    _check(_lib.ofv_graph_create_batched(h, len(pairs), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(g)),
           "ofv_graph_create_batched")
    return g.value


def ofv_batch_tuning(h: int):
    s, c, te, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check(_lib.ofv_batch_tuning(h, ctypes.byref(s), ctypes.byref(c), ctypes.byref(te), ctypes.byref(ms),
                                 ctypes.byref(t)), "ofv_batch_tuning")
    return {"schedule": s.value, "ctas_per_sm": c.value, "tile_edge": te.value, "ms": ms.value,
            "tuned": bool(t.value)}


def ofv_queue_selftest(timeout_us: int):
    """Returns (status, error_word) without raising."""
    w = ctypes.c_int()
    st = _lib.ofv_queue_selftest(timeout_us, ctypes.byref(w))
    return st, w.value


def ofv_graph_create(h: int, I1, I2, u, v) -> int:
    """Record ofv_compute(h, I1, I2, u, v) for these fixed buffers as a CUDA
    graph; replay it with ofv_graph_launch."""
    g = ctypes.c_void_p()
    _check(_lib.ofv_graph_create(h, _addr(I1), _addr(I2), _addr(u), _addr(v), ctypes.byref(g)), "ofv_graph_create")
    return g.value


def ofv_graph_launch(g: int, stream=None):
    _check(_lib.ofv_graph_launch(g, _stream(stream)), "ofv_graph_launch")


def ofv_graph_destroy(g: int):
    _check(_lib.ofv_graph_destroy(g), "ofv_graph_destroy")


def ofv_level_shape(h: int, level: int):
    H, W = ctypes.c_int(), ctypes.c_int()
    _check(_lib.ofv_level_shape(h, level, ctypes.byref(H), ctypes.byref(W)), "ofv_level_shape")
    return H.value, W.value


def ofv_read_level(h: int, frame: int, level: int, dst, stream=None):
    _check(_lib.ofv_read_level(h, frame, level, _addr(dst), _stream(stream)), "ofv_read_level")


def ofv_profile_enable(h: int, enable: bool):
    _check(_lib.ofv_profile_enable(h, 1 if enable else 0), "ofv_profile_enable")


def ofv_profile_read(h: int, k: int):
    ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(_lib.ofv_profile_read(h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)), "ofv_profile_read")
    return ms.value, n.value, b.value


def ofv_last_error() -> str:
    return _lib.ofv_last_error().decode()


def ofv_status_string(st: int) -> str:
    return _status_name(st)


def ofv_version() -> int:
    return _lib.ofv_version()


# --- convenience --------------------------------------------------------------
_IN_DTYPE = {OFV_IN_U8: "uint8", OFV_IN_U16: "uint16", OFV_IN_F32: "float32"}


class Flow:
    """Owns one ofv handle for H x W frames.

    ``Flow(H, W, **params)`` with ofv_params field names; ``flow(I1, I2)``
    returns (u, v) as new float32 CUDA tensors on the current stream."""

    def __init__(self, H: int, W: int, params: Params | None = None, **overrides):
        self.params = params or ofv_default_params(**overrides)
        self.H, self.W = H, W
        self.h = ofv_create(H, W, self.params)

    def __call__(self, I1, I2, u=None, v=None, stream=None):
        import torch
        for t in (I1, I2):
            if not (t.is_cuda and t.is_contiguous() and tuple(t.shape) == (self.H, self.W)):
                raise ValueError("frames must be contiguous CUDA tensors of shape (H, W)")
            if str(t.dtype).split(".")[-1] != _IN_DTYPE[self.params.input]:
                raise TypeError(f"frames must be {_IN_DTYPE[self.params.input]}")
        if u is None:
            u = torch.empty((self.H, self.W), dtype=torch.float32, device=I1.device)
        if v is None:
            v = torch.empty((self.H, self.W), dtype=torch.float32, device=I1.device)
        ofv_compute(self.h, I1, I2, u, v, stream)
        return u, v

    @staticmethod
    def apply(I1, I2, prefilter_w=None, params=None):
        """torch.autograd entry: differentiable (u, v) of (I1, I2); see
        ``autograd.apply``."""
        from .autograd import apply as _apply
        return _apply(I1, I2, prefilter_w, params)

    def close(self):
        if getattr(self, "h", None):
            ofv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
