"""FP64 CPU oracle of the optical-flow velocimetry estimator (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers; the estimator never imports
this package, and this package never imports the estimator.  The arithmetic
lives in ``ofv_oracle.c``; this module converts arrays and names defaults.

Default constants (readings of points the paper leaves open):
  eps_rel = 1e-6, eps_abs = 1e-20 (determinant guard), eps_n = 1e-2
  (normalization floor).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ofv_oracle.c")
_SRC_ADJ = os.path.join(_HERE, "ofv_oracle_adjoint.c")
_HDR = os.path.join(_HERE, "ofv_oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EPS_REL = 1e-6
EPS_ABS = 1e-20
EPS_N = 1e-2


def build(force: bool = False) -> str:
    """Compile liboracle.so beside its source (gcc, OpenMP over rows,
    no floating-point contraction so results match across hosts)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_ADJ), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               _SRC, _SRC_ADJ, "-o", _LIB_PATH + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("psl", ctypes.c_int), ("kr", ctypes.c_int), ("it", ctypes.c_int), ("nr", ctypes.c_int),
        ("bits", ctypes.c_int), ("prefilter", ctypes.c_int), ("w25", ctypes.c_void_p),
        ("eps_rel", ctypes.c_double), ("eps_abs", ctypes.c_double), ("eps_n", ctypes.c_double),
        ("increment_form", ctypes.c_int), ("win_sigma", ctypes.c_double),
        ("u_init", ctypes.c_void_p), ("v_init", ctypes.c_void_p), ("mask", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_scale.argtypes = [ctypes.c_int64, P, I, P]
            lib.orc_normalize.argtypes = [I, I, P, I, D, P]
            lib.orc_prefilter.argtypes = [I, I, P, P, P]
            lib.orc_reduce.argtypes = [I, I, P, P]
            lib.orc_bilinear.argtypes = [P, I, I, D, D]
            lib.orc_bilinear.restype = D
            lib.orc_central_diff.argtypes = [I, I, P, P, P]
            lib.orc_box_sum.argtypes = [I, I, P, I, P]
            lib.orc_window_sum.argtypes = [I, I, P, I, D, P]
            lib.orc_decimate_field.argtypes = [I, I, P, P, I, P, P]
            lib.orc_upsample.argtypes = [I, I, P, P, I, I, P, P]
            lib.orc_iterate.argtypes = [I, I, P, P, P, P, I, D, D, D, I, P, P, P, P, P]
            lib.orc_decimate_mask.argtypes = [I, I, P, I, P]
            lib.orc_iterate.restype = I
            lib.orc_ingest.argtypes = [I, I, P, ctypes.POINTER(_Params), P]
            lib.orc_ingest.restype = I
            lib.orc_pyramid.argtypes = [I, I, P, ctypes.POINTER(_Params), P]
            lib.orc_pyramid.restype = I
            lib.orc_flow.argtypes = [I, I, P, P, ctypes.POINTER(_Params), P, P, P, P]
            lib.orc_flow.restype = I
            lib.orc_flow_grad.argtypes = [I, I, P, P, ctypes.POINTER(_Params), P, P, P, P, P, P, P]
            lib.orc_flow_grad.restype = I
            lib.orc_vorticity.argtypes = [I, I, P, P, P]
            lib.orc_recirculation_count.argtypes = [I, I, P, P]
            lib.orc_recirculation_count.restype = ctypes.c_int64
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = I
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Params:
    """Estimator parameters (Sec. 2, Table 2): PSL pyramid sub-levels, KR
    kernel radius, IT Gauss-Newton iterations per level, NR normalization
    radius (0 = off).  Variants: increment_form, win_sigma > 0 (Gaussian
    window weights), init = (u0, v0) level-0 initial field (warm start),
    mask = level-0 region mask (nonzero = valid; masked output is NaN)."""
    psl: int = 2
    kr: int = 4
    it: int = 3
    nr: int = 0
    bits: int = 0
    prefilter: np.ndarray | None = None
    eps_rel: float = EPS_REL
    eps_abs: float = EPS_ABS
    eps_n: float = EPS_N
    increment_form: bool = False
    win_sigma: float = 0.0
    init: tuple | None = None
    mask: np.ndarray | None = None
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Params:
        s = _Params()
        s.psl, s.kr, s.it, s.nr, s.bits = self.psl, self.kr, self.it, self.nr, self.bits
        self._keep = []
        if self.prefilter is not None:
            w = _f64(self.prefilter).reshape(25)
            self._keep.append(w)
            s.prefilter, s.w25 = 1, w.ctypes.data
        else:
            s.prefilter, s.w25 = 0, None
        s.win_sigma = float(self.win_sigma)
        if self.init is not None:
            u0, v0 = _f64(self.init[0]), _f64(self.init[1])
            self._keep += [u0, v0]
            s.u_init, s.v_init = u0.ctypes.data, v0.ctypes.data
        else:
            s.u_init, s.v_init = None, None
        if self.mask is not None:
            m = np.ascontiguousarray(self.mask != 0, dtype=np.uint8)
            self._keep.append(m)
            s.mask = m.ctypes.data
        else:
            s.mask = None
        s.eps_rel, s.eps_abs, s.eps_n = self.eps_rel, self.eps_abs, self.eps_n
        s.increment_form = 1 if self.increment_form else 0
        return s


def level_sizes(H: int, W: int, psl: int):
    hs, ws = [H], [W]
    for _ in range(psl):
        hs.append((hs[-1] + 1) // 2)
        ws.append((ws[-1] + 1) // 2)
    return list(zip(hs, ws))


def scale(raw, bits: int) -> np.ndarray:
    raw = _f64(raw)
    out = np.empty_like(raw)
    _load().orc_scale(raw.size, _p(raw), bits, _p(out))
    return out


def normalize(I, nr: int, eps_n: float = EPS_N) -> np.ndarray:
    I = _f64(I)
    out = np.empty_like(I)
    _load().orc_normalize(I.shape[0], I.shape[1], _p(I), nr, eps_n, _p(out))
    return out


def prefilter(I, w25) -> np.ndarray:
    I = _f64(I)
    w = _f64(w25).reshape(25)
    out = np.empty_like(I)
    _load().orc_prefilter(I.shape[0], I.shape[1], _p(I), _p(w), _p(out))
    return out


def reduce(P) -> np.ndarray:
    P = _f64(P)
    H, W = P.shape
    out = np.empty(((H + 1) // 2, (W + 1) // 2))
    _load().orc_reduce(H, W, _p(P), _p(out))
    return out


def bilinear(P, px: float, py: float) -> float:
    P = _f64(P)
    return _load().orc_bilinear(_p(P), P.shape[0], P.shape[1], px, py)


def central_diff(P):
    P = _f64(P)
    dx = np.empty_like(P)
    dy = np.empty_like(P)
    _load().orc_central_diff(P.shape[0], P.shape[1], _p(P), _p(dx), _p(dy))
    return dx, dy


def box_sum(a, kr: int) -> np.ndarray:
    a = _f64(a)
    out = np.empty_like(a)
    _load().orc_box_sum(a.shape[0], a.shape[1], _p(a), kr, _p(out))
    return out


def window_sum(a, kr: int, sigma: float) -> np.ndarray:
    """Window sums with Gaussian weights exp(-(a^2+b^2)/(2 sigma^2)) (box for sigma <= 0)."""
    a = _f64(a)
    out = np.empty_like(a)
    _load().orc_window_sum(a.shape[0], a.shape[1], _p(a), kr, float(sigma), _p(out))
    return out


def decimate_field(u, v, level: int):
    """The level-`level` warm-start field from a level-0 field: V(2^l i, 2^l j) / 2^l."""
    u, v = _f64(u), _f64(v)
    H, W = u.shape
    h, w = level_sizes(H, W, level)[level]
    uc = np.empty((h, w)); vc = np.empty((h, w))
    _load().orc_decimate_field(H, W, _p(u), _p(v), level, _p(uc), _p(vc))
    return uc, vc


def decimate_mask(mask, level: int):
    """The level-`level` region mask: mask(2^l i, 2^l j) != 0 as 0 / 1."""
    m = np.ascontiguousarray(mask != 0, dtype=np.uint8)
    H, W = m.shape
    h, w = level_sizes(H, W, level)[level]
    out = np.empty((h, w), dtype=np.uint8)
    _load().orc_decimate_mask(H, W, _p(m), level, _p(out))
    return out


def upsample(uc, vc, H: int, W: int):
    uc, vc = _f64(uc), _f64(vc)
    u = np.empty((H, W))
    v = np.empty((H, W))
    _load().orc_upsample(uc.shape[0], uc.shape[1], _p(uc), _p(vc), H, W, _p(u), _p(v))
    return u, v


def iterate(P1, P2, u0, v0, kr: int, eps_rel: float = EPS_REL, eps_abs: float = EPS_ABS,
            increment_form: bool = False, win_sigma: float = 0.0, mask=None):
    """One Gauss-Newton iteration at one level: returns (u, v, ndet, guarded)."""
    P1, P2, u0, v0 = _f64(P1), _f64(P2), _f64(u0), _f64(v0)
    H, W = P1.shape
    u = np.empty((H, W)); v = np.empty((H, W)); nd = np.empty((H, W))
    g = np.empty((H, W), dtype=np.uint8)
    m = None if mask is None else np.ascontiguousarray(mask != 0, dtype=np.uint8)
    rc = _load().orc_iterate(H, W, _p(P1), _p(P2), _p(u0), _p(v0), kr, float(win_sigma), eps_rel, eps_abs,
                             1 if increment_form else 0, None if m is None else _p(m), _p(u), _p(v), _p(nd), _p(g))
    if rc:
        raise MemoryError("orc_iterate failed")
    return u, v, nd, g


def ingest(raw, params: Params) -> np.ndarray:
    raw = _f64(raw)
    out = np.empty_like(raw)
    c = params.c()
    if _load().orc_ingest(raw.shape[0], raw.shape[1], _p(raw), ctypes.byref(c), _p(out)):
        raise MemoryError("orc_ingest failed")
    return out


def pyramid(raw, params: Params):
    """Levels 0..PSL of one frame after ingest, as a list of arrays."""
    raw = _f64(raw)
    H, W = raw.shape
    sizes = level_sizes(H, W, params.psl)
    total = sum(h * w for h, w in sizes)
    out = np.empty(total)
    c = params.c()
    if _load().orc_pyramid(H, W, _p(raw), ctypes.byref(c), _p(out)):
        raise MemoryError("orc_pyramid failed")
    levels, off = [], 0
    for h, w in sizes:
        levels.append(out[off:off + h * w].reshape(h, w))
        off += h * w
    return levels


def flow(I1, I2, params: Params | None = None, diagnostics: bool = False):
    """Dense displacement (u, v) in px/frame at every pixel of the pair.

    With ``diagnostics`` also returns ndet (det/(Sxx+Syy)^2 of the last
    level-0 iteration) and guard0 (bit t set where level-0 iteration t kept V0)."""
    params = params or Params()
    a, b = _f64(I1), _f64(I2)
    if a.shape != b.shape or a.ndim != 2:
        raise ValueError("frames must be 2-D and of equal shape")
    H, W = a.shape
    u = np.empty((H, W)); v = np.empty((H, W)); nd = np.empty((H, W))
    g = np.empty((H, W), dtype=np.uint8)
    c = params.c()
    rc = _load().orc_flow(H, W, _p(a), _p(b), ctypes.byref(c), _p(u), _p(v), _p(nd), _p(g))
    if rc:
        raise RuntimeError(f"orc_flow failed ({rc})")
    if diagnostics:
        return u, v, nd, g
    return u, v


def flow_grad(I1, I2, params: Params, gu, gv):
    """Reverse mode: for a loss L with dL/du = gu and dL/dv = gv, returns
    (dL/dI1, dL/dI2, dL/dw25 or None, u, v).  NR must be 0."""
    a, b = _f64(I1), _f64(I2)
    gu, gv = _f64(gu), _f64(gv)
    H, W = a.shape
    g1 = np.empty((H, W)); g2 = np.empty((H, W)); u = np.empty((H, W)); v = np.empty((H, W))
    gw = np.zeros(25)
    c = params.c()
    rc = _load().orc_flow_grad(H, W, _p(a), _p(b), ctypes.byref(c), _p(gu), _p(gv), _p(g1), _p(g2), _p(gw),
                               _p(u), _p(v))
    if rc:
        raise RuntimeError(f"orc_flow_grad failed ({rc})")
    return g1, g2, (gw.reshape(5, 5) if params.prefilter is not None else None), u, v


def num_threads() -> int:
    """Threads the oracle's OpenMP loops run on (OMP_NUM_THREADS, else the host's cores)."""
    return int(_load().orc_num_threads())


def vorticity(u, v):
    """omega = dv/dx - du/dy of a field (u along columns, v along rows)."""
    u, v = _f64(u), _f64(v)
    out = np.empty_like(u)
    _load().orc_vorticity(u.shape[0], u.shape[1], _p(u), _p(v), _p(out))
    return out


def recirculation_count(u, mask=None):
    """Pixels of the region (mask != 0, or all) where u < 0 (Eq. 6 in pixels)."""
    u = _f64(u)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    return int(_load().orc_recirculation_count(u.shape[0], u.shape[1], _p(u), None if m is None else _p(m)))
