"""Seeded synthetic PIV inputs shared by the oracle tests, the GPU tests and
the benchmark.

The heavy lifting (field evaluation, particle rendering, noise and
quantisation) is in ``synth.c``; this module only marshals arguments and
states the workload recipes.  Nothing here computes any step of the optical
flow estimator.

Workload recipes (particle images shaped like the paper's workloads):

* ``rankine_pair``   -- 256x256 float32, Gaussian particles of FWHM 2.5 px at
  0.05 particles/px, peak intensity U[0.5, 1], Rankine vortex of core radius
  32 px and peak displacement 3 px at the image centre (Sec. 4.1).
* ``stream_frames``  -- time-resolved 12-bit uint16 sequence (frames F_0..F_n,
  pair i = (F_i, F_{i+1})), 0.08 ppp, FWHM U[2, 3] px, 1 % noise, Rankine
  vortex plus a uniform (1.3, -0.7) px shift.
* ``turbulence_pair`` -- 12-bit uint16, 0.1 ppp, displacement from a
  divergence-free random-Fourier-mode stream function with a k^-5/3 energy
  spectrum over wavelengths 8..1024 px, scaled to 2 px rms (stands in for
  the Madrid HIT DNS planes of Sec. 4.2, which are not available here).
* ``wake_pair``      -- 12-bit uint16, 0.1 ppp, potential flow round a
  cylinder of diameter 400 px plus a street of Lamb-Oseen vortices, scaled to
  a 4 px maximum (stands in for the cylinder-wake experiment of Sec. 7).
* ``smooth_pair``    -- sums of broad Gaussians (sigma 2 px), not quantised,
  uniformly translated; smooth enough for finite-difference checks.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))

OUT_F32, OUT_U16, OUT_U8 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile libsynth.so beside its source (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Field(ctypes.Structure):
    _fields_ = [
        ("ux", ctypes.c_double), ("uy", ctypes.c_double),
        ("rk_cx", ctypes.c_double), ("rk_cy", ctypes.c_double),
        ("rk_R", ctypes.c_double), ("rk_dmax", ctypes.c_double),
        ("turb_n", ctypes.c_int64),
        ("turb_kx", ctypes.c_void_p), ("turb_ky", ctypes.c_void_p),
        ("turb_amp", ctypes.c_void_p), ("turb_phase", ctypes.c_void_p),
        ("cyl_cx", ctypes.c_double), ("cyl_cy", ctypes.c_double),
        ("cyl_a", ctypes.c_double), ("cyl_uinf", ctypes.c_double),
        ("lo_n", ctypes.c_int64),
        ("lo_x", ctypes.c_void_p), ("lo_y", ctypes.c_void_p), ("lo_gamma", ctypes.c_void_p),
        ("lo_rc", ctypes.c_double),
        ("scale", ctypes.c_double),
        ("grid_h", ctypes.c_int64), ("grid_w", ctypes.c_int64),
        ("grid_u", ctypes.c_void_p), ("grid_v", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.syn_field_eval.argtypes = [ctypes.POINTER(_Field), ctypes.c_int64, P, P, P, P]
            lib.syn_particles.argtypes = [ctypes.c_uint64, ctypes.c_int64] + [ctypes.c_double] * 8 + [P] * 4
            lib.syn_render.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, P, P, P, P]
            lib.syn_finalize.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P]
            lib.syn_pair_positions.argtypes = [ctypes.POINTER(_Field), ctypes.c_int64, P, P, P, P, P, P]
            lib.syn_stream.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, P, P, P,
                                       ctypes.POINTER(_Field), ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P]
            lib.syn_stream.restype = ctypes.c_int
            lib.syn_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_double, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Field:
    """A displacement field d(x, y) in px/frame, attributed to the midpoint
    between the two exposures.  Parts add up; ``scale`` multiplies the sum."""

    def __init__(self):
        self._s = _Field()
        self._s.scale = 1.0
        self._keep = []

    # -- parts ---------------------------------------------------------
    def uniform(self, ux: float, uy: float) -> "Field":
        self._s.ux, self._s.uy = ux, uy
        return self

    def rankine(self, cx: float, cy: float, R: float, dmax: float) -> "Field":
        """Rankine vortex: azimuthal displacement dmax*r/R inside the core and
        dmax*R/r outside (Sec. 4.1 box, peak dmax at r = R); the two frames hold
        a particle rotated by -phi/2 and +phi/2 about the centre, phi = u_theta/r."""
        s = self._s
        s.rk_cx, s.rk_cy, s.rk_R, s.rk_dmax = cx, cy, R, dmax
        return self

    def modes(self, kx, ky, amp, phase) -> "Field":
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (kx, ky, amp, phase)]
        self._keep += arrs
        s = self._s
        s.turb_n = len(arrs[0])
        s.turb_kx, s.turb_ky, s.turb_amp, s.turb_phase = [a.ctypes.data for a in arrs]
        return self

    def cylinder(self, cx: float, cy: float, a: float, uinf: float) -> "Field":
        s = self._s
        s.cyl_cx, s.cyl_cy, s.cyl_a, s.cyl_uinf = cx, cy, a, uinf
        return self

    def lamb_oseen(self, xs, ys, gammas, rc: float) -> "Field":
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (xs, ys, gammas)]
        self._keep += arrs
        s = self._s
        s.lo_n = len(arrs[0])
        s.lo_x, s.lo_y, s.lo_gamma = [a.ctypes.data for a in arrs]
        s.lo_rc = rc
        return self

    def set_scale(self, scale: float) -> "Field":
        self._s.scale = scale
        return self

    def sampled(self, H: int, W: int) -> "Field":
        """This field sampled at every pixel centre of an H x W grid and
        interpolated bilinearly: cheap to evaluate for long particle streams."""
        u, v = self.grid(H, W)
        g = Field()
        g._keep = [np.ascontiguousarray(u), np.ascontiguousarray(v)]
        g._s.grid_h, g._s.grid_w = H, W
        g._s.grid_u, g._s.grid_v = g._keep[0].ctypes.data, g._keep[1].ctypes.data
        return g

    # -- evaluation ----------------------------------------------------
    def __call__(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        shape = np.broadcast(x, y).shape
        x = np.ascontiguousarray(np.broadcast_to(x, shape)).ravel()
        y = np.ascontiguousarray(np.broadcast_to(y, shape)).ravel()
        dx = np.empty_like(x)
        dy = np.empty_like(y)
        _load().syn_field_eval(ctypes.byref(self._s), x.size, _ptr(x), _ptr(y), _ptr(dx), _ptr(dy))
        return dx.reshape(shape), dy.reshape(shape)

    def grid(self, H: int, W: int):
        """Analytic displacement at every pixel centre (u along +x = columns,
        v along +y = rows), float64 H x W each."""
        yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
        return self(xx, yy)


def particles(seed: int, n: int, x0, x1, y0, y1, dmin, dmax, amin=0.5, amax=1.0):
    x = np.empty(n); y = np.empty(n); sg = np.empty(n); a = np.empty(n)
    _load().syn_particles(seed, n, x0, x1, y0, y1, dmin, dmax, amin, amax, _ptr(x), _ptr(y), _ptr(sg), _ptr(a))
    return x, y, sg, a


def render(H: int, W: int, x, y, sigma, amp) -> np.ndarray:
    img = np.zeros((H, W), dtype=np.float64)
    x, y, sigma, amp = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, sigma, amp)]
    _load().syn_render(H, W, x.size, _ptr(x), _ptr(y), _ptr(sigma), _ptr(amp), _ptr(img))
    return img


def finalize(img: np.ndarray, noise: float, seed: int, stream: int, bits: int, kind: int) -> np.ndarray:
    H, W = img.shape
    dt = {OUT_F32: np.float32, OUT_U16: np.uint16, OUT_U8: np.uint8}[kind]
    out = np.empty((H, W), dtype=dt)
    img = np.ascontiguousarray(img, dtype=np.float64)
    _load().syn_finalize(H, W, _ptr(img), noise, seed, stream, bits, kind, _ptr(out))
    return out


def _margin(field_max: float, dmax: float) -> float:
    sig = dmax / FWHM_PER_SIGMA
    return math.ceil(4.0 * sig + 2.0) + math.ceil(field_max) + 2.0


def particle_pair(H: int, W: int, field: Field, *, ppp: float, dmin: float, dmax: float,
                  seed: int, noise: float = 0.0, bits: int = 12, kind: int = OUT_U16,
                  field_max: float = 8.0, exclude=None):
    """One frame pair of particles displaced by ``field`` (midpoint convention).

    Particles fill the frame extended by a margin so the seeding density is
    uniform in the visible area; their count is ppp times the extended area.
    ``exclude(x, y) -> bool mask`` drops particles (e.g. inside a cylinder).
    Returns (I1, I2) as arrays of the requested output kind."""
    m = _margin(field_max, dmax)
    ext = (W + 2 * m) * (H + 2 * m)
    n = int(round(ppp * ext))
    x, y, sg, a = particles(seed, n, -m, W + m, -m, H + m, dmin, dmax)
    if exclude is not None:
        keep = ~exclude(x, y)
        x, y, sg, a = x[keep], y[keep], sg[keep], a[keep]
    dx, dy = field(x, y)
    I1 = render(H, W, x - 0.5 * dx, y - 0.5 * dy, sg, a)
    I2 = render(H, W, x + 0.5 * dx, y + 0.5 * dy, sg, a)
    F1 = finalize(I1, noise, seed + 1000003, 0, bits, kind)
    F2 = finalize(I2, noise, seed + 1000003, 1, bits, kind)
    return F1, F2


# ---------------------------------------------------------------------
# workload recipes
# ---------------------------------------------------------------------
def rankine_field(H: int, W: int, R: float = 32.0, dmax: float = 3.0, cx=None, cy=None) -> Field:
    return Field().rankine(W / 2.0 if cx is None else cx, H / 2.0 if cy is None else cy, R, dmax)


def rankine_pair(H: int = 256, W: int = 256, seed: int = 1, R: float = 32.0, dmax: float = 3.0,
                 ppp: float = 0.05, diameter: float = 2.5):
    """256x256 float32 Rankine pair: (I1, I2, truth_u, truth_v)."""
    f = rankine_field(H, W, R, dmax)
    I1, I2 = particle_pair(H, W, f, ppp=ppp, dmin=diameter, dmax=diameter, seed=seed,
                           noise=0.0, kind=OUT_F32, field_max=dmax)
    u, v = f.grid(H, W)
    return I1, I2, u, v


def translation_pair(H: int, W: int, d, seed: int = 7, ppp: float = 0.08, diameter: float = 2.5,
                     kind: int = OUT_F32, noise: float = 0.0, bits: int = 12):
    f = Field().uniform(float(d[0]), float(d[1]))
    return particle_pair(H, W, f, ppp=ppp, dmin=diameter, dmax=diameter, seed=seed, noise=noise,
                         kind=kind, bits=bits, field_max=abs(d[0]) + abs(d[1]))


def stream_field(H: int, W: int) -> Field:
    return Field().uniform(1.3, -0.7).rankine(W / 2.0, H / 2.0, 32.0, 3.0)


def stream_frames(H: int = 1024, W: int = 1024, n_frames: int = 1001, seed: int = 2,
                  ppp: float = 0.08, bits: int = 12, noise: float = 0.01, field: Field | None = None,
                  field_max: float = 5.0, exclude=None) -> np.ndarray:
    """Time-resolved 12-bit sequence (n_frames x H x W uint16) of particles
    advected by a steady field, by default a Rankine vortex (R 32 px, 3 px
    peak) plus a uniform (1.3, -0.7) px/frame shift.  Pair i is (F_i, F_{i+1}).
    ``exclude(x, y)`` drops particles whose starting position it flags."""
    f = stream_field(H, W) if field is None else field
    m = _margin(field_max, 3.0)
    n = int(round(ppp * (W + 2 * m) * (H + 2 * m)))
    x, y, sg, a = particles(seed, n, -m, W + m, -m, H + m, 2.0, 3.0)
    if exclude is not None:
        keep = ~exclude(x, y)
        x, y, sg, a = [np.ascontiguousarray(t[keep]) for t in (x, y, sg, a)]
        n = x.size
    out = np.empty((n_frames, H, W), dtype=np.uint16)
    rc = _load().syn_stream(H, W, n_frames, n, _ptr(x), _ptr(y), _ptr(sg), _ptr(a), ctypes.byref(f._s),
                            m, noise, seed + 1000003, bits, OUT_U16, _ptr(out))
    if rc != 0:
        raise MemoryError("syn_stream: allocation failed")
    return out


def turbulence_field(H: int, W: int, seed: int = 3, n_modes: int = 256, rms: float = 2.0,
                     lam_min: float = 8.0, lam_max: float = 1024.0) -> Field:
    """Divergence-free random-mode field: psi = sum A_n cos(k_n.x + phi_n),
    |k_n| log-spaced over wavelengths lam_min..lam_max, random directions and
    phases, A_n = sqrt(2 E(k_n) dk_n) / |k_n| with E(k) ~ k^(-5/3);
    u = dpsi/dy, v = -dpsi/dx; scaled to the requested rms |d| on the grid."""
    lib = _load()
    lam = lam_min * (lam_max / lam_min) ** (np.arange(n_modes) / (n_modes - 1.0))
    k = 2.0 * np.pi / lam
    dlnk = math.log(lam_max / lam_min) / (n_modes - 1.0)
    dk = k * dlnk
    E = k ** (-5.0 / 3.0)
    A = np.sqrt(2.0 * E * dk) / k
    th = np.empty(n_modes); ph = np.empty(n_modes)
    lib.syn_uniform(seed, 11, n_modes, 0.0, 2.0 * np.pi, _ptr(th))
    lib.syn_uniform(seed, 12, n_modes, 0.0, 2.0 * np.pi, _ptr(ph))
    f = Field().modes(k * np.cos(th), k * np.sin(th), A, ph)
    step = max(1, min(H, W) // 256)
    yy, xx = np.mgrid[0:H:step, 0:W:step].astype(np.float64)
    u, v = f(xx, yy)
    cur = math.sqrt(float(np.mean(u * u + v * v)))
    f.set_scale(rms / cur)
    return f


def turbulence_pair(H: int = 2048, W: int = 2048, seed: int = 3, ppp: float = 0.1, noise: float = 0.01,
                    bits: int = 12, kind: int = OUT_U16):
    f = turbulence_field(H, W, seed=seed)
    I1, I2 = particle_pair(H, W, f, ppp=ppp, dmin=2.0, dmax=3.0, seed=seed, noise=noise, bits=bits,
                           kind=kind, field_max=8.0)
    u, v = f.grid(H, W)
    return I1, I2, u, v


def wake_field(H: int = 4096, W: int = 5120, D: float = 400.0, cx: float = 1024.0, cy=None,
               dmax: float = 4.0, rc: float = 60.0):
    """Potential flow U(1 - a^2/z^2) round a cylinder of diameter D plus an
    alternating street of Lamb-Oseen vortices (core 60 px, spacing 1.2 D,
    lateral offset +-0.3 D) downstream, scaled so max |d| in the fluid is dmax.
    Returns (field, inside_cylinder(x, y) mask function)."""
    cy = H / 2.0 if cy is None else cy
    a = D / 2.0
    xs, ys, gs = [], [], []
    x = cx + D
    sign = 1.0
    gamma = 2.0 * np.pi * rc * 0.8
    while x < W + 1.2 * D:
        xs.append(x); ys.append(cy - sign * 0.3 * D); gs.append(sign * gamma)
        x += 1.2 * D
        sign = -sign
    f = Field().cylinder(cx, cy, a, 1.0).lamb_oseen(xs, ys, gs, rc)

    def inside(px, py):
        return (np.asarray(px) - cx) ** 2 + (np.asarray(py) - cy) ** 2 < a * a

    step = 4
    yy, xx = np.mgrid[0:H:step, 0:W:step].astype(np.float64)
    u, v = f(xx, yy)
    mag = np.sqrt(u * u + v * v)
    mag[inside(xx, yy)] = 0.0
    f.set_scale(dmax / float(mag.max()))
    return f, inside


def wake_pair(H: int = 4096, W: int = 5120, seed: int = 4, ppp: float = 0.1, noise: float = 0.01,
              bits: int = 12, kind: int = OUT_U16):
    f, inside = wake_field(H, W)
    I1, I2 = particle_pair(H, W, f, ppp=ppp, dmin=2.0, dmax=3.0, seed=seed, noise=noise, bits=bits,
                           kind=kind, field_max=8.0, exclude=inside)
    return I1, I2, f, inside


def smooth_pair(H: int, W: int, d, seed: int = 9, n_blobs=None, sigma: float = 2.0):
    """Sum of broad Gaussian blobs (sigma px), float64 and unquantised,
    translated by d with the midpoint convention.  Smooth and textured."""
    if n_blobs is None:
        n_blobs = max(4, (H * W) // 24)
    x, y, _, a = particles(seed, n_blobs, -8, W + 8, -8, H + 8, 1.0, 1.0)
    sg = np.full(n_blobs, sigma)
    I1 = render(H, W, x - 0.5 * d[0], y - 0.5 * d[1], sg, a)
    I2 = render(H, W, x + 0.5 * d[0], y + 0.5 * d[1], sg, a)
    s = max(I1.max(), I2.max())
    return I1 / s, I2 / s
