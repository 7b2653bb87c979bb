"""The synthetic input recipes hold what the design states for them.

These inputs stand in for the paper's images (Sec. 4.1 Rankine vortex,
Sec. 4.2 turbulence, Sec. 6 streams, Sec. 7 cylinder wake), so the
properties the tests and the benchmark rely on are pinned here: the Rankine
field of reading c12, the stream's uniform shift, the turbulence field's
zero divergence and rms, the particle-free cylinder of the wake, 12-bit
quantisation and seed determinism.
"""
import numpy as np
import pytest

import synth


def test_rankine_core_turns_by_a_constant_angle_and_peaks_at_r():
    # reading c12: a particle turns by phi = u_theta(r) / r about the centre,
    # -phi/2 and +phi/2 in the two frames; inside the core u_theta = dmax r / R,
    # so phi = dmax / R everywhere there and the displacement attributed to
    # the chord's midpoint (at radius r) is 2 r tan(phi / 2), azimuthal
    R, dmax, c = 32.0, 3.0, 128.0
    f = synth.rankine_field(256, 256, R=R, dmax=dmax)
    th = np.linspace(0.0, 2.0 * np.pi, 13)[:-1]
    for r in (2.0, 8.0, 16.0, 24.0):
        u, v = f(c + r * np.cos(th), c + r * np.sin(th))
        np.testing.assert_allclose(np.hypot(u, v), 2.0 * r * np.tan(dmax / R / 2.0), rtol=1e-12)
        np.testing.assert_allclose(u * np.cos(th) + v * np.sin(th), 0.0, atol=1e-12)  # no radial part
    # peak at r = R (up to the O(phi^2) chord correction) and dmax R / r outside
    u, v = f(c + R * np.cos(th), c + R * np.sin(th))
    assert np.all(np.abs(np.hypot(u, v) - dmax) < 0.01)
    u, v = f(c + 3 * R * np.cos(th), c + 3 * R * np.sin(th))
    np.testing.assert_allclose(np.hypot(u, v), dmax / 3.0, rtol=1e-3)
    # counter-clockwise in image coordinates (x right, y down): d = |d| (-sin, cos)
    u, v = f(np.array([c + 10.0]), np.array([c]))
    assert abs(u[0]) < 1e-12 and v[0] > 0


def test_stream_field_is_the_rankine_vortex_plus_the_uniform_shift():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 1024, 200), rng.uniform(0, 1024, 200)
    su, sv = synth.stream_field(1024, 1024)(x, y)
    ru, rv = synth.rankine_field(1024, 1024)(x, y)
    np.testing.assert_allclose(su - ru, 1.3, atol=1e-12)
    np.testing.assert_allclose(sv - rv, -0.7, atol=1e-12)


def test_turbulence_field_is_divergence_free_with_the_set_rms():
    H = W = 512
    f = synth.turbulence_field(H, W, seed=3)
    u, v = f.grid(H, W)
    rms = float(np.sqrt(np.mean(u * u + v * v)))
    assert abs(rms - 2.0) < 0.05, rms
    # divergence by central differences of the analytic field (step 1e-3 px)
    rng = np.random.default_rng(1)
    x, y, h = rng.uniform(0, W, 500), rng.uniform(0, H, 500), 1e-3
    dudx = (f(x + h, y)[0] - f(x - h, y)[0]) / (2 * h)
    dvdy = (f(x, y + h)[1] - f(x, y - h)[1]) / (2 * h)
    scale = float(np.sqrt(np.mean(dudx ** 2 + dvdy ** 2)))
    assert scale > 0.01
    assert float(np.abs(dudx + dvdy).max()) < 1e-5 * scale + 1e-9


def test_wake_has_no_particles_inside_the_cylinder():
    H, W = 1024, 2048
    I1, I2, f, inside = synth.wake_pair(H, W, seed=4)
    yy, xx = np.mgrid[0:H, 0:W]
    cx, cy, a = 1024.0, H / 2.0, 200.0
    deep = (xx - cx) ** 2 + (yy - cy) ** 2 < (a - 8.0) ** 2  # 8 px clear of the rim (blobs, displacement)
    assert inside(xx[deep], yy[deep]).all()
    for I in (I1, I2):
        assert I[deep].max() < 0.1 * 4095, "particle light inside the cylinder"
        assert I[~inside(xx, yy)].max() > 0.5 * 4095  # particles elsewhere


def test_stream_frames_are_12_bit_and_deterministic_per_seed():
    a = synth.stream_frames(96, 128, 4, seed=2)
    b = synth.stream_frames(96, 128, 4, seed=2)
    c = synth.stream_frames(96, 128, 4, seed=3)
    assert a.dtype == np.uint16 and a.shape == (4, 96, 128)
    assert a.max() <= 4095 and a.max() > 2000
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


@pytest.mark.parametrize("bits", [8, 12, 16])
def test_quantisation_uses_the_full_scale_of_the_bit_depth(bits):
    F = synth.stream_frames(64, 64, 2, seed=5, bits=bits)
    assert F.max() <= (1 << bits) - 1
    assert F.max() >= 0.4 * ((1 << bits) - 1)
