"""Pins of the oracle's estimator variants (CPU only): the Gaussian-weighted
window, the increment form of the Gauss-Newton step and the warm start of a
time-resolved sequence from an earlier field.

Independent routines: scipy.ndimage.correlate with the outer product of the
1-D weights (zero outside the image = the truncated window), numpy weighted
least squares for the one-step Lucas-Kanade solve, and numpy slicing for the
decimated warm-start field.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

RNG = np.random.default_rng(20251202)


def _particles(H, W, seed, ppp=0.06, diameter=2.5):
    n = int(ppp * H * W)
    x, y, _, a = synth.particles(seed, n, -4, W + 4, -4, H + 4, diameter, diameter)
    sg = np.full(n, diameter / synth.FWHM_PER_SIGMA)
    return synth.render(H, W, x, y, sg, a)


def _gauss1d(kr, sigma):
    d = np.arange(-kr, kr + 1, dtype=np.float64)
    return np.exp(-d * d / (2.0 * sigma * sigma))


# ---------------------------------------------------------------------------
# Gaussian window (variant of reading c1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,kr,sigma", [((12, 12), 1, 0.8), ((17, 23), 3, 1.5), ((40, 31), 6, 2.5),
                                            ((9, 33), 10, 4.0)])
def test_gaussian_window_equals_correlate_with_outer_weights(shape, kr, sigma):
    """Window sums with weights g(a) g(b), g(d) = exp(-d^2 / (2 sigma^2)),
    truncated at the border: scipy's correlate with the outer product and
    zeros outside the image."""
    a = RNG.standard_normal(shape)
    g = _gauss1d(kr, sigma)
    ref = ndimage.correlate(a, np.outer(g, g), mode="constant", cval=0.0)
    got = oracle.window_sum(a, kr, sigma)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_gaussian_window_tends_to_the_box_for_wide_sigma():
    """As sigma grows every weight tends to 1: the uniform box of reading c1."""
    a = RNG.standard_normal((20, 26))
    box = oracle.box_sum(a, 4)
    wide = oracle.window_sum(a, 4, 1e7)
    assert np.allclose(wide, box, rtol=1e-10, atol=1e-10)
    assert np.array_equal(oracle.window_sum(a, 4, 0.0), box)


def test_gaussian_window_one_step_is_weighted_lucas_kanade():
    """PSL = 0, IT = 1 from V = 0 with the Gaussian window: per window, the
    weighted least squares of G.V = -It with weights g(a) g(b)."""
    kr, sigma = 2, 1.2
    I1 = _particles(14, 14, seed=31, ppp=0.15)
    I2 = _particles(14, 14, seed=32, ppp=0.15) * 0.2 + I1 * 0.8
    u, v = oracle.flow(I1, I2, oracle.Params(psl=0, kr=kr, it=1, win_sigma=sigma))
    p1 = np.pad(I1, 1, mode="edge"); p2 = np.pad(I2, 1, mode="edge")
    gx = 0.25 * ((p1[1:-1, 2:] - p1[1:-1, :-2]) + (p2[1:-1, 2:] - p2[1:-1, :-2]))
    gy = 0.25 * ((p1[2:, 1:-1] - p1[:-2, 1:-1]) + (p2[2:, 1:-1] - p2[:-2, 1:-1]))
    it = I2 - I1
    g = _gauss1d(kr, sigma)
    for i in range(14):
        for j in range(14):
            rows, rhs, wts = [], [], []
            for a in range(-kr, kr + 1):
                for b in range(-kr, kr + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < 14 and 0 <= jj < 14:
                        rows.append([gx[ii, jj], gy[ii, jj]])
                        rhs.append(-it[ii, jj])
                        wts.append(g[a + kr] * g[b + kr])
            sw = np.sqrt(np.array(wts))
            sol = np.linalg.lstsq(np.array(rows) * sw[:, None], np.array(rhs) * sw, rcond=None)[0]
            assert abs(sol[0] - u[i, j]) < 1e-9 * max(1.0, abs(sol[0]))
            assert abs(sol[1] - v[i, j]) < 1e-9 * max(1.0, abs(sol[1]))


def test_gaussian_window_recovers_a_subpixel_translation():
    """For a uniform translation of a smooth image the weighted estimator
    lands where the box does: within the bias of bilinear interpolation
    (about 0.012 px mean for this image and shift, box and Gaussian alike)."""
    d = (0.35, -0.6)
    I1, I2 = synth.smooth_pair(64, 64, d, seed=9, sigma=2.0)
    u, v = oracle.flow(I1, I2, oracle.Params(psl=1, kr=4, it=6, win_sigma=2.0))
    s = (slice(12, -12), slice(12, -12))
    assert np.abs(u[s] - d[0]).mean() < 0.02 and np.abs(v[s] - d[1]).mean() < 0.02


# ---------------------------------------------------------------------------
# Increment form (reading c2's alternative)
# ---------------------------------------------------------------------------
def test_increment_form_from_zero_equals_direct_form():
    """From V0 = 0 the two forms solve the same system (r = -It)."""
    I1, I2, _, _ = synth.rankine_pair(40, 40, seed=6, R=10.0, dmax=1.0)
    P1 = np.asarray(I1, np.float64); P2 = np.asarray(I2, np.float64)
    z = np.zeros(P1.shape)
    a = oracle.iterate(P1, P2, z, z, 2)
    b = oracle.iterate(P1, P2, z, z, 2, increment_form=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_increment_form_step_is_v0_plus_the_lk_increment():
    """Increment form with a varying V0: V(m) = V0(m) + H^-1 sum G (-It),
    with G and It from the per-pixel warped samples; rebuilt here from
    scipy's bilinear map_coordinates and numpy sums on a 16x16 case."""
    kr = 1
    I1 = _particles(16, 16, seed=41, ppp=0.15)
    I2 = _particles(16, 16, seed=42, ppp=0.15) * 0.3 + I1 * 0.7
    yy, xx = np.mgrid[0:16, 0:16].astype(np.float64)
    u0 = 0.3 * np.sin(xx / 5.0); v0 = -0.2 * np.cos(yy / 4.0)
    u, v, _, _ = oracle.iterate(I1, I2, u0, v0, kr, increment_form=True)

    def samp(P, px, py):
        return ndimage.map_coordinates(P, [py, px], order=1, mode="nearest")

    pp1 = np.pad(I1, 1, mode="edge"); pp2 = np.pad(I2, 1, mode="edge")
    d1x = 0.5 * (pp1[1:-1, 2:] - pp1[1:-1, :-2]); d1y = 0.5 * (pp1[2:, 1:-1] - pp1[:-2, 1:-1])
    d2x = 0.5 * (pp2[1:-1, 2:] - pp2[1:-1, :-2]); d2y = 0.5 * (pp2[2:, 1:-1] - pp2[:-2, 1:-1])
    p1x, p1y = xx - u0 / 2, yy - v0 / 2
    p2x, p2y = xx + u0 / 2, yy + v0 / 2
    Gx = 0.5 * (samp(d1x, p1x, p1y) + samp(d2x, p2x, p2y))
    Gy = 0.5 * (samp(d1y, p1x, p1y) + samp(d2y, p2x, p2y))
    It = samp(I2, p2x, p2y) - samp(I1, p1x, p1y)
    for i in range(16):
        for j in range(16):
            sl = (slice(max(i - kr, 0), i + kr + 1), slice(max(j - kr, 0), j + kr + 1))
            Hm = np.array([[np.sum(Gx[sl] ** 2), np.sum(Gx[sl] * Gy[sl])],
                           [np.sum(Gx[sl] * Gy[sl]), np.sum(Gy[sl] ** 2)]])
            b = np.array([np.sum(-Gx[sl] * It[sl]), np.sum(-Gy[sl] * It[sl])])
            tr, det = Hm[0, 0] + Hm[1, 1], np.linalg.det(Hm)
            if not (tr > 1e-20) or det <= 1e-6 * tr * tr:
                exp = (u0[i, j], v0[i, j])
            else:
                du = np.linalg.solve(Hm, b)
                exp = (u0[i, j] + du[0], v0[i, j] + du[1])
            assert abs(exp[0] - u[i, j]) < 1e-9 and abs(exp[1] - v[i, j]) < 1e-9


# ---------------------------------------------------------------------------
# Warm start
# ---------------------------------------------------------------------------
def test_decimated_field_is_every_2l_th_sample_over_2l():
    u = RNG.standard_normal((37, 50)); v = RNG.standard_normal((37, 50))
    for level in (0, 1, 2, 3):
        uc, vc = oracle.decimate_field(u, v, level)
        f = 2 ** level
        assert uc.shape == oracle.level_sizes(37, 50, level)[level]
        assert np.array_equal(uc, u[::f, ::f] / f) and np.array_equal(vc, v[::f, ::f] / f)


@pytest.mark.parametrize("psl", [0, 2])
def test_warm_start_from_zero_is_the_cold_start_bitwise(psl):
    I1, I2, _, _ = synth.rankine_pair(48, 40, seed=8, R=10.0, dmax=1.2)
    z = np.zeros((48, 40))
    a = oracle.flow(I1, I2, oracle.Params(psl=psl, kr=3, it=2))
    b = oracle.flow(I1, I2, oracle.Params(psl=psl, kr=3, it=2, init=(z, z)))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_warm_start_reaches_a_shift_the_cold_start_misses():
    """A 4.6 px translation of particle images is beyond a single level's
    linearisation range: from zero, PSL 0 does not reach it (error above
    5 px); started within 0.3 px of the true field it converges to the
    particle-image accuracy (0.05 px).  Started from the negated field it
    does not, which pins the sign and the units of the initial field."""
    d = (4.6, -3.7)
    I1, I2 = synth.translation_pair(80, 80, d, seed=12)[:2]
    s = (slice(16, -16), slice(16, -16))
    p = dict(psl=0, kr=3, it=4)
    cold = oracle.flow(I1, I2, oracle.Params(**p))
    init = (np.full((80, 80), d[0] + 0.3), np.full((80, 80), d[1] - 0.3))
    warm = oracle.flow(I1, I2, oracle.Params(**p, init=init))
    wrong = oracle.flow(I1, I2, oracle.Params(**p, init=(-init[0], -init[1])))
    err = lambda f: np.hypot(f[0][s] - d[0], f[1][s] - d[1]).mean()
    assert err(warm) < 0.06
    assert err(cold) > 2.0 and err(wrong) > 2.0


def test_warm_start_with_pyramid_starts_the_coarsest_level_from_the_decimated_field():
    """PSL 1, IT 1 with an initial field is: one iteration at level 1 from the
    decimated field, the x2 up-sampling, one iteration at level 0."""
    I1, I2, _, _ = synth.rankine_pair(40, 36, seed=9, R=9.0, dmax=1.0)
    yy, xx = np.mgrid[0:40, 0:36].astype(np.float64)
    u0 = 0.4 + 0.1 * np.sin(xx / 6.0); v0 = -0.3 + 0.1 * np.cos(yy / 7.0)
    prm = oracle.Params(psl=1, kr=2, it=1)
    got = oracle.flow(I1, I2, oracle.Params(psl=1, kr=2, it=1, init=(u0, v0)))
    P1 = oracle.pyramid(I1, prm); P2 = oracle.pyramid(I2, prm)
    uc, vc = oracle.decimate_field(u0, v0, 1)
    a = oracle.iterate(P1[1], P2[1], uc, vc, 2)
    uu, vv = oracle.upsample(a[0], a[1], 40, 36)
    b = oracle.iterate(P1[0], P2[0], uu, vv, 2)
    assert np.array_equal(got[0], b[0]) and np.array_equal(got[1], b[1])


def test_reverse_mode_rejects_the_variants():
    I1, I2, _, _ = synth.rankine_pair(24, 24, seed=2, R=6.0, dmax=0.8)
    g = np.ones((24, 24))
    for kw in (dict(increment_form=True), dict(win_sigma=1.5), dict(init=(g, g))):
        with pytest.raises(RuntimeError):
            oracle.flow_grad(I1, I2, oracle.Params(psl=0, kr=2, it=1, **kw), g, g)


# ---------------------------------------------------------------------------
# Region mask
# ---------------------------------------------------------------------------
def test_decimated_mask_is_every_2l_th_sample():
    m = (RNG.random((37, 50)) > 0.3).astype(np.uint8) * 7
    for level in (0, 1, 2, 3):
        f = 2 ** level
        assert np.array_equal(oracle.decimate_mask(m, level), (m[::f, ::f] != 0).astype(np.uint8))


@pytest.mark.parametrize("psl", [0, 2])
def test_all_valid_mask_is_no_mask_bitwise(psl):
    I1, I2, _, _ = synth.rankine_pair(48, 40, seed=8, R=10.0, dmax=1.2)
    a = oracle.flow(I1, I2, oracle.Params(psl=psl, kr=3, it=2))
    b = oracle.flow(I1, I2, oracle.Params(psl=psl, kr=3, it=2, mask=np.ones((48, 40), np.uint8)))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_masked_one_step_is_lucas_kanade_over_the_valid_taps():
    """PSL 0, IT 1 from V = 0 with a mask: per window, least squares of
    G.V = -It over the valid taps only; masked pixels give no vector."""
    kr = 2
    I1 = _particles(14, 14, seed=51, ppp=0.15)
    I2 = _particles(14, 14, seed=52, ppp=0.15) * 0.2 + I1 * 0.8
    m = np.ones((14, 14), np.uint8)
    m[3:6, 4:9] = 0
    m[10:, 11:] = 0
    u, v = oracle.flow(I1, I2, oracle.Params(psl=0, kr=kr, it=1, mask=m))
    p1 = np.pad(I1, 1, mode="edge"); p2 = np.pad(I2, 1, mode="edge")
    gx = 0.25 * ((p1[1:-1, 2:] - p1[1:-1, :-2]) + (p2[1:-1, 2:] - p2[1:-1, :-2]))
    gy = 0.25 * ((p1[2:, 1:-1] - p1[:-2, 1:-1]) + (p2[2:, 1:-1] - p2[:-2, 1:-1]))
    it = I2 - I1
    for i in range(14):
        for j in range(14):
            if not m[i, j]:
                assert np.isnan(u[i, j]) and np.isnan(v[i, j])
                continue
            rows, rhs = [], []
            for a in range(-kr, kr + 1):
                for b in range(-kr, kr + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < 14 and 0 <= jj < 14 and m[ii, jj]:
                        rows.append([gx[ii, jj], gy[ii, jj]])
                        rhs.append(-it[ii, jj])
            sol = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
            assert abs(sol[0] - u[i, j]) < 1e-9 * max(1.0, abs(sol[0]))
            assert abs(sol[1] - v[i, j]) < 1e-9 * max(1.0, abs(sol[1]))


def test_masked_pixels_have_no_vector_and_a_full_mask_gives_none():
    I1, I2, _, _ = synth.rankine_pair(40, 48, seed=5, R=10.0, dmax=1.0)
    m = np.ones((40, 48), np.uint8)
    m[10:20, 5:30] = 0
    u, v = oracle.flow(I1, I2, oracle.Params(psl=2, kr=3, it=2, mask=m))
    assert np.isnan(u[m == 0]).all() and np.isnan(v[m == 0]).all()
    assert np.isfinite(u[m != 0]).all() and np.isfinite(v[m != 0]).all()
    u, v = oracle.flow(I1, I2, oracle.Params(psl=1, kr=3, it=2, mask=np.zeros((40, 48), np.uint8)))
    assert np.isnan(u).all() and np.isnan(v).all()


def test_a_masked_pixel_weighs_nothing_at_every_level():
    """Masking a pixel equals giving its products weight 0: with the whole
    level masked except a window, the solve uses that window's taps only,
    so the field inside a valid block is that of the block cut out with the
    truncated window (PSL 0, IT 1, V = 0; borders of the cut-out block act
    like image borders)."""
    I1 = _particles(32, 32, seed=61, ppp=0.12)
    I2 = _particles(32, 32, seed=62, ppp=0.12) * 0.25 + I1 * 0.75
    m = np.zeros((32, 32), np.uint8)
    m[8:24, 6:26] = 1
    u, v = oracle.flow(I1, I2, oracle.Params(psl=0, kr=2, it=1, mask=m))
    # the cut-out block sees its own image samples, but its central
    # differences at the block edge read pixels outside it: rebuild the
    # products on the full image and sum over valid taps only
    p1 = np.pad(I1, 1, mode="edge"); p2 = np.pad(I2, 1, mode="edge")
    gx = 0.25 * ((p1[1:-1, 2:] - p1[1:-1, :-2]) + (p2[1:-1, 2:] - p2[1:-1, :-2]))
    gy = 0.25 * ((p1[2:, 1:-1] - p1[:-2, 1:-1]) + (p2[2:, 1:-1] - p2[:-2, 1:-1]))
    r = -(I2 - I1)
    w = m.astype(np.float64)
    k = np.ones((5, 5))
    S = [ndimage.correlate(w * a, k, mode="constant") for a in (gx * gx, gx * gy, gy * gy, gx * r, gy * r)]
    sel = m != 0
    det = np.where(sel, S[0] * S[2] - S[1] ** 2, 1.0)
    eu = (S[2] * S[3] - S[1] * S[4]) / det
    ev = (S[0] * S[4] - S[1] * S[3]) / det
    assert np.allclose(u[sel], eu[sel], rtol=1e-9, atol=1e-12) and np.allclose(v[sel], ev[sel], rtol=1e-9, atol=1e-12)
