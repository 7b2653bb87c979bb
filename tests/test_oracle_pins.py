"""Pins of the FP64 oracle against facts fixed by the paper, by mathematics
or by independent library routines (CPU only).

Each test names what it pins.  Independent routines used: an integral image
(numpy cumsum) for window sums, scipy.ndimage.correlate / map_coordinates /
uniform_filter (mode 'nearest' is clamp-to-edge), numpy.linalg.lstsq for the
textbook Lucas-Kanade solve and a Nelder-Mead search for the SSD of Eq. 2.
"""
import numpy as np
import pytest
from scipy import ndimage, optimize

import oracle
import synth

RNG = np.random.default_rng(20250930)


def _particles(H, W, seed, ppp=0.06, diameter=2.5):
    n = int(ppp * H * W)
    x, y, _, a = synth.particles(seed, n, -4, W + 4, -4, H + 4, diameter, diameter)
    sg = np.full(n, diameter / synth.FWHM_PER_SIGMA)
    return synth.render(H, W, x, y, sg, a)


# ---------------------------------------------------------------------------
# Step 0 -- input scaling
# ---------------------------------------------------------------------------
def test_scale_maps_full_scale_counts_to_unit_interval():
    raw = np.array([[0.0, 4095.0, 2048.0]])
    out = oracle.scale(raw, 12)
    assert out[0, 0] == 0.0 and out[0, 1] == 1.0
    assert abs(out[0, 2] - 2048.0 / 4095.0) < 1e-16
    assert oracle.scale(np.array([[255.0]]), 8)[0, 0] == 1.0
    f = RNG.random((3, 4))
    assert np.array_equal(oracle.scale(f, 0), f)


# ---------------------------------------------------------------------------
# Window sums (Sec. 2: N(m) of radius KR) -- direct sums vs an integral image
# ---------------------------------------------------------------------------
def _integral_box(a, kr):
    H, W = a.shape
    S = np.zeros((H + 1, W + 1), dtype=np.int64)
    S[1:, 1:] = np.cumsum(np.cumsum(a.astype(np.int64), axis=0), axis=1)
    i = np.arange(H)[:, None]
    j = np.arange(W)[None, :]
    i0 = np.clip(i - kr, 0, H); i1 = np.clip(i + kr + 1, 0, H)
    j0 = np.clip(j - kr, 0, W); j1 = np.clip(j + kr + 1, 0, W)
    return S[i1, j1] - S[i0, j1] - S[i1, j0] + S[i0, j0]


@pytest.mark.parametrize("shape", [(12, 12), (17, 23), (64, 64)])
@pytest.mark.parametrize("kr", [1, 2, 4, 7, 10])
def test_box_sum_equals_integral_image_exactly(shape, kr):
    a = RNG.integers(-1000, 1000, size=shape)
    got = oracle.box_sum(a.astype(np.float64), kr)
    want = _integral_box(a, kr)
    assert np.array_equal(got, want.astype(np.float64))


def test_box_sum_real_values_separable_form():
    a = RNG.standard_normal((31, 19))
    kr = 3
    # separable: row sums then column sums with zero padding
    pad = np.pad(a, kr)
    rows = sum(pad[:, k:k + a.shape[1]] for k in range(2 * kr + 1))
    cols = sum(rows[k:k + a.shape[0], :] for k in range(2 * kr + 1))
    assert np.allclose(oracle.box_sum(a, kr), cols, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Pyramid (Sec. 2: Burt-Adelson reduction, each level halves H and W)
# ---------------------------------------------------------------------------
C5 = np.array([1, 4, 6, 4, 1]) / 16.0


def test_reduce_constant_is_constant():
    P = np.full((37, 22), 0.75)
    out = oracle.reduce(P)
    assert out.shape == (19, 11)
    assert np.all(out == 0.75)


def test_reduce_reproduces_linear_ramp_at_even_samples():
    H, W = 40, 33
    i, j = np.mgrid[0:H, 0:W].astype(np.float64)
    P = 0.25 + 0.0625 * i - 0.03125 * j
    out = oracle.reduce(P)
    ic, jc = np.mgrid[0:out.shape[0], 0:out.shape[1]].astype(np.float64)
    want = 0.25 + 0.0625 * (2 * ic) - 0.03125 * (2 * jc)
    inner = (slice(1, (H - 3) // 2 + 1), slice(1, (W - 3) // 2 + 1))
    assert np.allclose(out[inner], want[inner], atol=1e-14)


def test_reduce_impulse_response_is_the_kernel():
    P = np.zeros((32, 32))
    P[10, 10] = 1.0
    out = oracle.reduce(P)
    for ic in range(out.shape[0]):
        for jc in range(out.shape[1]):
            a, b = 10 - 2 * ic, 10 - 2 * jc
            want = C5[a + 2] * C5[b + 2] if (abs(a) <= 2 and abs(b) <= 2) else 0.0
            assert out[ic, jc] == want


@pytest.mark.parametrize("shape", [(16, 16), (17, 23), (9, 40)])
def test_reduce_matches_scipy_correlate_nearest(shape):
    P = RNG.random(shape)
    k2 = np.outer(C5, C5)
    full = ndimage.correlate(P, k2, mode="nearest")
    assert np.allclose(oracle.reduce(P), full[::2, ::2], atol=1e-14)


# ---------------------------------------------------------------------------
# Interpolation and gradients (readings c3, c4)
# ---------------------------------------------------------------------------
def test_bilinear_matches_map_coordinates_order1_nearest():
    P = RNG.random((13, 17))
    for _ in range(200):
        px = RNG.uniform(-3, 20)
        py = RNG.uniform(-3, 16)
        want = ndimage.map_coordinates(P, [[py], [px]], order=1, mode="nearest")[0]
        assert abs(oracle.bilinear(P, px, py) - want) < 1e-13


def test_bilinear_at_pixel_centres_returns_samples():
    P = RNG.random((7, 9))
    for i in range(7):
        for j in range(9):
            assert oracle.bilinear(P, float(j), float(i)) == P[i, j]


def test_central_diff_interior_is_numpy_gradient_and_edges_clamp():
    P = RNG.random((11, 14))
    dx, dy = oracle.central_diff(P)
    gy, gx = np.gradient(P)
    assert np.allclose(dx[:, 1:-1], gx[:, 1:-1], atol=1e-15)
    assert np.allclose(dy[1:-1, :], gy[1:-1, :], atol=1e-15)
    Pe = np.pad(P, 1, mode="edge")
    assert np.allclose(dx, 0.5 * (Pe[1:-1, 2:] - Pe[1:-1, :-2]), atol=1e-15)
    assert np.allclose(dy, 0.5 * (Pe[2:, 1:-1] - Pe[:-2, 1:-1]), atol=1e-15)


# ---------------------------------------------------------------------------
# Up-sampling and projection (Sec. 2 step 4)
# ---------------------------------------------------------------------------
def test_upsample_constant_doubles_exactly():
    uc = np.full((9, 12), 0.8125)
    vc = np.full((9, 12), -1.25)
    u, v = oracle.upsample(uc, vc, 17, 23)
    assert np.all(u == 1.625) and np.all(v == -2.5)


def test_upsample_matches_map_coordinates_at_half_positions():
    uc = RNG.standard_normal((10, 7))
    vc = RNG.standard_normal((10, 7))
    H, W = 19, 14
    u, v = oracle.upsample(uc, vc, H, W)
    yy, xx = np.mgrid[0:H, 0:W] / 2.0
    wu = 2 * ndimage.map_coordinates(uc, [yy, xx], order=1, mode="nearest")
    wv = 2 * ndimage.map_coordinates(vc, [yy, xx], order=1, mode="nearest")
    assert np.allclose(u, wu, atol=1e-14) and np.allclose(v, wv, atol=1e-14)


# ---------------------------------------------------------------------------
# Normalization and pre-filter (pre-processing; paper parity unpinned, the
# reading itself is pinned against library routines)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nr", [1, 2, 4])
def test_normalize_matches_uniform_filter_statistics(nr):
    I = RNG.random((23, 18))
    size = 2 * nr + 1
    ones = np.ones_like(I)
    cnt = ndimage.uniform_filter(ones, size, mode="constant") * size * size
    s1 = ndimage.uniform_filter(I, size, mode="constant") * size * size
    s2 = ndimage.uniform_filter(I * I, size, mode="constant") * size * size
    mu = s1 / cnt
    var = s2 / cnt - mu * mu
    want = (I - mu) / np.sqrt(var + oracle.EPS_N ** 2)
    assert np.allclose(oracle.normalize(I, nr), want, atol=1e-10)


def test_prefilter_matches_scipy_correlate_and_delta_is_identity():
    I = RNG.random((15, 21))
    w = RNG.standard_normal((5, 5))
    assert np.allclose(oracle.prefilter(I, w), ndimage.correlate(I, w, mode="nearest"), atol=1e-13)
    delta = np.zeros((5, 5)); delta[2, 2] = 1.0
    assert np.array_equal(oracle.prefilter(I, delta), I)


# ---------------------------------------------------------------------------
# Whole estimator: exact properties
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nr,pre", [(0, False), (2, False), (1, True)])
def test_zero_motion_gives_exactly_zero_flow(nr, pre):
    I = _particles(64, 80, seed=3)
    w = None
    if pre:
        w = RNG.standard_normal((5, 5)) * 0.1
        w[2, 2] += 1.0
    u, v = oracle.flow(I, I.copy(), oracle.Params(psl=2, kr=3, it=3, nr=nr, prefilter=w))
    assert np.all(u == 0.0) and np.all(v == 0.0)


def test_frame_swap_negates_flow_bitwise():
    I1, I2, _, _ = synth.rankine_pair(96, 96, seed=11, R=16.0, dmax=2.0)
    p = oracle.Params(psl=2, kr=4, it=3)
    u, v = oracle.flow(I1, I2, p)
    us, vs = oracle.flow(I2, I1, p)
    assert np.array_equal(us, -u) and np.array_equal(vs, -v)


def test_textureless_pair_is_guarded_and_keeps_zero():
    I = np.full((40, 40), 0.3)
    u, v, nd, g = oracle.flow(I, I * 1.01, oracle.Params(psl=1, kr=2, it=2), diagnostics=True)
    assert np.all(u == 0.0) and np.all(v == 0.0)
    assert np.all(nd == 0.0)
    assert np.all(g == 0b11)


@pytest.mark.parametrize("d", [(2, -1), (3, 2), (-1, 0), (4, -4), (0, 3)])
def test_integer_translation_is_recovered_exactly(d):
    """With V an integer vector the warped samples k -/+ V/2 fall on pixel
    centres or midpoints of both frames alike, so I2(k) = I1(k - d) makes the
    residual of Eq. 2 vanish at V = d: a zero-residual fixed point.  The
    pyramid reaches its basin, and Gauss-Newton then converges to d to
    rounding in the interior (the clamped border differs)."""
    big = _particles(200, 200, seed=5)
    I1 = big[40:168, 40:168]
    I2 = big[40 - d[1]:168 - d[1], 40 - d[0]:168 - d[0]]
    u, v = oracle.flow(I1, I2, oracle.Params(psl=2, kr=4, it=30))
    # the clamped border perturbs the fixed point by an amount that decays
    # with distance; 40 px in, it is below rounding
    s = (slice(40, -40), slice(40, -40))
    assert np.abs(u[s] - d[0]).max() < 1e-11
    assert np.abs(v[s] - d[1]).max() < 1e-11


def test_one_iteration_from_zero_is_textbook_lucas_kanade():
    """PSL = 0, IT = 1 starting from V = 0 reduces to Lucas-Kanade (Sec. 2):
    for each window, least squares of G.V = -It with G the frame-averaged
    central gradient.  12x12 with KR = 1, the shape of the worked example in
    the kernel-scale figure of Sec. 2."""
    I1 = _particles(12, 12, seed=21, ppp=0.15)
    I2 = _particles(12, 12, seed=22, ppp=0.15) * 0.2 + I1 * 0.8
    u, v = oracle.flow(I1, I2, oracle.Params(psl=0, kr=1, it=1))
    p1 = np.pad(I1, 1, mode="edge"); p2 = np.pad(I2, 1, mode="edge")
    gx = 0.25 * ((p1[1:-1, 2:] - p1[1:-1, :-2]) + (p2[1:-1, 2:] - p2[1:-1, :-2]))
    gy = 0.25 * ((p1[2:, 1:-1] - p1[:-2, 1:-1]) + (p2[2:, 1:-1] - p2[:-2, 1:-1]))
    it = I2 - I1
    for i in range(12):
        for j in range(12):
            rows, rhs = [], []
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < 12 and 0 <= jj < 12:
                        rows.append([gx[ii, jj], gy[ii, jj]])
                        rhs.append(-it[ii, jj])
            sol = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
            assert abs(sol[0] - u[i, j]) < 1e-9 * max(1.0, abs(sol[0]))
            assert abs(sol[1] - v[i, j]) < 1e-9 * max(1.0, abs(sol[1]))


def test_direct_and_increment_forms_agree_for_constant_field():
    """Reading c2: the direct form H V = sum G (G.V0 - It) equals the
    increment form V0 + H^-1 sum G (-It) whenever V0 is constant over the
    window."""
    I1, I2, _, _ = synth.rankine_pair(48, 48, seed=4, R=12.0, dmax=1.0)
    P1 = np.asarray(I1, np.float64); P2 = np.asarray(I2, np.float64)
    u0 = np.full(P1.shape, 0.37); v0 = np.full(P1.shape, -0.21)
    a = oracle.iterate(P1, P2, u0, v0, 3)
    b = oracle.iterate(P1, P2, u0, v0, 3, increment_form=True)
    assert np.allclose(a[0], b[0], atol=1e-10) and np.allclose(a[1], b[1], atol=1e-10)


def test_converged_field_is_near_the_literal_ssd_minimum():
    """Eq. 2 taken literally: for each window the SSD of the bilinearly
    warped frames is minimised over a constant V by Nelder-Mead.  The
    Gauss-Newton fixed point uses the sampled central-difference gradient
    rather than the exact derivative of the bilinear interpolant, so with a
    non-zero residual the two stationary points differ slightly; on smooth
    images (sigma 2 px) the difference measured is about 1e-3 px."""
    d = (0.3, -0.45)
    I1, I2 = synth.smooth_pair(64, 64, d, seed=9, sigma=2.0)
    u, v = oracle.flow(I1, I2, oracle.Params(psl=0, kr=4, it=10))

    def ssd(V, m):
        i, j = m
        ys, xs = np.mgrid[i - 4:i + 5, j - 4:j + 5].astype(float)
        A = ndimage.map_coordinates(I1, [ys - V[1] / 2, xs - V[0] / 2], order=1, mode="nearest")
        B = ndimage.map_coordinates(I2, [ys + V[1] / 2, xs + V[0] / 2], order=1, mode="nearest")
        return float(np.sum((A - B) ** 2))

    for m in [(20, 20), (30, 25), (40, 44), (25, 40), (32, 32)]:
        res = optimize.minimize(ssd, x0=[0.0, 0.0], args=(m,), method="Nelder-Mead",
                                options=dict(xatol=1e-9, fatol=1e-18, maxiter=4000))
        assert abs(res.x[0] - u[m]) < 3e-3 and abs(res.x[1] - v[m]) < 3e-3
        # and both are within the bilinear bias of the true shift
        assert abs(u[m] - d[0]) < 0.03 and abs(v[m] - d[1]) < 0.03


# ---------------------------------------------------------------------------
# Whole estimator: recovery of analytic fields
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d", [(0.30, -0.45), (1.3, -0.7), (2.6, 1.9)])
def test_subpixel_translation_of_particles(d):
    """Uniform sub-pixel translation of particle images (FWHM 2.5 px).  The
    error is dominated by the bias of bilinear interpolation of small
    particles, measured at 0.03-0.05 px mean; sign or axis mistakes would
    give errors of the order of |d|."""
    I1, I2 = synth.translation_pair(128, 128, d, seed=7)
    u, v = oracle.flow(I1, I2, oracle.Params(psl=2, kr=4, it=3))
    e = np.hypot(u - d[0], v - d[1])[12:-12, 12:-12]
    assert e.mean() < 0.06
    assert np.percentile(e, 99) < 0.12


def test_rankine_vortex_recovered_away_from_core():
    """256x256, 0.05 ppp, FWHM 2.5 px, R = 32 px, 3 px peak, PSL 2, KR 4,
    IT 3.  The paper reports best-case mean errors of 0.048-0.27 px on its
    Rankine images (Sec. 6, Table 4) and sub-pixel errors for D/R <= 0.7;
    here D/R = 3/32."""
    I1, I2, tu, tv = synth.rankine_pair()
    u, v = oracle.flow(I1, I2, oracle.Params(psl=2, kr=4, it=3))
    err = np.hypot(u - tu, v - tv)
    yy, xx = np.mgrid[0:256, 0:256]
    r = np.hypot(xx - 128, yy - 128)
    border = 2 * 4 + 2
    far = (r >= 48) & (xx >= border) & (xx < 256 - border) & (yy >= border) & (yy < 256 - border)
    assert err[far].mean() < 0.05
    assert err.mean() < 0.27
    assert err.max() < 1.0
