"""Pins of the FP64 oracle's reverse mode (CPU only).

The paper defines no derivative of the estimator; the reverse mode is the
chain rule through the forward steps, local normalization included.  It is pinned against the forward
oracle itself by central finite differences of L = sum(gu*u + gv*v) along
random directions (a check that shares no arithmetic with the reverse code),
and by facts any gradient must satisfy: linearity in (gu, gv), the input
scale factor of the intensity range, and zero gradients where every pixel
is guarded.
"""
import numpy as np
import pytest

import oracle
import synth


def _loss(I1, I2, p, gu, gv):
    u, v = oracle.flow(I1, I2, p)
    return float(np.sum(gu * u) + np.sum(gv * v))


def _fd_dir(fun, x, d, h):
    """Central difference along d with one Richardson step (error O(h^4))."""
    c1 = (fun(x + h * d) - fun(x - h * d)) / (2 * h)
    c2 = (fun(x + 0.5 * h * d) - fun(x - 0.5 * h * d)) / h
    return (4.0 * c2 - c1) / 3.0


H_NR = 1e-7  # finite-difference step with local normalization


def _case(H, W, seed, shift=(0.7, -0.4)):
    I1, I2 = synth.smooth_pair(H, W, shift, seed=seed)
    rng = np.random.default_rng(seed)
    gu = rng.standard_normal((H, W))
    gv = rng.standard_normal((H, W))
    return I1, I2, gu, gv, rng


@pytest.mark.parametrize("psl,kr,it", [(1, 2, 2), (0, 3, 1), (2, 1, 3)])
def test_frame_gradients_match_finite_differences(psl, kr, it):
    H, W = 36, 40
    I1, I2, gu, gv, rng = _case(H, W, seed=11 + psl)
    p = oracle.Params(psl=psl, kr=kr, it=it)
    g1, g2, gw, u, v = oracle.flow_grad(I1, I2, p, gu, gv)
    assert gw is None
    u0, v0 = oracle.flow(I1, I2, p)
    assert np.array_equal(u, u0) and np.array_equal(v, v0)
    for frame in (0, 1):
        d = rng.standard_normal((H, W))
        if frame == 0:
            fd = _fd_dir(lambda X: _loss(X, I2, p, gu, gv), I1, d, 1e-6)
            an = float(np.sum(g1 * d))
        else:
            fd = _fd_dir(lambda X: _loss(I1, X, p, gu, gv), I2, d, 1e-6)
            an = float(np.sum(g2 * d))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (frame, fd, an)


def test_single_pixel_perturbations_match_finite_differences():
    # entries of the gradient one by one at the border, the corner and inside
    H, W = 24, 28
    I1, I2, gu, gv, _ = _case(H, W, seed=5)
    p = oracle.Params(psl=1, kr=2, it=2)
    g1, g2, _, _, _ = oracle.flow_grad(I1, I2, p, gu, gv)
    for (i, j) in [(0, 0), (0, 13), (H - 1, W - 1), (12, 14), (7, 0)]:
        d = np.zeros((H, W))
        d[i, j] = 1.0
        fd1 = _fd_dir(lambda X: _loss(X, I2, p, gu, gv), I1, d, 1e-6)
        fd2 = _fd_dir(lambda X: _loss(I1, X, p, gu, gv), I2, d, 1e-6)
        assert abs(fd1 - g1[i, j]) <= 1e-6 * max(1.0, abs(g1[i, j])), (i, j, fd1, g1[i, j])
        assert abs(fd2 - g2[i, j]) <= 1e-6 * max(1.0, abs(g2[i, j])), (i, j, fd2, g2[i, j])


def test_prefilter_weight_gradient_matches_finite_differences():
    H, W = 34, 38
    I1, I2, gu, gv, rng = _case(H, W, seed=21)
    w = np.zeros((5, 5))
    w[2, 2] = 0.6
    w[1:4, 1:4] += 0.05
    w += 0.01 * rng.standard_normal((5, 5))
    p = oracle.Params(psl=1, kr=3, it=2, prefilter=w)
    g1, g2, gw, _, _ = oracle.flow_grad(I1, I2, p, gu, gv)
    assert gw.shape == (5, 5)

    def lw(wx):
        return _loss(I1, I2, oracle.Params(psl=1, kr=3, it=2, prefilter=wx), gu, gv)

    for _ in range(2):
        d = rng.standard_normal((5, 5))
        fd = _fd_dir(lw, w, d, 1e-6)
        an = float(np.sum(gw * d))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
    # frames through the pre-filter
    d = rng.standard_normal((H, W))
    fd = _fd_dir(lambda X: _loss(X, I2, p, gu, gv), I1, d, 1e-6)
    assert abs(fd - float(np.sum(g1 * d))) <= 1e-6 * max(1.0, abs(fd))


def test_gradient_is_linear_in_the_output_gradient():
    H, W = 30, 32
    I1, I2, gu, gv, rng = _case(H, W, seed=3)
    hu, hv = rng.standard_normal((H, W)), rng.standard_normal((H, W))
    p = oracle.Params(psl=1, kr=2, it=2, prefilter=np.full((5, 5), 0.04))
    a = oracle.flow_grad(I1, I2, p, gu, gv)
    b = oracle.flow_grad(I1, I2, p, hu, hv)
    c = oracle.flow_grad(I1, I2, p, gu - 2.0 * hu, gv - 2.0 * hv)
    for k in range(3):
        ref = a[k] - 2.0 * b[k]
        assert np.max(np.abs(c[k] - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))


def test_counts_input_scales_the_gradient_by_the_full_scale():
    # I = raw / (2^bits - 1): dL/draw = dL/dI / 4095 for 12-bit counts
    H, W = 28, 30
    I1, I2, gu, gv, _ = _case(H, W, seed=8)
    raw1, raw2 = I1 * 4095.0, I2 * 4095.0
    pf = oracle.Params(psl=1, kr=2, it=2)
    pb = oracle.Params(psl=1, kr=2, it=2, bits=12)
    f1, f2, _, uf, _ = oracle.flow_grad(I1, I2, pf, gu, gv)
    r1, r2, _, ur, _ = oracle.flow_grad(raw1, raw2, pb, gu, gv)
    assert np.max(np.abs(ur - uf)) < 1e-9
    assert np.max(np.abs(r1 * 4095.0 - f1)) <= 1e-8 * max(1.0, np.max(np.abs(f1)))
    assert np.max(np.abs(r2 * 4095.0 - f2)) <= 1e-8 * max(1.0, np.max(np.abs(f2)))


def test_zero_output_gradient_gives_zero():
    H, W = 20, 20
    I1, I2, _, _, _ = _case(H, W, seed=2)
    z = np.zeros((H, W))
    g1, g2, gw, _, _ = oracle.flow_grad(I1, I2, oracle.Params(psl=1, kr=2, it=2, prefilter=np.eye(5) * 0.2), z, z)
    assert not g1.any() and not g2.any() and not gw.any()


def test_constant_frames_give_zero_gradient():
    # constant frames: every window sum is 0, every pixel is guarded and keeps
    # V0 = 0, and the field is locally independent of the images
    H, W = 20, 22
    I1 = np.full((H, W), 0.3)
    I2 = np.full((H, W), 0.3)
    rng = np.random.default_rng(1)
    gu, gv = rng.standard_normal((H, W)), rng.standard_normal((H, W))
    g1, g2, gw, u, v = oracle.flow_grad(I1, I2, oracle.Params(psl=1, kr=2, it=2, prefilter=np.eye(5) * 0.2), gu, gv)
    assert not u.any() and not v.any()
    assert not g1.any() and not g2.any() and not gw.any()


@pytest.mark.parametrize("nr,with_prefilter", [(1, False), (2, False), (2, True)])
def test_normalization_gradients_match_finite_differences(nr, with_prefilter):
    """Local normalization (Sec. 2, step 1; radius NR) in the chain: frame
    gradients along random directions and single pixels at the corner, the
    border and inside, and the pre-filter weights, whose input is then the
    normalized frame.  Normalization divides by the local deviation (a few
    hundredths here), which magnifies an input step by up to ~100 at the
    warped samples; the step is 1e-7 so that the finite difference stays
    inside one bilinear cell (at 1e-6 one direction crosses a cell edge)."""
    H, W = 30, 34
    I1, I2, gu, gv, rng = _case(H, W, seed=40 + nr)
    w = None
    if with_prefilter:
        w = np.zeros((5, 5))
        w[2, 2] = 0.7
        w[1:4, 1:4] += 0.04
        w += 0.01 * rng.standard_normal((5, 5))
    p = oracle.Params(psl=1, kr=2, it=2, nr=nr, prefilter=w)
    g1, g2, gw, u, v = oracle.flow_grad(I1, I2, p, gu, gv)
    u0, v0 = oracle.flow(I1, I2, p)
    assert np.array_equal(u, u0) and np.array_equal(v, v0)
    for frame in (0, 1):
        d = rng.standard_normal((H, W))
        if frame == 0:
            fd = _fd_dir(lambda X: _loss(X, I2, p, gu, gv), I1, d, H_NR)
            an = float(np.sum(g1 * d))
        else:
            fd = _fd_dir(lambda X: _loss(I1, X, p, gu, gv), I2, d, H_NR)
            an = float(np.sum(g2 * d))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (frame, fd, an)
    for (i, j) in [(0, 0), (H - 1, 5), (15, 17)]:
        d = np.zeros((H, W))
        d[i, j] = 1.0
        fd = _fd_dir(lambda X: _loss(X, I2, p, gu, gv), I1, d, H_NR)
        assert abs(fd - g1[i, j]) <= 1e-6 * max(1.0, abs(g1[i, j])), (i, j, fd, g1[i, j])
    if with_prefilter:
        def lw(wx):
            return _loss(I1, I2, oracle.Params(psl=1, kr=2, it=2, nr=nr, prefilter=wx), gu, gv)
        d = rng.standard_normal((5, 5))
        fd = _fd_dir(lw, w, d, 1e-6)
        an = float(np.sum(gw * d))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_normalization_adjoint_of_a_constant_offset_is_zero():
    """Normalization removes the local mean: adding a constant to a frame
    changes nothing, so the gradient sums to zero over every box-closed
    direction -- in particular along the constant direction."""
    H, W = 26, 28
    I1, I2, gu, gv, _ = _case(H, W, seed=9)
    p = oracle.Params(psl=1, kr=2, it=2, nr=2)
    g1, g2, _, _, _ = oracle.flow_grad(I1, I2, p, gu, gv)
    assert abs(g1.sum()) <= 1e-9 * np.abs(g1).sum()
    assert abs(g2.sum()) <= 1e-9 * np.abs(g2).sum()
