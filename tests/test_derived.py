"""Quantities derived from the fields (Sec. 7): vorticity, the
recirculation area of Eq. 6 and point probes.

CPU pins of the oracle: numpy.gradient (an independent finite-difference
gradient with the same interior/border scheme), exactness on linear fields
(solid-body rotation has omega = 2 Omega everywhere, borders included) and
a brute-force count.  GPU parity (marked gpu): the CUDA kernels against the
oracle on the same FP32 fields -- vorticity within FP32 rounding of the two
differences, the recirculation count bit-exact (both compare the same FP32
values with 0).
"""
import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(7)


def test_vorticity_matches_numpy_gradient():
    for H, W in [(1, 1), (1, 5), (4, 1), (2, 2), (17, 23), (64, 48)]:
        u = RNG.standard_normal((H, W))
        v = RNG.standard_normal((H, W))
        ref = np.zeros((H, W))
        if W > 1:
            ref += np.gradient(v, axis=1)
        if H > 1:
            ref -= np.gradient(u, axis=0)
        assert np.max(np.abs(oracle.vorticity(u, v) - ref)) <= 1e-15


def test_solid_body_rotation_has_uniform_vorticity():
    H, W, om = 31, 40, 0.013
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    u = -om * (y - 15.3)
    v = om * (x - 19.7)
    w = oracle.vorticity(u, v)
    assert np.max(np.abs(w - 2 * om)) < 1e-15
    # a uniform translation has none
    assert not oracle.vorticity(np.full((H, W), 1.3), np.full((H, W), -0.7)).any()


def test_rankine_core_vorticity():
    # inside the core of the Rankine vortex the field is a solid-body rotation
    H = W = 128
    f = synth.rankine_field(H, W, R=32.0, dmax=3.0)
    u, v = f.grid(H, W)
    w = oracle.vorticity(u, v)
    # u_theta = dmax r / R inside the core: omega = 2 dmax / R
    assert abs(w[64, 64] - 2 * 3.0 / 32.0) < 2e-3


def test_recirculation_count_is_a_brute_force_count():
    u = RNG.standard_normal((37, 29))
    u[3, 4] = 0.0   # H(-0) = 0
    u[5, 6] = -0.0  # -0 < 0 is false
    mask = RNG.random((37, 29)) < 0.6
    assert oracle.recirculation_count(u) == int(np.sum(u < 0))
    assert oracle.recirculation_count(u, mask) == int(np.sum((u < 0) & mask))
    assert oracle.recirculation_count(np.ones((5, 5))) == 0


# ---------------------------------------------------------------------------
# GPU parity
# ---------------------------------------------------------------------------
def _fields(n, H, W, seed):
    r = np.random.default_rng(seed)
    u = r.standard_normal((n, H, W)).astype(np.float32)
    v = r.standard_normal((n, H, W)).astype(np.float32)
    return u, v


@pytest.mark.gpu
@pytest.mark.parametrize("n,H,W,pad", [(1, 1, 1, 5), (3, 2, 7, 5), (2, 97, 130, 5), (5, 256, 320, 5),
                                       (4, 64, 96, 4), (2, 3, 8, 0)])
def test_gpu_vorticity_matches_oracle(n, H, W, pad):
    torch = pytest.importorskip("torch")
    import paper_2509_25924_gb300 as ofv
    u, v = _fields(n, H, W, seed=H + W)
    dev = torch.device("cuda:0")
    stride = H * W + pad  # padded fields (a multiple of 4 takes the 16-byte path)
    tu = torch.zeros(n * stride + 5, device=dev)
    tv = torch.zeros_like(tu)
    for k in range(n):
        tu[k * stride:k * stride + H * W] = torch.from_numpy(u[k].ravel()).to(dev)
        tv[k * stride:k * stride + H * W] = torch.from_numpy(v[k].ravel()).to(dev)
    om = torch.full_like(tu, 7.0)
    ofv.ofv_vorticity(H, W, n, tu, tv, stride, om)
    torch.cuda.synchronize()
    got = om.cpu().numpy()
    for k in range(n):
        ref = oracle.vorticity(u[k].astype(np.float64), v[k].astype(np.float64))
        g = got[k * stride:k * stride + H * W].reshape(H, W)
        assert np.max(np.abs(g - ref)) <= 2e-6 * max(1.0, np.max(np.abs(ref)))
        assert np.all(got[k * stride + H * W:(k + 1) * stride] == 7.0)  # padding untouched


@pytest.mark.gpu
@pytest.mark.parametrize("masked,H,W", [(False, 301, 257), (True, 301, 257), (False, 300, 256), (True, 300, 256)])
def test_gpu_recirculation_count_is_exact(masked, H, W):
    torch = pytest.importorskip("torch")
    import paper_2509_25924_gb300 as ofv
    n = 6
    u, _ = _fields(n, H, W, seed=3)
    u[0] = np.abs(u[0])       # no recirculation
    u[1] = -np.abs(u[1]) - 1  # all of it
    u[2, 0, 0] = 0.0
    mask = (RNG.random((H, W)) < 0.5).astype(np.uint8) if masked else None
    dev = torch.device("cuda:0")
    tu = torch.from_numpy(u).to(dev)
    tm = torch.from_numpy(mask).to(dev) if masked else None
    counts = torch.full((n,), -1, dtype=torch.int64, device=dev)
    ofv.ofv_recirculation_area(H, W, n, tu, H * W, tm, counts)
    torch.cuda.synchronize()
    got = counts.cpu().numpy()
    for k in range(n):
        assert got[k] == oracle.recirculation_count(u[k].astype(np.float64), mask)


def test_probe_oracle_is_scipy_bilinear():
    """A probe is the estimator's bilinear interpolation (clamp-to-edge):
    scipy's map_coordinates(order=1, mode='nearest') at the same points."""
    from scipy import ndimage
    f = RNG.standard_normal((23, 31))
    pts = np.concatenate([RNG.uniform(-3, 34, (40, 2)), [[0, 0], [30, 22], [12.5, 7.25], [-0.5, 22.7]]])
    got = np.array([oracle.bilinear(f, x, y) for x, y in pts])
    ref = ndimage.map_coordinates(f, [pts[:, 1], pts[:, 0]], order=1, mode="nearest")
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.gpu
def test_gpu_probes_match_the_oracle_bilinear():
    torch = pytest.importorskip("torch")
    import paper_2509_25924_gb300 as ofv
    n, H, W, npts = 4, 77, 131, 300
    u, v = _fields(n, H, W, seed=11)
    u[2, 10, 20] = np.nan  # a pixel without a vector
    pts = np.concatenate([RNG.uniform(-4, W + 4, (npts - 4, 1)), RNG.uniform(-4, H + 4, (npts - 4, 1))], axis=1)
    pts = np.concatenate([pts, [[20.0, 10.0], [20.5, 10.5], [0.0, 0.0], [W - 1.0, H - 1.0]]]).astype(np.float32)
    dev = torch.device("cuda:0")
    tu = torch.from_numpy(u).to(dev); tv = torch.from_numpy(v).to(dev)
    out = torch.full((n, npts, 2), 7.0, device=dev)
    ofv.ofv_probe(H, W, n, tu, tv, H * W, npts, torch.from_numpy(pts).to(dev), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k in range(n):
        for p, (x, y) in enumerate(pts.astype(np.float64)):
            ru = oracle.bilinear(u[k].astype(np.float64), x, y)
            rv = oracle.bilinear(v[k].astype(np.float64), x, y)
            if np.isnan(ru):
                assert np.isnan(got[k, p, 0])
                continue
            assert abs(got[k, p, 0] - ru) <= 2e-6 * max(1.0, abs(ru)) and abs(got[k, p, 1] - rv) <= 2e-6 * max(1.0, abs(rv))
