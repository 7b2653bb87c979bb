"""GPU parity of the reverse mode: ofv_backward through the C ABI, and the
torch.autograd wrapper, vs the FP64 oracle's reverse mode on the same seeded
inputs.

Tolerance (written here): relative L2 error of each gradient
||g_gpu - g_oracle|| / ||g_oracle|| <= 1e-4 for FP32 storage (measured 2e-7
to 2e-6 on smooth pairs and particle images, 8e-6 for the pre-filter
weights) and 5e-3 for FP16 level storage (measured 6e-4).  The gradient
multiplies FP32 round-off by the condition number of each 2x2 system and by
the slopes of the bilinear cells, so it is compared in the aggregate rather
than element by element; float atomics make the last bits vary between
runs.  A finite difference of the GPU forward pass along random pre-filter
directions checks the GPU gradient without the oracle (h = 3e-3, measured
1.6e-4 relative, bound 2e-3).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2509_25924_gb300 as ofv  # noqa: E402
from paper_2509_25924_gb300.autograd import flow_fn  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
_IN = {np.dtype(np.float32): ofv.OFV_IN_F32, np.dtype(np.uint16): ofv.OFV_IN_U16,
       np.dtype(np.uint8): ofv.OFV_IN_U8}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def gpu_grad(I1, I2, gu, gv, w25=None, bits=12, **kw):
    H, W = I1.shape
    kw.setdefault("input", _IN[I1.dtype])
    kw.setdefault("bit_depth", bits)
    if w25 is not None:
        kw["prefilter"] = 1
    h = ofv.ofv_create(H, W, ofv.ofv_default_params(**kw))
    try:
        t1 = torch.from_numpy(np.ascontiguousarray(I1)).to(DEV)
        t2 = torch.from_numpy(np.ascontiguousarray(I2)).to(DEV)
        if w25 is not None:
            ofv.ofv_set_prefilter(h, torch.tensor(np.asarray(w25, np.float32).reshape(25), device=DEV))
        tgu = torch.from_numpy(gu.astype(np.float32)).to(DEV)
        tgv = torch.from_numpy(gv.astype(np.float32)).to(DEV)
        g1 = torch.empty((H, W), dtype=torch.float32, device=DEV)
        g2 = torch.empty_like(g1)
        gw = torch.empty(25, dtype=torch.float32, device=DEV)
        ofv.ofv_backward(h, t1, t2, tgu, tgv, g1, g2, gw)
        torch.cuda.synchronize()
        return g1.cpu().numpy(), g2.cpu().numpy(), gw.cpu().numpy().reshape(5, 5)
    finally:
        ofv.ofv_destroy(h)


def oracle_grad(I1, I2, gu, gv, w25=None, bits=12, psl=2, kr=4, it=3, nr=0):
    b = bits if I1.dtype != np.float32 else 0
    p = oracle.Params(psl=psl, kr=kr, it=it, nr=nr, bits=b, prefilter=w25)
    g1, g2, gw, _, _ = oracle.flow_grad(I1.astype(np.float64), I2.astype(np.float64), p, gu, gv)
    return g1, g2, gw


def _smooth(H, W, seed, shift=(0.8, -0.5)):
    I1, I2 = synth.smooth_pair(H, W, shift, seed=seed)
    rng = np.random.default_rng(seed)
    return (I1.astype(np.float32), I2.astype(np.float32),
            rng.standard_normal((H, W)), rng.standard_normal((H, W)))


@pytest.mark.parametrize("H,W,psl,kr,it", [(64, 72, 1, 2, 2), (97, 83, 2, 4, 3), (48, 48, 0, 3, 1),
                                           (80, 96, 1, 12, 2)])
def test_frame_gradients_match_oracle(H, W, psl, kr, it):
    I1, I2, gu, gv = _smooth(H, W, seed=H + W)
    g1, g2, _ = gpu_grad(I1, I2, gu, gv, levels_psl=psl, kernel_radius=kr, iterations=it)
    o1, o2, _ = oracle_grad(I1, I2, gu, gv, psl=psl, kr=kr, it=it)
    assert _rel(g1, o1) <= 1e-4, _rel(g1, o1)
    assert _rel(g2, o2) <= 1e-4, _rel(g2, o2)


def test_prefilter_weight_gradient_matches_oracle():
    H, W = 70, 66
    I1, I2, gu, gv = _smooth(H, W, seed=4)
    rng = np.random.default_rng(4)
    w = np.zeros((5, 5))
    w[2, 2] = 0.6
    w[1:4, 1:4] += 0.05
    w = (w + 0.01 * rng.standard_normal((5, 5))).astype(np.float32)
    g1, g2, gw = gpu_grad(I1, I2, gu, gv, w25=w, levels_psl=1, kernel_radius=3, iterations=2)
    o1, o2, ow = oracle_grad(I1, I2, gu, gv, w25=w.astype(np.float64), psl=1, kr=3, it=2)
    assert _rel(gw, ow) <= 1e-4, _rel(gw, ow)
    assert _rel(g1, o1) <= 1e-4 and _rel(g2, o2) <= 1e-4


def test_prefilter_gradient_matches_gpu_finite_differences():
    # central differences of the GPU forward pass (FP32) along random
    # directions of the 25 weights, against ofv_backward
    H, W = 70, 66
    I1, I2, gu, gv = _smooth(H, W, seed=4)
    rng = np.random.default_rng(4)
    w = np.zeros((5, 5))
    w[2, 2] = 0.6
    w[1:4, 1:4] += 0.05
    w = (w + 0.01 * rng.standard_normal((5, 5))).astype(np.float32)
    _, _, gw = gpu_grad(I1, I2, gu, gv, w25=w, levels_psl=1, kernel_radius=3, iterations=2)
    p = ofv.ofv_default_params(input=ofv.OFV_IN_F32, prefilter=1, levels_psl=1, kernel_radius=3, iterations=2)
    h = ofv.ofv_create(H, W, p)
    try:
        t1 = torch.from_numpy(I1).to(DEV)
        t2 = torch.from_numpy(I2).to(DEV)
        u = torch.empty((H, W), device=DEV)
        v = torch.empty_like(u)

        def loss(wx):
            ofv.ofv_set_prefilter(h, torch.tensor(wx.reshape(25), dtype=torch.float32, device=DEV))
            ofv.ofv_compute(h, t1, t2, u, v)
            torch.cuda.synchronize()
            return float((u.double().cpu().numpy() * gu).sum() + (v.double().cpu().numpy() * gv).sum())

        for trial in range(2):
            d = np.random.default_rng(100 + trial).standard_normal((5, 5))
            fd = (loss(w + 3e-3 * d) - loss(w - 3e-3 * d)) / 6e-3
            an = float((gw * d).sum())
            assert abs(fd - an) <= 2e-3 * abs(an), (fd, an)
    finally:
        ofv.ofv_destroy(h)


@pytest.mark.parametrize("dtype,bits", [(np.uint16, 12), (np.uint8, 8)])
def test_particle_images_counts_input(dtype, bits):
    kind = synth.OUT_U16 if dtype == np.uint16 else synth.OUT_U8
    I1, I2 = synth.particle_pair(160, 176, synth.rankine_field(160, 176), ppp=0.05, dmin=2.5, dmax=2.5, seed=6,
                                 noise=0.01, kind=kind, bits=bits, field_max=3.0)
    assert I1.dtype == dtype
    rng = np.random.default_rng(6)
    gu, gv = rng.standard_normal(I1.shape), rng.standard_normal(I1.shape)
    g1, g2, _ = gpu_grad(I1, I2, gu, gv, bits=bits)
    o1, o2, _ = oracle_grad(I1, I2, gu, gv, bits=bits)
    assert _rel(g1, o1) <= 1e-4, _rel(g1, o1)
    assert _rel(g2, o2) <= 1e-4, _rel(g2, o2)


@pytest.mark.parametrize("storage,tol", [(ofv.OFV_STORE_F16, 5e-3), (ofv.OFV_STORE_BF16, 4e-2)])
def test_reduced_storage_gradient(storage, tol):
    # level images rounded to 11 (FP16) or 8 (BF16) significant bits
    I1, I2, gu, gv = _smooth(64, 80, seed=9)
    g1, g2, _ = gpu_grad(I1, I2, gu, gv, storage=storage, levels_psl=1, kernel_radius=3, iterations=2)
    o1, o2, _ = oracle_grad(I1, I2, gu, gv, psl=1, kr=3, it=2)
    assert _rel(g1, o1) <= tol and _rel(g2, o2) <= tol, (_rel(g1, o1), _rel(g2, o2))


def test_zero_output_gradient_gives_zero():
    I1, I2, _, _ = _smooth(48, 56, seed=2)
    z = np.zeros(I1.shape)
    g1, g2, gw = gpu_grad(I1, I2, z, z, w25=np.full((5, 5), 0.04, np.float32), levels_psl=1, kernel_radius=2,
                          iterations=2)
    assert not g1.any() and not g2.any() and not gw.any()


@pytest.mark.parametrize("nr,with_prefilter", [(1, False), (2, False), (2, True)])
def test_normalization_gradients_match_oracle(nr, with_prefilter):
    """Reverse mode through local normalization (Sec. 2 step 1): frames and
    pre-filter weights against the FP64 reverse mode."""
    H, W = 72, 84
    I1, I2, gu, gv = _smooth(H, W, seed=30 + nr)
    w = None
    if with_prefilter:
        w = np.zeros((5, 5), np.float32)
        w[2, 2] = 0.7
        w[1:4, 1:4] += 0.04
    g1, g2, gw = gpu_grad(I1, I2, gu, gv, w25=w, norm_radius=nr, levels_psl=1, kernel_radius=3, iterations=2)
    o1, o2, ow = oracle_grad(I1, I2, gu, gv, w25=None if w is None else w.astype(np.float64), psl=1, kr=3, it=2,
                             nr=nr)
    assert _rel(g1, o1) <= 1e-4, _rel(g1, o1)
    assert _rel(g2, o2) <= 1e-4, _rel(g2, o2)
    if with_prefilter:
        assert _rel(gw, ow) <= 1e-4, _rel(gw, ow)


def test_paper_parameters_gradient_matches_oracle():
    """8-bit particle images with the paper's benchmark parameters (NR 2,
    KR 10, IT 3; Sec. 6), PSL 1."""
    I1, I2 = synth.particle_pair(150, 170, synth.rankine_field(150, 170), ppp=0.05, dmin=2.5, dmax=2.5, seed=8,
                                 noise=0.01, kind=synth.OUT_U8, bits=8, field_max=3.0)
    rng = np.random.default_rng(8)
    gu, gv = rng.standard_normal(I1.shape), rng.standard_normal(I1.shape)
    g1, g2, _ = gpu_grad(I1, I2, gu, gv, bits=8, norm_radius=2, levels_psl=1, kernel_radius=10, iterations=3)
    o1, o2, _ = oracle_grad(I1, I2, gu, gv, bits=8, psl=1, kr=10, it=3, nr=2)
    assert _rel(g1, o1) <= 1e-4, _rel(g1, o1)
    assert _rel(g2, o2) <= 1e-4, _rel(g2, o2)


def test_autograd_function_matches_c_abi_and_oracle():
    H, W = 72, 80
    I1, I2, gu, gv = _smooth(H, W, seed=12)
    w = np.zeros((5, 5), np.float32)
    w[2, 2] = 0.7
    w[1:4, 1:4] += 0.03
    flow = ofv.Flow(H, W, input=ofv.OFV_IN_F32, prefilter=1, levels_psl=1, kernel_radius=3, iterations=2)
    try:
        t1 = torch.from_numpy(I1).to(DEV).requires_grad_(True)
        t2 = torch.from_numpy(I2).to(DEV).requires_grad_(True)
        tw = torch.from_numpy(w).to(DEV).requires_grad_(True)
        u, v = flow_fn(flow, t1, t2, tw)
        loss = (u * torch.from_numpy(gu.astype(np.float32)).to(DEV)).sum() + \
               (v * torch.from_numpy(gv.astype(np.float32)).to(DEV)).sum()
        loss.backward()
        o1, o2, ow = oracle_grad(I1, I2, gu, gv, w25=w.astype(np.float64), psl=1, kr=3, it=2)
        assert _rel(t1.grad.cpu().numpy(), o1) <= 1e-4
        assert _rel(t2.grad.cpu().numpy(), o2) <= 1e-4
        assert _rel(tw.grad.cpu().numpy(), ow) <= 1e-4
        # forward of the autograd node is the plain estimator
        ou, ov = oracle.flow(I1.astype(np.float64), I2.astype(np.float64),
                             oracle.Params(psl=1, kr=3, it=2, prefilter=w.astype(np.float64)))
        assert np.max(np.abs(u.detach().cpu().numpy() - ou)) < 1e-3
    finally:
        flow.close()


def test_prefilter_training_step_lowers_the_loss():
    # a few gradient steps on the pre-filter weights against a known field
    H, W = 96, 96
    d = (1.3, -0.6)
    I1, I2 = synth.smooth_pair(H, W, d, seed=31)
    I1, I2 = I1.astype(np.float32), I2.astype(np.float32)
    flow = ofv.Flow(H, W, input=ofv.OFV_IN_F32, prefilter=1, levels_psl=1, kernel_radius=4, iterations=1)
    try:
        t1 = torch.from_numpy(I1).to(DEV)
        t2 = torch.from_numpy(I2).to(DEV)
        w = torch.zeros((5, 5), device=DEV)
        w[2, 2] = 1.0
        w[0, 0] = 0.3  # a bad start: the ideal filter is symmetric
        w.requires_grad_(True)
        opt = torch.optim.SGD([w], lr=5e-2)
        losses = []
        for _ in range(6):
            opt.zero_grad()
            u, v = flow_fn(flow, t1, t2, w)
            loss = ((u - d[0]) ** 2).mean() + ((v - d[1]) ** 2).mean()
            loss.backward()
            losses.append(float(loss))
            opt.step()
        # FP64 reverse mode with the same steps: 0.00993 -> 0.00911
        assert losses[-1] < 0.97 * losses[0], losses
    finally:
        flow.close()


def test_flow_apply_entry_matches_flow_fn():
    H, W = 64, 72
    I1, I2, gu, gv = _smooth(H, W, seed=21)
    w = np.zeros((5, 5), np.float32)
    w[2, 2] = 0.8
    w[2, 1] = w[2, 3] = 0.1
    params = dict(levels_psl=1, kernel_radius=3, iterations=2)
    tgu = torch.from_numpy(gu.astype(np.float32)).to(DEV)
    tgv = torch.from_numpy(gv.astype(np.float32)).to(DEV)
    grads = []
    for use_apply in (True, False):
        t1 = torch.from_numpy(I1).to(DEV).requires_grad_(True)
        t2 = torch.from_numpy(I2).to(DEV).requires_grad_(True)
        tw = torch.from_numpy(w).to(DEV).requires_grad_(True)
        if use_apply:
            u, v = ofv.Flow.apply(t1, t2, tw, params)
        else:
            flow = ofv.Flow(H, W, input=ofv.OFV_IN_F32, prefilter=1, **params)
            u, v = flow_fn(flow, t1, t2, tw)
        ((u * tgu).sum() + (v * tgv).sum()).backward()
        grads.append((u.detach().cpu().numpy(), t1.grad.cpu().numpy(), tw.grad.cpu().numpy()))
        if not use_apply:
            flow.close()
    assert np.array_equal(grads[0][0], grads[1][0])
    assert _rel(grads[0][1], grads[1][1]) <= 1e-5 and _rel(grads[0][2], grads[1][2]) <= 1e-5
