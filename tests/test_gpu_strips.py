"""The strip-decomposed field (ofv_compute_strips) on one GPU.

One field is computed as N horizontal strips, each with its own pyramids
and fields: a strip computes its image rows plus a redundant halo from the
input rows around it, and after every Gauss-Newton iteration copies the
rows of the new field its next iteration reads from the strips that own
them -- the decomposition that spreads one large field over several GPUs
(the paper's "2 or 3 GPUs", Conclusions), run here strip after strip on the
one GPU a call gets.  The strips own whole tile rows of the block kernel's
grid at every level, so the result must equal ofv_compute's bitwise.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2509_25924_gb300 as ofv  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _both(I1, I2, nstrips, max_disp, w25=None, **kw):
    H, W = I1.shape
    p = ofv.ofv_default_params(**kw)
    h = ofv.ofv_create(H, W, p)
    try:
        if w25 is not None:
            ofv.ofv_set_prefilter(h, torch.tensor(np.asarray(w25, np.float32).reshape(25), device=DEV))
        t1 = torch.from_numpy(np.ascontiguousarray(I1)).to(DEV)
        t2 = torch.from_numpy(np.ascontiguousarray(I2)).to(DEV)
        u = torch.full((H, W), float("nan"), device=DEV)
        v = torch.full((H, W), float("nan"), device=DEV)
        ofv.ofv_compute(h, t1, t2, u, v)
        us = torch.full((H, W), float("nan"), device=DEV)
        vs = torch.full((H, W), float("nan"), device=DEV)
        ofv.ofv_compute_strips(h, nstrips, max_disp, t1, t2, us, vs)  # grows the strip workspace
        # then fill every workspace with NaN bytes: a row read before it was
        # written would show up in the second result
        ofv.ofv_debug_poison(h)
        us.fill_(float("nan"))
        vs.fill_(float("nan"))
        ofv.ofv_compute_strips(h, nstrips, max_disp, t1, t2, us, vs)
        torch.cuda.synchronize()
        return (u, v), (us, vs)
    finally:
        ofv.ofv_destroy(h)


@pytest.mark.parametrize("nstrips", [2, 4])
def test_21mp_wake_strips_are_bitwise_the_single_field(nstrips):
    I1, I2, _, _ = synth.wake_pair(seed=4)
    (u, v), (us, vs) = _both(I1, I2, nstrips, 8)
    assert torch.isfinite(us).all() and torch.isfinite(vs).all()
    assert torch.equal(us, u) and torch.equal(vs, v)


def test_1mp_stream_pair_three_strips():
    F = synth.stream_frames(1024, 1024, 2, seed=2)
    (u, v), (us, vs) = _both(F[0], F[1], 3, 8)
    assert torch.equal(us, u) and torch.equal(vs, v)


@pytest.mark.parametrize("storage", [ofv.OFV_STORE_F32, ofv.OFV_STORE_F16])
def test_small_field_more_strips_than_coarse_tile_rows(storage):
    """300 x 200 in 5 strips: the coarsest level has two tile rows, so three
    strips own nothing there; normalization and the pre-filter widen the
    input rows each strip ingests."""
    I1, I2, _, _ = synth.rankine_pair(300, 200, seed=5)
    w = np.zeros(25, np.float32)
    w[12] = 0.8
    w[[7, 11, 13, 17]] = 0.05
    (u, v), (us, vs) = _both(I1, I2, 5, 6, w25=w, input=ofv.OFV_IN_F32, storage=storage, norm_radius=2, prefilter=1)
    assert torch.equal(us, u) and torch.equal(vs, v)


def test_paper_parameters_two_strips():
    """8-bit input, NR 2, KR 10 (64-px tiles), IT 3, PSL 2 on 1 Mp."""
    F = synth.stream_frames(1024, 1024, 2, seed=7, ppp=0.05, bits=8).astype(np.uint8)
    (u, v), (us, vs) = _both(F[0], F[1], 2, 8, input=ofv.OFV_IN_U8, bit_depth=8, norm_radius=2, kernel_radius=10)
    assert torch.equal(us, u) and torch.equal(vs, v)


@pytest.mark.parametrize("kr,edge", [(4, 32), (10, 32), (6, 32)])
def test_alternative_tile_edge_strips(kr, edge):
    """The strips own whole rows of the tile grid of the shape tile_edge
    selects."""
    F = synth.stream_frames(700, 900, 2, seed=11)
    (u, v), (us, vs) = _both(F[0], F[1], 3, 8, kernel_radius=kr, tile_edge=edge)
    assert torch.equal(us, u) and torch.equal(vs, v)


def test_strips_refuse_a_mask_and_bad_counts():
    h = ofv.ofv_create(128, 128, ofv.ofv_default_params(input=ofv.OFV_IN_F32))
    try:
        t = torch.zeros((128, 128), device=DEV)
        u = torch.empty_like(t)
        v = torch.empty_like(t)
        with pytest.raises(ofv.OfvError) as ei:
            ofv.ofv_compute_strips(h, 0, 8, t, t, u, v)
        assert ei.value.status == ofv.OFV_ERR_INVALID_ARG
        ofv.ofv_set_mask(h, torch.ones((128, 128), dtype=torch.uint8, device=DEV))
        with pytest.raises(ofv.OfvError) as ei:
            ofv.ofv_compute_strips(h, 2, 8, t, t, u, v)
        assert ei.value.status == ofv.OFV_ERR_UNSUPPORTED
    finally:
        ofv.ofv_destroy(h)
